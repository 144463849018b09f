// plane_tail.cu -- the tail D_uz D_uy of a kick (Eq. 4 for i = 2, 3) in one pass over
// f for FP32 velocity cubes too large for one CTA (n_uy = n_uz = 48).
//
// A (cell, j_x) plane of the velocity cube holds n_uy rows (j_y) of n_uz cells (j_z),
// contiguous in f (Listing 1: u_z innermost), and both sweeps stay inside it.  A
// block stages four planes of one spatial cell in shared memory (rows padded to
// n_uz + 1 floats, so that a warp walking columns and a warp walking rows both hit 32
// different banks), 48 threads per plane march its columns (D_uy), then its rows
// (D_uz), and the block writes the planes back: f is read and written once for the
// two sweeps instead of twice.  Each line is marched in shared memory through a
// window of five cells in registers (march_strided, one body for both sweeps, faces in
// blocks of 8), the arithmetic of march_regs in the same order, so the result equals the
// separate u_y and u_z sweeps bit for bit.
// The stride of a line (its axis and the sign of its Courant number) is a run-time
// value: one march body for both axes and signs (four compile-time bodies measured
// slower: 43.9 against 41.0 ms on the 48^3 x 48^3 run).
#include "vk_lines.cuh"

namespace vk {

namespace {

constexpr int kPlanesPerBlock = 4;

template <int NU> constexpr int plane_pitch() { return NU + 1; }
template <int NU> constexpr size_t plane_smem() { return size_t(kPlanesPerBlock) * NU * plane_pitch<NU>() * sizeof(float); }

template <int NU>
__global__ void __launch_bounds__(kPlanesPerBlock * NU) plane_tail_kernel(float *__restrict__ f, const __grid_constant__ PlaneTailArgs a)
{
    constexpr int P = plane_pitch<NU>(), Q = NU * NU / 4; // 16-byte chunks per plane
    extern __shared__ __align__(16) float plane_s[];
    const long long p0 = a.plane0 + blockIdx.x * (long long)kPlanesPerBlock; // first plane of the block
    const long long pend = a.plane0 + a.nplanes;
    // stage the planes (a plane is NU rows of NU floats, contiguous; NU % 4 == 0, so a
    // 16-byte chunk never straddles two rows)
    for (int k = threadIdx.x; k < kPlanesPerBlock * Q; k += blockDim.x) {
        const int q = k / Q, e = 4 * (k - q * Q), row = e / NU, col = e - row * NU;
        if (p0 + q < pend) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(f + (p0 + q) * NU * NU) + (k - q * Q));
            float *s = plane_s + (q * NU + row) * P + col;
            s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
        }
    }
    __syncthreads();
    // the block's planes belong to one spatial cell (the host checks n_ux % 4 == 0)
    const long long cell = p0 / a.nux;
    const int q = threadIdx.x / NU, l = threadIdx.x - q * NU;
    float *plane = plane_s + q * NU * P;
    bool bad = false;
    // D_uy (column l, rows 0 .. NU-1), then D_uz (row l): one march body for both
#pragma unroll 1
    for (int ax = 0; ax < 2; ++ax) {
        const LineCoefT<float> k = ax == 0 ? a.coef_y[cell] : a.coef_z[cell];
        if (p0 + q < pend && k.nd >= 0) {
            // from the far end when the Courant number is negative
            const bool neg = k.nd & 1;
            const int step = ax == 0 ? P : 1;
            float *first = plane + (ax == 0 ? l : l * P) + (neg ? (NU - 1) * step : 0);
            const float sum = march_strided<NU>(first, neg ? -step : step, to_lim(k));
            bad |= !(sum >= 0.f) || isinf(sum);
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < kPlanesPerBlock * Q; k += blockDim.x) {
        const int qq = k / Q, e = 4 * (k - qq * Q), row = e / NU, col = e - row * NU;
        if (p0 + qq < pend) {
            const float *s = plane_s + (qq * NU + row) * P + col;
            reinterpret_cast<float4 *>(f + (p0 + qq) * NU * NU)[k - qq * Q] = make_float4(s[0], s[1], s[2], s[3]);
        }
    }
    if (bad) atomicOr(a.err, ERR_NAN);
}

} // namespace

bool plane_tail_supported(int nuy, int nuz, int nux, int dtype)
{
    return dtype == 1 && nuy == nuz && nuz == 48 && nux % kPlanesPerBlock == 0;
}

cudaError_t launch_plane_tail(float *f, const PlaneTailArgs &a, int nu, cudaStream_t st)
{
    if (a.nplanes <= 0) return cudaSuccess;
    if (nu != 48 || a.plane0 % kPlanesPerBlock || a.nplanes % kPlanesPerBlock) return cudaErrorInvalidValue;
    const long long blocks = a.nplanes / kPlanesPerBlock;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    const cudaError_t e = cudaFuncSetAttribute(plane_tail_kernel<48>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               int(plane_smem<48>()));
    if (e != cudaSuccess) return e;
    plane_tail_kernel<48><<<unsigned(blocks), kPlanesPerBlock * 48, plane_smem<48>(), st>>>(f, a);
    return cudaGetLastError();
}

} // namespace vk
