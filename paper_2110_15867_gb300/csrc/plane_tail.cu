// plane_tail.cu -- the tail D_uz D_uy of a kick (Eq. 4 for i = 2, 3) in one pass over
// f for velocity cubes too large for one CTA (n_uy = n_uz = 48).
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
// 16-bit storage: the planes are decoded into FP32 as they are staged; D_uy's result
// stays FP32 and each row is encoded once, after D_uz, with a refreshed line scale (the
// rounding points of the fused tail of smaller cubes, not of the separate sweeps).
#include "vk_lines.cuh"

namespace vk {

namespace {

constexpr int kPlanesPerBlock = 4;

template <int NU> constexpr int plane_pitch() { return NU + 1; }
template <int NU> constexpr size_t plane_smem() { return size_t(kPlanesPerBlock) * NU * plane_pitch<NU>() * sizeof(float); }

template <int NU, typename T>
__global__ void __launch_bounds__(kPlanesPerBlock * NU) plane_tail_kernel(T *__restrict__ f, const __grid_constant__ PlaneTailArgs a)
{
    constexpr bool CODED = sizeof(T) == 2;
    constexpr int P = plane_pitch<NU>(), PER = 16 / int(sizeof(T)), Q = NU * NU / PER; // 16-byte chunks per plane
    extern __shared__ __align__(16) float plane_s[];
    const long long p0 = a.plane0 + blockIdx.x * (long long)kPlanesPerBlock; // first plane of the block
    const long long pend = a.plane0 + a.nplanes;
    // stage the planes (a plane is NU rows of NU values, contiguous; NU % PER == 0, so a
    // 16-byte chunk never straddles two rows); codes are decoded with their row's scale
    for (int k = threadIdx.x; k < kPlanesPerBlock * Q; k += blockDim.x) {
        const int q = k / Q, e = PER * (k - q * Q), row = e / NU, col = e - row * NU;
        if (p0 + q < pend) {
            float *s = plane_s + (q * NU + row) * P + col;
            if constexpr (CODED) {
                float v[PER];
                Chunk<T>::get(reinterpret_cast<const unsigned char *>(f + (p0 + q) * NU * NU) + 16 * (k - q * Q),
                              a.scale[(p0 + q) * NU + row], v);
#pragma unroll
                for (int i = 0; i < PER; ++i) s[i] = v[i];
            } else {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(f + (p0 + q) * NU * NU) + (k - q * Q));
                s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
            }
        }
    }
    __syncthreads();
    // the block's planes belong to one spatial cell (the host checks n_ux % 4 == 0)
    const long long cell = p0 / a.nux;
    const int q = threadIdx.x / NU, l = threadIdx.x - q * NU;
    float *plane = plane_s + q * NU * P;
    bool bad = false, any = false;
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
            any = true;
        }
        __syncthreads();
    }
    if constexpr (CODED) {
        // thread l encodes row l (a u_z line) of its plane as the u_z sweep does: the new
        // scale is the row's largest value; stochastic rounding with the stream that sweep
        // draws for the line.  A plane neither sweep touched keeps its codes.
        if (p0 + q < pend && any) {
            const long long line = (p0 + q) * NU + l;
            const float *s = plane + l * P;
            float v[NU], m = 0.f;
#pragma unroll
            for (int j = 0; j < NU; ++j) {
                v[j] = s[j];
                m = fmaxf(m, v[j]);
            }
            m = coded_scale<T>(m);
            a.scale[line] = m;
            const float inv = inv_scale(m);
            unsigned rng = sr_bits((unsigned long long)line * NU, a.seed);
            unsigned char *dst = reinterpret_cast<unsigned char *>(f + line * NU);
#pragma unroll
            for (int c = 0; c < NU / PER; ++c) {
                float e[PER];
#pragma unroll
                for (int i = 0; i < PER; ++i) e[i] = v[PER * c + i];
                Chunk<T>::put(dst + 16 * c, inv, e, rng);
            }
        }
    } else {
        for (int k = threadIdx.x; k < kPlanesPerBlock * Q; k += blockDim.x) {
            const int qq = k / Q, e = 4 * (k - qq * Q), row = e / NU, col = e - row * NU;
            if (p0 + qq < pend) {
                const float *s = plane_s + (qq * NU + row) * P + col;
                reinterpret_cast<float4 *>(f + (p0 + qq) * NU * NU)[k - qq * Q] = make_float4(s[0], s[1], s[2], s[3]);
            }
        }
    }
    if (bad) atomicOr(a.err, ERR_NAN);
}

} // namespace

bool plane_tail_supported(int nuy, int nuz, int nux, int dtype)
{
    return dtype >= 1 && dtype <= 3 && nuy == nuz && nuz == 48 && nux % kPlanesPerBlock == 0;
}

template <typename T> static cudaError_t launch_plane_tail_t(T *f, const PlaneTailArgs &a, long long blocks, cudaStream_t st)
{
    const cudaError_t e = cudaFuncSetAttribute(plane_tail_kernel<48, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               int(plane_smem<48>()));
    if (e != cudaSuccess) return e;
    plane_tail_kernel<48, T><<<unsigned(blocks), kPlanesPerBlock * 48, plane_smem<48>(), st>>>(f, a);
    return cudaGetLastError();
}

cudaError_t launch_plane_tail(void *f, const PlaneTailArgs &a, int nu, int dtype, cudaStream_t st)
{
    if (a.nplanes <= 0) return cudaSuccess;
    if (nu != 48 || a.plane0 % kPlanesPerBlock || a.nplanes % kPlanesPerBlock) return cudaErrorInvalidValue;
    if (dtype != 1 && !a.scale) return cudaErrorInvalidValue;
    const long long blocks = a.nplanes / kPlanesPerBlock;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    switch (dtype) {
    case 1: return launch_plane_tail_t(static_cast<float *>(f), a, blocks, st);
    case 2: return launch_plane_tail_t(static_cast<__nv_bfloat16 *>(f), a, blocks, st);
    case 3: return launch_plane_tail_t(static_cast<__half *>(f), a, blocks, st);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace vk
