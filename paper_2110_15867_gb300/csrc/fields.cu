// fields.cu -- the small spatial-grid kernels around the sweeps
// (Yoshikawa, Tanaka & Yoshida, SC'21):
//   * velocity-sweep coefficients: g_i = d phi / d x_i by the periodic
//     4th-order central difference (the "differentiating" of the PM potential,
//     Sec. 4.1.2) and the Courant number nu = -g_i dt / du of Eq. (4);
//   * the density moment rho_nu(x) = int f d^3u (Sec. 4.1.3: every spatial
//     cell holds its whole velocity cube, so the moment needs no exchange);
//   * the total mass (compensated FP64);
//   * the periodic Poisson solve of Eq. (2) by discrete Fourier transform
//     (the convolution method of Sec. 4.1.2 on one GPU).
#include <type_traits>

#include "vk_common.cuh"

namespace vk {

// ----------------------------------------------------------------------------
// velocity-sweep coefficients
// ----------------------------------------------------------------------------

template <typename C>
__global__ void velocity_coef_kernel(GridDims g, const float *__restrict__ phi, double dt, int mask,
                                     LineCoefT<C> *cx, LineCoefT<C> *cy, LineCoefT<C> *cz, unsigned *err)
{
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int iz = int(c % g.n[2]);
        const int iy = int((c / g.n[2]) % g.n[1]);
        const int ix = int(c / ((long long)g.n[2] * g.n[1]));
        const int idx[3] = {ix, iy, iz};
        LineCoefT<C> *outs[3] = {cx, cy, cz};
        for (int d = 0; d < 3; ++d) {
            if (!(mask & (1 << d))) continue;
            double v[5];
            for (int o = -2; o <= 2; ++o) {
                int q[3] = {idx[0], idx[1], idx[2]};
                q[d] = (q[d] + o + 2 * g.n[d]) % g.n[d];
                v[o + 2] = (double)phi[((long long)q[0] * g.n[1] + q[1]) * g.n[2] + q[2]];
            }
            const double h = g.L / g.n[d];
            const double grad = (8.0 * (v[3] - v[1]) - (v[4] - v[0])) / (12.0 * h);
            const double du = 2.0 * g.V / g.nu[d];
            const double nu = -grad * dt / du;
            LineCoefT<C> k = make_line_coef<C>(nu);
            if (!(fabs(nu) < 1.0)) { // also catches NaN
                k.nd = -1;
                atomicOr(err, ERR_CFL);
            }
            outs[d][c] = k;
        }
    }
}

cudaError_t launch_velocity_coef(const GridDims &g, const float *phi, double dt, int mask, void *coef_x,
                                 void *coef_y, void *coef_z, int dtype, unsigned *err, cudaStream_t st)
{
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    const int threads = 256;
    const int blocks = int((ncell + threads - 1) / threads < 4096 ? (ncell + threads - 1) / threads : 4096);
    if (dtype == 0)
        velocity_coef_kernel<double><<<blocks, threads, 0, st>>>(
            g, phi, dt, mask, (LineCoefT<double> *)coef_x, (LineCoefT<double> *)coef_y,
            (LineCoefT<double> *)coef_z, err);
    else
        velocity_coef_kernel<float><<<blocks, threads, 0, st>>>(
            g, phi, dt, mask, (LineCoefT<float> *)coef_x, (LineCoefT<float> *)coef_y,
            (LineCoefT<float> *)coef_z, err);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// moment
// ----------------------------------------------------------------------------

// Neumaier step in the working precision: (s, c) accumulates x exactly up to
// the second-order term; s + c is formed only in FP64.
__device__ __forceinline__ void neumaier(float &s, float &c, float x)
{
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// One CTA per spatial cell (grid-stride): FP32 compensated partial sums over
// 16-byte vectors, combined in FP64 across the CTA in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) moment_kernel(GridDims g, const T *__restrict__ f, double *rho)
{
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long cube = (long long)g.nu[0] * g.nu[1] * g.nu[2];
    const double du3 = (2.0 * g.V / g.nu[0]) * (2.0 * g.V / g.nu[1]) * (2.0 * g.V / g.nu[2]);
    __shared__ double part[8];
    for (long long c = blockIdx.x; c < ncell; c += gridDim.x) {
        const T *q = f + c * cube;
        double tot;
        if (sizeof(T) == 8) {
            double s = 0.0, e = 0.0;
            for (long long k = threadIdx.x; k < cube; k += blockDim.x) {
                const double x = (double)q[k];
                const double t = s + x;
                e += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
                s = t;
            }
            tot = s + e;
        } else {
            float s = 0.f, e = 0.f;
            const float4 *q4 = reinterpret_cast<const float4 *>(q);
            const long long n4 = cube / 4;
            for (long long k = threadIdx.x; k < n4; k += blockDim.x) {
                const float4 v = q4[k];
                neumaier(s, e, v.x);
                neumaier(s, e, v.y);
                neumaier(s, e, v.z);
                neumaier(s, e, v.w);
            }
            tot = (double)s + (double)e;
        }
        tot = warp_sum_d(tot);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = tot;
        __syncthreads();
        if (threadIdx.x == 0) {
            double r = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += part[w];
            rho[c] = du3 * r;
        }
        __syncthreads();
    }
}

// 16-bit storage: value = code * scale of its u_z line; 16-byte vectors of 8
// codes never straddle a line (n_uz is a multiple of 8).
template <typename T>
__global__ void __launch_bounds__(256) moment_coded_kernel(GridDims g, const T *__restrict__ f,
                                                           const float *__restrict__ scale, double *rho)
{
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    const int nuz = g.nu[2];
    const long long lines = (long long)g.nu[0] * g.nu[1];
    const long long cube = lines * nuz;
    const double du3 = (2.0 * g.V / g.nu[0]) * (2.0 * g.V / g.nu[1]) * (2.0 * g.V / g.nu[2]);
    __shared__ double part[8];
    // 16-byte vectors per line: 2 or 4 (n_uz 16 or 32, a shift), else 3, 5 or 6 (n_uz 24, 40, 48)
    const int vpl = nuz / 8, vshift = nuz == 32 ? 2 : 1;
    const bool pow2 = nuz == 16 || nuz == 32;
    for (long long c = blockIdx.x; c < ncell; c += gridDim.x) {
        const uint4 *q = reinterpret_cast<const uint4 *>(f + c * cube);
        const float *sc = scale + c * lines;
        float s = 0.f, e = 0.f;
        for (int k = threadIdx.x; k < int(cube / 8); k += blockDim.x) {
            const uint4 v = q[k];
            const unsigned u[4] = {v.x, v.y, v.z, v.w};
            // eight codes of 8 (BF16) or 11 (FP16) significant bits: their FP32 sum is
            // exact or off by the last bit
            float t = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 x;
                if (std::is_same<T, __nv_bfloat16>::value)
                    x = make_float2(__uint_as_float(u[j] << 16), __uint_as_float(u[j] & 0xffff0000u));
                else
                    x = __half22float2(*reinterpret_cast<const __half2 *>(&u[j]));
                t += x.x + x.y;
            }
            // the product and its rounding error (exact, by FMA) both enter the sum
            const float w = sc[pow2 ? k >> vshift : k / vpl];
            const float pr = t * w;
            neumaier(s, e, pr);
            e += fmaf(t, w, -pr);
        }
        double tot = warp_sum_d((double)s + (double)e);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = tot;
        __syncthreads();
        if (threadIdx.x == 0) {
            double r = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += part[w];
            rho[c] = du3 * r;
        }
        __syncthreads();
    }
}

cudaError_t launch_moment_coded(const GridDims &g, const void *f, const float *scale, int dtype, double *rho,
                                cudaStream_t st, int sm_count)
{
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long blocks = ncell < (long long)sm_count * 8 ? ncell : (long long)sm_count * 8;
    if (dtype == 2)
        moment_coded_kernel<__nv_bfloat16><<<int(blocks), 256, 0, st>>>(g, (const __nv_bfloat16 *)f, scale, rho);
    else
        moment_coded_kernel<__half><<<int(blocks), 256, 0, st>>>(g, (const __half *)f, scale, rho);
    return cudaGetLastError();
}

cudaError_t launch_moment(const GridDims &g, const void *f, int dtype, double *rho, cudaStream_t st,
                          int sm_count)
{
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long blocks = ncell < (long long)sm_count * 8 ? ncell : (long long)sm_count * 8;
    if (dtype == 0)
        moment_kernel<double><<<int(blocks), 256, 0, st>>>(g, (const double *)f, rho);
    else
        moment_kernel<float><<<int(blocks), 256, 0, st>>>(g, (const float *)f, rho);
    return cudaGetLastError();
}

// The moment fused into the x sweep: the velocity cube of spatial cell
// x cells_per_row + c arrives as nparts partial sums (in the storage type) laid out
// [c][part][x]; rho = du^3 x their sum in FP64 in a fixed order.  One block per c:
// 4 groups of 64 threads (x) take every 4th part, then one group adds the 4 sums.
template <typename P>
__global__ void __launch_bounds__(256) moment_finish_kernel(const P *__restrict__ mpart, int nparts, int nx,
                                                            long long cells_per_row, double du3, double *rho)
{
    __shared__ double red[4][64];
    const int tx = threadIdx.x & 63, grp = threadIdx.x >> 6;
    for (long long c = blockIdx.x; c < cells_per_row; c += gridDim.x) {
        const P *q = mpart + c * nparts * (long long)nx;
        for (int x0 = 0; x0 < nx; x0 += 64) {
            const int x = x0 + tx;
            double s = 0.0;
            if (x < nx)
                for (int k = grp; k < nparts; k += 4) s += double(q[(long long)k * nx + x]);
            red[grp][tx] = s;
            __syncthreads();
            if (grp == 0 && x < nx) rho[x * cells_per_row + c] = du3 * (((red[0][tx] + red[1][tx]) + red[2][tx]) + red[3][tx]);
            __syncthreads();
        }
    }
}

cudaError_t launch_moment_finish(const void *mpart, int dtype, int nparts, int nx, long long cells_per_row, double du3,
                                 double *rho, cudaStream_t st, int sm_count)
{
    const long long blocks = cells_per_row < (long long)sm_count * 8 ? cells_per_row : (long long)sm_count * 8;
    if (dtype == 0)
        moment_finish_kernel<double><<<int(blocks), 256, 0, st>>>((const double *)mpart, nparts, nx, cells_per_row,
                                                                     du3, rho);
    else
        moment_finish_kernel<float><<<int(blocks), 256, 0, st>>>((const float *)mpart, nparts, nx, cells_per_row, du3,
                                                                    rho);
    return cudaGetLastError();
}

// Adjoint of the moment: rho(x) = du^3 sum_u f(x, u), so dL/df(x, u) =
// du^3 dL/drho(x) for every u.  lam (+)= that, 16 bytes per thread and step.
template <typename T>
__global__ void __launch_bounds__(256) moment_adjoint_kernel(GridDims g, const double *__restrict__ dLdrho, T *lam,
                                                             int accumulate)
{
    constexpr int V = 16 / int(sizeof(T));
    const long long cube = (long long)g.nu[0] * g.nu[1] * g.nu[2];
    const long long nvec = (long long)g.n[0] * g.n[1] * g.n[2] * cube / V;
    const double du3 = (2.0 * g.V / g.nu[0]) * (2.0 * g.V / g.nu[1]) * (2.0 * g.V / g.nu[2]);
    uint4 *q = reinterpret_cast<uint4 *>(lam);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvec; i += (long long)gridDim.x * blockDim.x) {
        const T v = T(du3 * dLdrho[(i * V) / cube]); // a 16-byte vector never straddles a cell (cube % 64 == 0)
        uint4 u = accumulate ? q[i] : make_uint4(0, 0, 0, 0);
        T *e = reinterpret_cast<T *>(&u);
#pragma unroll
        for (int k = 0; k < V; ++k) e[k] += v;
        q[i] = u;
    }
}

cudaError_t launch_moment_adjoint(const GridDims &g, const double *dLdrho, int dtype, void *lam, int accumulate,
                                  cudaStream_t st, int sm_count)
{
    const int threads = 256;
    const int blocks = sm_count * 8;
    if (dtype == 0)
        moment_adjoint_kernel<double><<<blocks, threads, 0, st>>>(g, dLdrho, (double *)lam, accumulate);
    else
        moment_adjoint_kernel<float><<<blocks, threads, 0, st>>>(g, dLdrho, (float *)lam, accumulate);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// velocity moments: density, mean velocity, velocity dispersion tensor
// ----------------------------------------------------------------------------
// Sec. 4.1.3 keeps each spatial cell's velocity cube in one place so that these
// need no communication.  Per cell: S0 = sum f, S1_i = sum u_i f, S2_ij = sum
// u_i u_j f over the velocity cell centres; rho = du^3 S0, umean_i = S1_i / S0,
// sigma2_ij = S2_ij / S0 - umean_i umean_j (0 where S0 = 0).

// 16 bytes of storage -> N values (x the row's scale for 16-bit codes)
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    static constexpr int N = 4;
    __device__ static void get(const uint4 &u, float, float (&o)[4])
    {
        o[0] = __uint_as_float(u.x); o[1] = __uint_as_float(u.y);
        o[2] = __uint_as_float(u.z); o[3] = __uint_as_float(u.w);
    }
};
template <> struct Vec16<double> {
    static constexpr int N = 2;
    __device__ static void get(const uint4 &u, double, double (&o)[2])
    {
        o[0] = __hiloint2double(int(u.y), int(u.x));
        o[1] = __hiloint2double(int(u.w), int(u.z));
    }
};
template <> struct Vec16<__nv_bfloat16> {
    static constexpr int N = 8;
    __device__ static void get(const uint4 &u, float sc, float (&o)[8])
    {
        const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            o[2 * q] = __fmul_rn(__uint_as_float(w[q] << 16), sc);
            o[2 * q + 1] = __fmul_rn(__uint_as_float(w[q] & 0xffff0000u), sc);
        }
    }
};
template <> struct Vec16<__half> {
    static constexpr int N = 8;
    __device__ static void get(const uint4 &u, float sc, float (&o)[8])
    {
        const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 h = __half22float2(*reinterpret_cast<const __half2 *>(&w[q]));
            o[2 * q] = __fmul_rn(h.x, sc);
            o[2 * q + 1] = __fmul_rn(h.y, sc);
        }
    }
};

// compensated accumulator in the working precision
template <typename C> struct NSum {
    C s, c;
    __device__ void add(C x)
    {
        const C t = s + x;
        c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __device__ double get() const { return (double)s + (double)c; }
};

// One warp per spatial cell: each lane sums every 32nd 16-byte vector of the
// cube, then the ten sums are combined across the warp in FP64 in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) moments_kernel(GridDims g, const T *__restrict__ f,
                                                      const float *__restrict__ scale, double *rho, double *umean,
                                                      double *sigma2)
{
    using C = typename Compute<T>::type;
    constexpr int N = Vec16<T>::N;
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    const int nux = g.nu[0], nuy = g.nu[1], nuz = g.nu[2];
    const int nvec = nux * nuy * nuz / N; // 16-byte vectors per cube
    const int vrow = nuz / N;             // per u_z line
    const double du3 = (2.0 * g.V / nux) * (2.0 * g.V / nuy) * (2.0 * g.V / nuz);
    // n / d as a multiply-high by floor((2^32 - 1) / d) + 1: exact while n d < 2^32
    // (here n < 2^21, d <= 128)
    const unsigned mv = 0xffffffffu / unsigned(vrow) + 1u, my = 0xffffffffu / unsigned(nuy) + 1u;
    auto div_vrow = [&](int n) { return vrow == 1 ? n : int(__umulhi(unsigned(n), mv)); };
    auto div_nuy = [&](int n) { return int(__umulhi(unsigned(n), my)); };
    __shared__ C su[3][kMaxVel]; // velocity cell centres, formed in FP64 and rounded once
    for (int j = threadIdx.x; j < kMaxVel; j += blockDim.x)
        for (int d = 0; d < 3; ++d) su[d][j] = j < g.nu[d] ? C(-g.V + (j + 0.5) * (2.0 * g.V / g.nu[d])) : C(0);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long cell = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); cell < ncell; cell += warps) {
        const uint4 *q = reinterpret_cast<const uint4 *>(f + cell * (long long)nvec * N);
        const float *sc = scale ? scale + cell * nux * nuy : nullptr;
        // S0 compensated; the other nine sums in the working precision
        NSum<C> s0{C(0), C(0)};
        C acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = C(0);
#pragma unroll 4
        for (int k = lane; k < nvec; k += 32) {
            const int row = div_vrow(k), jz0 = (k - row * vrow) * N;
            const int jx = div_nuy(row), jy = row - jx * nuy;
            C v[N];
            Vec16<T>::get(q[k], sc ? sc[row] : 1.f, v);
            const C ux = su[0][jx], uy = su[1][jy];
            C t0 = C(0), t1 = C(0), t2 = C(0);
#pragma unroll
            for (int e = 0; e < N; ++e) {
                const C uz = su[2][jz0 + e];
                const C w = uz * v[e];
                t0 += v[e];
                t1 += w;
                t2 += uz * w;
            }
            s0.add(t0);
            acc[0] += ux * t0;
            acc[1] += uy * t0;
            acc[2] += t1;
            acc[3] += ux * ux * t0;
            acc[4] += uy * uy * t0;
            acc[5] += t2;
            acc[6] += ux * uy * t0;
            acc[7] += ux * t1;
            acc[8] += uy * t1;
        }
        double S[10];
        S[0] = warp_sum_d(s0.get());
#pragma unroll
        for (int k = 1; k < 10; ++k) S[k] = warp_sum_d((double)acc[k - 1]);
        if (lane == 0) {
            const double S0 = S[0], inv = S0 != 0.0 ? 1.0 / S0 : 0.0;
            const double m[3] = {S[1] * inv, S[2] * inv, S[3] * inv};
            // S index of sigma2 component k (xx, yy, zz, xy, xz, yz) and its pair
            const int si[6] = {4, 5, 6, 7, 8, 9}, pi[6] = {0, 1, 2, 0, 0, 1}, pj[6] = {0, 1, 2, 1, 2, 2};
            if (rho) rho[cell] = du3 * S0;
            if (umean)
                for (int i = 0; i < 3; ++i) umean[i * ncell + cell] = m[i];
            if (sigma2)
                for (int k = 0; k < 6; ++k)
                    sigma2[k * ncell + cell] = S0 != 0.0 ? S[si[k]] * inv - m[pi[k]] * m[pj[k]] : 0.0;
        }
    }
}

cudaError_t launch_moments(const GridDims &g, const void *f, const float *scale, int dtype, double *rho,
                           double *umean, double *sigma2, cudaStream_t st, int sm_count)
{
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long need = (ncell + 7) / 8; // 8 warps (cells) per block
    // one wave of resident blocks: each warp strides over the cells, so a second, partial
    // wave would leave most of the SMs idle for its whole length
    const void *kern = dtype == 0 ? (const void *)moments_kernel<double>
                       : dtype == 1 ? (const void *)moments_kernel<float>
                       : dtype == 2 ? (const void *)moments_kernel<__nv_bfloat16>
                                    : (const void *)moments_kernel<__half>;
    int per_sm = 0;
    const cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
    if (oe != cudaSuccess) return oe;
    if (per_sm < 1) per_sm = 1;
    const long long wave = (long long)sm_count * per_sm;
    const long long blocks = need < wave ? need : wave;
    switch (dtype) {
    case 0: moments_kernel<double><<<int(blocks), 256, 0, st>>>(g, (const double *)f, nullptr, rho, umean, sigma2); break;
    case 1: moments_kernel<float><<<int(blocks), 256, 0, st>>>(g, (const float *)f, nullptr, rho, umean, sigma2); break;
    case 2:
        moments_kernel<__nv_bfloat16><<<int(blocks), 256, 0, st>>>(g, (const __nv_bfloat16 *)f, scale, rho, umean, sigma2);
        break;
    default: moments_kernel<__half><<<int(blocks), 256, 0, st>>>(g, (const __half *)f, scale, rho, umean, sigma2); break;
    }
    return cudaGetLastError();
}

// y += x (FP64), or y = x when x_only
__global__ void axpy_kernel(long long n, const double *__restrict__ x, double *y, int assign)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = assign ? x[i] : y[i] + x[i];
}

cudaError_t launch_add(long long n, const double *x, double *y, bool assign, cudaStream_t st)
{
    const int threads = 256;
    const int blocks = int((n + threads - 1) / threads < 4096 ? (n + threads - 1) / threads : 4096);
    axpy_kernel<<<blocks, threads, 0, st>>>(n, x, y, assign ? 1 : 0);
    return cudaGetLastError();
}

// dx dy dz * sum rho, Neumaier in FP64 per thread, fixed-order combine
__global__ void __launch_bounds__(1024) mass_kernel(GridDims g, const double *__restrict__ rho, double *out)
{
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    double s = 0.0, e = 0.0;
    for (long long k = threadIdx.x; k < ncell; k += blockDim.x) {
        const double x = rho[k];
        const double t = s + x;
        e += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __shared__ double ps[1024], pe[1024];
    ps[threadIdx.x] = s;
    pe[threadIdx.x] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, E = 0.0;
        for (unsigned i = 0; i < blockDim.x; ++i) {
            const double x = ps[i];
            const double t = S + x;
            E += (fabs(S) >= fabs(x)) ? ((S - t) + x) : ((x - t) + S);
            S = t;
            E += pe[i];
        }
        *out = (S + E) * (g.L / g.n[0]) * (g.L / g.n[1]) * (g.L / g.n[2]);
    }
}

cudaError_t launch_mass(const GridDims &g, const double *rho, double *out, cudaStream_t st)
{
    mass_kernel<<<1, 1024, 0, st>>>(g, rho, out);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Poisson, Eq. (2)
// ----------------------------------------------------------------------------

__global__ void poisson_load_kernel(long long n, const double *__restrict__ rho, const double *__restrict__ bg,
                                    double2 *z)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[i] = make_double2(rho[i] + (bg ? bg[i] : 0.0), 0.0);
}

// DFT along dimension d: out[.., k, ..] = sum_m in[.., m, ..] e^{sign 2 pi i k m / n_d},
// factored once (Cooley-Tukey) as n = n1 n2 with m = n2 m1 + m2 and k = k1 + n1 k2:
//   Y[k1][m2] = W_n^{m2 k1} sum_{m1} x[n2 m1 + m2] W_{n1}^{m1 k1},
//   X[k1 + n1 k2] = sum_{m2} Y[k1][m2] W_{n2}^{m2 k2},
// n (n1 + n2 + 1) complex products per line instead of n^2 (n1 = 1 for a prime n: the
// plain sum).  W_{n1} = W_n^{n2}, W_{n2} = W_n^{n1}: one twiddle table per axis.  A
// block holds `lines` lines of the axis in shared memory, n threads per line.
__global__ void __launch_bounds__(256) dft_axis_kernel(GridDims g, int d, int sign, int n1, int lines,
                                                       const double2 *__restrict__ in, double2 *out,
                                                       const double2 *__restrict__ tw)
{
    extern __shared__ double2 dft_smem[];
    const long long n0 = g.n[0], nn1 = g.n[1], nn2 = g.n[2];
    const long long st[3] = {nn1 * nn2, nn2, 1};
    const int n = g.n[d], n2 = n / n1;
    const long long nlines = n0 * nn1 * nn2 / n;
    // the other two dimensions of a line, in memory order
    const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;
    const long long nb = g.n[db];
    const int li = threadIdx.x / n, k = threadIdx.x % n; // this thread: line li of the block, index k
    double2 *x = dft_smem + li * n, *y = dft_smem + lines * n + li * n;
    for (long long l0 = blockIdx.x * (long long)lines; l0 < nlines; l0 += (long long)gridDim.x * lines) {
        const long long line = l0 + li;
        const bool act = li < lines && line < nlines;
        long long base = 0;
        if (act) {
            base = (line / nb) * st[da] + (line % nb) * st[db];
            x[k] = in[base + k * st[d]];
        }
        __syncthreads();
        if (act) {
            // stage 1 for (k1, m2) = (k / n2, k % n2)
            const int k1 = k / n2, m2 = k % n2;
            double sr = 0.0, si = 0.0;
            int q = 0; // (n2 m1 k1) mod n
            for (int m1 = 0; m1 < n1; ++m1) {
                const double2 v = x[n2 * m1 + m2], w = tw[q];
                const double wi = sign * w.y;
                sr += v.x * w.x - v.y * wi;
                si += v.x * wi + v.y * w.x;
                q += n2 * k1; // < n
                if (q >= n) q -= n;
            }
            const double2 w = tw[(m2 * k1) % n];
            const double wi = sign * w.y;
            y[k] = make_double2(sr * w.x - si * wi, sr * wi + si * w.x); // Y[k1][m2] at k1 n2 + m2
        }
        __syncthreads();
        if (act) {
            // stage 2 for output k = k1 + n1 k2
            const int k1 = k % n1, k2 = k / n1;
            double sr = 0.0, si = 0.0;
            int q = 0; // (n1 m2 k2) mod n
            for (int m2 = 0; m2 < n2; ++m2) {
                const double2 v = y[k1 * n2 + m2], w = tw[q];
                const double wi = sign * w.y;
                sr += v.x * w.x - v.y * wi;
                si += v.x * wi + v.y * w.x;
                q += n1 * k2; // < n
                if (q >= n) q -= n;
            }
            out[base + k * st[d]] = make_double2(sr, si);
        }
        __syncthreads();
    }
}

// the factor n1 of n used by dft_axis_kernel: its largest divisor <= sqrt(n)
static int dft_n1(int n)
{
    int best = 1;
    for (int f = 2; f * f <= n; ++f)
        if (n % f == 0) best = f;
    return best;
}

__global__ void poisson_scale_kernel(GridDims g, double2 *z, double fac)
{
    const long long n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    const long long total = n0 * n1 * n2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long id[3] = {i / (n1 * n2), (i / n2) % n1, i % n2};
        double k2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const long long nd = g.n[d];
            const long long w = id[d] < (nd + 1) / 2 ? id[d] : id[d] - nd; // integer wave number
            const double k = 2.0 * M_PI * (double)w / g.L;
            k2 += k * k;
        }
        const double s = (k2 == 0.0) ? 0.0 : -fac / k2;
        z[i] = make_double2(z[i].x * s, z[i].y * s);
    }
}

// FP32 phi (the field the kicks read) or FP64 (the adjoint's dL/drho)
__global__ void poisson_store_kernel(long long n, const double2 *__restrict__ z, float *phi, double *phi64)
{
    const double inv = 1.0 / (double)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (phi) phi[i] = (float)(z[i].x * inv);
        if (phi64) phi64[i] = z[i].x * inv;
    }
}

cudaError_t launch_poisson(const GridDims &g, const PoissonScratch &ps, const double *rho, const double *bg,
                           double a, double four_pi_G, float *phi, cudaStream_t st, double *phi64)
{
    const long long n = (long long)g.n[0] * g.n[1] * g.n[2];
    const int threads = 256;
    const int blocks = int((n + threads - 1) / threads < 8192 ? (n + threads - 1) / threads : 8192);
    poisson_load_kernel<<<blocks, threads, 0, st>>>(n, rho, bg, ps.z0);
    double2 *a0 = ps.z0, *a1 = ps.z1;
    auto dft = [&](int d, int sign) {
        const int nd = g.n[d], lines = 256 / nd; // nd <= 256
        const long long nlines = n / nd;
        const long long nb = (nlines + lines - 1) / lines;
        const int grid = int(nb < 8192 ? nb : 8192);
        dft_axis_kernel<<<grid, lines * nd, 2 * lines * nd * sizeof(double2), st>>>(g, d, sign, dft_n1(nd), lines, a0,
                                                                                   a1, ps.tw[d]);
        double2 *t = a0; a0 = a1; a1 = t;
    };
    for (int d = 2; d >= 0; --d) dft(d, -1);
    poisson_scale_kernel<<<blocks, threads, 0, st>>>(g, a0, four_pi_G * a * a);
    for (int d = 0; d < 3; ++d) dft(d, +1);
    poisson_store_kernel<<<blocks, threads, 0, st>>>(n, a0, phi, phi64);
    return cudaGetLastError();
}

} // namespace vk
