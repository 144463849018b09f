// vk_common.cuh -- device building blocks of libvlasov (sm_103a).
//
//  * PTX wrappers: mbarrier, TMA tensor copies (cp.async.bulk.tensor), bulk
//    async groups, proxy fences, the global timer used by bounded waits.
//  * SL-MPP5 (Sec. 4.2 of Yoshikawa, Tanaka & Yoshida, SC'21): the
//    conservative semi-Lagrangian fractional flux, the Suresh-Huynh
//    monotonicity-preserving constraint and the positivity clamp, and the
//    march of one line in shared memory.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vk_kernels.h"

namespace vk {

// A bounded wait gives up after this much wall time or this many polls.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr unsigned kWaitLimitPolls = 1u << 26;

// ----------------------------------------------------------------------------
// PTX wrappers
// ----------------------------------------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with the given parity; false if the wait ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (unsigned it = 1; it < kWaitLimitPolls; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0 && globaltimer() - t0 > kWaitLimitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0,
                                            int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0,
                                            int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int c0, int c1)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1)
                 : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int c0, int c1,
                                             int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

__device__ __forceinline__ void bulk_wait_read_all()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// barrier among the consumer warps only (named barrier 1)
__device__ __forceinline__ void consumer_sync(int nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// ----------------------------------------------------------------------------
// storage <-> compute conversions
// ----------------------------------------------------------------------------

template <typename T> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };

__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_c(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T from_c(typename Compute<T>::type v);
template <> __device__ __forceinline__ float from_c<float>(float v) { return v; }
template <> __device__ __forceinline__ double from_c<double>(double v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_c<__half>(float v) { return __float2half_rn(v); }

// ----------------------------------------------------------------------------
// min / max with three inputs (one instruction for f32 on sm_100+)
// ----------------------------------------------------------------------------

__device__ __forceinline__ float mn3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float mx3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ double mn3(double a, double b, double c) { return fmin(a, fmin(b, c)); }
__device__ __forceinline__ double mx3(double a, double b, double c) { return fmax(a, fmax(b, c)); }
__device__ __forceinline__ float mn2(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float mx2(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double mn2(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ double mx2(double a, double b) { return fmax(a, b); }

// minmod: 0 unless all arguments share a sign, else the one of least magnitude
template <typename C> __device__ __forceinline__ C minmod2(C a, C b)
{
    return mx2(mn2(a, b), C(0)) + mn2(mx2(a, b), C(0));
}

template <typename C> __device__ __forceinline__ C minmod4(C a, C b, C c, C d)
{
    const C lo = mn2(mn3(a, b, c), d);
    const C hi = mx2(mx3(a, b, c), d);
    return mx2(lo, C(0)) + mn2(hi, C(0));
}

// ----------------------------------------------------------------------------
// SL-MPP5 line coefficients
// ----------------------------------------------------------------------------

template <typename C> struct Lim {
    C w0, w1, w2, w3, w4, s, alpha;
};

template <typename C> __device__ __forceinline__ Lim<C> to_lim(const LineCoefT<C> &k)
{
    return Lim<C>{k.w[0], k.w[1], k.w[2], k.w[3], k.w[4], k.s, k.alpha};
}

// Fractional flux through the downwind face of the donor c0 (local frame, flow
// toward +index): SL reconstruction mean fbar, Suresh-Huynh constraint on
// fbar with the given alpha (skipped when fbar lies between c0 and the MP
// bound), then s * fbar clamped to [0, c0] (positivity).
// dm4m / dm4p are the limited curvatures at the upwind / downwind faces.
template <typename C>
__device__ __forceinline__ C sl_mpp5_flux(const Lim<C> &k, C cm2, C cm1, C c0, C cp1, C cp2, C dm4m,
                                          C dm4p)
{
    const C fbar = k.w0 * cm2 + k.w1 * cm1 + k.w2 * c0 + k.w3 * cp1 + k.w4 * cp2;
    const C dlm = c0 - cm1;
    const C dlp = cp1 - c0;
    const C up = k.alpha * dlm;
    const C fmp = c0 + minmod2(dlp, up);
    const C ful = c0 + up;
    const C fmd = C(0.5) * (c0 + cp1 - dm4p);
    const C flc = c0 + C(0.5) * dlm + C(4.0 / 3.0) * dm4m;
    const C fmin = mx2(mn3(c0, cp1, fmd), mn3(c0, ful, flc));
    const C fmax = mn2(mx3(c0, cp1, fmd), mx3(c0, ful, flc));
    // fmin <= c0 <= fmax, so the median of (fbar, fmin, fmax) is a clamp
    const C clamp = mn2(mx2(fbar, fmin), fmax);
    const C v = ((fbar - c0) * (fbar - fmp) <= C(0)) ? fbar : clamp;
    return mn2(mx2(k.s * v, C(0)), c0);
}

// limited curvature at the face between two cells with curvatures d0, d1
template <typename C> __device__ __forceinline__ C dm4(C d0, C d1)
{
    return minmod4(C(4) * d0 - d1, C(4) * d1 - d0, d0, d1);
}

// ----------------------------------------------------------------------------
// one line in shared memory
// ----------------------------------------------------------------------------

// Advance the line p[0], p[step], ..., p[(L-1) step] (local frame: flow toward
// +index) by the fractional part of the Courant number, in place:
// c_i <- c_i - (F_{i+1/2} - F_{i-1/2}).  PERIODIC selects the position-space
// seam; otherwise ghost cells are 0 and both outer faces carry no flux.
// Returns the sum of the new values (used for the NaN / sign check).
// Requires L >= 4.
template <typename T, bool PERIODIC, typename C>
__device__ __forceinline__ C march_line(T *p, long step, int L, const Lim<C> &k)
{
    const C s0 = to_c(p[0]);
    const C s1 = to_c(p[step]);
    C cm2, cm1, c0, cp1, dcur, dm4m, Fm;
    if (PERIODIC) {
        const C a = to_c(p[(long)(L - 3) * step]);
        const C b = to_c(p[(long)(L - 2) * step]);
        const C c = to_c(p[(long)(L - 1) * step]);
        const C dmm = a - C(2) * b + c;
        const C dm = b - C(2) * c + s0;
        const C d0 = c - C(2) * s0 + s1;
        const C dm4_mm = dm4(dmm, dm);
        const C dm4_m = dm4(dm, d0);
        Fm = sl_mpp5_flux(k, a, b, c, s0, s1, dm4_mm, dm4_m); // face -1/2, donor c_{-1}
        cm2 = b;
        cm1 = c;
        dcur = d0;
        dm4m = dm4_m;
    } else {
        const C dm = s0;               // c_{-2} - 2 c_{-1} + c_0 with zero ghosts
        const C d0 = s1 - C(2) * s0;   // c_{-1} - 2 c_0 + c_1
        cm2 = C(0);
        cm1 = C(0);
        dcur = d0;
        dm4m = dm4(dm, d0);
        Fm = C(0);
    }
    c0 = s0;
    cp1 = s1;
    C sum = C(0);
#pragma unroll 4
    for (int i = 0; i < L - 2; ++i) {
        const C cp2 = to_c(p[(long)(i + 2) * step]);
        const C dn = c0 - C(2) * cp1 + cp2;
        const C dm4p = dm4(dcur, dn);
        const C F = sl_mpp5_flux(k, cm2, cm1, c0, cp1, cp2, dm4m, dm4p);
        const C out = c0 + (Fm - F);
        p[(long)i * step] = from_c<T>(out);
        sum += out;
        cm2 = cm1;
        cm1 = c0;
        c0 = cp1;
        cp1 = cp2;
        dcur = dn;
        dm4m = dm4p;
        Fm = F;
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const C cp2 = PERIODIC ? (t == 0 ? s0 : s1) : C(0);
        const C dn = c0 - C(2) * cp1 + cp2;
        const C dm4p = dm4(dcur, dn);
        C F = sl_mpp5_flux(k, cm2, cm1, c0, cp1, cp2, dm4m, dm4p);
        if (!PERIODIC && t == 1) F = C(0); // outer velocity face
        const C out = c0 + (Fm - F);
        p[(long)(L - 2 + t) * step] = from_c<T>(out);
        sum += out;
        cm2 = cm1;
        cm1 = c0;
        c0 = cp1;
        cp1 = cp2;
        dcur = dn;
        dm4m = dm4p;
        Fm = F;
    }
    return sum;
}

// rotate the line right by r positions (0 <= r < L): q[i] <- q[i - r]
template <typename T> __device__ __forceinline__ void rotate_line(T *p, long step, int L, int r)
{
    auto rev = [&](int a, int b) { // reverse [a, b)
        for (int i = a, j = b - 1; i < j; ++i, --j) {
            const T t = p[(long)i * step];
            p[(long)i * step] = p[(long)j * step];
            p[(long)j * step] = t;
        }
    };
    if (r == 0) return;
    rev(0, L - r);
    rev(L - r, L);
    rev(0, L);
}

} // namespace vk
