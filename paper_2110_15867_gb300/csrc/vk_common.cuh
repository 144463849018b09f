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

// Non-blocking probe: has the phase with this parity completed?
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
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

// wait until at most n (0..7) of the most recent bulk groups are still reading shared memory
__device__ __forceinline__ void bulk_wait_read_at_most(unsigned n)
{
    switch (n) {
    case 0: asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.bulk.wait_group.read 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.bulk.wait_group.read 4;" ::: "memory"); break;
    case 5: asm volatile("cp.async.bulk.wait_group.read 5;" ::: "memory"); break;
    case 6: asm volatile("cp.async.bulk.wait_group.read 6;" ::: "memory"); break;
    default: asm volatile("cp.async.bulk.wait_group.read 7;" ::: "memory"); break;
    }
}

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

// ----------------------------------------------------------------------------
// 16-bit storage codec: stochastic rounding to BF16 / FP16
// ----------------------------------------------------------------------------
// Re-encoding f after every sweep with round-to-nearest drops or biases the
// small per-sweep updates; stochastic rounding keeps each encode unbiased in
// expectation.  Random bits: the 32-bit finalizer of MurmurHash3 (Appleby)
// seeds one stream per line of the march from the element index and a
// per-sweep seed; the stream then advances with the 32-bit linear congruential
// generator of Numerical Recipes (a = 1664525, c = 1013904223), whose upper 16
// bits feed one value each.  A run is reproducible.

__device__ __forceinline__ unsigned fmix32(unsigned h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ unsigned sr_bits(unsigned long long elem, unsigned seed)
{
    return fmix32(unsigned(elem) ^ unsigned(elem >> 32) * 0x9e3779b9u ^ seed * 0x85ebca6bu);
}

__device__ __forceinline__ unsigned lcg_next(unsigned &x)
{
    x = x * 1664525u + 1013904223u;
    return x;
}


// Two non-negative FP32 values -> packed bf16x2 with stochastic rounding: the upper 16
// bits of two LCG steps are added below the BF16 mantissa of x and of y, and one byte
// permute packs the two upper halves.
__device__ __forceinline__ unsigned sr_pack_bf16x2(float x, float y, unsigned &rng)
{
    const unsigned r1 = lcg_next(rng) >> 16, r2 = lcg_next(rng) >> 16;
    return __byte_perm(__float_as_uint(x) + r1, __float_as_uint(y) + r2, 0x7632);
}

// Line scales of the 16-bit codec.  coded_scale: the scale a refresh stores for a line
// whose largest value is m; BF16 keeps at least 2^-64, so that a line left empty can
// still take in mass from the sweeps that keep the scale (BF16 carries 8 significant
// bits at any exponent: codes up to 2^64 x its largest value stay finite, and values
// down to 2^-190 stay representable); FP16 has 5 exponent bits and keeps m itself.
// inv_scale: 1 / s for encoding, 0 for s = 0 and for a subnormal s, whose reciprocal
// would overflow (such a line holds nothing above 2^-126; its values encode as 0).
template <typename T> __device__ __forceinline__ float coded_scale(float m) { return m; }
template <> __device__ __forceinline__ float coded_scale<__nv_bfloat16>(float m) { return fmaxf(m, 0x1p-64f); }
__device__ __forceinline__ float inv_scale(float s) { return s >= 0x1p-126f ? __fdividef(1.f, s) : 0.f; }

// Two non-negative FP32 values -> packed f16x2 with stochastic rounding: 13 of the upper
// 16 bits of two LCG steps are added below the FP16 mantissa (13 bits below FP32's), and
// one round-toward-zero conversion packs both (x in the lower half).
__device__ __forceinline__ unsigned sr_pack_f16x2(float x, float y, unsigned &rng)
{
    const unsigned r1 = (lcg_next(rng) >> 16) & 0x1fffu, r2 = (lcg_next(rng) >> 16) & 0x1fffu;
    const float xr = __uint_as_float(__float_as_uint(x) + r1), yr = __uint_as_float(__float_as_uint(y) + r2);
    unsigned out;
    asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(out) : "f"(yr), "f"(xr));
    return out;
}

// ----------------------------------------------------------------------------
// arithmetic on float, double and float2 (two independent lines in packed FP32:
// add / sub / mul / fma use the f32x2 instructions of sm_100+, min / max / select
// act per component)
// ----------------------------------------------------------------------------

#define VK_F2_BINOP(name, op)                                                                        \
    __device__ __forceinline__ float2 name(float2 a, float2 b)                                        \
    {                                                                                                 \
        float2 d;                                                                                     \
        asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t" op     \
            " rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"                                                    \
            : "=f"(d.x), "=f"(d.y)                                                                    \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                                \
        return d;                                                                                     \
    }
VK_F2_BINOP(vadd, "add.rn.f32x2")
VK_F2_BINOP(vsub, "sub.rn.f32x2")
VK_F2_BINOP(vmul, "mul.rn.f32x2")
#undef VK_F2_BINOP

// a * b + c
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ float2 mn2(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ float2 mx2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ float2 mn3(float2 a, float2 b, float2 c)
{
    return make_float2(mn3(a.x, b.x, c.x), mn3(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 mx3(float2 a, float2 b, float2 c)
{
    return make_float2(mx3(a.x, b.x, c.x), mx3(a.y, b.y, c.y));
}

template <typename X> __device__ __forceinline__ X splat(double v);
template <> __device__ __forceinline__ float splat<float>(double v) { return float(v); }
template <> __device__ __forceinline__ double splat<double>(double v) { return v; }
template <> __device__ __forceinline__ float2 splat<float2>(double v) { return make_float2(float(v), float(v)); }

// minmod: 0 unless all arguments share a sign, else the one of least magnitude;
// = median(lo, 0, hi) with lo / hi the smallest / largest argument
template <typename X> __device__ __forceinline__ X minmod4(X a, X b, X c, X d)
{
    const X lo = mn2(mn3(a, b, c), d);
    const X hi = mx2(mx3(a, b, c), d);
    return mn2(mx2(lo, splat<X>(0.0)), hi);
}

// ----------------------------------------------------------------------------
// SL-MPP5 line coefficients
// ----------------------------------------------------------------------------

template <typename X> struct Lim {
    X w0, w1, w2, w3, w4, s, alpha;
};

template <typename C> __device__ __forceinline__ Lim<C> to_lim(const LineCoefT<C> &k)
{
    return Lim<C>{k.w[0], k.w[1], k.w[2], k.w[3], k.w[4], k.s, k.alpha};
}

// two lines in one packed pair
__device__ __forceinline__ Lim<float2> to_lim2(const LineCoefT<float> &a, const LineCoefT<float> &b)
{
    return Lim<float2>{make_float2(a.w[0], b.w[0]), make_float2(a.w[1], b.w[1]), make_float2(a.w[2], b.w[2]),
                       make_float2(a.w[3], b.w[3]), make_float2(a.w[4], b.w[4]), make_float2(a.s, b.s),
                       make_float2(a.alpha, b.alpha)};
}

// Fractional flux through the downwind face of the donor c0 (local frame, flow
// toward +index): SL reconstruction mean fbar, Suresh-Huynh monotonicity
// constraint on fbar with the given alpha, then s * fbar clamped to [0, c0]
// (positivity).  dm4m / dm4p are the limited curvatures at the upwind /
// downwind faces of the donor.
//
// Suresh & Huynh keep fbar when it lies between c0 and the MP bound
// f_MP = c0 + minmod(cp1 - c0, alpha (c0 - cm1)) and otherwise take
// median(fbar, fmin, fmax).  f_MP is the median of (c0, cp1, f_UL), and every
// one of the sets bounding fmin and fmax contains c0 together with cp1 or f_UL,
// so [c0, f_MP] lies inside [fmin, fmax] (both are pure selections, exactly so
// in floating point): the constraint is the clamp of fbar to [fmin, fmax].
template <typename X>
__device__ __forceinline__ X sl_mpp5_flux(const Lim<X> &k, X cm2, X cm1, X c0, X cp1, X cp2, X dm4m, X dm4p)
{
    const X fbar = vfma(k.w4, cp2, vfma(k.w3, cp1, vfma(k.w2, c0, vfma(k.w1, cm1, vmul(k.w0, cm2)))));
    const X dlm = vsub(c0, cm1);
    const X ful = vfma(k.alpha, dlm, c0);
    const X fmd = vmul(splat<X>(0.5), vsub(vadd(c0, cp1), dm4p));
    const X flc = vfma(splat<X>(4.0 / 3.0), dm4m, vfma(splat<X>(0.5), dlm, c0));
    // clamp(fbar, fmin, fmax) with fmin = max(A, B), fmax = min(C, D): by associativity
    // of max and min, min(max(fbar, A, B), C, D) -- two 3-input operations instead of four
    const X v = mn3(mx3(fbar, mn3(c0, cp1, fmd), mn3(c0, ful, flc)), mx3(c0, cp1, fmd), mx3(c0, ful, flc));
    return mn2(mx2(vmul(k.s, v), splat<X>(0.0)), c0);
}

// limited curvature at the face between two cells with curvatures d0, d1
template <typename X> __device__ __forceinline__ X dm4(X d0, X d1)
{
    const X four = splat<X>(4.0);
    return minmod4(vsub(vmul(four, d0), d1), vsub(vmul(four, d1), d0), d0, d1);
}

// curvature c_{i-1} - 2 c_i + c_{i+1}
template <typename X> __device__ __forceinline__ X curv(X a, X b, X c)
{
    return vadd(vfma(splat<X>(-2.0), b, a), c);
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
        const C dmm = curv(a, b, c);
        const C dm = curv(b, c, s0);
        const C d0 = curv(c, s0, s1);
        const C dm4_mm = dm4(dmm, dm);
        const C dm4_m = dm4(dm, d0);
        Fm = sl_mpp5_flux(k, a, b, c, s0, s1, dm4_mm, dm4_m); // face -1/2, donor c_{-1}
        cm2 = b;
        cm1 = c;
        dcur = d0;
        dm4m = dm4_m;
    } else {
        const C dm = s0;                       // c_{-2} - 2 c_{-1} + c_0 with zero ghosts
        const C d0 = curv(C(0), s0, s1);       // c_{-1} - 2 c_0 + c_1
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
        const C dn = curv(c0, cp1, cp2);
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
        const C dn = curv(c0, cp1, cp2);
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
