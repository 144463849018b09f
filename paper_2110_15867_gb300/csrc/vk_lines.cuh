// vk_lines.cuh -- pieces shared by the kernels that hold whole velocity lines in
// registers (sweep_lines.cu, kick_cube.cu): 16-byte chunks of a line <-> FP32 values
// (decoded with the line scale for 16-bit codes, re-encoded with stochastic
// rounding), single values of 16-bit codes, and the march of one zero-flux line of
// Eq. (4) held in registers.
#pragma once

#include "vk_common.cuh"

namespace vk {

// 16-byte chunk <-> values (times / divided by the line scale for 16-bit codes)
template <typename T> struct Chunk;
template <> struct Chunk<float> {
    __device__ static void get(const unsigned char *p, float s, float (&o)[4])
    {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    }
    __device__ static void put(unsigned char *p, float, const float (&o)[4], unsigned &)
    {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <> struct Chunk<__nv_bfloat16> {
    __device__ static void get(const unsigned char *p, float s, float (&o)[8])
    {
        const uint4 a = *reinterpret_cast<const uint4 *>(p);
        const unsigned w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            o[2 * q] = __fmul_rn(__uint_as_float(w[q] << 16), s);
            o[2 * q + 1] = __fmul_rn(__uint_as_float(w[q] & 0xffff0000u), s);
        }
    }
    // rng: stochastic-rounding stream of the line
    __device__ static void put(unsigned char *p, float inv, const float (&o)[8], unsigned &rng)
    {
        unsigned w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = sr_pack_bf16x2(o[2 * q] * inv, o[2 * q + 1] * inv, rng);
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
};
template <> struct Chunk<__half> {
    __device__ static void get(const unsigned char *p, float s, float (&o)[8])
    {
        const uint4 a = *reinterpret_cast<const uint4 *>(p);
        const unsigned w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[q]));
            o[2 * q] = __fmul_rn(f.x, s);
            o[2 * q + 1] = __fmul_rn(f.y, s);
        }
    }
    __device__ static void put(unsigned char *p, float inv, const float (&o)[8], unsigned &rng)
    {
        unsigned w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = sr_pack_f16x2(o[2 * q] * inv, o[2 * q + 1] * inv, rng);
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
};

template <> struct Chunk<double> {
    __device__ static void get(const unsigned char *p, float, double (&o)[2])
    {
        const double2 a = *reinterpret_cast<const double2 *>(p);
        o[0] = a.x; o[1] = a.y;
    }
    __device__ static void put(unsigned char *p, float, const double (&o)[2], unsigned &)
    {
        *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
    }
};

#define CODED_RNG_INIT(e, seed) (sizeof(T) == 2 ? sr_bits((e), (seed)) : 0u)

// Advance both lines of the pair (forward local frame; zero-flux faces).
// X = float2: two lines as one packed pair; X = float: one line.
template <int NU, typename X>
__device__ __forceinline__ X march_regs(X (&v)[NU], const Lim<X> &lim)
{
    const X zero = splat<X>(0.0);
    X d[NU];
#pragma unroll
    for (int i = 0; i < NU; ++i)
        d[i] = curv(i > 0 ? v[i - 1] : zero, v[i], i + 1 < NU ? v[i + 1] : zero);
    const X dm = v[0]; // curvature of the ghost cell -1: 0 - 0 + c_0
    // F[k] = flux through face k - 1/2, k = 1 .. NU-1 (outer faces carry nothing)
    X Fprev = zero, sum = zero;
    X dm4m = dm4(dm, d[0]);
    X out[NU];
#pragma unroll
    for (int i = 0; i < NU; ++i) {
        X F = zero;
        X dm4p = zero;
        if (i + 1 < NU) {
            const X cm2 = i >= 2 ? v[i - 2] : zero;
            const X cm1 = i >= 1 ? v[i - 1] : zero;
            const X cp2 = i + 2 < NU ? v[i + 2] : zero;
            dm4p = dm4(d[i], d[i + 1]);
            F = sl_mpp5_flux(lim, cm2, cm1, v[i], v[i + 1], cp2, dm4m, dm4p);
        }
        out[i] = vadd(v[i], vsub(Fprev, F));
        sum = vadd(sum, out[i]);
        Fprev = F;
        dm4m = dm4p;
    }
#pragma unroll
    for (int i = 0; i < NU; ++i) v[i] = out[i];
    return sum;
}


// The zero-flux line p[0], p[st], ..., p[(NU - 1) st] (forward local frame) advanced in
// place: march_regs with the line read a window ahead and each cell written at its own
// face (never read again).  Returns the sum of the new values.
template <int NU> __device__ __forceinline__ float march_strided(float *p, int st, const Lim<float> &lim)
{
    static_assert(NU >= 4, "lines of at least 4 cells");
    float cm2 = 0.f, cm1 = 0.f, c0 = p[0], cp1 = p[st], cp2 = p[2 * st];
    float db = curv(0.f, c0, cp1);  // curvature of cell 0
    float dm4m = dm4(c0, db);       // face -1/2: the ghost cell -1 has curvature 0 - 0 + c_0
    float Fprev = 0.f, sum = 0.f;
    // blocks of 8 faces: a fully unrolled 48-face body per sweep missed in the instruction cache
#pragma unroll 8
    for (int i = 0; i < NU; ++i) {
        float F = 0.f, dm4p = 0.f, dc = 0.f;
        if (i + 1 < NU) {
            dc = curv(c0, cp1, cp2); // curvature of cell i + 1
            dm4p = dm4(db, dc);
            F = sl_mpp5_flux(lim, cm2, cm1, c0, cp1, cp2, dm4m, dm4p);
        }
        const float out = vadd(c0, vsub(Fprev, F));
        p[i * st] = out;
        sum = vadd(sum, out);
        Fprev = F;
        dm4m = dm4p;
        db = dc;
        cm2 = cm1;
        cm1 = c0;
        c0 = cp1;
        cp1 = cp2;
        cp2 = i + 3 < NU ? p[(i + 3) * st] : 0.f;
    }
    return sum;
}

// A single value of a line (strided access): decode with the scale of its u_z line,
// encode with one stochastic-rounding draw (16 random bits; v >= 0).  Every decode is
// a rounded product (__fmul_rn): a plain product may be contracted into the first sum
// that uses it, depending on the code around it, and the kernels that share a
// rounding point (the one-pass kick, the fused tail, the separate sweeps) must agree
// bit for bit.
template <typename T> struct RegCodec;
template <> struct RegCodec<float> {
    __device__ static float get(float c, float) { return c; }
    __device__ static float put(float v, float, unsigned) { return v; }
};
template <> struct RegCodec<__nv_bfloat16> {
    __device__ static float get(__nv_bfloat16 c, float s) { return __fmul_rn(__bfloat162float(c), s); }
    __device__ static __nv_bfloat16 put(float v, float inv, unsigned r16)
    {
        const unsigned b = (__float_as_uint(v * inv) + r16) >> 16; // stochastic rounding (v >= 0)
        return __ushort_as_bfloat16((unsigned short)b);
    }
};
template <> struct RegCodec<__half> {
    __device__ static float get(__half c, float s) { return __fmul_rn(__half2float(c), s); }
    __device__ static __half put(float v, float inv, unsigned r16)
    {
        return __float2half_rz(__uint_as_float(__float_as_uint(v * inv) + (r16 & 0x1fffu)));
    }
};

} // namespace vk
