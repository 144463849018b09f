// codec.cu -- encode and decode of the 16-bit storage of f (BF16 or FP16 codes with
// one FP32 scale per u_z line).  The paper stores f in FP32 (Sec. 5.1); this
// storage is the library's own reduced-precision mode, and these two kernels are
// the only way into and out of it.
//
// Encode of one u_z line v_0 .. v_{n-1} (FP64 or FP32 values):
//   w_k   = v_k rounded to FP32 (round to nearest even),
//   m     = max_k w_k (a shuffle reduction over the lanes that hold the line),
//   s     = max(m, 0), raised to at least 2^-64 for BF16 codes (the floor the sweeps
//           keep, so that an empty line can take in mass again),
//   c_k   = RN16(w_k / s) with the IEEE FP32 quotient, or 0 where s = 0,
// RN16 = round to nearest even into BF16 or FP16.  Decode: c_k x s, exact in FP64,
// rounded to nearest even in FP32.
#include "vk_common.cuh"

namespace vk {

namespace {

template <typename T> __device__ __forceinline__ T rn16(float q);
template <> __device__ __forceinline__ __nv_bfloat16 rn16<__nv_bfloat16>(float q) { return __float2bfloat16_rn(q); }
template <> __device__ __forceinline__ __half rn16<__half>(float q) { return __float2half_rn(q); }

template <typename T> __device__ __forceinline__ float floor_scale(float m) { return fmaxf(m, 0.f); }
template <> __device__ __forceinline__ float floor_scale<__nv_bfloat16>(float m) { return fmaxf(m, 0x1p-64f); }

// G lanes per line (a power of two, 4 .. 32), E elements per lane (E G >= nuz).  A warp
// holds 32 / G lines; lines are taken by warps in a grid-stride loop.
template <typename S, typename T, int E>
__global__ void __launch_bounds__(256) encode_kernel(long long nlines, int nuz, int G, const S *__restrict__ src,
                                                     T *__restrict__ codes, float *__restrict__ scale)
{
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;       // lane within its line group
    const int grp = lane / G;       // line of the warp this lane works on
    const int lpw = 32 / G;         // lines per warp
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long w0 = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (long long base = w0 * lpw; base < nlines; base += warps * lpw) {
        const long long line = base + grp;
        const bool live = line < nlines;
        float w[E];
        float m = -INFINITY; // lanes past the end of the line hold no value
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = sub + e * G;
            w[e] = 0.f;
            if (live && k < nuz) {
                w[e] = (float)src[line * nuz + k];
                m = fmaxf(m, w[e]);
            }
        }
        // max over the G lanes of the group
        for (int o = G >> 1; o > 0; o >>= 1) {
            const float t = __shfl_xor_sync(0xffffffffu, m, o);
            m = fmaxf(m, t);
        }
        if (!live) continue;
        const float s = floor_scale<T>(m);
        if (sub == 0) scale[line] = s;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = sub + e * G;
            if (k < nuz) codes[line * nuz + k] = s == 0.f ? rn16<T>(0.f) : rn16<T>(w[e] / s);
        }
    }
}

template <typename T> __device__ __forceinline__ float from16(T c);
template <> __device__ __forceinline__ float from16<__nv_bfloat16>(__nv_bfloat16 c) { return __bfloat162float(c); }
template <> __device__ __forceinline__ float from16<__half>(__half c) { return __half2float(c); }

template <typename T, typename D>
__global__ void __launch_bounds__(256) decode_kernel(long long nlines, int nuz, const T *__restrict__ codes,
                                                     const float *__restrict__ scale, D *__restrict__ dst)
{
    const long long n = nlines * nuz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const D c = (D)from16<T>(codes[i]);
        const D s = (D)scale[i / nuz];
        dst[i] = c * s;
    }
}

template <typename S, typename T>
cudaError_t encode_t(long long nlines, int nuz, const void *src, void *codes, float *scale, cudaStream_t st,
                     int sm_count)
{
    int G = 4;
    while (G < nuz && G < 32) G <<= 1;
    const int E = (nuz + G - 1) / G;
    const long long groups = (nlines + 32 / G - 1) / (32 / G);
    const long long blocks_needed = (groups + 7) / 8;
    const int blocks = int(blocks_needed < (long long)sm_count * 16 ? blocks_needed : (long long)sm_count * 16);
    if (blocks <= 0) return cudaSuccess;
    const S *s = (const S *)src;
    T *c = (T *)codes;
    switch (E) {
    case 1: encode_kernel<S, T, 1><<<blocks, 256, 0, st>>>(nlines, nuz, G, s, c, scale); break;
    case 2: encode_kernel<S, T, 2><<<blocks, 256, 0, st>>>(nlines, nuz, G, s, c, scale); break;
    case 3: encode_kernel<S, T, 3><<<blocks, 256, 0, st>>>(nlines, nuz, G, s, c, scale); break;
    default: encode_kernel<S, T, 4><<<blocks, 256, 0, st>>>(nlines, nuz, G, s, c, scale); break;
    }
    return cudaGetLastError();
}

template <typename T, typename D>
cudaError_t decode_t(long long nlines, int nuz, const void *codes, const float *scale, void *dst, cudaStream_t st,
                     int sm_count)
{
    const long long n = nlines * nuz;
    const long long need = (n + 255) / 256;
    const int blocks = int(need < (long long)sm_count * 16 ? need : (long long)sm_count * 16);
    if (blocks <= 0) return cudaSuccess;
    decode_kernel<T, D><<<blocks, 256, 0, st>>>(nlines, nuz, (const T *)codes, scale, (D *)dst);
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_encode(long long nlines, int nuz, const void *src, int src_dtype, void *codes, int code_dtype,
                          float *scale, cudaStream_t st, int sm_count)
{
    const bool bf = code_dtype == 2;
    if (src_dtype == 0)
        return bf ? encode_t<double, __nv_bfloat16>(nlines, nuz, src, codes, scale, st, sm_count)
                  : encode_t<double, __half>(nlines, nuz, src, codes, scale, st, sm_count);
    return bf ? encode_t<float, __nv_bfloat16>(nlines, nuz, src, codes, scale, st, sm_count)
              : encode_t<float, __half>(nlines, nuz, src, codes, scale, st, sm_count);
}

cudaError_t launch_decode(long long nlines, int nuz, const void *codes, int code_dtype, const float *scale, void *dst,
                          int dst_dtype, cudaStream_t st, int sm_count)
{
    const bool bf = code_dtype == 2;
    if (dst_dtype == 0)
        return bf ? decode_t<__nv_bfloat16, double>(nlines, nuz, codes, scale, dst, st, sm_count)
                  : decode_t<__half, double>(nlines, nuz, codes, scale, dst, st, sm_count);
    return bf ? decode_t<__nv_bfloat16, float>(nlines, nuz, codes, scale, dst, st, sm_count)
              : decode_t<__half, float>(nlines, nuz, codes, scale, dst, st, sm_count);
}

} // namespace vk
