// kick_cube.cu -- one kick of Eq. (5), D_uz D_uy D_ux, in a single pass over f.
//
// Every spatial cell owns its whole velocity cube (Listing 1: u_z innermost) and a
// kick never leaves the cell (Sec. 4.1.3: the velocity sweeps need no exchange), so
// a CTA can take one cube of NU^3 cells (NU = n_ux = n_uy = n_uz = 16 or 32) into
// shared memory, run the three velocity sweeps of Eq. (4) on it, and write it back
// once: f is read and written once per kick instead of once per sweep.
//
// Shared memory holds three half-cube buffers (NU / 2 planes of constant j_x each;
// at NU = 32 in FP32, 64 KB each) that rotate: while a cube sits in two of them,
// the third receives the first half of the next cube, and once the first half of
// the current cube has been swept and stored, its buffer receives the second half
// of the next cube.  Half-cube number j (two per cube, in the order the CTA takes
// its cubes) always lives in buffer j % 3.  One producer thread drives the TMA
// engine (loads with transaction-count mbarriers, bulk stores); every wait is
// bounded.  Rows (u_z lines) are stored with the TMA 32/64/128-byte swizzle, so
// the three access patterns are free of bank conflicts:
//   D_ux: thread = line (j_y, j_z), walks j_x across both halves (one value per
//         row, lanes on consecutive j_z: one row segment per warp access);
//   D_uy: a warp owns whole planes of a half; lane = column j_z, walks j_y;
//   D_uz: the same warp, lane = row j_y, reads its row in 16-byte chunks.
// Each line is marched in registers by the same SL-MPP5 code (march_regs) as the
// separate sweeps, so the result equals D_uz D_uy D_ux run as separate kernels,
// bit for bit.  16-bit storage keeps the rounding points of the separate path:
// D_ux encodes its result with the line scales it decoded with (one stochastic
// draw per value, the stream of the u_x register-line kernel), D_uy writes FP32
// into a per-warp plane buffer, D_uz takes its rows from there, refreshes each row
// scale to the row's largest value and encodes with the stream of the u_z kernel.
#include "vk_lines.cuh"

namespace vk {

namespace {

template <int NU, typename T> struct Cube {
    static constexpr int es = int(sizeof(T));
    static constexpr bool coded = sizeof(T) == 2;
    static constexpr int rowbytes = NU * es;
    static constexpr int chunks = rowbytes / 16;
    static constexpr int per = 16 / es;
    static constexpr int half_rows = NU * NU / 2; // u_z lines of half a cube
    static constexpr unsigned half_bytes = unsigned(half_rows) * rowbytes;
    static constexpr int box_rows = half_rows < 256 ? half_rows : 256;
    static constexpr int boxes = half_rows / box_rows;
    static constexpr unsigned scale_bytes = coded ? unsigned(half_rows) * 4u : 0u;
    static constexpr int threads = NU * NU / 2; // consumer threads
    static constexpr int warps = threads / 32;
    static constexpr int planes_per_warp = 32 / NU; // of each half
    static constexpr int pitch = NU + 1;            // FP32 plane buffer: floats per row
    static constexpr int plane_floats = NU * pitch; // NU = 16: the two planes of a warp fall on complementary banks
    static constexpr unsigned plane_bytes = coded ? unsigned(warps * planes_per_warp * plane_floats) * 4u : 0u;
    // 16-bit: per warp, the inverse scales of the rows its D_ux lines cross (32)
    static constexpr unsigned inv_bytes = coded ? unsigned(warps) * 32u * 4u : 0u;
    static constexpr size_t smem = 128 + 1024 + 3 * size_t(half_bytes) + 3 * size_t(scale_bytes) + plane_bytes + inv_bytes;
    // swizzled byte offset of 16-byte chunk j of row r / of element c of row r
    __device__ static int off(int r, int j) { return r * rowbytes + 16 * (j ^ ((r * rowbytes >> 7) & (chunks - 1))); }
    __device__ static int eoff(int r, int c) { return off(r, c / per) + (c % per) * es; }
};

// D_ux on line (jy, jz) of the cube in halves h[0], h[1] (scales s[0], s[1]); e0 =
// index of the line's first element in f (16-bit stochastic-rounding stream).
// Returns true when the line sum is negative, NaN or infinite.
template <int NU, typename T, bool NEG>
__device__ __forceinline__ bool cube_ux(unsigned char *const (&h)[2], const float *const (&s)[2], const float *inv_jx,
                                        int jy, int jz, const Lim<float> &lim, unsigned long long e0, unsigned seed)
{
    using G = Cube<NU, T>;
    constexpr int HP = NU / 2; // planes per half
    float v[NU];
#pragma unroll
    for (int jx = 0; jx < NU; ++jx) {
        const int r = (jx % HP) * NU + jy;
        const T c = *reinterpret_cast<const T *>(h[jx / HP] + G::eoff(r, jz));
        v[NEG ? NU - 1 - jx : jx] = RegCodec<T>::get(c, G::coded ? s[jx / HP][r] : 1.f);
    }
    const float sum = march_regs<NU, float>(v, lim);
    unsigned rng = G::coded ? sr_bits(e0, seed) : 0u;
#pragma unroll
    for (int jx = 0; jx < NU; ++jx) {
        const int r = (jx % HP) * NU + jy;
        float inv = 1.f;
        unsigned rb = 0u;
        if (G::coded) {
            inv = inv_jx[jx]; // u_x keeps the scales
            rb = lcg_next(rng) >> 16;
        }
        *reinterpret_cast<T *>(h[jx / HP] + G::eoff(r, jz)) = RegCodec<T>::put(v[NEG ? NU - 1 - jx : jx], inv, rb);
    }
    return !(sum >= 0.f) || isinf(sum);
}

// D_uy on column jz of plane jxl (within half buffer hb, scales sb): FP32 in place, or
// decoded into the FP32 plane buffer pl (row pitch Cube::pitch) for 16-bit codes.
template <int NU, typename T, bool NEG>
__device__ __forceinline__ bool cube_uy(unsigned char *hb, const float *sb, float *pl, int jxl, int jz,
                                        const Lim<float> &lim)
{
    using G = Cube<NU, T>;
    float v[NU];
#pragma unroll
    for (int jy = 0; jy < NU; ++jy) {
        const int r = jxl * NU + jy;
        const T c = *reinterpret_cast<const T *>(hb + G::eoff(r, jz));
        v[NEG ? NU - 1 - jy : jy] = RegCodec<T>::get(c, G::coded ? sb[r] : 1.f);
    }
    const float sum = march_regs<NU, float>(v, lim);
#pragma unroll
    for (int jy = 0; jy < NU; ++jy) {
        const float x = v[NEG ? NU - 1 - jy : jy];
        if constexpr (G::coded) pl[jy * G::pitch + jz] = x;
        else *reinterpret_cast<float *>(hb + G::eoff(jxl * NU + jy, jz)) = x;
    }
    return !(sum >= 0.f) || isinf(sum);
}

// D_uz on row jy of plane jxl: from the half buffer (FP32) or from the FP32 plane
// buffer (16-bit codes, whose row scale is then refreshed and the row encoded).
template <int NU, typename T, bool NEG>
__device__ __forceinline__ bool cube_uz(unsigned char *hb, float *sb, const float *pl, int jxl, int jy,
                                        const Lim<float> &lim, unsigned long long e0, unsigned seed)
{
    using G = Cube<NU, T>;
    const int r = jxl * NU + jy;
    float v[NU];
    if constexpr (G::coded) {
#pragma unroll
        for (int jz = 0; jz < NU; ++jz) v[NEG ? NU - 1 - jz : jz] = pl[jy * G::pitch + jz];
    } else {
#pragma unroll
        for (int j = 0; j < G::chunks; ++j) {
            float a[4];
            Chunk<float>::get(hb + G::off(r, j), 1.f, a);
#pragma unroll
            for (int q = 0; q < 4; ++q) v[NEG ? NU - 1 - (4 * j + q) : 4 * j + q] = a[q];
        }
    }
    const float sum = march_regs<NU, float>(v, lim);
    float inv = 1.f;
    if constexpr (G::coded) {
        float m = 0.f;
#pragma unroll
        for (int l = 0; l < NU; ++l) m = fmaxf(m, v[l]);
        m = coded_scale<T>(m);
        sb[r] = m;
        inv = inv_scale(m);
    }
    unsigned rng = G::coded ? sr_bits(e0, seed) : 0u;
#pragma unroll
    for (int j = 0; j < G::chunks; ++j) {
        float a[G::per];
#pragma unroll
        for (int q = 0; q < G::per; ++q) a[q] = v[NEG ? NU - 1 - (G::per * j + q) : G::per * j + q];
        Chunk<T>::put(hb + G::off(r, j), inv, a, rng);
    }
    return !(sum >= 0.f) || isinf(sum);
}

template <int NU, typename T>
__global__ void __launch_bounds__(Cube<NU, T>::threads + kProducer, NU == 32 ? 1 : 4)
    kick_cube_kernel(const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap smap,
                     const __grid_constant__ KickArgs a)
{
    using G = Cube<NU, T>;
    constexpr int NT = G::threads;
    constexpr unsigned tx_bytes = G::half_bytes + G::scale_bytes;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem); // 3: a half-cube buffer holds its data
    uint64_t *done = full + 3;                           // 3: the consumers are done with a half
    uint64_t *uxd = done + 3;                            // D_ux of the current cube is complete
    unsigned char *bufs = smem + 128 + ((1024u - ((smem_u32(smem) + 128u) & 1023u)) & 1023u);
    auto hbuf = [&](unsigned j) { return bufs + size_t(G::half_bytes) * (j % 3); };
    auto sbuf = [&](unsigned j) {
        return reinterpret_cast<float *>(bufs + 3 * size_t(G::half_bytes) + size_t(G::scale_bytes) * (j % 3));
    };
    float *planes = reinterpret_cast<float *>(bufs + 3 * size_t(G::half_bytes) + 3 * size_t(G::scale_bytes));
    float *invs = reinterpret_cast<float *>(bufs + 3 * size_t(G::half_bytes) + 3 * size_t(G::scale_bytes) +
                                            G::plane_bytes); // 16-bit: 32 per warp

    if (threadIdx.x == 0) {
        for (int q = 0; q < 3; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&done[q], NT);
        }
        mbar_init(uxd, NT);
        fence_barrier_init();
    }
    __syncthreads();

    const long long Gd = gridDim.x, b = blockIdx.x;
    const unsigned n_my = unsigned(a.ncells > b ? (a.ncells - b + Gd - 1) / Gd : 0);
    const unsigned halves = 2 * n_my;
    auto first_row = [&](unsigned j) {
        const long long cube = a.cell0 + b + (long long)(j / 2) * Gd;
        return cube * (NU * NU) + (j % 2) * G::half_rows;
    };

    if (threadIdx.x >= NT) {
        // producer: one thread drives the TMA engine
        if (threadIdx.x != NT) return;
        auto load = [&](unsigned j) {
            uint64_t *bar = &full[j % 3];
            mbar_arrive_expect_tx(bar, tx_bytes);
            const long long r0 = first_row(j);
            for (int q = 0; q < G::boxes; ++q)
                tma_load_2d(hbuf(j) + q * G::box_rows * G::rowbytes, &fmap, bar, 0, int(r0 + q * G::box_rows));
            if (G::coded) tma_load_2d(sbuf(j), &smap, bar, 0, int(r0 / NU));
        };
        unsigned loaded = 0;
        for (; loaded < 3 && loaded < halves; ++loaded) load(loaded);
        bool ok = true;
        for (unsigned j = 0; j < halves; ++j) {
            if (!mbar_wait_bounded(&done[j % 3], (j / 3) & 1u)) {
                ok = false;
                break;
            }
            const long long r0 = first_row(j);
            for (int q = 0; q < G::boxes; ++q)
                tma_store_2d(&fmap, hbuf(j) + q * G::box_rows * G::rowbytes, 0, int(r0 + q * G::box_rows));
            if (G::coded) tma_store_2d(&smap, sbuf(j), 0, int(r0 / NU));
            bulk_commit();
            if (loaded < halves) {
                bulk_wait_read_all(); // the buffer of half j is free once the store has read it
                load(loaded++);
            }
        }
        bulk_wait_all();
        if (!ok) {
            atomicOr(a.err, ERR_TIMEOUT);
            // let the loads in flight land before the CTA exits
            for (unsigned j = 0; j < loaded; ++j) mbar_wait_bounded(&full[j % 3], (j / 3) & 1u);
        }
        return;
    }

    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    float *pl = planes + (w * G::planes_per_warp + lane / NU) * G::plane_floats; // 16-bit: this lane's plane
    bool bad = false;
    for (unsigned k = 0; k < n_my; ++k) {
        const unsigned j0 = 2 * k, j1 = 2 * k + 1;
        const bool got = mbar_wait_bounded(&full[j0 % 3], (j0 / 3) & 1u) && mbar_wait_bounded(&full[j1 % 3], (j1 / 3) & 1u);
        if (!__all_sync(0xffffffffu, got)) {
            atomicOr(a.err, ERR_TIMEOUT);
            return;
        }
        const long long cube = a.cell0 + b + (long long)k * Gd;
        unsigned char *const h[2] = {hbuf(j0), hbuf(j1)};
        float *const s[2] = {sbuf(j0), sbuf(j1)};
        const unsigned long long e_cube = (unsigned long long)cube * (NU * NU * NU);
        // one Courant number per cell and axis: every branch below is CTA-uniform
        const LineCoefT<float> kx = a.coef_x[cube];
        if (kx.nd >= 0) {
            const Lim<float> lim = to_lim(kx);
            const float *const sc[2] = {s[0], s[1]};
#pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                const int line = q * NT + t, jy = line / NU, jz = line % NU;
                const unsigned long long e0 = e_cube + (unsigned long long)line;
                // 16-bit: the warp's lines cross NU rows per j_y (32 / NU values of j_y): each
                // lane forms the inverse scale of one of them once, for the whole warp
                float *wi = invs + w * 32;
                if constexpr (G::coded) {
                    __syncwarp();
                    const int jy_l = (q * NT + w * 32) / NU + lane / NU, jx = lane % NU;
                    wi[lane] = inv_scale(sc[jx / (NU / 2)][(jx % (NU / 2)) * NU + jy_l]);
                    __syncwarp();
                }
                const float *inv_jx = wi + (lane / NU) * NU;
                bad |= (kx.nd & 1) ? cube_ux<NU, T, true>(h, sc, inv_jx, jy, jz, lim, e0, a.seed_x)
                                   : cube_ux<NU, T, false>(h, sc, inv_jx, jy, jz, lim, e0, a.seed_x);
            }
        }
        // every D_ux line crosses every plane: all of them finish before D_uy
        mbar_arrive(uxd);
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(uxd, k & 1u))) {
            atomicOr(a.err, ERR_TIMEOUT);
            return;
        }
        const LineCoefT<float> ky = a.coef_y[cube], kz = a.coef_z[cube];
        const int jxl = w * G::planes_per_warp + lane / NU, c = lane % NU;
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh) {
            unsigned char *const hb = hh ? h[1] : h[0]; // selects, not a dynamically indexed array
            float *const sb = hh ? s[1] : s[0];
            if (ky.nd >= 0) {
                const Lim<float> lim = to_lim(ky);
                bad |= (ky.nd & 1) ? cube_uy<NU, T, true>(hb, sb, pl, jxl, c, lim)
                                   : cube_uy<NU, T, false>(hb, sb, pl, jxl, c, lim);
            } else if (G::coded) {
                // no D_uy: the plane buffer takes the decoded values as they are
#pragma unroll 4
                for (int jy = 0; jy < NU; ++jy) {
                    const int r = jxl * NU + jy;
                    pl[jy * G::pitch + c] = RegCodec<T>::get(*reinterpret_cast<const T *>(hb + G::eoff(r, c)), sb[r]);
                }
            }
            __syncwarp();
            const unsigned long long e0 = e_cube + (unsigned long long)((hh * (NU / 2) + jxl) * NU + c) * NU;
            if (kz.nd >= 0) {
                const Lim<float> lim = to_lim(kz);
                bad |= (kz.nd & 1) ? cube_uz<NU, T, true>(hb, sb, pl, jxl, c, lim, e0, a.seed_z)
                                   : cube_uz<NU, T, false>(hb, sb, pl, jxl, c, lim, e0, a.seed_z);
            } else if (G::coded && ky.nd >= 0) {
                // D_uy changed the plane but D_uz does not run: encode it with the row's scale
                // refreshed as the u_z sweep would not; keep the stored scale, round to nearest
                const int r = jxl * NU + c;
                const float inv = inv_scale(sb[r]);
#pragma unroll 4
                for (int jz = 0; jz < NU; ++jz)
                    *reinterpret_cast<T *>(hb + G::eoff(r, jz)) = from_c<T>(pl[c * G::pitch + jz] * inv);
            }
            __syncwarp();
            fence_proxy_async();
            mbar_arrive(&done[(2 * k + hh) % 3]);
        }
    }
    if (bad) atomicOr(a.err, ERR_NAN);
}

template <int NU, typename T> const void *kick_kernel() { return (const void *)kick_cube_kernel<NU, T>; }

const void *kick_kernel_for(int nu, int dtype)
{
    switch (dtype) {
    case 1: return nu == 32 ? kick_kernel<32, float>() : kick_kernel<16, float>();
    case 2: return nu == 32 ? kick_kernel<32, __nv_bfloat16>() : kick_kernel<16, __nv_bfloat16>();
    case 3: return nu == 32 ? kick_kernel<32, __half>() : kick_kernel<16, __half>();
    default: return nullptr;
    }
}

template <int NU> size_t smem_for(int dtype)
{
    return dtype == 1 ? Cube<NU, float>::smem : Cube<NU, __nv_bfloat16>::smem;
}

template <int NU> int threads_for() { return Cube<NU, float>::threads + kProducer; }

} // namespace

bool kick_cube_supported(int nux, int nuy, int nuz, int dtype)
{
    return nux == nuy && nuy == nuz && (nuz == 16 || nuz == 32) && dtype >= 1 && dtype <= 3;
}

int kick_cube_box_rows(int nu) { return nu * nu / 2 < 256 ? nu * nu / 2 : 256; }

size_t kick_cube_smem(int nu, int dtype) { return nu == 32 ? smem_for<32>(dtype) : smem_for<16>(dtype); }

int occupancy_kick_cube(int nu, int dtype)
{
    const void *k = kick_kernel_for(nu, dtype);
    if (!k) return 0;
    const size_t smem = kick_cube_smem(nu, dtype);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) return 0;
    int n = 0;
    const int threads = nu == 32 ? threads_for<32>() : threads_for<16>();
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_kick_cube(const CUtensorMap &fmap, const CUtensorMap &smap, const KickArgs &a, int nu, int dtype,
                             int grid, cudaStream_t st)
{
    if (a.ncells <= 0 || grid <= 0) return cudaSuccess;
    const void *k = kick_kernel_for(nu, dtype);
    if (!k || !a.coef_x || !a.coef_y || !a.coef_z) return cudaErrorInvalidValue;
    // row coordinates of the tensor maps are 32-bit
    if ((a.cell0 + a.ncells) * (long long)nu * nu > 0x7fffffffll) return cudaErrorInvalidValue;
    const size_t smem = kick_cube_smem(nu, dtype);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    KickArgs args = a;
    void *params[] = {const_cast<CUtensorMap *>(&fmap), const_cast<CUtensorMap *>(&smap), &args};
    const int threads = nu == 32 ? threads_for<32>() : threads_for<16>();
    return cudaLaunchKernel(k, dim3(grid), dim3(threads), params, smem, st);
}

} // namespace vk
