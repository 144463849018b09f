// sweep_lines.cu -- SL-MPP5 sweeps with whole lines in registers: u_z lines of
// n_uz = 16 or 32 cells (FP32, BF16, FP16), the fused kick tail, and strided
// u_x / u_y lines of 16 or 32 cells.
//
// Eq. (4) for i = 3 (Yoshikawa, Tanaka & Yoshida, SC'21).  A u_z line is one
// row of n_uz contiguous cells, 64 or 128 bytes.  TMA loads a box of 256 rows
// with the 64-/128-byte hardware swizzle: 16-byte chunk j of row r lands at
// chunk j ^ ((r * rowbytes >> 7) & (rowbytes / 16 - 1)), so eight threads that
// each read a 16-byte chunk of eight consecutive rows hit eight different bank
// groups.  Each of 256 consumer threads (line_sweep1_kernel) owns one row of
// the tile, pulls it into registers, marches it fully unrolled (the orientation
// is a warp-uniform branch: all 256 rows of a tile share a spatial cell), and
// writes it back for the TMA store.  This replaces the shared-memory transpose
// of sweep_contig.cu, the GPU analogue of the paper's load-and-transpose (LAT,
// Sec. 4.3), for these line lengths.
//
// Fused kick tail (FUSE_Y, n_uy = n_uz): a tile of 256 rows is 256 / n_uy
// whole (cell, j_x) planes of n_uy rows (j_y) by n_uz columns (j_z), so the
// u_y lines of the tile are its columns.  Before the u_z sweep each consumer
// thread walks one column down a plane (D_uy, Eq. 4 for i = 2); the u_z sweep
// then reads the updated tile: D_uz D_uy in one pass over f instead of two.
// 16-bit storage: the columns are decoded with their rows' scales and the D_uy
// result goes to an FP32 copy of the tile (same swizzled layout), from which the
// u_z rows are read; only the D_uz result is encoded (one rounding per kick
// tail instead of two).
#include "vk_lines.cuh"

namespace vk {

constexpr int kLineRows = 256;              // rows per tile, one per consumer thread
constexpr int kLineRing = 2;                // tile slots

template <int NU, typename T> struct LineGeom {
    static constexpr int rowbytes = NU * int(sizeof(T));
    static constexpr int chunks = rowbytes / 16;
    static constexpr int per = 16 / int(sizeof(T)); // elements per 16-byte chunk
    // swizzled byte offset of 16-byte chunk j of row r
    __device__ static int off(int r, int j) { return r * rowbytes + 16 * (j ^ ((r * rowbytes >> 7) & (chunks - 1))); }
};

// One row per consumer thread: a tile of 256 rows, 256 consumer threads and one
// producer warp.
constexpr int kLine1Threads = kLineRows;

// D_uy on the tile's planes for the one-row kernel (FP32, n_uy = n_uz = NU):
// warp w later sweeps rows 32w..32w+31 along u_z, whole planes; lane l walks
// column l % NU of the plane that starts at row 32w + (l / NU) NU.
template <int NU, bool NEG>
__device__ __forceinline__ bool plane_column1(unsigned char *base, int tid, const Lim<float> &lim)
{
    using G_ = LineGeom<NU, float>;
    const int w = tid >> 5, l = tid & 31;
    const int r_first = 32 * w + (l / NU) * NU, c = l % NU;
    float v[NU];
#pragma unroll
    for (int i = 0; i < NU; ++i)
        v[NEG ? NU - 1 - i : i] =
            *reinterpret_cast<const float *>(base + G_::off(r_first + i, c / G_::per) + (c % G_::per) * 4);
    const float sum = march_regs<NU, float>(v, lim);
#pragma unroll
    for (int i = 0; i < NU; ++i)
        *reinterpret_cast<float *>(base + G_::off(r_first + i, c / G_::per) + (c % G_::per) * 4) =
            v[NEG ? NU - 1 - i : i];
    return !(sum >= 0.f) || isinf(sum);
}

// The same for 16-bit codes: lane l of warp w decodes column l % NU of the plane
// at row 32w + (l / NU) NU (row 32w + i has the scale held by lane i), marches it
// in FP32 and writes it to the FP32 tile copy `wide`.
template <int NU, typename T, bool NEG>
__device__ __forceinline__ bool plane_column1_coded(const unsigned char *base, unsigned char *wide, int tid,
                                                   const Lim<float> &lim, float s_own)
{
    using GT = LineGeom<NU, T>;
    using GF = LineGeom<NU, float>;
    const int w = tid >> 5, l = tid & 31;
    const int j0 = (l / NU) * NU, r_first = 32 * w + j0, c = l % NU;
    float v[NU];
#pragma unroll
    for (int i = 0; i < NU; ++i) {
        const float s = __shfl_sync(0xffffffffu, s_own, j0 + i);
        const T code = *reinterpret_cast<const T *>(base + GT::off(r_first + i, c / GT::per) + (c % GT::per) * 2);
        v[NEG ? NU - 1 - i : i] = __fmul_rn(float(code), s);
    }
    const float sum = march_regs<NU, float>(v, lim);
#pragma unroll
    for (int i = 0; i < NU; ++i)
        *reinterpret_cast<float *>(wide + GF::off(r_first + i, c / GF::per) + (c % GF::per) * 4) =
            v[NEG ? NU - 1 - i : i];
    return !(sum >= 0.f) || isinf(sum);
}

template <int NU, typename T, bool FUSE_Y>
__global__ void __launch_bounds__(kLine1Threads + kProducer, 3)
    line_sweep1_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap dmap,
                       const __grid_constant__ ContigArgs<float> args)
{
    constexpr int S = kLineRing;
    constexpr unsigned slot_bytes = kLineRows * NU * sizeof(T);
    constexpr bool CODED = sizeof(T) == 2;
    using G_ = LineGeom<NU, T>;
    constexpr int PER = G_::per;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *done = full + S;
    unsigned char *ring = smem + 128 + ((1024u - ((smem_u32(smem) + 128u) & 1023u)) & 1023u);
    auto slot = [&](unsigned e) { return ring + slot_bytes * (e % S); };
    unsigned char *wide = ring + slot_bytes * S; // FP32 copy of a 16-bit tile after D_uy (fused only)

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&done[s], kLine1Threads);
        }
        fence_barrier_init();
    }
    __syncthreads();

    const long long Gd = gridDim.x, b = blockIdx.x;
    const unsigned n_my = unsigned((args.num_tiles > b) ? (args.num_tiles - b + Gd - 1) / Gd : 0);

    if (threadIdx.x < kProducer) {
        if (threadIdx.x != 0) return;
        unsigned loaded = 0, retired = 0;
        bool ok = true;
        while (retired < n_my) {
            bool progress = false;
            while (retired < loaded && mbar_test_wait(&done[retired % S], (retired / S) & 1u)) {
                tma_store_2d(&dmap, slot(retired), 0, int((args.tile0 + b + (long long)retired * Gd) * kLineRows));
                bulk_commit();
                ++retired;
                progress = true;
            }
            if (loaded < n_my && loaded < retired + S) {
                if (loaded >= unsigned(S)) bulk_wait_read_at_most(retired - 1u - (loaded - S));
                const unsigned st = loaded % S;
                mbar_arrive_expect_tx(&full[st], slot_bytes);
                tma_load_2d(slot(loaded), &map, &full[st], 0, int((args.tile0 + b + (long long)loaded * Gd) * kLineRows));
                ++loaded;
                progress = true;
            }
            if (!progress && !mbar_wait_bounded(&done[retired % S], (retired / S) & 1u)) {
                ok = false;
                break;
            }
        }
        bulk_wait_all();
        if (!ok) {
            atomicOr(args.err, ERR_TIMEOUT);
            for (unsigned t = retired; t < loaded; ++t) mbar_wait_bounded(&full[t % S], (t / S) & 1u);
        }
        return;
    }

    const int r = threadIdx.x - kProducer;
    for (unsigned k = 0; k < n_my; ++k) {
        const unsigned st = k % S;
        // all lanes of a warp leave together (the fused pass synchronises the warp)
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[st], (k / S) & 1u))) {
            atomicOr(args.err, ERR_TIMEOUT);
            break;
        }
        const long long row0 = (args.tile0 + b + (long long)k * Gd) * kLineRows;
        unsigned char *base = slot(k);
        // rows of a tile are whole planes of one spatial cell: tile-uniform
        const float sc = CODED && row0 + r < args.rows ? args.scale[row0 + r] : 1.f;
        bool from_wide = false; // 16-bit fused: the u_z rows come from the FP32 copy
        if constexpr (FUSE_Y) {
            const LineCoefT<float> ky = args.cell_coef_y[fdiv(unsigned(row0), args.div_rpc)];
            if (row0 < args.rows && ky.nd >= 0) {
                bool bad;
                if constexpr (CODED) {
                    bad = (ky.nd & 1) ? plane_column1_coded<NU, T, true>(base, wide, r, to_lim(ky), sc)
                                      : plane_column1_coded<NU, T, false>(base, wide, r, to_lim(ky), sc);
                    from_wide = true;
                } else {
                    bad = (ky.nd & 1) ? plane_column1<NU, true>(base, r, to_lim(ky))
                                      : plane_column1<NU, false>(base, r, to_lim(ky));
                }
                if (bad) atomicOr(args.err, ERR_NAN);
            }
            __syncwarp();
        }
        if (row0 + r < args.rows) {
            const LineCoefT<float> kc = args.cell_coef[fdiv(unsigned(row0 + r), args.div_rpc)];
            if (kc.nd >= 0) {
                const bool neg = kc.nd & 1; // one orientation per spatial cell: warp-uniform
                unsigned rng = CODED_RNG_INIT((unsigned long long)(row0 + r) * NU, args.seed);
                float v[NU];
                if (from_wide) {
                    using GF = LineGeom<NU, float>;
#pragma unroll
                    for (int j = 0; j < GF::chunks; ++j) {
                        float a[4];
                        Chunk<float>::get(wide + GF::off(r, j), 1.f, a);
#pragma unroll
                        for (int q = 0; q < 4; ++q) v[neg ? NU - 1 - (4 * j + q) : 4 * j + q] = a[q];
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < G_::chunks; ++j) {
                        float a[PER];
                        Chunk<T>::get(base + G_::off(r, j), sc, a);
#pragma unroll
                        for (int q = 0; q < PER; ++q) v[neg ? NU - 1 - (PER * j + q) : PER * j + q] = a[q];
                    }
                }
                const float sum = march_regs<NU, float>(v, to_lim(kc));
                float inv = 1.f;
                if (CODED) {
                    // new scale: the line's largest value
                    float m = 0.f;
#pragma unroll
                    for (int l = 0; l < NU; ++l) m = fmaxf(m, v[l]);
                    m = coded_scale<T>(m);
                    args.scale[row0 + r] = m;
                    inv = inv_scale(m);
                }
#pragma unroll
                for (int j = 0; j < G_::chunks; ++j) {
                    float a[PER];
#pragma unroll
                    for (int q = 0; q < PER; ++q) a[q] = v[neg ? NU - 1 - (PER * j + q) : PER * j + q];
                    Chunk<T>::put(base + G_::off(r, j), inv, a, rng);
                }
                if (!(sum >= 0.f) || isinf(sum)) atomicOr(args.err, ERR_NAN);
            }
        }
        fence_proxy_async();
        mbar_arrive(&done[st]);
    }
}

// ----------------------------------------------------------------------------
// strided zero-flux lines in registers (u_x, u_y)
// ----------------------------------------------------------------------------
// Thread t owns line t: outer = t / n_inner, inner = t % n_inner, cell i of the line
// at (outer L + i) n_inner + inner.  Neighbouring threads own neighbouring columns,
// so each of the L loads (and stores) of a warp is one coalesced segment; all loads
// are issued before the march.  A negative Courant number reverses the register
// order (the march always flows toward +index).  16-bit codes: cell i decodes with
// the scale of its u_z line (line0 + i Iz, Iz = n_inner / nuz u_z lines per row of
// the swept axis), which the sweep keeps, and encodes back with stochastic rounding.

template <int L, typename T>
__global__ void __launch_bounds__(256, L > 32 ? 2 : 3) reg_lines_kernel(const T *__restrict__ src, T *dst,
                                                          const __grid_constant__ RegLineArgs a)
{
    constexpr bool CODED = sizeof(T) == 2;
    const long long t = a.line0 + blockIdx.x * 256ll + threadIdx.x;
    if (t >= a.line0 + a.nlines) return;
    long long outer, cell;
    if (a.line0 + a.nlines <= 0xffffffffll) { // every line index of the launch fits 32 bits
        outer = fdiv(unsigned(t), a.div_inner);
        cell = fdiv(unsigned(outer), a.div_opc);
    } else {
        outer = t / a.n_inner;
        cell = outer / a.outer_per_cell;
    }
    const long long inner = t - outer * a.n_inner;
    const long long base = outer * L * a.n_inner + inner;
    const LineCoefT<float> kc = a.cell_coef[cell];
    const T *p = src + base;
    T *q = dst + base;
    if (kc.nd < 0) {
        // Courant number out of range (flagged by the constants kernel): unchanged
        if (q != p)
#pragma unroll
            for (int i = 0; i < L; ++i) q[i * a.n_inner] = p[i * a.n_inner];
        return;
    }
    // 16-bit: the u_z line of cell i is zl + i Iz (inner < n_inner < 2^32)
    const long long Iz = CODED ? a.n_inner / a.nuz : 0;
    const long long zl = CODED ? outer * L * Iz + fdiv(unsigned(inner), a.div_nuz) : 0;
    const bool neg = kc.nd & 1; // one orientation per spatial cell
    float v[L];
#pragma unroll
    for (int i = 0; i < L; ++i) v[i] = RegCodec<T>::get(p[i * a.n_inner], CODED ? __ldg(a.scale + zl + i * Iz) : 1.f);
    if (neg) {
#pragma unroll
        for (int i = 0; i < L / 2; ++i) { const float t0 = v[i]; v[i] = v[L - 1 - i]; v[L - 1 - i] = t0; }
    }
    const float sum = march_regs<L, float>(v, to_lim(kc));
    if (neg) {
#pragma unroll
        for (int i = 0; i < L / 2; ++i) { const float t0 = v[i]; v[i] = v[L - 1 - i]; v[L - 1 - i] = t0; }
    }
    unsigned rng = CODED ? sr_bits((unsigned long long)base, a.seed) : 0u;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        float inv = 1.f;
        unsigned r = 0u;
        if (CODED) {
            inv = inv_scale(__ldg(a.scale + zl + i * Iz));
            r = lcg_next(rng) >> 16;
        }
        q[i * a.n_inner] = RegCodec<T>::put(v[i], inv, r);
    }
    if (!(sum >= 0.f) || isinf(sum)) atomicOr(a.err, ERR_NAN);
}

bool reg_lines_supported(int L) { return L == 16 || L == 32 || L == 48; }

template <typename T> static cudaError_t launch_reg_t(const void *src, void *dst, const RegLineArgs &a, unsigned blocks,
                                                      cudaStream_t st)
{
    const T *s = static_cast<const T *>(src);
    T *d = static_cast<T *>(dst);
    if (a.L == 32) reg_lines_kernel<32, T><<<blocks, 256, 0, st>>>(s, d, a);
    else if (a.L == 16) reg_lines_kernel<16, T><<<blocks, 256, 0, st>>>(s, d, a);
    else if (a.L == 48) reg_lines_kernel<48, T><<<blocks, 256, 0, st>>>(s, d, a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_reg_lines(const void *src, void *dst, const RegLineArgs &args, int dtype, cudaStream_t st)
{
    if (args.nlines <= 0) return cudaSuccess;
    const long long blocks = (args.nlines + 255) / 256;
    if (blocks > 0x7fffffffll || args.n_inner <= 0 || args.n_inner > 0xffffffffll || args.outer_per_cell <= 0 ||
        args.outer_per_cell > 0xffffffffll)
        return cudaErrorInvalidValue;
    RegLineArgs a = args;
    a.div_inner = make_fastdiv(unsigned(a.n_inner));
    a.div_opc = make_fastdiv(unsigned(a.outer_per_cell));
    a.div_nuz = make_fastdiv(unsigned(a.nuz > 0 ? a.nuz : 1));
    switch (dtype) {
    case 1: return launch_reg_t<float>(src, dst, a, unsigned(blocks), st);
    case 2: return launch_reg_t<__nv_bfloat16>(src, dst, a, unsigned(blocks), st);
    case 3: return launch_reg_t<__half>(src, dst, a, unsigned(blocks), st);
    default: return cudaErrorInvalidValue;
    }
}

// ----------------------------------------------------------------------------
// u_z rows staged per warp (other line lengths)
// ----------------------------------------------------------------------------
// Each warp owns 32 consecutive rows: it copies them to shared memory with
// coalesced 16-byte loads, each lane marches its own row in registers, and the
// warp copies the rows back.  A row takes NU es / 16 chunks of 16 bytes; the
// pitch is rounded up to an odd number of chunks, so that the 8 lanes of a phase
// reading chunk j of their rows hit 8 different groups of 4 banks.  16-bit codes:
// the row decodes with its scale, the sweep sets the scale to the row's largest
// new value and encodes with stochastic rounding (one stream per row and sweep).
template <int NU, typename T> constexpr int rows_chunks() { return NU * int(sizeof(T)) / 16; }
template <int NU, typename T> constexpr int rows_pitch() { return rows_chunks<NU, T>() | 1; } // in chunks
template <int NU, typename T> constexpr size_t rows_sweep_smem() { return size_t(256) * rows_pitch<NU, T>() * 16; }

template <int NU, typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2) rows_sweep_kernel(const T *__restrict__ src, T *dst,
                                                                                const __grid_constant__ RowsArgs a)
{
    using C = typename Compute<T>::type;
    constexpr bool CODED = sizeof(T) == 2;
    constexpr int CH = rows_chunks<NU, T>(), PC = rows_pitch<NU, T>(), PER = 16 / int(sizeof(T));
    static_assert(CH * 16 == NU * int(sizeof(T)), "a row is whole 16-byte chunks");
    extern __shared__ __align__(16) uint4 rows_sw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint4 *sr = rows_sw + w * 32 * PC;
    const long long r0 = a.row0 + (blockIdx.x * 8ll + w) * 32; // the warp's first row
    const long long left = a.row0 + a.nrows - r0;
    const int nrows = left >= 32 ? 32 : (left > 0 ? int(left) : 0);
    const uint4 *g = reinterpret_cast<const uint4 *>(src + r0 * NU);
    uint4 *o = reinterpret_cast<uint4 *>(dst + r0 * NU);
#pragma unroll
    for (int k = lane; k < 32 * CH; k += 32) {
        const int row = k / CH, col = k % CH;
        if (row < nrows) sr[row * PC + col] = __ldg(g + k);
    }
    __syncwarp();
    if (lane < nrows) {
        const long long row = r0 + lane;
        // FP32 rows keep the plain division: measured 22.1 ms per u_z sweep on 48^3 x 48^3
        // against 24.2 with the divider (16-bit rows: 19.5 with it against 21.6)
        const long long cell = sizeof(T) == 4 ? row / a.rows_per_cell : (long long)fdiv(unsigned(row), a.div_rpc);
        const LineCoefT<C> kc = static_cast<const LineCoefT<C> *>(a.cell_coef)[cell];
        if (kc.nd >= 0) {
            const bool neg = kc.nd & 1; // one orientation per spatial cell
            unsigned char *mine = reinterpret_cast<unsigned char *>(sr + lane * PC);
            const float sc = CODED ? a.scale[row] : 1.f;
            C v[NU];
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                C e[PER];
                Chunk<T>::get(mine + 16 * q, sc, e);
#pragma unroll
                for (int j = 0; j < PER; ++j) v[neg ? NU - 1 - (PER * q + j) : PER * q + j] = e[j];
            }
            const C sum = march_regs<NU, C>(v, to_lim(kc));
            float inv = 1.f;
            if constexpr (CODED) {
                // new scale: the row's largest value
                float m = 0.f;
#pragma unroll
                for (int l = 0; l < NU; ++l) m = fmaxf(m, v[l]);
                m = coded_scale<T>(m);
                a.scale[row] = m;
                inv = inv_scale(m);
            }
            unsigned rng = CODED_RNG_INIT((unsigned long long)row * NU, a.seed);
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                C e[PER];
#pragma unroll
                for (int j = 0; j < PER; ++j) e[j] = v[neg ? NU - 1 - (PER * q + j) : PER * q + j];
                Chunk<T>::put(mine + 16 * q, inv, e, rng);
            }
            if (!(sum >= C(0)) || isinf(sum)) atomicOr(a.err, ERR_NAN);
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = lane; k < 32 * CH; k += 32) {
        const int row = k / CH, col = k % CH;
        if (row < nrows) o[k] = sr[row * PC + col];
    }
}

bool rows_sweep_supported(int L, int dtype) { return dtype >= 0 && dtype <= 3 && (L == 24 || L == 40 || L == 48); }

template <int NU, typename T>
static cudaError_t launch_rows_t(const void *src, void *dst, const RowsArgs &a, cudaStream_t st)
{
    const long long blocks = (a.nrows + 255) / 256;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    const cudaError_t e = cudaFuncSetAttribute(rows_sweep_kernel<NU, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               int(rows_sweep_smem<NU, T>()));
    if (e != cudaSuccess) return e;
    rows_sweep_kernel<NU, T><<<unsigned(blocks), 256, rows_sweep_smem<NU, T>(), st>>>(static_cast<const T *>(src),
                                                                                     static_cast<T *>(dst), a);
    return cudaGetLastError();
}

template <typename T> static cudaError_t launch_rows_len(const void *src, void *dst, const RowsArgs &a, cudaStream_t st)
{
    switch (a.L) {
    case 24: return launch_rows_t<24, T>(src, dst, a, st);
    case 40: return launch_rows_t<40, T>(src, dst, a, st);
    case 48: return launch_rows_t<48, T>(src, dst, a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rows_sweep(const void *src, void *dst, const RowsArgs &args, int dtype, cudaStream_t st)
{
    if (args.nrows <= 0) return cudaSuccess;
    if ((dtype == 2 || dtype == 3) && !args.scale) return cudaErrorInvalidValue;
    // row indices (u_z lines) stay below 2^31 (checked at init)
    if (args.row0 + args.nrows + 255 > 0xffffffffll || args.rows_per_cell <= 0 || args.rows_per_cell > 0xffffffffll)
        return cudaErrorInvalidValue;
    RowsArgs a = args;
    a.div_rpc = make_fastdiv(unsigned(a.rows_per_cell));
    switch (dtype) {
    case 0: return launch_rows_len<double>(src, dst, a, st);
    case 1: return launch_rows_len<float>(src, dst, a, st);
    case 2: return launch_rows_len<__nv_bfloat16>(src, dst, a, st);
    case 3: return launch_rows_len<__half>(src, dst, a, st);
    default: return cudaErrorInvalidValue;
    }
}

static const void *line_kernel_for(int nu, int dtype, bool fuse_y)
{
    if (fuse_y && dtype == 2)
        return nu == 32 ? (const void *)line_sweep1_kernel<32, __nv_bfloat16, true>
                        : (const void *)line_sweep1_kernel<16, __nv_bfloat16, true>;
    if (fuse_y && dtype == 3)
        return nu == 32 ? (const void *)line_sweep1_kernel<32, __half, true> : (const void *)line_sweep1_kernel<16, __half, true>;
    if (fuse_y) return nu == 32 ? (const void *)line_sweep1_kernel<32, float, true> : (const void *)line_sweep1_kernel<16, float, true>;
    if (dtype == 2)
        return nu == 32 ? (const void *)line_sweep1_kernel<32, __nv_bfloat16, false>
                        : (const void *)line_sweep1_kernel<16, __nv_bfloat16, false>;
    if (dtype == 3)
        return nu == 32 ? (const void *)line_sweep1_kernel<32, __half, false> : (const void *)line_sweep1_kernel<16, __half, false>;
    return nu == 32 ? (const void *)line_sweep1_kernel<32, float, false> : (const void *)line_sweep1_kernel<16, float, false>;
}

// the ring of tiles, plus the FP32 tile copy of the 16-bit fused pass
size_t line_sweep_smem(int nu, int es, bool fuse_y)
{
    return 128 + 1024 + (size_t)kLineRing * kLineRows * nu * es + (fuse_y && es == 2 ? (size_t)kLineRows * nu * 4 : 0);
}

bool line_sweep_fused_supported(int dtype) { return dtype >= 1 && dtype <= 3; }

bool line_sweep_supported(int nu, long long rows_per_cell)
{
    return (nu == 16 || nu == 32) && rows_per_cell % kLineRows == 0;
}

cudaError_t launch_line_sweep(const CUtensorMap &map, const CUtensorMap &dmap, const ContigArgs<float> &a_in, int nu,
                              int dtype, int grid, cudaStream_t st, bool fuse_y)
{
    if (fuse_y && (!line_sweep_fused_supported(dtype) || !a_in.cell_coef_y)) return cudaErrorInvalidValue;
    // row indices (u_z lines) stay below 2^31 (checked at init), a tile's rows below rows + 256
    if (a_in.rows + 256 > 0xffffffffll || a_in.rows_per_cell <= 0 || a_in.rows_per_cell > 0xffffffffll)
        return cudaErrorInvalidValue;
    ContigArgs<float> a = a_in;
    a.div_rpc = make_fastdiv(unsigned(a.rows_per_cell));
    const void *k = line_kernel_for(nu, dtype, fuse_y);
    const size_t smem = line_sweep_smem(nu, dtype == 1 ? 4 : 2, fuse_y);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<CUtensorMap *>(&map), const_cast<CUtensorMap *>(&dmap), &a};
    const int threads = kLine1Threads + kProducer;
    return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, st);
}

int occupancy_line_sweep(int nu, int dtype, bool fuse_y)
{
    const void *k = line_kernel_for(nu, dtype, fuse_y);
    const size_t smem = line_sweep_smem(nu, dtype == 1 ? 4 : 2, fuse_y);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) return 0;
    int n = 0;
    const int threads = kLine1Threads + kProducer;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
    return n;
}

int line_sweep_rows_per_tile() { return kLineRows; }

} // namespace vk
