// sweep_tile.cu -- position sweeps D_x, D_y, D_z of Eq. (3) (periodic lines,
// |nu| < 1) on FP32 storage with whole lines staged in shared memory.
//
// f is viewed as [O][L][I] (slower axes, the swept axis of L cells, the faster
// axes) and the faster axes I are cut into tiles of 256 contiguous columns: a
// tile holds every cell of 256 lines (L rows of 1 KB), loaded and stored by one
// TMA box {32, 8, L} of the 4D view [O][L][I / 32][32] with the 128-byte swizzle,
// so that 16-byte chunk j of the 128-byte unit u of a row lands at chunk
// j ^ (u & 7).  A thread owns one column (one line of Eq. 3, whose Courant number
// nu_j = u_j dt / (a^2 dx) depends only on the column's velocity index j) and
// marches it fully unrolled in registers with a sliding five-cell window, reading
// each row once and writing it back in place (SL-MPP5, the same code as every
// other sweep).  Groups of 256 threads work on different tiles; a ring of at
// least groups + 1 tile slots (up to 192 KB), filled and drained by one producer
// thread, keeps the next tiles loading while the groups march theirs.  The orientation of a line
// is its sign of nu.  In the x and y sweeps it is the same for whole tiles, which
// march with a fixed direction; in the z sweep (n_uz = 32), where the sign flips in
// the middle of every u_z line, warps take the 16 columns of one sign of two u_z
// lines four units apart (no bank conflicts under the swizzle) and each warp marches
// with a fixed direction.  Both bodies run side by side on an SM, which fits the
// instruction cache once lines of more than 32 cells march in blocks of 8 faces.
// Tiles that mix signs take the direction per column at run time.  For the x sweep the group's
// warps also add up every marched tile's rows into per-cell partials of rho_nu (the
// moment of Eq. 5 is taken right after this sweep), in the order of the streamed
// sweep's moment warp.
// The same tiles serve the u_x sweep of Eq. (4) (ZF): f viewed as [cell][u_x][u_y u_z],
// zero-flux lines, one Courant number per tile (the cell's), marched through a window of
// five cells (march_strided, the arithmetic of the other velocity sweeps).
#include "vk_lines.cuh"

namespace vk {

namespace {

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, const void *src, int c0, int c1, int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// thread groups (256 columns each) marching tiles at once; the ring holds one slot more
template <int L> constexpr int tile_groups() { return L <= 48 ? 3 : 2; }
template <int L> constexpr unsigned tile_bytes() { return unsigned(L) * 1024u; }
// ring slots: one more than the groups, more for short lines (up to 192 KB of tiles), so
// that several tile loads are in flight while the groups march
template <int L> constexpr int tile_slots()
{
    return (196608 / tile_bytes<L>() > 12 ? 12 : int(196608 / tile_bytes<L>())) > tile_groups<L>() + 1
               ? (196608 / tile_bytes<L>() > 12 ? 12 : int(196608 / tile_bytes<L>()))
               : tile_groups<L>() + 1;
}
// barriers (256 B), the velocity-column table, alignment to 1 KB, the ring
constexpr size_t kTileHeader = 256 + kMaxVel * sizeof(LineCoefT<float>);
template <int L> constexpr size_t tile_smem() { return kTileHeader + 1024 + size_t(tile_slots<L>()) * tile_bytes<L>(); }

// March the periodic line p[0], p[st], ..., p[(L - 1) st] (flow toward +index) in place;
// st < 0 walks a line with a negative Courant number from its far end.  DIR = +1 / -1 fixes
// the stride at compile time; DIR = 0 takes it at run time, one body for both
// orientations (for tiles whose CTAs meet both signs of u and cannot take them sign by
// sign).  Returns the sum of the new values.
// Faces marched per loop iteration: lines up to 32 cells unroll completely; longer lines
// in blocks of 8 faces, so that the code of a march stays inside the instruction cache.
template <int L> constexpr int march_unroll() { return L <= 32 ? L : 8; }

template <int L, int DIR>
__device__ __forceinline__ float march_tile(float *p, int st_rt, const Lim<float> &lim)
{
    const int st = DIR == 0 ? st_rt : DIR * 256; // rows are 256 floats apart
    const float a = p[(L - 3) * st], b = p[(L - 2) * st], c = p[(L - 1) * st];
    const float s0 = p[0], s1 = p[st];
    const float dmm = curv(a, b, c), dm = curv(b, c, s0), d0 = curv(c, s0, s1);
    float dm4m = dm4(dm, d0);
    float Fm = sl_mpp5_flux(lim, a, b, c, s0, s1, dm4(dmm, dm), dm4m); // face -1/2, donor c_{-1}
    float cm2 = b, cm1 = c, c0 = s0, cp1 = s1, dcur = d0, sum = 0.f;
    auto face = [&](float cp2, float *dst) {
        const float dn = curv(c0, cp1, cp2);
        const float dm4p = dm4(dcur, dn);
        const float F = sl_mpp5_flux(lim, cm2, cm1, c0, cp1, cp2, dm4m, dm4p);
        const float out = c0 + (Fm - F);
        *dst = out;
        sum += out;
        cm2 = cm1;
        cm1 = c0;
        c0 = cp1;
        cp1 = cp2;
        dcur = dn;
        dm4m = dm4p;
        Fm = F;
    };
#pragma unroll march_unroll<L>()
    for (int i = 0; i < L - 2; ++i) face(p[(i + 2) * st], p + i * st);
    face(s0, p + (L - 2) * st); // the last two faces take the first two cells' old values
    face(s1, p + (L - 1) * st);
    return sum;
}

// The logical 16-byte chunks lane and lane + 32 of a swizzled 1-KB row (chunk j of unit u
// is stored at chunk j ^ (u & 7) of that unit), summed in the order the streamed x sweep
// sums its unswizzled rows: the partial sums agree bit for bit.
__device__ __forceinline__ float lane_row_sum1k(const float *row, int lane)
{
    const float4 *q = reinterpret_cast<const float4 *>(row);
    const int u = lane >> 3, j = lane & 7;
    const float4 x = q[u * 8 + (j ^ u)], y = q[(u + 4) * 8 + (j ^ (u + 4))];
    return ((x.x + x.y) + (x.z + x.w)) + ((y.x + y.y) + (y.z + y.w));
}

// rows v0..v3 of 32 lanes each -> lane l holds the total of row l >> 3 (a fixed butterfly)
__device__ __forceinline__ float rows4_sum(float v0, float v1, float v2, float v3, int lane)
{
    constexpr unsigned kAll = 0xffffffffu;
    const bool hi = lane & 16, odd = lane & 8;
    float k0 = hi ? v2 : v0, k1 = hi ? v3 : v1;
    k0 += __shfl_xor_sync(kAll, hi ? v0 : v2, 16);
    k1 += __shfl_xor_sync(kAll, hi ? v1 : v3, 16);
    float k = odd ? k1 : k0;
    k += __shfl_xor_sync(kAll, odd ? k0 : k1, 8);
    k += __shfl_xor_sync(kAll, k, 4);
    k += __shfl_xor_sync(kAll, k, 2);
    k += __shfl_xor_sync(kAll, k, 1);
    return k;
}

// SIGNED: every warp's columns have one sign of u (TileArgs::tile_sign), marched with a fixed direction.
// ZF: a u_x sweep (zero-flux lines, the tile's cell's coefficients)
template <int L, bool MOMENT, bool SIGNED, bool ZF = false>
__global__ void __launch_bounds__(tile_groups<L>() * 256 + kProducer, 1)
    tile_sweep_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap dmap,
                      const __grid_constant__ TileArgs a)
{
    constexpr int NG = tile_groups<L>(), S = tile_slots<L>(), NT = NG * 256;
    constexpr unsigned TB = tile_bytes<L>();
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem); // S: the slot holds its tile
    uint64_t *done = full + S;                           // S: the tile's group is done with it
    uint64_t *marched = done + S;                        // NG: every column of the group's tile is marched
    LineCoefT<float> *tab = reinterpret_cast<LineCoefT<float> *>(smem + 256);
    static_assert((2 * S + NG) * 8 <= 256, "barriers fit ahead of the table");
    unsigned char *ring = smem + kTileHeader + ((1024u - ((smem_u32(smem) + unsigned(kTileHeader)) & 1023u)) & 1023u);
    auto slot = [&](unsigned k) { return reinterpret_cast<float *>(ring + size_t(TB) * (k % S)); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&done[s], 256);
        }
        for (int g = 0; g < NG; ++g) mbar_init(&marched[g], 256);
        fence_barrier_init();
    }
    for (int j = threadIdx.x; j < a.nvel; j += blockDim.x) tab[j] = a.table[j];
    __syncthreads();

    const long long G = gridDim.x, b = blockIdx.x;
    const unsigned n_my = unsigned(a.num_tiles > b ? (a.num_tiles - b + G - 1) / G : 0);
    auto coords = [&](unsigned k, int &u0, int &o) {
        const long long t = a.tile0 + b + (long long)k * G;
        const long long oq = t / a.tiles_inner;
        u0 = int((t - oq * a.tiles_inner) * 8); // first 32-column unit of the tile
        o = int(oq);
    };

    if (threadIdx.x >= NT) {
        // producer: one thread drives the TMA engine
        if (threadIdx.x != NT) return;
        auto load = [&](unsigned k) {
            int u0, o;
            coords(k, u0, o);
            mbar_arrive_expect_tx(&full[k % S], TB);
            tma_load_4d(slot(k), &map, &full[k % S], 0, u0, 0, o);
        };
        unsigned loaded = 0;
        for (; loaded < unsigned(S) && loaded < n_my; ++loaded) load(loaded);
        bool ok = true;
        for (unsigned k = 0; k < n_my; ++k) {
            if (!mbar_wait_bounded(&done[k % S], (k / S) & 1u)) {
                ok = false;
                break;
            }
            int u0, o;
            coords(k, u0, o);
            tma_store_4d(&dmap, slot(k), 0, u0, 0, o);
            bulk_commit();
            if (loaded < n_my) {
                bulk_wait_read_all(); // the slot is free once the store has read it
                load(loaded++);
            }
        }
        bulk_wait_all();
        if (!ok) {
            atomicOr(a.err, ERR_TIMEOUT);
            for (unsigned k = 0; k < loaded; ++k) mbar_wait_bounded(&full[k % S], (k / S) & 1u);
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int grp = threadIdx.x >> 8, tid = threadIdx.x & 255, w = tid >> 5, lane = tid & 31;
    int unit, e; // the thread's column: 32-column unit of the tile and position in it
    if (a.zperm) {
        // z sweep, n_uz = 32: warps 0-3 take u_z < 0 (e < 16), warps 4-7 u_z > 0, each
        // warp the same half of units w % 4 and w % 4 + 4
        unit = (w & 3) + (lane < 16 ? 0 : 4);
        e = (w >> 2) * 16 + (lane & 15);
    } else {
        unit = w;
        e = lane;
    }
    // swizzled offset of the column inside a 1-KB row, in floats
    const int coff = unit * 32 + (((e >> 2) ^ (unit & 7)) << 2) + (e & 3);
    bool bad = false;
    for (unsigned k = grp; k < n_my; k += NG) {
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[k % S], (k / S) & 1u))) {
            atomicOr(a.err, ERR_TIMEOUT);
            return;
        }
        int u0, o;
        coords(k, u0, o);
        const long long inner = 32ll * (u0 + unit) + e;
        const LineCoefT<float> kc = ZF ? a.cell_coef[o] : tab[(inner / a.vstride) % a.nvel];
        float *p = slot(k) + coff;
        if (kc.nd >= 0) {
            const Lim<float> lim = to_lim(kc);
            // a negative Courant number is the mirror image: march the line from its far end
            const bool neg = kc.nd & 1;
            float sum;
            if constexpr (ZF) sum = march_strided<L>(neg ? p + (L - 1) * 256 : p, neg ? -256 : 256, lim);
            else if constexpr (!SIGNED) sum = march_tile<L, 0>(neg ? p + (L - 1) * 256 : p, neg ? -256 : 256, lim);
            else if (neg) sum = march_tile<L, -1>(p + (L - 1) * 256, 0, lim); // one sign per tile
            else sum = march_tile<L, 1>(p, 0, lim);
            bad |= !(sum >= 0.f) || isinf(sum);
        }
        if constexpr (MOMENT) {
            // x sweep: once the group's tile is marched, warp w adds up rows 4q .. 4q + 3 for
            // q = w, w + 8, ...: row x of the tile whose first column is c0 adds to spatial
            // cell x (n_inner / cube) + c0 / cube as its partial (c0 % cube) / 256, stored at
            // mpart[((c0 / cube) nparts + part) L + x]
            const unsigned j = k / NG; // the group's tile count: the phase of its barrier
            mbar_arrive(&marched[grp]);
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&marched[grp], j & 1u))) {
                atomicOr(a.err, ERR_TIMEOUT);
                return;
            }
            const long long c0 = 32ll * u0;
            float *base = static_cast<float *>(a.mpart) + ((c0 / a.cube) * a.nparts + (c0 % a.cube) / 256) * (long long)L;
            const float *q = slot(k);
#pragma unroll
            for (int r = 4 * w; r < L; r += 32) {
                const float tot = rows4_sum(lane_row_sum1k(q + r * 256, lane), lane_row_sum1k(q + (r + 1) * 256, lane),
                                            lane_row_sum1k(q + (r + 2) * 256, lane),
                                            lane_row_sum1k(q + (r + 3) * 256, lane), lane);
                if ((lane & 7) == 0) base[r + (lane >> 3)] = tot;
            }
        }
        fence_proxy_async();
        mbar_arrive(&done[k % S]);
    }
    if (bad) atomicOr(a.err, ERR_NAN);
}

// ----------------------------------------------------------------------------
// 16-bit storage (BF16 / FP16 codes, one FP32 scale per u_z line of 32 or 48 cells)
// ----------------------------------------------------------------------------
// The same tiles, 512-byte rows of codes (no swizzle) plus the tile's scales (box
// {8 u_z lines, L rows} for n_uz = 32); a position sweep and a u_x sweep keep every scale.  Each value decodes as
// code x scale, the line is marched in FP32 and every value is encoded back with
// stochastic rounding (one stream per column and sweep, one draw per value in march
// order).  z sweep: warp w takes the columns of one sign of units 2 (w % 4) and
// 2 (w % 4) + 1 (adjacent 64-byte units fall on disjoint banks).
// n_uz = 48: a tile's 256 columns fall on 6 or 7 u_z lines, starting anywhere in one; its
// scale box starts at the line index rounded down to a multiple of 4 (the 16-byte rule of
// TMA) and spans 12 lines.  n_uz = 32: the 8 lines of the tile exactly.
template <int NZ> constexpr int tile16_scale_lines() { return NZ == 32 ? 8 : 12; }
template <int L> constexpr unsigned tile16_codes() { return unsigned(L) * 512u; }
template <int L, int NZ = 32> constexpr unsigned tile16_slot()
{
    return (tile16_codes<L>() + unsigned(L) * 4u * unsigned(tile16_scale_lines<NZ>()) + 127u) & ~127u;
}
template <int L, int NZ = 32> constexpr int tile16_slots()
{
    return (196608 / tile16_slot<L, NZ>() > 12 ? 12 : int(196608 / tile16_slot<L, NZ>())) > tile_groups<L>() + 1
               ? (196608 / tile16_slot<L, NZ>() > 12 ? 12 : int(196608 / tile16_slot<L, NZ>()))
               : tile_groups<L>() + 1;
}
// after the ring: per consumer warp, the inverse scales of the (up to two) u_z lines its
// columns belong to, one per row, formed once per tile instead of once per value
template <int L> constexpr size_t tile16_inv_bytes() { return size_t(tile_groups<L>()) * 8 * 2 * L * sizeof(float); }
template <int L, int NZ = 32> constexpr size_t tile16_smem()
{
    return kTileHeader + 1024 + size_t(tile16_slots<L, NZ>()) * tile16_slot<L, NZ>() + tile16_inv_bytes<L>();
}

template <int L, int DIR, typename T, int SX = 8>
__device__ __forceinline__ float march_tile16(T *p, const float *sp, const float *ip, int st_rt, const Lim<float> &lim,
                                              unsigned rng)
{
    const int st = DIR == 0 ? st_rt : DIR * 256;                // rows are 256 codes apart
    const int ss = DIR == 0 ? (st_rt > 0 ? SX : -SX) : DIR * SX; // and SX scales
    const int is = DIR == 0 ? (st_rt > 0 ? 1 : -1) : DIR;     // and 1 inverse scale
    auto get = [&](int i) { return RegCodec<T>::get(p[i * st], sp[i * ss]); };
    const float a = get(L - 3), b = get(L - 2), c = get(L - 1);
    const float s0 = get(0), s1 = get(1);
    const float dmm = curv(a, b, c), dm = curv(b, c, s0), d0 = curv(c, s0, s1);
    float dm4m = dm4(dm, d0);
    float Fm = sl_mpp5_flux(lim, a, b, c, s0, s1, dm4(dmm, dm), dm4m);
    float cm2 = b, cm1 = c, c0 = s0, cp1 = s1, dcur = d0, sum = 0.f;
    auto face = [&](float cp2, int i) {
        const float dn = curv(c0, cp1, cp2);
        const float dm4p = dm4(dcur, dn);
        const float F = sl_mpp5_flux(lim, cm2, cm1, c0, cp1, cp2, dm4m, dm4p);
        const float out = c0 + (Fm - F);
        p[i * st] = RegCodec<T>::put(out, ip[i * is], lcg_next(rng) >> 16);
        sum += out;
        cm2 = cm1;
        cm1 = c0;
        c0 = cp1;
        cp1 = cp2;
        dcur = dn;
        dm4m = dm4p;
        Fm = F;
    };
#pragma unroll march_unroll<L>()
    for (int i = 0; i < L - 2; ++i) face(get(i + 2), i);
    face(s0, L - 2);
    face(s1, L - 1);
    return sum;
}

// march_strided on codes: a value is decoded (the scale of its row) as it enters the
// window and a new value encoded (the inverse scale of its row, one stochastic-rounding
// draw per cell in walk order) at its own face.  st, ss, is: the strides between rows of
// codes, scales and inverse scales (negative for a line walked from its far end).
template <int L, typename T>
__device__ __forceinline__ float march_tile16_zf(T *p, int st, const float *sp, int ss, const float *ip, int is,
                                                 const Lim<float> &lim, unsigned rng)
{
    static_assert(L >= 4, "lines of at least 4 cells");
    auto get = [&](int i) { return RegCodec<T>::get(p[i * st], sp[i * ss]); };
    float cm2 = 0.f, cm1 = 0.f, c0 = get(0), cp1 = get(1), cp2 = get(2);
    float db = curv(0.f, c0, cp1); // curvature of cell 0
    float dm4m = dm4(c0, db);      // face -1/2: the ghost cell -1 has curvature 0 - 0 + c_0
    float Fprev = 0.f, sum = 0.f;
#pragma unroll 8
    for (int i = 0; i < L; ++i) {
        float F = 0.f, dm4p = 0.f, dc = 0.f;
        if (i + 1 < L) {
            dc = curv(c0, cp1, cp2); // curvature of cell i + 1
            dm4p = dm4(db, dc);
            F = sl_mpp5_flux(lim, cm2, cm1, c0, cp1, cp2, dm4m, dm4p);
        }
        const float out = vadd(c0, vsub(Fprev, F));
        p[i * st] = RegCodec<T>::put(out, ip[i * is], lcg_next(rng) >> 16);
        sum = vadd(sum, out);
        Fprev = F;
        dm4m = dm4p;
        db = dc;
        cm2 = cm1;
        cm1 = c0;
        c0 = cp1;
        cp1 = cp2;
        cp2 = i + 3 < L ? get(i + 3) : 0.f;
    }
    return sum;
}

template <int L, typename T, bool SIGNED, int NZ = 32, bool ZF = false>
__global__ void __launch_bounds__(tile_groups<L>() * 256 + kProducer, 1)
    tile_sweep16_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap smap,
                        const __grid_constant__ TileArgs a)
{
    constexpr int NG = tile_groups<L>(), S = tile16_slots<L, NZ>(), NT = NG * 256, SX = tile16_scale_lines<NZ>();
    constexpr unsigned CB = tile16_codes<L>(), SB = tile16_slot<L, NZ>();
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *done = full + S;
    LineCoefT<float> *tab = reinterpret_cast<LineCoefT<float> *>(smem + 256);
    static_assert(2 * S * 8 <= 256, "barriers fit ahead of the table");
    unsigned char *ring = smem + kTileHeader + ((1024u - ((smem_u32(smem) + unsigned(kTileHeader)) & 1023u)) & 1023u);
    auto slot = [&](unsigned k) { return reinterpret_cast<T *>(ring + size_t(SB) * (k % S)); };
    auto sslot = [&](unsigned k) { return reinterpret_cast<float *>(ring + size_t(SB) * (k % S) + CB); };
    float *winv = reinterpret_cast<float *>(ring + size_t(SB) * S);
    static_assert(tile16_smem<L, NZ>() <= 227 * 1024, "the tiles and inverse scales fit shared memory");

    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&done[q], 256);
        }
        fence_barrier_init();
    }
    for (int j = threadIdx.x; j < a.nvel; j += blockDim.x) tab[j] = a.table[j];
    __syncthreads();

    const long long G = gridDim.x, b = blockIdx.x;
    const unsigned n_my = unsigned(a.num_tiles > b ? (a.num_tiles - b + G - 1) / G : 0);
    auto coords = [&](unsigned k, int &u0, int &o) {
        const long long t = a.tile0 + b + (long long)k * G;
        const long long oq = t / a.tiles_inner;
        u0 = int((t - oq * a.tiles_inner) * 8);
        o = int(oq);
    };
    // first u_z line of the tile's scale box (n_uz = 32: its first line exactly)
    auto line0 = [&](int u0) { return NZ == 32 ? u0 : int(32ll * u0 / NZ / 4 * 4); };

    if (threadIdx.x >= NT) {
        if (threadIdx.x != NT) return;
        auto load = [&](unsigned k) {
            int u0, o;
            coords(k, u0, o);
            mbar_arrive_expect_tx(&full[k % S], CB + unsigned(L) * 4u * unsigned(SX));
            tma_load_4d(slot(k), &map, &full[k % S], 0, u0, 0, o);
            tma_load_3d(sslot(k), &smap, &full[k % S], line0(u0), 0, o);
        };
        unsigned loaded = 0;
        for (; loaded < unsigned(S) && loaded < n_my; ++loaded) load(loaded);
        bool ok = true;
        for (unsigned k = 0; k < n_my; ++k) {
            if (!mbar_wait_bounded(&done[k % S], (k / S) & 1u)) {
                ok = false;
                break;
            }
            int u0, o;
            coords(k, u0, o);
            tma_store_4d(&map, slot(k), 0, u0, 0, o); // the scales stay as they are
            bulk_commit();
            if (loaded < n_my) {
                bulk_wait_read_all();
                load(loaded++);
            }
        }
        bulk_wait_all();
        if (!ok) {
            atomicOr(a.err, ERR_TIMEOUT);
            for (unsigned k = 0; k < loaded; ++k) mbar_wait_bounded(&full[k % S], (k / S) & 1u);
        }
        return;
    }

    const int grp = threadIdx.x >> 8, tid = threadIdx.x & 255, w = tid >> 5, lane = tid & 31;
    int unit, e;
    if (a.zperm) {
        unit = ((w & 3) << 1) + (lane >> 4);
        e = (w >> 2) * 16 + (lane & 15);
    } else {
        unit = w;
        e = lane;
    }
    // this warp's inverse scales: [h][row] for the (up to two) u_z lines of its columns
    float *wi = winv + (grp * 8 + w) * 2 * L;
    bool bad = false;
    for (unsigned k = grp; k < n_my; k += NG) {
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[k % S], (k / S) & 1u))) {
            atomicOr(a.err, ERR_TIMEOUT);
            return;
        }
        int u0, o;
        coords(k, u0, o);
        const long long inner = 32ll * (u0 + unit) + e;
        const LineCoefT<float> kc = ZF ? a.cell_coef[o] : tab[(inner / a.vstride) % a.nvel];
        T *p = slot(k) + unit * 32 + e;
        // the scale box column of this thread's u_z line, the warp's first such column and
        // how many the warp spans (n_uz = 32: units are lines, two under zperm)
        int col, first, nlines;
        if constexpr (NZ == 32) {
            col = unit;
            first = a.zperm ? ((w & 3) << 1) : w;
            nlines = a.zperm ? 2 : 1;
        } else {
            // (no zperm: the warp's 32 columns are contiguous, on one or two lines)
            const long long x0 = line0(u0), c0 = 32ll * (u0 + w);
            col = int(inner / NZ - x0);
            first = int(c0 / NZ - x0);
            nlines = int((c0 + 31) / NZ - c0 / NZ) + 1;
        }
        const float *sp = sslot(k) + col;
        const float *ip_col = wi + (col - first) * L;
        __syncwarp(); // every lane is done with the previous tile's inverses
        for (int idx = lane; idx < nlines * L; idx += 32) {
            const int h = idx / L, r = idx - h * L;
            wi[idx] = inv_scale(sslot(k)[r * SX + first + h]);
        }
        __syncwarp();
        if (kc.nd >= 0) {
            const Lim<float> lim = to_lim(kc);
            const bool neg = kc.nd & 1;
            // the column's stream, from the index of its first cell
            const unsigned rng = sr_bits((unsigned long long)((long long)o * L * a.n_inner + inner), a.seed);
            float sum;
            if constexpr (ZF)
                sum = march_tile16_zf<L, T>(neg ? p + (L - 1) * 256 : p, neg ? -256 : 256, neg ? sp + (L - 1) * SX : sp,
                                            neg ? -SX : SX, neg ? ip_col + (L - 1) : ip_col, neg ? -1 : 1, lim, rng);
            else if constexpr (!SIGNED)
                sum = march_tile16<L, 0, T, SX>(neg ? p + (L - 1) * 256 : p, neg ? sp + (L - 1) * SX : sp,
                                                neg ? ip_col + (L - 1) : ip_col, neg ? -256 : 256, lim, rng);
            else if (neg)
                sum = march_tile16<L, -1, T, SX>(p + (L - 1) * 256, sp + (L - 1) * SX, ip_col + (L - 1), 0, lim, rng);
            else sum = march_tile16<L, 1, T, SX>(p, sp, ip_col, 0, lim, rng);
            bad |= !(sum >= 0.f) || isinf(sum);
        }
        fence_proxy_async();
        mbar_arrive(&done[k % S]);
    }
    if (bad) atomicOr(a.err, ERR_NAN);
}

template <int L, typename T, int NZ = 32> const void *tile16_kernel(bool sign)
{
    return sign ? (const void *)tile_sweep16_kernel<L, T, true, NZ> : (const void *)tile_sweep16_kernel<L, T, false, NZ>;
}

template <typename T> const void *tile16_kernel_for(int L, bool sign, int nuz)
{
    if (nuz == 48) return L == 48 ? tile16_kernel<48, T, 48>(sign) : nullptr;
    if (nuz != 32) return nullptr;
    switch (L) {
    case 16: return tile16_kernel<16, T>(sign);
    case 24: return tile16_kernel<24, T>(sign);
    case 32: return tile16_kernel<32, T>(sign);
    case 48: return tile16_kernel<48, T>(sign);
    case 64: return tile16_kernel<64, T>(sign);
    case 96: return tile16_kernel<96, T>(sign);
    default: return nullptr;
    }
}

size_t tile16_smem_for(int L, int nuz)
{
    if (nuz == 48) return tile16_smem<48, 48>();
    switch (L) {
    case 16: return tile16_smem<16>();
    case 24: return tile16_smem<24>();
    case 32: return tile16_smem<32>();
    case 48: return tile16_smem<48>();
    case 64: return tile16_smem<64>();
    default: return tile16_smem<96>();
    }
}

template <int L> const void *tile_kernel(bool moment, bool sign)
{
    if (sign) return moment ? (const void *)tile_sweep_kernel<L, true, true> : (const void *)tile_sweep_kernel<L, false, true>;
    return moment ? (const void *)tile_sweep_kernel<L, true, false> : (const void *)tile_sweep_kernel<L, false, false>;
}

const void *tile_kernel_for(int L, bool moment, bool sign = true)
{
    switch (L) {
    case 16: return tile_kernel<16>(moment, sign);
    case 24: return tile_kernel<24>(moment, sign);
    case 32: return tile_kernel<32>(moment, sign);
    case 48: return tile_kernel<48>(moment, sign);
    case 64: return tile_kernel<64>(moment, sign);
    default: return nullptr;
    }
}

size_t tile_smem_for(int L)
{
    switch (L) {
    case 16: return tile_smem<16>();
    case 24: return tile_smem<24>();
    case 32: return tile_smem<32>();
    case 48: return tile_smem<48>();
    default: return tile_smem<64>();
    }
}

int tile_threads_for(int L, bool) { return (L <= 48 ? 3 : 2) * 256 + kProducer; }

// u_x sweeps (zero-flux lines, one direction per tile): lines of 48 cells
const void *tile_kernel_zf(int L, int dtype, int nuz)
{
    if (L != 48) return nullptr;
    if (dtype == 1) return (const void *)tile_sweep_kernel<48, false, true, true>;
    if (nuz != 48) return nullptr;
    if (dtype == 2) return (const void *)tile_sweep16_kernel<48, __nv_bfloat16, true, 48, true>;
    if (dtype == 3) return (const void *)tile_sweep16_kernel<48, __half, true, 48, true>;
    return nullptr;
}

const void *tile_kernel_any(int L, int dtype, bool moment, bool sign, int nuz)
{
    if (dtype == 2) return moment ? nullptr : tile16_kernel_for<__nv_bfloat16>(L, sign, nuz);
    if (dtype == 3) return moment ? nullptr : tile16_kernel_for<__half>(L, sign, nuz);
    return tile_kernel_for(L, moment, sign);
}

} // namespace

bool tile_sweep_supported(int L, long long n_inner, int dtype, int nuz)
{
    if (n_inner % 256 != 0 || !tile_kernel_any(L, dtype, false, true, nuz)) return false;
    return dtype == 1 || ((dtype == 2 || dtype == 3) && n_inner % nuz == 0);
}

bool tile_sweep_zf_supported(int L, long long n_inner, int dtype, int nuz)
{
    return n_inner % 256 == 0 && n_inner % nuz == 0 && tile_kernel_zf(L, dtype, nuz) != nullptr;
}

int occupancy_tile_sweep(int L, int dtype, bool moment, int nuz)
{
    const void *k = tile_kernel_any(L, dtype, moment, true, nuz);
    if (!k) return 0;
    const size_t smem = dtype == 1 ? tile_smem_for(L) : tile16_smem_for(L, nuz);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, tile_threads_for(L, moment), smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_tile_sweep(const CUtensorMap &map, const CUtensorMap &dmap, const CUtensorMap &smap,
                              const TileArgs &a, int dtype, int grid, cudaStream_t st)
{
    if (a.num_tiles <= 0 || grid <= 0) return cudaSuccess;
    const bool moment = a.mpart != nullptr, zf = a.cell_coef != nullptr;
    const void *k = zf ? tile_kernel_zf(a.L, dtype, a.nuz) : tile_kernel_any(a.L, dtype, moment, a.tile_sign != 0, a.nuz);
    if (!k || (!zf && (a.nvel <= 0 || a.vstride <= 0)) || a.nvel > kMaxVel || a.tiles_inner <= 0 || (zf && moment))
        return cudaErrorInvalidValue;
    if (moment && (dtype != 1 || a.cube % 256 || a.nparts <= 0)) return cudaErrorInvalidValue;
    if (dtype != 1 && (a.zperm && a.nuz != 32)) return cudaErrorInvalidValue;
    const size_t smem = dtype == 1 ? tile_smem_for(a.L) : tile16_smem_for(a.L, a.nuz);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    // FP32: (map, dmap, args); 16-bit: in place (map, smap, args)
    void *params[] = {const_cast<CUtensorMap *>(&map),
                      const_cast<CUtensorMap *>(dtype == 1 ? &dmap : &smap), const_cast<TileArgs *>(&a)};
    return cudaLaunchKernel(k, dim3(grid), dim3(tile_threads_for(a.L, moment)), params, smem, st);
}

} // namespace vk
