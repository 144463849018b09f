// sweep_stream.cu -- SL-MPP5 sweeps along a strided axis (x, y, z; u_x, u_y when
// their lines are not marched in registers), lines streamed through shared
// memory in chunks of rows; the x sweep can also sum the velocity moment.
//
// Eq. (3) (position advection, periodic) and Eq. (4) (velocity advection,
// zero-flux faces) of Yoshikawa, Tanaka & Yoshida, SC'21, for Courant numbers
// with no whole-cell part (|nu| < 1 on every line; sweep_strided.cu handles
// whole-cell shifts).
//
// f is the 3D tensor [O][L][I] (slower axes, swept axis, faster axes).  A CTA
// owns a block of columns -- {W inner} x {P outer} -- and walks it down the
// swept axis in chunks of R rows: TMA box {W, R, P}.  Each consumer thread owns
// two adjacent columns (one packed FP32 pair, or one column in FP64) and keeps
// its sliding window in registers, so a column needs only R rows of shared
// memory in flight instead of its whole line: more CTAs fit per SM.
//
// Ring of S chunk slots.  For a periodic line the first entry of a block is a
// "prologue" box starting at row L-3 (its first three rows are the upwind
// neighbours of row 0; the rest lies outside the tensor and reads as zero).
// Producer (warp 0, lane 0): loads entries in order into the ring and, before
// reusing a slot, waits until the consumers release it and TMA-stores it back
// in place when it holds a chunk.  Consumers: the output of row i is final
// after row i + 2 has been read, so a chunk is released (done barrier) when its
// last row has been written.  Every wait is bounded.
#include "vk_common.cuh"

namespace vk {

constexpr int kStreamMinBlocks = 4; // resident CTAs per SM the streamed sweep is compiled for

// Per-thread view of the storage of its column(s): load a row as the compute
// vector X and store X back.  FP32 / FP64 store f itself.  BF16 / FP16 store
// f / scale with one FP32 scale per u_z line; the scale of the row comes from
// shared memory (staged by TMA with the chunk), `sp` points at it.
// NC: consumer threads per CTA; a CTA's block is V * NC columns wide.
template <typename T> struct Lane;
template <> struct Lane<float> {
    using X = float2; // two columns per thread
    static constexpr int V = 2, NC = kStreamConsumers;
    __device__ static X load(const float *p, const float *) { return *reinterpret_cast<const float2 *>(p); }
    __device__ static void store(float *p, X v, const float *, unsigned &) { *reinterpret_cast<float2 *>(p) = v; }
    __device__ static bool bad(X s) { return !(s.x >= 0.f) || !(s.y >= 0.f) || isinf(s.x) || isinf(s.y); }
};
template <> struct Lane<double> {
    using X = double;
    static constexpr int V = 1, NC = kStreamConsumers;
    __device__ static X load(const double *p, const float *) { return *p; }
    __device__ static void store(double *p, X v, const float *, unsigned &) { *p = v; }
    __device__ static bool bad(X s) { return !(s >= 0.0) || isinf(s); }
};
template <> struct Lane<__nv_bfloat16> {
    using X = float2;
    static constexpr int V = 2, NC = kStreamConsumers;
    __device__ static X load(const __nv_bfloat16 *p, const float *sp)
    {
        const unsigned u = *reinterpret_cast<const unsigned *>(p);
        const float s = *sp;
        // a bf16 is the upper half of an FP32
        return vmul(make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u)), make_float2(s, s));
    }
    // rows are stored in order, so the rounding stream advances once per row
    __device__ static void store(__nv_bfloat16 *p, X v, const float *sp, unsigned &rng)
    {
        const float inv = inv_scale(*sp);
        *reinterpret_cast<unsigned *>(p) = sr_pack_bf16x2(v.x * inv, v.y * inv, rng);
    }
    __device__ static bool bad(X s) { return Lane<float>::bad(s); }
};
template <> struct Lane<__half> {
    using X = float2;
    static constexpr int V = 2, NC = kStreamConsumers;
    __device__ static X load(const __half *p, const float *sp)
    {
        const float2 h = __half22float2(*reinterpret_cast<const __half2 *>(p));
        const float s = *sp;
        return vmul(h, make_float2(s, s));
    }
    __device__ static void store(__half *p, X v, const float *sp, unsigned &rng)
    {
        const float inv = inv_scale(*sp);
        *reinterpret_cast<unsigned *>(p) = sr_pack_f16x2(v.x * inv, v.y * inv, rng);
    }
    __device__ static bool bad(X s) { return Lane<float>::bad(s); }
};

template <typename C, typename X> struct PairLim;
template <> struct PairLim<float, float> {
    __device__ static Lim<float> make(const LineCoefT<float> &a, const LineCoefT<float> &) { return to_lim(a); }
};
template <> struct PairLim<float, float2> {
    __device__ static Lim<float2> make(const LineCoefT<float> &a, const LineCoefT<float> &b) { return to_lim2(a, b); }
};
template <> struct PairLim<double, double> {
    __device__ static Lim<double> make(const LineCoefT<double> &a, const LineCoefT<double> &) { return to_lim(a); }
};

// March one block's column(s) down the line in physical row order, reading the
// rows from the ring (chunk c of the line is ring entry ec + c; a periodic
// line's prologue entry e holds rows L-3..L-1 first).  NEG selects the
// orientation: the flux through face i+1/2 has donor i (nu > 0) or donor i+1
// with the mirrored stencil (nu < 0); either way rows are consumed in order and
// a chunk is released once its last row has been written.  Returns the sum of
// the new values.
template <typename T> __host__ __device__ constexpr int stream_rows() { return sizeof(T) == 2 ? 2 * kStreamRows : kStreamRows; }

template <typename T, bool PERIODIC, bool NEG, typename X, typename SlotPtr, typename ScalePtr, typename Acq,
          typename Rel>
__device__ __forceinline__ X march_stream(const Lim<X> &lim, unsigned e, unsigned ec, int coff, int soff, int L, int W,
                                          int Wl, unsigned &rng, SlotPtr slot_ptr, ScalePtr scale_ptr, Acq acquire,
                                          Rel release, bool &alive)
{
    using LN = Lane<T>;
    constexpr int R = stream_rows<T>();
    const X zero = splat<X>(0.0);
    auto row_ptr = [&](int r) { return slot_ptr(ec + unsigned(r / R)) + coff + (r % R) * W; };
    auto srow_ptr = [&](int r) { return scale_ptr(ec + unsigned(r / R)) + soff + (r % R) * Wl; };
    X p3 = zero, p2 = zero, p1 = zero; // c_{-3}, c_{-2}, c_{-1}
    if (PERIODIC) {
        if (!acquire(e)) return zero;
        const T *q = slot_ptr(e) + coff;
        const float *qs = scale_ptr(e) + soff;
        p3 = LN::load(q, qs);
        p2 = LN::load(q + W, qs + Wl);
        p1 = LN::load(q + 2 * W, qs + 2 * Wl);
        release(e);
    }
    if (!acquire(ec)) return zero; // rows 0..3 lie in chunk 0 (R >= 4)
    const X s0 = LN::load(row_ptr(0), srow_ptr(0));
    const X s1 = LN::load(row_ptr(1), srow_ptr(1));
    X sum = zero;
    // Rows i whose look-ahead rows i + LA all lie inside the line and whose chunk
    // is complete are marched chunk by chunk with compile-time offsets (chunk c is
    // "simple" when c R + R - 1 + LA < L); the rest row by row.
    if (!NEG) {
        constexpr int LA = 2;
        // window c_{i-2} .. c_{i+2}, donor c_i
        X cm2, cm1, c0 = s0, cp1 = s1, dcur, dm4m, Fm;
        const X dm = curv(p2, p1, s0);
        const X d0 = curv(p1, s0, s1);
        dm4m = dm4(dm, d0);
        if (PERIODIC) Fm = sl_mpp5_flux(lim, p3, p2, p1, s0, s1, dm4(curv(p3, p2, p1), dm), dm4m);
        else Fm = zero;
        cm2 = p2;
        cm1 = p1;
        dcur = d0;
        auto face = [&](X cp2, T *dst, const float *dsc) {
            const X dn = curv(c0, cp1, cp2);
            const X dm4p = dm4(dcur, dn);
            const X F = sl_mpp5_flux(lim, cm2, cm1, c0, cp1, cp2, dm4m, dm4p);
            const X out = vadd(c0, vsub(Fm, F));
            LN::store(dst, out, dsc, rng);
            sum = vadd(sum, out);
            cm2 = cm1;
            cm1 = c0;
            c0 = cp1;
            cp1 = cp2;
            dcur = dn;
            dm4m = dm4p;
            Fm = F;
        };
        const int nsimple = (L - LA + 1) / R - 1 > 0 ? (L - LA + 1) / R - 1 : 0;
        for (int c = 0; c < nsimple; ++c) {
            T *cur = slot_ptr(ec + unsigned(c)) + coff;
            T *nxt = slot_ptr(ec + unsigned(c + 1)) + coff;
            const float *scur = scale_ptr(ec + unsigned(c)) + soff;
            const float *snxt = scale_ptr(ec + unsigned(c + 1)) + soff;
            if (!acquire(ec + unsigned(c + 1))) return zero;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const X cp2 = (q + LA < R) ? LN::load(cur + (q + LA) * W, scur + (q + LA) * Wl)
                                          : LN::load(nxt + (q + LA - R) * W, snxt + (q + LA - R) * Wl);
                face(cp2, cur + q * W, scur + q * Wl);
            }
            release(ec + unsigned(c));
        }
        for (int i = nsimple * R; i < L; ++i) {
            const int r = i + LA;
            X cp2;
            if (r < L) {
                if (r % R == 0 && !acquire(ec + unsigned(r / R))) return zero;
                cp2 = LN::load(row_ptr(r), srow_ptr(r));
            } else {
                cp2 = PERIODIC ? (r == L ? s0 : s1) : zero;
            }
            if (!PERIODIC && i == L - 1) {
                // outer velocity face: nothing crosses it
                const X out = vadd(c0, Fm);
                LN::store(row_ptr(i), out, srow_ptr(i), rng);
                sum = vadd(sum, out);
            } else {
                face(cp2, row_ptr(i), srow_ptr(i));
            }
            if (i % R == R - 1 || i == L - 1) release(ec + unsigned(i / R));
        }
    } else {
        constexpr int LA = 3;
        // window c_{i-1} .. c_{i+3}, donor c_{i+1}, flux toward -index
        // curvatures are summed in the marching order (toward -index), as every kernel
        // that walks a line with a negative Courant number from its far end sums them
        const X s2 = LN::load(row_ptr(2), srow_ptr(2));
        const X dmn = curv(s0, p1, p2); // d_{-1}
        const X d0 = curv(s1, s0, p1);
        const X d1 = curv(s2, s1, s0);
        X dm4a = dm4(d0, d1);           // limited curvature at face i+1/2
        X Fm;                            // mass moving left through face i-1/2
        if (PERIODIC) Fm = sl_mpp5_flux(lim, s2, s1, s0, p1, p2, dm4a, dm4(dmn, d0));
        else Fm = zero;
        X cm1 = p1, c0 = s0, cp1 = s1, cp2 = s2, d_1 = d1;
        auto face = [&](X cp3, T *dst, const float *dsc) {
            const X d_2 = curv(cp3, cp2, cp1);
            const X dm4b = dm4(d_1, d_2); // face i+3/2
            const X F = sl_mpp5_flux(lim, cp3, cp2, cp1, c0, cm1, dm4b, dm4a);
            const X out = vadd(c0, vsub(F, Fm));
            LN::store(dst, out, dsc, rng);
            sum = vadd(sum, out);
            cm1 = c0;
            c0 = cp1;
            cp1 = cp2;
            cp2 = cp3;
            d_1 = d_2;
            dm4a = dm4b;
            Fm = F;
        };
        const int nsimple = (L - LA + 1) / R - 1 > 0 ? (L - LA + 1) / R - 1 : 0;
        for (int c = 0; c < nsimple; ++c) {
            T *cur = slot_ptr(ec + unsigned(c)) + coff;
            T *nxt = slot_ptr(ec + unsigned(c + 1)) + coff;
            const float *scur = scale_ptr(ec + unsigned(c)) + soff;
            const float *snxt = scale_ptr(ec + unsigned(c + 1)) + soff;
            if (!acquire(ec + unsigned(c + 1))) return zero;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const X cp3 = (q + LA < R) ? LN::load(cur + (q + LA) * W, scur + (q + LA) * Wl)
                                          : LN::load(nxt + (q + LA - R) * W, snxt + (q + LA - R) * Wl);
                face(cp3, cur + q * W, scur + q * Wl);
            }
            release(ec + unsigned(c));
        }
        for (int i = nsimple * R; i < L; ++i) {
            const int r = i + LA;
            X cp3;
            if (r < L) {
                if (r % R == 0 && !acquire(ec + unsigned(r / R))) return zero;
                cp3 = LN::load(row_ptr(r), srow_ptr(r));
            } else {
                cp3 = PERIODIC ? (r == L ? s0 : (r == L + 1 ? s1 : s2)) : zero;
            }
            if (!PERIODIC && i == L - 1) {
                const X out = vsub(c0, Fm); // nothing enters through the outer face
                LN::store(row_ptr(i), out, srow_ptr(i), rng);
                sum = vadd(sum, out);
            } else {
                face(cp3, row_ptr(i), srow_ptr(i));
            }
            if (i % R == R - 1 || i == L - 1) release(ec + unsigned(i / R));
        }
    }
    return sum;
}

// ----------------------------------------------------------------------------
// velocity moment fused into the x sweep
// ----------------------------------------------------------------------------
// A moment warp sums every released chunk's rows (4 rows x W values, all in one
// spatial cell's velocity cube) while the producer stores the chunk: a lane adds
// its two 16-byte chunks of a row pairwise, then the warp adds the lanes pairwise in a fixed
// order (FP32 storage: FP32, at most 8 roundings deep; FP64: FP64).  The first two
// levels halve the rows each lane holds, the last three add within groups of 8
// lanes, so lane l ends with the total of row l >> 3.  The producer reloads a slot
// only after the moment warp has summed it.
__device__ __forceinline__ float lane_row_sum(const float *row, int lane)
{
    // 16-byte chunks lane and lane + 32: each quarter warp reads 128 contiguous bytes
    const float4 *q = reinterpret_cast<const float4 *>(row);
    const float4 a = q[lane], b = q[lane + 32];
    return ((a.x + a.y) + (a.z + a.w)) + ((b.x + b.y) + (b.z + b.w));
}
__device__ __forceinline__ double lane_row_sum(const double *row, int lane)
{
    const double2 *q = reinterpret_cast<const double2 *>(row);
    const double2 a = q[lane], b = q[lane + 32];
    return (a.x + a.y) + (b.x + b.y);
}
template <typename T> __device__ __forceinline__ float lane_row_sum(const T *, int) { return 0.f; }

template <typename A> __device__ __forceinline__ A rows4_warp_sum(A v0, A v1, A v2, A v3, int lane)
{
    constexpr unsigned kAll = 0xffffffffu;
    const bool hi = lane & 16, odd = lane & 8;
    A k0 = hi ? v2 : v0, k1 = hi ? v3 : v1;
    k0 += __shfl_xor_sync(kAll, hi ? v0 : v2, 16);
    k1 += __shfl_xor_sync(kAll, hi ? v1 : v3, 16);
    A k = odd ? k1 : k0;
    k += __shfl_xor_sync(kAll, odd ? k0 : k1, 8);
    k += __shfl_xor_sync(kAll, k, 4);
    k += __shfl_xor_sync(kAll, k, 2);
    k += __shfl_xor_sync(kAll, k, 1);
    return k;
}

// threads ahead of the consumers: the producer warp, and the moment warp if any
template <bool MOMENT> __host__ __device__ constexpr int stream_head() { return kProducer + (MOMENT ? 32 : 0); }

template <typename T, bool PERIODIC, bool MOMENT = false>
__global__ void __launch_bounds__(Lane<T>::NC + stream_head<MOMENT>(), kStreamMinBlocks)
    stream_sweep_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap dmap,
                        const __grid_constant__ CUtensorMap smap,
                        const __grid_constant__ StreamArgs<typename Compute<T>::type> args)
{
    constexpr bool CODED = sizeof(T) == 2;
    using C = typename Compute<T>::type;
    using LN = Lane<T>;
    using X = typename LN::X;
    constexpr int V = LN::V;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int S = kStreamRing;
    constexpr int R = stream_rows<T>();
    const int L = args.L, W = args.W, P = args.P;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *done = full + S;
    int4 *meta = reinterpret_cast<int4 *>(done + S); // per slot: store coordinates, is-chunk flag
    uint64_t *summed = reinterpret_cast<uint64_t *>(meta + S); // the moment warp has read the slot
    constexpr int kHead = stream_head<MOMENT>();
    static_assert(3 * S * sizeof(uint64_t) + S * sizeof(int4) <= 512, "ring barriers and meta fit ahead of the table");
    LineCoefT<C> *tab = reinterpret_cast<LineCoefT<C> *>(smem + 512);
    const size_t tab_bytes = (args.coef_mode == 0) ? ((sizeof(LineCoefT<C>) * args.nvel + 127) & ~size_t(127)) : 0;
    unsigned char *ring = smem + 512 + tab_bytes;
    const int slot_elems = W * R * P;
    const unsigned code_bytes = unsigned(slot_elems * sizeof(T));
    const unsigned slot_pitch = (code_bytes + 127u) & ~127u;
    auto slot_ptr = [&](unsigned e) { return reinterpret_cast<T *>(ring + slot_pitch * (e & (S - 1))); };
    // 16-bit storage: the scales of the chunk's u_z lines, box {Wl, R, P} starting at line
    // (c0 / n_uz) & ~3 (16-byte aligned), wide enough for every line the block touches
    const int nuz = CODED ? int(args.nuz) : 1;
    const int Wl = CODED ? args.swidth : 0;
    const unsigned scale_bytes = CODED ? unsigned(Wl * R * P * 4) : 0u;
    const unsigned scale_pitch = (scale_bytes + 127u) & ~127u;
    unsigned char *sring = ring + size_t(slot_pitch) * S;
    auto scale_ptr = [&](unsigned e) { return reinterpret_cast<float *>(sring + scale_pitch * (e & (S - 1))); };
    const unsigned slot_bytes = code_bytes + scale_bytes; // transaction bytes of one entry
    const int nC = (L + R - 1) / R;                // chunks per line
    const int E = nC + (PERIODIC ? 1 : 0);         // ring entries per block

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&done[s], Lane<T>::NC);
            if (MOMENT) mbar_init(&summed[s], 1);
        }
        fence_barrier_init();
    }
    if (args.coef_mode == 0)
        for (int j = threadIdx.x; j < args.nvel; j += blockDim.x) tab[j] = args.table[j];
    __syncthreads();

    const long long G = gridDim.x, b = blockIdx.x;
    const long long n_my = (args.num_blocks > b) ? (args.num_blocks - b + G - 1) / G : 0;

    if (threadIdx.x < kProducer) {
        if (threadIdx.x != 0) return;
        // Entries are loaded in order into slot e % S and retired in order: once the
        // consumers release an entry its chunk is stored back (one bulk group per
        // entry, empty for a prologue), without waiting.  A slot is reloaded only
        // after the store of its previous entry has read the slot out.
        const unsigned total = unsigned(n_my) * unsigned(E);
        unsigned loaded = 0, retired = 0;
        long long k = 0;
        int j = 0, c0 = 0, c2 = 0;
        bool ok = true;
        while (retired < total) {
            bool progress = false;
            while (retired < loaded && mbar_test_wait(&done[retired & (S - 1)], (retired / S) & 1u)) {
                const int4 m = meta[retired & (S - 1)];
                if (m.w) tma_store_3d(&dmap, slot_ptr(retired), m.x, m.y, m.z);
                bulk_commit();
                ++retired;
                progress = true;
            }
            if (loaded < total && loaded < retired + S) {
                // the store of entry loaded - S is group loaded - S of `retired` groups
                if (loaded >= unsigned(S)) bulk_wait_read_at_most(retired - 1u - (loaded - S));
                if (MOMENT && loaded >= unsigned(S) &&
                    !mbar_wait_bounded(&summed[loaded & (S - 1)], ((loaded - S) / S) & 1u)) {
                    ok = false;
                    break;
                }
                if (j == 0) {
                    const long long t = args.tile0 + b + k * G;
                    c0 = int((t % args.tiles_inner) * W);
                    c2 = int((t / args.tiles_inner) * P);
                }
                const int ch = PERIODIC ? j - 1 : j;
                const int c1 = ch >= 0 ? ch * R : L - 3;
                const unsigned st = loaded & (S - 1);
                meta[st] = make_int4(c0, c1, c2, ch >= 0);
                mbar_arrive_expect_tx(&full[st], slot_bytes);
                tma_load_3d(slot_ptr(loaded), &map, &full[st], c0, c1, c2);
                if (CODED) {
                    if (args.scale_rank == 3)
                        tma_load_3d(scale_ptr(loaded), &smap, &full[st], (c0 / nuz) & ~3, c1, c2);
                    else
                        tma_load_2d(scale_ptr(loaded), &smap, &full[st], c1, c2);
                }
                ++loaded;
                if (++j == E) { j = 0; ++k; }
                progress = true;
            }
            if (!progress && !mbar_wait_bounded(&done[retired & (S - 1)], (retired / S) & 1u)) {
                ok = false;
                break;
            }
        }
        bulk_wait_all();
        if (!ok) {
            atomicOr(args.err, ERR_TIMEOUT);
            for (unsigned t = retired; t < loaded; ++t) mbar_wait_bounded(&full[t & (S - 1)], (t / S) & 1u);
        }
        return;
    }

    if (MOMENT && threadIdx.x < kHead) {
        // ------------------------------------------------------------ moment warp
        // entries in order: wait for the consumers' release, sum the chunk's rows
        // (row x of the block at inner offset c0 adds to spatial cell
        // x (n_inner / cube) + c0 / cube as its partial (c0 % cube) / W, stored at
        // mpart[((c0 / cube) nparts + part) L + x]), then free the slot for reloading
        using A = decltype(lane_row_sum((const T *)nullptr, 0));
        const int lane = threadIdx.x & 31;
        const int cube = int(args.cube);
        const unsigned total = unsigned(n_my) * unsigned(E);
        A *base = nullptr;
        int base_c0 = -1;
        for (unsigned en = 0; en < total; ++en) {
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&done[en & (S - 1)], (en / S) & 1u));
            if (!ok) {
                if (lane == 0) atomicOr(args.err, ERR_TIMEOUT);
                return;
            }
            const int4 m = meta[en & (S - 1)];
            if (m.w) {
                if (m.x != base_c0) {
                    base_c0 = m.x;
                    base = static_cast<A *>(args.mpart) +
                           ((long long)(m.x / cube) * args.nparts + (m.x % cube) / W) * (long long)L;
                }
                const T *q = slot_ptr(en);
                const A z = A(0);
                const A tot = rows4_warp_sum(lane_row_sum(q, lane), m.y + 1 < L ? lane_row_sum(q + W, lane) : z,
                                             m.y + 2 < L ? lane_row_sum(q + 2 * W, lane) : z,
                                             m.y + 3 < L ? lane_row_sum(q + 3 * W, lane) : z, lane);
                const int r = lane >> 3;
                if ((lane & 7) == 0 && m.y + r < L) base[m.y + r] = tot;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&summed[en & (S - 1)]);
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int tid = threadIdx.x - kHead;
    int col;  // first of this thread's V columns inside the block
    if (args.perm_line > 0) {
        // z sweep: the Courant number changes sign in the middle of each velocity
        // line; threads [0, H) take the columns with u_z < 0 and [Hp, Hp + H) those
        // with u_z > 0, so that whole warps march with one orientation (Hp: H rounded
        // up to whole warps when both halves still fit, e.g. 60 -> 64 for 5 lines of 48)
        const int Lz = args.perm_line, q = Lz / (2 * V);   // pairs per half line
        const int lines = W / Lz, H = lines * q;
        const int Hw = (H + 31) & ~31, Hp = 2 * Hw <= LN::NC ? Hw : H;
        const int tt = tid < Hp ? tid : tid - Hp;
        col = (tt / q) * Lz + (tid < Hp ? 0 : Lz / 2) + V * (tt % q);
        if (tt >= H || tid >= Hp + H) col = W * P;          // idle thread
    } else {
        col = tid * V;
    }
    const int w = col % W, p = col / W;
    const bool has_col = col < W * P;
    const int coff = p * R * W + w;          // column offset inside a slot; rows are W apart
    bool alive = true;
    unsigned e = 0;                          // next ring entry
    auto acquire = [&](unsigned ee) {
        if (!mbar_wait_bounded(&full[ee & (S - 1)], (ee / S) & 1u)) {
            atomicOr(args.err, ERR_TIMEOUT);
            alive = false;
        }
        return alive;
    };
    auto release = [&](unsigned ee) {
        fence_proxy_async();
        mbar_arrive(&done[ee & (S - 1)]);
    };

    for (long long k = 0; k < n_my && alive; ++k) {
        const long long t = args.tile0 + b + k * G;
        long long tq;  // tile row (outer block) of tile t
        if (args.fast32) tq = fdiv(unsigned(t), args.div_tiles);
        else tq = t / args.tiles_inner;
        const long long tr = t - tq * args.tiles_inner;
        const long long inner = tr * W + w;
        const long long outer = tq * P + p;
        bool work = has_col && inner < args.n_inner && outer < args.n_outer;
        Lim<X> lim{};
        bool neg = false;
        if (work) {
            LineCoefT<C> ka, kb;
            if (args.coef_mode == 0) {
                // velocity column of each of the thread's columns: (inner / vstride) % nvel
                if (args.fast32) {
                    const unsigned qa = fdiv(unsigned(inner), args.div_vstride);
                    const unsigned qb = fdiv(unsigned(inner + V - 1), args.div_vstride);
                    ka = tab[qa - fdiv(qa, args.div_nvel) * unsigned(args.nvel)];
                    kb = tab[qb - fdiv(qb, args.div_nvel) * unsigned(args.nvel)];
                } else {
                    ka = tab[(inner / args.vstride) % args.nvel];
                    kb = tab[((inner + V - 1) / args.vstride) % args.nvel];
                }
            } else {
                ka = args.cell_coef[args.fast32 ? (long long)fdiv(unsigned(outer), args.div_opc)
                                                : outer / args.outer_per_cell];
                kb = ka;
            }
            if (ka.nd < 0 || kb.nd < 0) work = false; // Courant number out of range: leave as is
            neg = ka.nd & 1;
            lim = PairLim<C, X>::make(ka, kb);
        }
        const unsigned ec = e + (PERIODIC ? 1u : 0u); // entry of chunk 0
        if (!work) {
            // keep the barrier phases in step with the other consumers
            for (int j = 0; j < E && alive; ++j)
                if (acquire(e + unsigned(j))) release(e + unsigned(j));
            e += E;
            continue;
        }
        // 16-bit storage: a rounding stream per column pair and block, from the element index
        unsigned rng = CODED ? sr_bits((unsigned long long)(outer * L * args.n_inner + inner), args.seed) : 0u;
        // this column's line in a scale slot
        const int c0 = int(tr * W);
        const int soff = CODED ? (p * R * Wl + (c0 + w) / nuz - ((c0 / nuz) & ~3)) : 0;
        X sum;
        if (neg)
            sum = march_stream<T, PERIODIC, true>(lim, e, ec, coff, soff, L, W, Wl, rng, slot_ptr, scale_ptr, acquire,
                                                  release, alive);
        else
            sum = march_stream<T, PERIODIC, false>(lim, e, ec, coff, soff, L, W, Wl, rng, slot_ptr, scale_ptr, acquire,
                                                   release, alive);
        if (!alive) break;
        if (LN::bad(sum)) atomicOr(args.err, ERR_NAN);
        e += unsigned(E);
    }
}

// the dividers of the consumers' per-block index arithmetic (fast32 when every index fits)
template <typename C> static void set_stream_dividers(StreamArgs<C> &a)
{
    const long long lim = 0xffffffffll - 1024;
    a.fast32 = a.tile0 + a.num_blocks < lim && a.n_inner < lim && a.n_outer < lim && a.tiles_inner > 0 &&
               a.vstride > 0 && a.vstride < lim && a.outer_per_cell > 0 && a.outer_per_cell < lim;
    if (!a.fast32) return;
    a.div_tiles = make_fastdiv(unsigned(a.tiles_inner));
    a.div_vstride = make_fastdiv(unsigned(a.vstride));
    a.div_nvel = make_fastdiv(unsigned(a.nvel > 0 ? a.nvel : 1));
    a.div_opc = make_fastdiv(unsigned(a.outer_per_cell));
}

template <typename T>
static cudaError_t launch_stream_t(const CUtensorMap &map, const CUtensorMap &dmap, const CUtensorMap &smap,
                                   const StreamArgs<typename Compute<T>::type> &a_in, int grid, size_t smem,
                                   cudaStream_t st)
{
    StreamArgs<typename Compute<T>::type> a = a_in;
    set_stream_dividers(a);
    auto kern = a.periodic ? stream_sweep_kernel<T, true> : stream_sweep_kernel<T, false>;
    int threads = Lane<T>::NC + stream_head<false>();
    if constexpr (sizeof(T) != 2)
        if (a.mpart) {
            kern = stream_sweep_kernel<T, true, true>; // the x sweep with the moment
            threads = Lane<T>::NC + stream_head<true>();
        }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, threads, smem, st>>>(map, dmap, smap, a);
    return cudaGetLastError();
}

cudaError_t launch_stream_f32(const CUtensorMap &map, const CUtensorMap &dmap, const StreamArgs<float> &a, int grid,
                              size_t smem, cudaStream_t st)
{
    return launch_stream_t<float>(map, dmap, map, a, grid, smem, st);
}

cudaError_t launch_stream_f64(const CUtensorMap &map, const CUtensorMap &dmap, const StreamArgs<double> &a, int grid,
                              size_t smem, cudaStream_t st)
{
    return launch_stream_t<double>(map, dmap, map, a, grid, smem, st);
}

cudaError_t launch_stream_bf16(const CUtensorMap &map, const CUtensorMap &smap, const StreamArgs<float> &a, int grid,
                               size_t smem, cudaStream_t st)
{
    return launch_stream_t<__nv_bfloat16>(map, map, smap, a, grid, smem, st);
}

cudaError_t launch_stream_f16(const CUtensorMap &map, const CUtensorMap &smap, const StreamArgs<float> &a, int grid,
                              size_t smem, cudaStream_t st)
{
    return launch_stream_t<__half>(map, map, smap, a, grid, smem, st);
}

template <typename T> static const void *stream_ptr(int periodic)
{
    return periodic ? (const void *)stream_sweep_kernel<T, true> : (const void *)stream_sweep_kernel<T, false>;
}

int stream_columns_per_thread(int dtype) { return dtype == 0 ? 1 : 2; }
int stream_consumers(int) { return kStreamConsumers; }

int occupancy_stream(int dtype, int periodic, size_t smem)
{
    const void *k = dtype == 0 ? stream_ptr<double>(periodic)
                    : dtype == 1 ? stream_ptr<float>(periodic)
                    : dtype == 2 ? stream_ptr<__nv_bfloat16>(periodic)
                                 : stream_ptr<__half>(periodic);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, stream_consumers(dtype) + kProducer, smem) != cudaSuccess)
        return 0;
    return n;
}

} // namespace vk
