// vlasov_api.cu -- host side of the C ABI declared in include/vlasov.h.
//
// Owns the context: argument checks, the TMA tensor maps of f for each sweep
// axis, the tile / pipeline geometry, the scratch buffers, and the order of
// the kernels of one split step (Eq. 5 of Yoshikawa, Tanaka & Yoshida, SC'21).
#include <cudaTypedefs.h>

#include <mutex>
#include <new>
#include <vector>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "../../include/vlasov.h"
#include "vk_common.cuh"
#include "vk_kernels.h"

using namespace vk;

namespace {

thread_local char g_init_error[256] = "";

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Parameters of a tiled tensor map, kept so the same view can be encoded for
// another array of the same shape (out-of-place sweeps, recorded inputs).
struct MapSpec {
    CUtensorMapDataType type;
    cuuint32_t rank;
    cuuint64_t gdim[4];
    cuuint64_t gstr[3];
    cuuint32_t box[4];
    CUtensorMapSwizzle swz;
    CUtensorMapL2promotion promo;
};

CUresult encode_spec(CUtensorMap *m, const MapSpec &s, const void *base)
{
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return encode_fn()(m, s.type, s.rank, const_cast<void *>(base), s.gdim, s.gstr, s.box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, s.swz, s.promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

MapSpec spec3(CUtensorMapDataType type, long long I, long long L, long long O, size_t es, int W, int R, int P)
{
    MapSpec s{};
    s.type = type;
    s.rank = 3;
    s.gdim[0] = (cuuint64_t)I; s.gdim[1] = (cuuint64_t)L; s.gdim[2] = (cuuint64_t)O;
    s.gstr[0] = (cuuint64_t)(I * es); s.gstr[1] = (cuuint64_t)(I * L * es);
    s.box[0] = (cuuint32_t)W; s.box[1] = (cuuint32_t)R; s.box[2] = (cuuint32_t)P;
    s.swz = CU_TENSOR_MAP_SWIZZLE_NONE;
    s.promo = CU_TENSOR_MAP_L2_PROMOTION_L2_256B;
    return s;
}

// rows of L elements: box {L, R rows}
MapSpec spec_rows(CUtensorMapDataType type, long long L, long long rows, size_t es, int R, CUtensorMapSwizzle swz)
{
    MapSpec s{};
    s.type = type;
    s.rank = 2;
    s.gdim[0] = (cuuint64_t)L; s.gdim[1] = (cuuint64_t)rows;
    s.gstr[0] = (cuuint64_t)(L * es);
    s.box[0] = (cuuint32_t)L; s.box[1] = (cuuint32_t)R;
    s.swz = swz;
    s.promo = CU_TENSOR_MAP_L2_PROMOTION_L2_256B;
    return s;
}

// f as [O][L][I / 32][32] FP32 with box {32, 8, L, 1}: the tiles of the staged position sweeps
MapSpec spec_tiles(long long I, long long L, long long O)
{
    MapSpec s{};
    s.type = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    s.rank = 4;
    s.gdim[0] = 32; s.gdim[1] = (cuuint64_t)(I / 32); s.gdim[2] = (cuuint64_t)L; s.gdim[3] = (cuuint64_t)O;
    s.gstr[0] = 128; s.gstr[1] = (cuuint64_t)(I * 4); s.gstr[2] = (cuuint64_t)(I * L * 4);
    s.box[0] = 32; s.box[1] = 8; s.box[2] = (cuuint32_t)L; s.box[3] = 1;
    s.swz = CU_TENSOR_MAP_SWIZZLE_128B;
    s.promo = CU_TENSOR_MAP_L2_PROMOTION_L2_256B;
    return s;
}

struct AxisPlan {
    CUtensorMap map;
    MapSpec spec;
    int L, W, P, stages, grid;
    long long n_inner, n_outer, num_tiles;
    int tiles_inner;
    size_t smem;
};

} // namespace

constexpr int kMaxSlabs = 16; // x-slabs of the pipelined host-buffer step

struct vlasov_ctx {
    vlasov_grid g;
    GridDims gd;
    void *f;
    float *scale; // 16-bit storage: FP32 scale per u_z line (caller-owned)
    cudaStream_t stream;
    size_t es;
    int sm_count;
    long long ncell; // spatial cells
    AxisPlan plan[6];
    AxisPlan splan[5];   // streamed sweeps (|nu| < 1), axes 0..4
    int perm_line[5];
    int splan_R[5];
    CUtensorMap smap[5]; // 16-bit storage: scale array seen like f, the u_z line collapsed
    int scale_rank[5];
    int swidth[5]; // inner extent of each axis' scale box
    // u_z with whole lines in registers
    bool use_lines;
    CUtensorMap lmap;
    MapSpec lspec;
    // kick tail D_uz D_uy fused in the u_z line kernel (n_uy = n_uz)
    bool can_fuse_kick;
    bool can_plane_tail; // the kick tail over staged (cell, j_x) planes (n_uy = n_uz = 48)
    int fuse_kick; // vlasov_set_fused_kick: 0 separate sweeps, 1 fused tail, 2 whole kick in one pass
    // position sweeps with whole lines staged per tile (see vlasov_set_position_tiles)
    // staged tiles of the x, y, z sweeps and (index 3) of the u_x sweep
    bool tile_ok[4], use_tiles;
    CUtensorMap tmap[4], tsmap[4]; // tsmap: 16-bit storage, the scales of a tile
    MapSpec tspec[4];
    int tgrid[4];
    long long ttiles_inner[4], tn_outer[4];
    // the whole kick D_uz D_uy D_ux in one pass (n_ux = n_uy = n_uz = 16 or 32)
    bool can_kick_cube;
    CUtensorMap kmap, ksmap;
    int kgrid;
    int lgrid_fused;
    long long lrows, ltiles;
    int lgrid;
    // scratch
    unsigned *d_err;
    void *d_coef[3];
    double *d_rho;
    double *d_mass;
    PoissonScratch ps;
    // adjoint scratch, allocated on first use: the inputs of sweeps 1..8 of a
    // step, dL/dg per velocity axis, lambda of a whole-cell-shift position sweep
    void *d_rec[8];
    double *d_dLdg;
    void *d_lam_tmp;
    double *d_sc; // self-consistent adjoint: dL/dphi^{n+1} and dL/drho (2 * ncell)
    double *d_part; // adjoint: per-block sums of dL/dnu (deterministic per-cell reduction)
    size_t part_len;
    void *d_mpart; // the moment fused into the x sweep: per-cell partial sums (storage type)
    bool fuse_moment;
    // vlasov_step_host: sweeps restricted to the x-planes [slab_x0, slab_x1) (all if empty)
    int slab_x0, slab_x1;
    long long splan_tpp[5]; // tiles per x-plane of the streamed sweeps (0: a block spans planes)
    long long ltpp;         // the same for the u_z line kernel
    cudaStream_t copy_stream;                // uploads
    cudaStream_t down_stream;                // downloads
    cudaEvent_t slab_ev[2 * kMaxSlabs + 2];
    cudaEvent_t down_ev[kMaxSlabs + 1];      // after each slab's download; [kMaxSlabs]: after the last
    bool slab_ev_ok;
    // downloads of the last vlasov_step_host that the context stream has not been made
    // to wait for (0: none), and their slab size: the next vlasov_step_host with the
    // same slabs orders each upload after the download of its own slab only; any other
    // call queues the wait for all of them first (settle)
    int pending_slabs;
    size_t pending_slab_bytes;
    int adj_arrays; // f-sized scratch arrays vlasov_step_adjoint may use: 8, 4 or 0 (8 if they fit, else 4)
    char msg[256];
    unsigned sweeps; // sweeps queued so far: the stochastic-rounding seed of the next one
    // per-part timers
    bool timers_on;
    struct Pending { int kind; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double acc_ms[VLASOV_T_KINDS];
    long long launches[VLASOV_T_KINDS];
};

// Bracket the kernels queued between construction and destruction with events
// (when timers are on) and count them.
struct PartTimer {
    vlasov_ctx *c;
    int kind;
    cudaEvent_t a = nullptr;
    PartTimer(vlasov_ctx *c_, int kind_, int nlaunch) : c(c_), kind(kind_)
    {
        c->launches[kind] += nlaunch;
        if (!c->timers_on) return;
        a = take();
        cudaEventRecord(a, c->stream);
    }
    cudaEvent_t take()
    {
        cudaEvent_t e = nullptr;
        if (!c->pool.empty()) { e = c->pool.back(); c->pool.pop_back(); }
        else cudaEventCreate(&e);
        return e;
    }
    ~PartTimer()
    {
        if (!a) return;
        cudaEvent_t b = take();
        cudaEventRecord(b, c->stream);
        c->pending.push_back({kind, a, b});
    }
};

static int fail(vlasov_ctx *c, int code, const char *fmt, ...)
{
    char *dst = c ? c->msg : g_init_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return code;
}

static int cuda_fail(vlasov_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, VLASOV_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define VK_CUDA(ctx, call)                                                                                  \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);                                          \
    } while (0)

// queue on the context stream the wait for the downloads of the last vlasov_step_host
static int settle(vlasov_ctx *c)
{
    if (c->pending_slabs) {
        c->pending_slabs = 0;
        VK_CUDA(c, cudaStreamWaitEvent(c->stream, c->down_ev[kMaxSlabs], 0));
    }
    return VLASOV_OK;
}

#define VK_SETTLE(ctx)                                                                                      \
    do {                                                                                                    \
        if (int rc_ = settle(ctx)) return rc_;                                                              \
    } while (0)

static CUtensorMapDataType tmap_type(int dtype)
{
    switch (dtype) {
    case VLASOV_F64: return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    case VLASOV_F32: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    case VLASOV_BF16: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    default: return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    }
}

// Plan the sweeps of the axes whose bits are set in mask (all six by default): tensor
// maps, tile geometry and launch grids.
static int plan_axes(vlasov_ctx *c, int mask = 0x3f)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return fail(c, VLASOV_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const long long d6[6] = {c->g.nx, c->g.ny, c->g.nz, c->g.nux, c->g.nuy, c->g.nuz};
    const size_t es = c->es;
    const size_t kSmemBudget = 200 * 1024;
    const bool coded = c->g.dtype == VLASOV_BF16 || c->g.dtype == VLASOV_F16;
    // whole-line kernels (whole-cell shifts, u_z lines of other lengths): FP32 / FP64 only
    for (int ax = 0; ax < 6 && !coded; ++ax) {
        if (!(mask >> ax & 1)) continue;
        AxisPlan &p = c->plan[ax];
        p.L = int(d6[ax]);
        long long I = 1, O = 1;
        for (int k = ax + 1; k < 6; ++k) I *= d6[k];
        for (int k = 0; k < ax; ++k) O *= d6[k];
        p.n_inner = I;
        p.n_outer = O;
        CUresult r;
        if (ax < 5) {
            int W, P;
            if (I >= kConsumers) { W = kConsumers; P = 1; }
            else { W = int(I); P = kConsumers / W; if (P > O) P = int(O); }
            while ((size_t)W * p.L * P * es > 96 * 1024 && W * P > 32) {
                if (P > 1) P = (P + 1) / 2;
                else W /= 2;
            }
            p.W = W;
            p.P = P;
            p.tiles_inner = int((I + W - 1) / W);
            p.num_tiles = (long long)p.tiles_inner * ((O + P - 1) / P);
            const size_t tile = ((size_t)W * p.L * P * es + 127) & ~size_t(127);
            const size_t tab = ax < 3 ? ((sizeof(LineCoefT<double>) * kMaxVel + 127) & ~size_t(127)) : 0;
            int S = int((kSmemBudget - 128 - tab) / tile);
            S = S < 2 ? 2 : (S > 4 ? 4 : S);
            p.stages = S;
            p.smem = 128 + tab + (size_t)S * tile;
            p.spec = spec3(tmap_type(c->g.dtype), I, p.L, O, es, W, p.L, P);
            r = encode_spec(&p.map, p.spec, c->f);
            const int occ = occupancy_strided(c->g.dtype == VLASOV_F64 ? 0 : 1, ax < 3, p.smem);
            if (occ <= 0) return fail(c, VLASOV_ECUDA, "axis %d: a CTA does not fit (%zu B shared memory)", ax, p.smem);
            p.grid = int(p.num_tiles < (long long)occ * c->sm_count ? p.num_tiles : (long long)occ * c->sm_count);
        } else {
            const long long rows = O * 1; // one row per (cell, jx, jy)
            p.W = p.L;
            p.P = kConsumers; // rows per tile
            p.n_outer = rows;
            p.num_tiles = (rows + kConsumers - 1) / kConsumers;
            p.tiles_inner = 1;
            const size_t ces = c->g.dtype == VLASOV_F64 ? 8 : 4;
            const size_t tile = ((size_t)p.L * kConsumers * es + 127) & ~size_t(127);
            const size_t bbuf = (size_t)p.L * (kConsumers + 1) * ces;
            int S = int((kSmemBudget - 128 - bbuf) / tile);
            S = S < 2 ? 2 : (S > 4 ? 4 : S);
            p.stages = S;
            p.smem = 128 + (size_t)S * tile + bbuf;
            p.spec = spec_rows(tmap_type(c->g.dtype), p.L, rows, es, kConsumers, CU_TENSOR_MAP_SWIZZLE_NONE);
            r = encode_spec(&p.map, p.spec, c->f);
            const int occ = occupancy_contig(c->g.dtype == VLASOV_F64 ? 0 : 1, p.smem);
            // u_z rows of 24, 40 or 48 cells never take the transposing kernel
            if (occ <= 0 && rows_sweep_supported(int(c->g.nuz), c->g.dtype)) {
                p.grid = 0;
                continue;
            }
            if (occ <= 0) return fail(c, VLASOV_ECUDA, "axis 5: a CTA does not fit (%zu B shared memory)", p.smem);
            p.grid = int(p.num_tiles < (long long)occ * c->sm_count ? p.num_tiles : (long long)occ * c->sm_count);
        }
        if (r != CUDA_SUCCESS) return fail(c, VLASOV_ECUDA, "axis %d: cuTensorMapEncodeTiled failed (%d)", ax, int(r));
    }
    // streamed sweeps: blocks of V * consumers columns, chunks of R rows, a ring of S slots
    const int V = stream_columns_per_thread(c->g.dtype); // columns per consumer thread
    const int cols = V * stream_consumers(c->g.dtype);
    for (int ax = 0; ax < 5; ++ax) {
        if (!(mask >> ax & 1)) continue;
        AxisPlan &p = c->splan[ax];
        p.L = int(d6[ax]);
        long long I = 1, O = 1;
        for (int k = ax + 1; k < 6; ++k) I *= d6[k];
        for (int k = 0; k < ax; ++k) O *= d6[k];
        p.n_inner = I;
        p.n_outer = O;
        int W, P;
        c->perm_line[ax] = 0;
        if (ax == 2 && c->g.nuz <= cols) {
            // the z sweep's Courant number changes sign inside each u_z line: whole lines per block
            W = (cols / c->g.nuz) * c->g.nuz;
            P = 1;
            c->perm_line[ax] = c->g.nuz;
        } else if (I >= cols) { W = cols; P = 1; }
        else { W = int(I); P = cols / W; if (P > O) P = int(O); }
        const int R = coded ? 2 * kStreamRows : kStreamRows; // the kernels' stream_rows<T>()
        const int S = kStreamRing;
        p.W = W;
        p.P = P;
        p.stages = S;
        p.tiles_inner = int((I + W - 1) / W);
        p.num_tiles = (long long)p.tiles_inner * ((O + P - 1) / P);
        const size_t slot = ((size_t)W * R * P * es + 127) & ~size_t(127);
        const size_t csz = c->g.dtype == VLASOV_F64 ? sizeof(LineCoefT<double>) : sizeof(LineCoefT<float>);
        const size_t tab = ax < 3 ? ((csz * (size_t)d6[3 + ax] + 127) & ~size_t(127)) : 0;
        size_t sslot = 0;
        if (coded) {
            // scales of the lines of one chunk: box {Wl, R, P} over [O][L][I / nuz] from line
            // (c0 / nuz) & ~3 of a block at inner offset c0 (the u_y sweep has I = nuz: box
            // {R, P} over [O][L]).  Wl = W / nuz when that is a multiple of 4 (every c0 / nuz
            // then is one too), else it covers the up to 3 lines ahead of c0's own line and
            // the ceil((W - 1) / nuz) + 1 lines a block of W columns can touch.
            const int nuz = int(c->g.nuz);
            int Wl = 1;
            if (ax < 4) {
                Wl = (W % nuz == 0 && (W / nuz) % 4 == 0) ? W / nuz : 3 + (W - 1 + nuz - 1) / nuz + 1;
                Wl = (Wl + 3) & ~3;
            } else if (I != nuz || W != nuz) {
                return fail(c, VLASOV_EINVAL, "axis %d: u_y blocks must be whole u_z lines", ax);
            }
            c->swidth[ax] = Wl;
            sslot = ((size_t)Wl * R * P * 4 + 127) & ~size_t(127);
            CUresult rs;
            if (ax < 4) {
                const cuuint64_t sdim[3] = {(cuuint64_t)(I / nuz), (cuuint64_t)p.L, (cuuint64_t)O};
                const cuuint64_t sstr[2] = {(cuuint64_t)(I / nuz * 4), (cuuint64_t)(I / nuz * p.L * 4)};
                const cuuint32_t sbox[3] = {(cuuint32_t)Wl, (cuuint32_t)R, (cuuint32_t)P};
                const cuuint32_t sest[3] = {1, 1, 1};
                rs = enc(&c->smap[ax], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->scale, sdim, sstr, sbox, sest,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                c->scale_rank[ax] = 3;
            } else {
                const cuuint64_t sdim[2] = {(cuuint64_t)p.L, (cuuint64_t)O};
                const cuuint64_t sstr[1] = {(cuuint64_t)(p.L * 4)};
                const cuuint32_t sbox[2] = {(cuuint32_t)R, (cuuint32_t)P};
                const cuuint32_t sest[2] = {1, 1};
                rs = enc(&c->smap[ax], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->scale, sdim, sstr, sbox, sest,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                c->scale_rank[ax] = 2;
            }
            if (rs != CUDA_SUCCESS) return fail(c, VLASOV_ECUDA, "axis %d: scale tensor map failed (%d)", ax, int(rs));
        }
        p.smem = 512 + tab + (size_t)S * (slot + sslot);
        p.grid = R; // rows per chunk (kept here; the launch grid is computed below)
        p.spec = spec3(tmap_type(c->g.dtype), I, p.L, O, es, W, R, P);
        const CUresult r = encode_spec(&p.map, p.spec, c->f);
        if (r != CUDA_SUCCESS) return fail(c, VLASOV_ECUDA, "axis %d: stream tensor map failed (%d)", ax, int(r));
        const int occ = occupancy_stream(c->g.dtype, ax < 3, p.smem);
        if (occ <= 0) return fail(c, VLASOV_ECUDA, "axis %d: a streamed CTA does not fit (%zu B)", ax, p.smem);
        p.grid = int(p.num_tiles < (long long)occ * c->sm_count ? p.num_tiles : (long long)occ * c->sm_count);
        c->splan_R[ax] = R;
        const long long opp = p.n_outer / c->g.nx; // outer lines per x-plane
        c->splan_tpp[ax] = (p.n_outer % c->g.nx == 0 && opp % P == 0) ? (opp / P) * p.tiles_inner : 0;
    }
    // u_z: register lines when a line is 32, 64 or 128 bytes (FP32 / 16-bit, n_uz 16 or 32)
    c->use_lines = (mask >> 5 & 1) && c->g.dtype != VLASOV_F64 &&
                   line_sweep_supported(c->g.nuz, (long long)c->g.nux * c->g.nuy);
    if (c->use_lines) {
        const int nu = c->g.nuz, rpt = line_sweep_rows_per_tile();
        c->lrows = c->ncell * c->g.nux * c->g.nuy;
        c->ltiles = (c->lrows + rpt - 1) / rpt;
        const size_t rowbytes = nu * es;
        const CUtensorMapSwizzle sw = rowbytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                      : rowbytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                       : CU_TENSOR_MAP_SWIZZLE_32B;
        c->lspec = spec_rows(tmap_type(c->g.dtype), nu, c->lrows, es, rpt, sw);
        const CUresult r = encode_spec(&c->lmap, c->lspec, c->f);
        if (r != CUDA_SUCCESS) return fail(c, VLASOV_ECUDA, "u_z line tensor map failed (%d)", int(r));
        const int occ = occupancy_line_sweep(nu, c->g.dtype);
        if (occ <= 0) return fail(c, VLASOV_ECUDA, "u_z line sweep CTA does not fit");
        c->lgrid = int(c->ltiles < (long long)occ * c->sm_count ? c->ltiles : (long long)occ * c->sm_count);
        const long long rpp = c->lrows / c->g.nx; // u_z rows per x-plane
        c->ltpp = rpp % rpt == 0 ? rpp / rpt : 0;
    }
    for (int ax = 0; ax < 4; ++ax) {
        c->tile_ok[ax] = false;
        if (!(mask >> ax & 1) || c->g.dtype == VLASOV_F64) continue;
        long long I = 1, O = 1;
        for (int k = ax + 1; k < 6; ++k) I *= d6[k];
        for (int k = 0; k < ax; ++k) O *= d6[k];
        // u_x: [cell][u_x][u_y u_z], zero-flux lines of 48 (lines of 16 and 32 take the
        // one-pass kick or the register lines)
        const bool ok = ax == 3 ? tile_sweep_zf_supported(int(d6[ax]), I, c->g.dtype, int(c->g.nuz))
                                : tile_sweep_supported(int(d6[ax]), I, c->g.dtype, int(c->g.nuz));
        if (!ok || O > 0x7fffffffll || I / 32 > 0x7fffffffll) continue;
        c->tspec[ax] = spec_tiles(I, d6[ax], O);
        if (coded) {
            // codes: 512-byte rows of 32-code units, no swizzle; scales: one per u_z line, a
            // tile's 8 lines (n_uz = 32) or the 12 from its first line rounded down to a
            // multiple of 4 (n_uz = 48: the 6 or 7 lines of its 256 columns)
            const long long nl = I / c->g.nuz;
            c->tspec[ax].type = tmap_type(c->g.dtype);
            c->tspec[ax].gstr[0] = 64; c->tspec[ax].gstr[1] = (cuuint64_t)(I * 2); c->tspec[ax].gstr[2] = (cuuint64_t)(I * d6[ax] * 2);
            c->tspec[ax].swz = CU_TENSOR_MAP_SWIZZLE_NONE;
            MapSpec ss{};
            ss.type = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
            ss.rank = 3;
            ss.gdim[0] = (cuuint64_t)nl; ss.gdim[1] = (cuuint64_t)d6[ax]; ss.gdim[2] = (cuuint64_t)O;
            ss.gstr[0] = (cuuint64_t)(nl * 4); ss.gstr[1] = (cuuint64_t)(nl * d6[ax] * 4);
            ss.box[0] = c->g.nuz == 32 ? 8 : 12; ss.box[1] = (cuuint32_t)d6[ax]; ss.box[2] = 1;
            ss.swz = CU_TENSOR_MAP_SWIZZLE_NONE;
            ss.promo = CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
            if (encode_spec(&c->tsmap[ax], ss, c->scale) != CUDA_SUCCESS) continue;
        }
        if (encode_spec(&c->tmap[ax], c->tspec[ax], c->f) != CUDA_SUCCESS) continue;
        const int occ = occupancy_tile_sweep(int(d6[ax]), c->g.dtype, ax == 0 && !coded, int(c->g.nuz));
        if (occ <= 0) continue;
        c->ttiles_inner[ax] = I / 256;
        c->tn_outer[ax] = O;
        const long long tiles = O * (I / 256);
        c->tgrid[ax] = int(tiles < (long long)occ * c->sm_count ? tiles : (long long)occ * c->sm_count);
        c->tile_ok[ax] = true;
    }
    c->can_kick_cube = (mask & 0x38) == 0x38 && kick_cube_supported(c->g.nux, c->g.nuy, c->g.nuz, c->g.dtype) &&
                       c->ncell * c->g.nux * c->g.nuy < (1ll << 31);
    if (c->can_kick_cube) {
        // f as rows of nu values (u_z lines), a box of half a cube's rows (at most 256)
        const int nu = c->g.nuz;
        const size_t rowbytes = nu * es;
        const CUtensorMapSwizzle sw = rowbytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                      : rowbytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                       : CU_TENSOR_MAP_SWIZZLE_32B;
        const MapSpec ks = spec_rows(tmap_type(c->g.dtype), nu, c->ncell * nu * nu, es, kick_cube_box_rows(nu), sw);
        CUresult r = encode_spec(&c->kmap, ks, c->f);
        if (r != CUDA_SUCCESS) return fail(c, VLASOV_ECUDA, "kick tensor map failed (%d)", int(r));
        if (coded) {
            // the scales as [ncell nu][nu] (one row per j_x plane), half a cube per box
            const MapSpec ss = spec_rows(CU_TENSOR_MAP_DATA_TYPE_FLOAT32, nu, c->ncell * nu, 4, nu / 2,
                                         CU_TENSOR_MAP_SWIZZLE_NONE);
            r = encode_spec(&c->ksmap, ss, c->scale);
            if (r != CUDA_SUCCESS) return fail(c, VLASOV_ECUDA, "kick scale tensor map failed (%d)", int(r));
        } else {
            c->ksmap = c->kmap; // not read
        }
        const int occ = occupancy_kick_cube(nu, c->g.dtype);
        if (occ <= 0) return fail(c, VLASOV_ECUDA, "one-pass kick CTA does not fit");
        c->kgrid = int(c->ncell < (long long)occ * c->sm_count ? c->ncell : (long long)occ * c->sm_count);
    }
    c->can_fuse_kick = c->use_lines && (mask >> 4 & 1) && line_sweep_fused_supported(c->g.dtype) &&
                       c->g.nuy == c->g.nuz;
    if (c->can_fuse_kick) {
        const int occ = occupancy_line_sweep(c->g.nuz, c->g.dtype, true);
        if (occ <= 0) return fail(c, VLASOV_ECUDA, "fused kick CTA does not fit");
        c->lgrid_fused = int(c->ltiles < (long long)occ * c->sm_count ? c->ltiles : (long long)occ * c->sm_count);
    }
    c->can_plane_tail = !c->can_fuse_kick && (mask >> 4 & 1) && (mask >> 5 & 1) &&
                        plane_tail_supported(c->g.nuy, c->g.nuz, c->g.nux, c->g.dtype);
    return VLASOV_OK;
}

static void free_scratch(vlasov_ctx *c)
{
    cudaFree(c->d_err);
    for (int d = 0; d < 3; ++d) cudaFree(c->d_coef[d]);
    cudaFree(c->d_rho);
    cudaFree(c->d_mass);
    cudaFree(c->ps.z0);
    cudaFree(c->ps.z1);
    for (int d = 0; d < 3; ++d) cudaFree(c->ps.tw[d]);
    for (int k = 0; k < 8; ++k) cudaFree(c->d_rec[k]);
    cudaFree(c->d_dLdg);
    cudaFree(c->d_lam_tmp);
    cudaFree(c->d_sc);
    cudaFree(c->d_part);
    cudaFree(c->d_mpart);
    if (c->slab_ev_ok) {
        for (auto e : c->slab_ev) cudaEventDestroy(e);
        for (auto e : c->down_ev) cudaEventDestroy(e);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->down_stream) cudaStreamDestroy(c->down_stream);
}

extern "C" int vlasov_init(vlasov_ctx **out, const vlasov_grid *g, void *f_dev, float *scale_dev, void *stream)
{
    if (!out || !g || !f_dev) return fail(nullptr, VLASOV_EINVAL, "vlasov_init: null argument");
    *out = nullptr;
    const int dims[6] = {g->nx, g->ny, g->nz, g->nux, g->nuy, g->nuz};
    for (int k = 0; k < 3; ++k)
        if (dims[k] < 4 || dims[k] > 256) return fail(nullptr, VLASOV_EINVAL, "spatial size %d outside [4, 256]", dims[k]);
    for (int k = 3; k < 6; ++k)
        if (dims[k] < 4 || dims[k] > kMaxVel || dims[k] % 4)
            return fail(nullptr, VLASOV_EINVAL, "velocity size %d must be a multiple of 4 in [4, %d]", dims[k], kMaxVel);
    if (!(g->L > 0) || !(g->V > 0)) return fail(nullptr, VLASOV_EINVAL, "L and V must be positive");
    if (g->dtype < VLASOV_F64 || g->dtype > VLASOV_F16) return fail(nullptr, VLASOV_EINVAL, "unknown dtype %d", g->dtype);
    const bool coded = g->dtype == VLASOV_BF16 || g->dtype == VLASOV_F16;
    if (!coded && scale_dev) return fail(nullptr, VLASOV_EINVAL, "scale_dev must be NULL for FP32/FP64 storage");
    if (coded) {
        if (!scale_dev || reinterpret_cast<uintptr_t>(scale_dev) % 16)
            return fail(nullptr, VLASOV_EINVAL, "16-bit storage needs a 16-byte aligned scale_dev");
        if (!line_sweep_supported(g->nuz, (long long)g->nux * g->nuy) && !rows_sweep_supported(g->nuz, g->dtype))
            return fail(nullptr, VLASOV_EINVAL,
                        "16-bit storage needs nuz = 16 or 32 with nux * nuy a multiple of 256, or nuz = 24, 40 or 48");
    }
    if (reinterpret_cast<uintptr_t>(f_dev) % 16) return fail(nullptr, VLASOV_EINVAL, "f_dev must be 16-byte aligned");
    const long long ncell = (long long)g->nx * g->ny * g->nz;
    const long long cube = (long long)g->nux * g->nuy * g->nuz;
    if (ncell * g->nux * g->nuy >= (1ll << 31)) return fail(nullptr, VLASOV_EINVAL, "too many u_z lines for 32-bit TMA coordinates");
    if (ncell * cube / g->nx >= (1ll << 32)) return fail(nullptr, VLASOV_EINVAL, "grid too large for 32-bit TMA extents");

    vlasov_ctx *c = new (std::nothrow) vlasov_ctx();
    if (!c) return fail(nullptr, VLASOV_ENOMEM, "out of host memory");
    c->g = *g;
    c->f = f_dev;
    c->scale = coded ? scale_dev : nullptr;
    c->stream = (cudaStream_t)stream;
    c->es = g->dtype == VLASOV_F64 ? 8 : (coded ? 2 : 4);
    c->ncell = ncell;
    c->fuse_kick = 2; // see vlasov_set_fused_kick
    c->use_tiles = true; // see vlasov_set_position_tiles
    c->fuse_moment = true; // see vlasov_set_fused_moment
    c->slab_x0 = c->slab_x1 = 0;
    c->gd.n[0] = g->nx; c->gd.n[1] = g->ny; c->gd.n[2] = g->nz;
    c->gd.nu[0] = g->nux; c->gd.nu[1] = g->nuy; c->gd.nu[2] = g->nuz;
    c->gd.L = g->L;
    c->gd.V = g->V;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        fail(nullptr, VLASOV_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
        delete c;
        return VLASOV_ECUDA;
    }
    const size_t coef_bytes = (size_t)ncell * (g->dtype == VLASOV_F64 ? sizeof(LineCoefT<double>) : sizeof(LineCoefT<float>));
    bool ok = cudaMalloc(&c->d_err, sizeof(unsigned)) == cudaSuccess;
    for (int d = 0; d < 3 && ok; ++d) ok = cudaMalloc(&c->d_coef[d], coef_bytes) == cudaSuccess;
    ok = ok && cudaMalloc(&c->d_rho, sizeof(double) * ncell) == cudaSuccess;
    ok = ok && cudaMalloc(&c->d_mass, sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&c->ps.z0, sizeof(double2) * ncell) == cudaSuccess;
    ok = ok && cudaMalloc(&c->ps.z1, sizeof(double2) * ncell) == cudaSuccess;
    for (int d = 0; d < 3 && ok; ++d) {
        const int n = dims[d];
        ok = cudaMalloc(&c->ps.tw[d], sizeof(double2) * n) == cudaSuccess;
        if (!ok) break;
        double2 *h = new double2[n];
        for (int q = 0; q < n; ++q) h[q] = make_double2(cos(2.0 * M_PI * q / n), sin(2.0 * M_PI * q / n));
        ok = cudaMemcpy(c->ps.tw[d], h, sizeof(double2) * n, cudaMemcpyHostToDevice) == cudaSuccess;
        delete[] h;
    }
    ok = ok && cudaMemset(c->d_err, 0, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_scratch(c);
        delete c;
        return fail(nullptr, VLASOV_ENOMEM, "device scratch allocation failed");
    }
    const int rc = plan_axes(c);
    if (rc != VLASOV_OK) {
        snprintf(g_init_error, sizeof g_init_error, "%s", c->msg);
        free_scratch(c);
        delete c;
        return rc;
    }
    *out = c;
    return VLASOV_OK;
}

extern "C" void vlasov_destroy(vlasov_ctx *c)
{
    if (!c) return;
    settle(c);
    cudaStreamSynchronize(c->stream);
    free_scratch(c);
    for (auto &p : c->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : c->pool) cudaEventDestroy(e);
    delete c;
}

static size_t f_bytes(const vlasov_ctx *c) { return (size_t)c->ncell * c->g.nux * c->g.nuy * c->g.nuz * c->es; }

extern "C" int vlasov_upload(vlasov_ctx *c, const void *f_host)
{
    if (!c || !f_host) return c ? fail(c, VLASOV_EINVAL, "vlasov_upload: null host buffer") : VLASOV_EINVAL;
    VK_SETTLE(c);
    const size_t bytes = (size_t)c->ncell * c->g.nux * c->g.nuy * c->g.nuz * c->es;
    VK_CUDA(c, cudaMemcpyAsync(c->f, f_host, bytes, cudaMemcpyHostToDevice, c->stream));
    return VLASOV_OK;
}

extern "C" int vlasov_download(vlasov_ctx *c, void *f_host)
{
    if (!c || !f_host) return c ? fail(c, VLASOV_EINVAL, "vlasov_download: null host buffer") : VLASOV_EINVAL;
    VK_SETTLE(c);
    const size_t bytes = (size_t)c->ncell * c->g.nux * c->g.nuy * c->g.nuz * c->es;
    VK_CUDA(c, cudaMemcpyAsync(f_host, c->f, bytes, cudaMemcpyDeviceToHost, c->stream));
    return VLASOV_OK;
}

extern "C" int vlasov_enable_timers(vlasov_ctx *c, int on)
{
    if (!c) return VLASOV_EINVAL;
    c->timers_on = on != 0;
    return VLASOV_OK;
}

extern "C" int vlasov_read_timers(vlasov_ctx *c, double *ms, long long *launches, int nkinds)
{
    if (!c || nkinds < 0) return VLASOV_EINVAL;
    VK_SETTLE(c);
    VK_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto &p : c->pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) c->acc_ms[p.kind] += t;
        c->pool.push_back(p.a);
        c->pool.push_back(p.b);
    }
    c->pending.clear();
    for (int k = 0; k < nkinds && k < VLASOV_T_KINDS; ++k) {
        if (ms) ms[k] = c->acc_ms[k];
        if (launches) launches[k] = c->launches[k];
    }
    for (int k = 0; k < VLASOV_T_KINDS; ++k) { c->acc_ms[k] = 0.0; c->launches[k] = 0; }
    return VLASOV_OK;
}

extern "C" int vlasov_set_stream(vlasov_ctx *c, void *stream)
{
    if (!c) return VLASOV_EINVAL;
    c->stream = (cudaStream_t)stream;
    return VLASOV_OK;
}

extern "C" int vlasov_set_f(vlasov_ctx *c, void *f_dev, float *scale_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    if (!f_dev || reinterpret_cast<uintptr_t>(f_dev) % 16) return fail(c, VLASOV_EINVAL, "vlasov_set_f: f_dev must be 16-byte aligned");
    const bool coded = c->g.dtype == VLASOV_BF16 || c->g.dtype == VLASOV_F16;
    if (coded != (scale_dev != nullptr) || (scale_dev && reinterpret_cast<uintptr_t>(scale_dev) % 16))
        return fail(c, VLASOV_EINVAL, "vlasov_set_f: scale_dev must be a 16-byte aligned array exactly for 16-bit storage");
    if (f_dev == c->f && scale_dev == c->scale) return VLASOV_OK;
    c->f = f_dev;
    c->scale = scale_dev;
    return plan_axes(c); // re-encode the tensor maps for the new arrays
}

template <typename C> static void fill_stream_args(StreamArgs<C> &A, const vlasov_ctx *c, int ax)
{
    const AxisPlan &p = c->splan[ax];
    A.L = p.L; A.W = p.W; A.P = p.P; A.R = c->splan_R[ax]; A.stages = p.stages;
    A.tiles_inner = p.tiles_inner; A.periodic = ax < 3; A.perm_line = c->perm_line[ax];
    A.n_inner = p.n_inner; A.n_outer = p.n_outer; A.num_blocks = p.num_tiles;
    A.tile0 = 0;
    if (c->slab_x1 > c->slab_x0) {
        // the x-planes [slab_x0, slab_x1) are whole tiles (vlasov_step_host checks)
        A.tile0 = c->slab_x0 * c->splan_tpp[ax];
        A.num_blocks = (c->slab_x1 - c->slab_x0) * c->splan_tpp[ax];
    }
    A.err = c->d_err;
    A.scale = c->scale;
    A.nuz = c->g.nuz;
    A.seed = c->sweeps;
    A.scale_rank = c->scale_rank[ax];
    A.swidth = c->swidth[ax];
}

// Tensor maps of one plan for a sweep that reads src and writes dst (both
// arrays of c's shape; the plan's own map where one is c->f).
struct SweepMaps {
    CUtensorMap in, out;
};

static int sweep_maps(vlasov_ctx *c, const CUtensorMap &own, const MapSpec &spec, const void *src, void *dst,
                      SweepMaps &m)
{
    if (src == c->f) m.in = own;
    else if (encode_spec(&m.in, spec, src) != CUDA_SUCCESS) return fail(c, VLASOV_ECUDA, "tensor map of a sweep input failed");
    if (dst == c->f) m.out = own;
    else if (encode_spec(&m.out, spec, dst) != CUDA_SUCCESS) return fail(c, VLASOV_ECUDA, "tensor map of a sweep output failed");
    return VLASOV_OK;
}

// streamed launch for the storage type of c (the arguments use FP32 constants unless FP64)
// persistent grid of a streamed launch: no more CTAs than tiles
static int stream_grid(const vlasov_ctx *c, int ax, long long tiles)
{
    const int g = c->splan[ax].grid;
    return int(tiles < g ? tiles : g);
}

static cudaError_t launch_stream_any(const vlasov_ctx *c, int ax, const StreamArgs<float> &A, const SweepMaps &m)
{
    const AxisPlan &sp = c->splan[ax];
    const int grid = stream_grid(c, ax, A.num_blocks);
    if (grid <= 0) return cudaSuccess;
    switch (c->g.dtype) {
    case VLASOV_BF16: return launch_stream_bf16(sp.map, c->smap[ax], A, grid, sp.smem, c->stream);
    case VLASOV_F16: return launch_stream_f16(sp.map, c->smap[ax], A, grid, sp.smem, c->stream);
    default: return launch_stream_f32(m.in, m.out, A, grid, sp.smem, c->stream);
    }
}

static bool coded(const vlasov_ctx *c) { return c->g.dtype == VLASOV_BF16 || c->g.dtype == VLASOV_F16; }

static long long velocity_cube(const vlasov_ctx *c) { return (long long)c->g.nux * c->g.nuy * c->g.nuz; }

// Partial sums per spatial cell of the moment fused into the x sweep: one per block
// (W columns) of the velocity cube.
static int moment_parts(const vlasov_ctx *c) { return int(velocity_cube(c) / c->splan[0].W); }

// Can the streamed x sweep sum its output rows into the velocity moment?  Its
// moment warp sums chunks of 4 rows x W values (32 bytes a lane), which must lie
// in one spatial cell's velocity cube (W | cube, one plane per block); the partial
// sums need ncell x cube / W values.
// The per-cell partial sums of the fused moment (ncell x cube / W values of the storage
// type, W = the 1-KB blocks of the x sweep), allocated on first use.
static bool moment_buffer(vlasov_ctx *c)
{
    if (!c->d_mpart) {
        if (cudaMalloc(&c->d_mpart, (size_t)c->es * c->ncell * (velocity_cube(c) * c->es / 1024)) != cudaSuccess) {
            cudaGetLastError();
            c->d_mpart = nullptr;
            c->fuse_moment = false; // no room: the separate moment kernel from here on
            return false;
        }
    }
    return true;
}

static bool fused_moment_ok(vlasov_ctx *c, int ax)
{
    if (ax != 0 || !c->fuse_moment || coded(c)) return false;
    const AxisPlan &sp = c->splan[0];
    const long long cube = velocity_cube(c);
    if (sp.P != 1 || c->splan_R[0] != 4 || (long long)sp.W * c->es != 1024 || cube % sp.W) return false;
    return moment_buffer(c);
}

// position sweep from src to dst (NULL, NULL: c->f in place) with per-velocity-column
// constants from nu_j = u_j dt / (a^2 dx).  With rho_fused (x sweep only) the sweep
// also writes the velocity moment of its output to rho_fused when it can, and then
// sets *fused.
static int run_position(vlasov_ctx *c, int ax, double dt, double a, const void *src = nullptr, void *dst = nullptr,
                        double *rho_fused = nullptr, bool *fused = nullptr)
{
    ++c->sweeps;
    if (!src) src = c->f;
    if (!dst) dst = c->f;
    if (!(a > 0) || !isfinite(dt) || !isfinite(a)) return fail(c, VLASOV_EINVAL, "sweep %d: need finite dt and a > 0", ax);
    if (coded(c) && (src != c->f || dst != c->f)) return fail(c, VLASOV_EINVAL, "16-bit storage sweeps in place only");
    const AxisPlan &p = c->plan[ax];
    const int nvel = (&c->g.nux)[ax];
    const double du = 2.0 * c->g.V / nvel;
    const double dx = c->g.L / (&c->g.nx)[ax];
    long long vstride = 1;
    for (int k = ax + 1; k < 3; ++k) vstride *= (&c->g.nux)[k];
    double numax = 0.0;
    for (int j = 0; j < nvel; ++j) numax = fmax(numax, fabs((-c->g.V + (j + 0.5) * du) * dt / (a * a * dx)));
    SweepMaps m;
    int rc;
    if (numax < 1.0 && c->use_tiles && c->tile_ok[ax]) {
        // no whole-cell shift: whole lines staged per tile
        TileArgs A{};
        A.L = (&c->g.nx)[ax];
        A.n_inner = c->ttiles_inner[ax] * 256;
        A.n_outer = c->tn_outer[ax];
        A.tiles_inner = c->ttiles_inner[ax];
        A.tile0 = 0;
        A.num_tiles = A.n_outer * A.tiles_inner;
        if (c->slab_x1 > c->slab_x0) {
            const long long tpp = A.num_tiles / c->g.nx; // tiles per x-plane (y and z sweeps)
            A.tile0 = c->slab_x0 * tpp;
            A.num_tiles = (c->slab_x1 - c->slab_x0) * tpp;
        }
        A.vstride = vstride;
        A.nvel = nvel;
        A.nuz = int(c->g.nuz);
        A.zperm = ax == 2 && c->g.nuz == 32;
        // Tiles have one sign of u when its runs (vstride nvel / 2 columns: u_j < 0 exactly for
        // j < nvel / 2) are whole tiles; the march then takes a fixed direction per tile (D_x,
        // D_y: every thread of a tile the same), as it does per warp in the z sweep, whose
        // warps hold the columns of one sign of u_z.  Both unrolled bodies run side by side on
        // an SM (lines of more than 32 cells march in blocks of 8 faces, which fit the
        // instruction cache).  Otherwise the direction is taken per column at run time.
        const long long run = vstride * nvel / 2;
        const int grid = int(A.num_tiles < c->tgrid[ax] ? A.num_tiles : c->tgrid[ax]);
        A.tile_sign = A.zperm || (nvel % 2 == 0 && run % 256 == 0);
        A.err = c->d_err;
        A.seed = c->sweeps;
        for (int j = 0; j < nvel; ++j) A.table[j] = make_line_coef<float>((-c->g.V + (j + 0.5) * du) * dt / (a * a * dx));
        const long long cube = velocity_cube(c);
        const bool fm = rho_fused && ax == 0 && !coded(c) && c->fuse_moment && cube % 256 == 0 && moment_buffer(c);
        if (fm) { A.mpart = c->d_mpart; A.cube = cube; A.nparts = int(cube / 256); }
        if (coded(c)) m.in = m.out = c->tmap[ax]; // 16-bit sweeps run in place (checked above)
        else if ((rc = sweep_maps(c, c->tmap[ax], c->tspec[ax], src, dst, m))) return rc;
        cudaError_t e;
        {
            PartTimer t(c, ax, 1);
            e = launch_tile_sweep(m.in, m.out, c->tsmap[ax], A, c->g.dtype, grid, c->stream);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "position sweep launch");
        if (fm) {
            const double du3 = (2.0 * c->g.V / c->g.nux) * (2.0 * c->g.V / c->g.nuy) * (2.0 * c->g.V / c->g.nuz);
            PartTimer t(c, VLASOV_T_MOMENT, 1);
            e = launch_moment_finish(c->d_mpart, 1, int(cube / 256), c->g.nx, c->ncell / c->g.nx, du3, rho_fused,
                                     c->stream, c->sm_count);
            if (e != cudaSuccess) return cuda_fail(c, e, "moment launch");
            if (fused) *fused = true;
        }
        return VLASOV_OK;
    }
    if (numax < 1.0) {
        // no whole-cell shift on any line: streamed sweep
        const AxisPlan &sp = c->splan[ax];
        if (!coded(c) && (rc = sweep_maps(c, sp.map, sp.spec, src, dst, m))) return rc;
        const bool fm = rho_fused && fused_moment_ok(c, ax);
        const long long cube = velocity_cube(c);
        cudaError_t e;
        if (c->g.dtype == VLASOV_F64) {
            StreamArgs<double> A{};
            fill_stream_args(A, c, ax);
            A.vstride = vstride; A.nvel = nvel; A.coef_mode = 0; A.outer_per_cell = 1; A.cell_coef = nullptr;
            for (int j = 0; j < nvel; ++j) A.table[j] = make_line_coef<double>((-c->g.V + (j + 0.5) * du) * dt / (a * a * dx));
            if (fm) { A.mpart = c->d_mpart; A.cube = cube; A.nparts = moment_parts(c); }
            PartTimer t(c, ax, 1);
            e = A.num_blocks > 0 ? launch_stream_f64(m.in, m.out, A, stream_grid(c, ax, A.num_blocks), sp.smem, c->stream) : cudaSuccess;
        } else {
            StreamArgs<float> A{};
            fill_stream_args(A, c, ax);
            A.vstride = vstride; A.nvel = nvel; A.coef_mode = 0; A.outer_per_cell = 1; A.cell_coef = nullptr;
            for (int j = 0; j < nvel; ++j) A.table[j] = make_line_coef<float>((-c->g.V + (j + 0.5) * du) * dt / (a * a * dx));
            if (fm) { A.mpart = c->d_mpart; A.cube = cube; A.nparts = moment_parts(c); }
            PartTimer t(c, ax, 1);
            e = launch_stream_any(c, ax, A, m);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "position sweep launch");
        if (fm) {
            const double du3 = (2.0 * c->g.V / c->g.nux) * (2.0 * c->g.V / c->g.nuy) * (2.0 * c->g.V / c->g.nuz);
            PartTimer t(c, VLASOV_T_MOMENT, 1);
            e = launch_moment_finish(c->d_mpart, c->g.dtype == VLASOV_F64 ? 0 : 1, moment_parts(c), c->g.nx,
                                     c->ncell / c->g.nx, du3, rho_fused, c->stream, c->sm_count);
            if (e != cudaSuccess) return cuda_fail(c, e, "moment launch");
            if (fused) *fused = true;
        }
        return VLASOV_OK;
    }
    if (coded(c)) return fail(c, VLASOV_EINVAL, "sweep %d: |nu| = %.3g >= 1 needs FP32 or FP64 storage", ax, numax);
    if (c->slab_x1 > c->slab_x0) return fail(c, VLASOV_EINVAL, "sweep %d: a whole-cell shift cannot run on an x-slab", ax);
    if ((rc = sweep_maps(c, p.map, p.spec, src, dst, m))) return rc;
    cudaError_t e;
    if (c->g.dtype == VLASOV_F64) {
        StridedArgs<double> A{};
        A.L = p.L; A.W = p.W; A.P = p.P; A.stages = p.stages; A.tiles_inner = p.tiles_inner; A.periodic = 1;
        A.n_inner = p.n_inner; A.n_outer = p.n_outer; A.num_tiles = p.num_tiles;
        A.vstride = vstride; A.nvel = nvel; A.coef_mode = 0; A.outer_per_cell = 1; A.cell_coef = nullptr;
        A.err = c->d_err;
        for (int j = 0; j < nvel; ++j) A.table[j] = make_line_coef<double>((-c->g.V + (j + 0.5) * du) * dt / (a * a * dx));
        PartTimer t(c, ax, 1);
        e = launch_strided_f64(m.in, m.out, A, p.grid, p.smem, c->stream);
    } else {
        StridedArgs<float> A{};
        A.L = p.L; A.W = p.W; A.P = p.P; A.stages = p.stages; A.tiles_inner = p.tiles_inner; A.periodic = 1;
        A.n_inner = p.n_inner; A.n_outer = p.n_outer; A.num_tiles = p.num_tiles;
        A.vstride = vstride; A.nvel = nvel; A.coef_mode = 0; A.outer_per_cell = 1; A.cell_coef = nullptr;
        A.err = c->d_err;
        for (int j = 0; j < nvel; ++j) A.table[j] = make_line_coef<float>((-c->g.V + (j + 0.5) * du) * dt / (a * a * dx));
        PartTimer t(c, ax, 1);
        e = launch_strided_f32(m.in, m.out, A, p.grid, p.smem, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "position sweep launch");
    return VLASOV_OK;
}

// the u_z line kernel's tiles of the current x-slab (all tiles when none is set)
static void line_slab(const vlasov_ctx *c, ContigArgs<float> &A)
{
    A.tile0 = 0;
    if (c->slab_x1 > c->slab_x0) {
        A.tile0 = c->slab_x0 * c->ltpp;
        A.num_tiles = (c->slab_x1 - c->slab_x0) * c->ltpp;
    }
}

static int line_grid(const vlasov_ctx *, int grid, long long tiles) { return int(tiles < grid ? tiles : grid); }

// u_x / u_y on FP32 or 16-bit storage with lines of 16, 32 or 48 cells: the register-line
// kernel, unless the u_x staged tiles take the sweep (run_tile_ux)
static bool use_reg_lines(const vlasov_ctx *c, int ax)
{
    if (c->g.dtype == VLASOV_F64 || (ax != 3 && ax != 4)) return false;
    const int L = (&c->g.nux)[ax - 3];
    // FP32 u_x lines of 48 cells stream faster (48^3 x 48^3: 20.7 ms against 22.3 in registers;
    // u_y 23.8 streamed against 22.0, BF16 u_x 29.6 / 28.6 and u_y 33.7 / 27.8; on staged
    // tiles u_x takes 16.6 ms in FP32 and 21.8 ms in BF16)
    if (L == 48 && ax == 3 && c->g.dtype == VLASOV_F32) return false;
    return reg_lines_supported(L);
}

// the u_x sweep on staged tiles of [cell][u_x][u_y u_z] (zero-flux lines; each tile's
// columns take the coefficients of its cell)
static int run_tile_ux(vlasov_ctx *c, const void *src, void *dst)
{
    TileArgs A{};
    A.L = int(c->g.nux);
    A.n_inner = c->ttiles_inner[3] * 256;
    A.n_outer = c->tn_outer[3];
    A.tiles_inner = c->ttiles_inner[3];
    A.tile0 = 0;
    A.num_tiles = A.n_outer * A.tiles_inner;
    if (c->slab_x1 > c->slab_x0) {
        const long long tpp = A.num_tiles / c->g.nx; // tiles per x-plane
        A.tile0 = c->slab_x0 * tpp;
        A.num_tiles = (c->slab_x1 - c->slab_x0) * tpp;
    }
    if (A.num_tiles <= 0) return VLASOV_OK;
    A.vstride = 1;
    A.nvel = 0;
    A.nuz = int(c->g.nuz);
    A.tile_sign = 1;
    A.err = c->d_err;
    A.seed = c->sweeps;
    A.cell_coef = (const LineCoefT<float> *)c->d_coef[0];
    SweepMaps m;
    int rc;
    if (coded(c)) m.in = m.out = c->tmap[3]; // in place (checked by the caller)
    else if ((rc = sweep_maps(c, c->tmap[3], c->tspec[3], src, dst, m))) return rc;
    const int grid = int(A.num_tiles < c->tgrid[3] ? A.num_tiles : c->tgrid[3]);
    PartTimer t(c, 3, 1);
    const cudaError_t e = launch_tile_sweep(m.in, m.out, c->tsmap[3], A, c->g.dtype, grid, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "u_x tile sweep launch");
    return VLASOV_OK;
}

// velocity sweep from src to dst (NULL, NULL: c->f in place) with the per-cell
// constants already in d_coef[ax - 3]
static int run_velocity(vlasov_ctx *c, int ax, const void *src = nullptr, void *dst = nullptr)
{
    ++c->sweeps;
    if (!src) src = c->f;
    if (!dst) dst = c->f;
    if (coded(c) && (src != c->f || dst != c->f)) return fail(c, VLASOV_EINVAL, "16-bit storage sweeps in place only");
    if (ax == 3 && c->use_tiles && c->tile_ok[3]) return run_tile_ux(c, src, dst);
    const AxisPlan &p = c->plan[ax];
    const void *coef = c->d_coef[ax - 3];
    SweepMaps m;
    int rc;
    cudaError_t e;
    if (ax < 5 && use_reg_lines(c, ax)) {
        const AxisPlan &sp = c->splan[ax];
        RegLineArgs A{};
        A.L = sp.L; A.n_inner = sp.n_inner; A.n_outer = sp.n_outer; A.outer_per_cell = sp.n_outer / c->ncell;
        A.cell_coef = (const LineCoefT<float> *)coef; A.err = c->d_err;
        A.line0 = 0; A.nlines = sp.n_outer * sp.n_inner;
        if (c->slab_x1 > c->slab_x0) {
            const long long lpp = sp.n_outer / c->g.nx * sp.n_inner; // lines per x-plane
            A.line0 = c->slab_x0 * lpp;
            A.nlines = (c->slab_x1 - c->slab_x0) * lpp;
        }
        A.scale = c->scale; A.nuz = int(c->g.nuz); A.seed = c->sweeps;
        PartTimer t(c, ax, 1);
        e = launch_reg_lines(src, dst, A, c->g.dtype, c->stream);
    } else if (ax < 5) {
        const AxisPlan &sp = c->splan[ax];
        if (!coded(c) && (rc = sweep_maps(c, sp.map, sp.spec, src, dst, m))) return rc;
        const long long opc = sp.n_outer / c->ncell;
        PartTimer t(c, ax, 1);
        if (c->g.dtype == VLASOV_F64) {
            StreamArgs<double> A{};
            fill_stream_args(A, c, ax);
            A.vstride = 1; A.nvel = 0; A.coef_mode = 1; A.outer_per_cell = opc;
            A.cell_coef = (const LineCoefT<double> *)coef;
            e = A.num_blocks > 0 ? launch_stream_f64(m.in, m.out, A, stream_grid(c, ax, A.num_blocks), sp.smem, c->stream) : cudaSuccess;
        } else {
            StreamArgs<float> A{};
            fill_stream_args(A, c, ax);
            A.vstride = 1; A.nvel = 0; A.coef_mode = 1; A.outer_per_cell = opc;
            A.cell_coef = (const LineCoefT<float> *)coef;
            e = launch_stream_any(c, ax, A, m);
        }
    } else if (c->use_lines) {
        if ((rc = sweep_maps(c, c->lmap, c->lspec, src, dst, m))) return rc;
        ContigArgs<float> A{};
        A.L = c->g.nuz; A.R = line_sweep_rows_per_tile(); A.stages = 0; A.rows = c->lrows; A.num_tiles = c->ltiles;
        A.rows_per_cell = (long long)c->g.nux * c->g.nuy; A.cell_coef = (const LineCoefT<float> *)coef; A.err = c->d_err;
        A.scale = c->scale;
        A.seed = c->sweeps;
        line_slab(c, A);
        PartTimer t(c, ax, 1);
        e = A.num_tiles > 0 ? launch_line_sweep(m.in, m.out, A, c->g.nuz, c->g.dtype, line_grid(c, c->lgrid, A.num_tiles), c->stream)
                            : cudaSuccess;
    } else if (rows_sweep_supported(int(c->g.nuz), c->g.dtype)) {
        RowsArgs A{};
        A.L = int(c->g.nuz);
        A.rows_per_cell = (long long)c->g.nux * c->g.nuy;
        A.row0 = 0;
        A.nrows = c->ncell * A.rows_per_cell;
        if (c->slab_x1 > c->slab_x0) {
            const long long rpp = A.nrows / c->g.nx; // rows per x-plane
            A.row0 = c->slab_x0 * rpp;
            A.nrows = (c->slab_x1 - c->slab_x0) * rpp;
        }
        A.cell_coef = coef;
        A.err = c->d_err;
        A.scale = c->scale;
        A.seed = c->sweeps;
        PartTimer t(c, ax, 1);
        e = launch_rows_sweep(src, dst, A, c->g.dtype, c->stream);
    } else {
        if (c->slab_x1 > c->slab_x0) return fail(c, VLASOV_EINVAL, "u_z sweep: the transposing kernel cannot run on an x-slab");
        if ((rc = sweep_maps(c, p.map, p.spec, src, dst, m))) return rc;
        const long long rpc = (long long)c->g.nux * c->g.nuy;
        PartTimer t(c, ax, 1);
        if (c->g.dtype == VLASOV_F64) {
            ContigArgs<double> A{};
            A.L = p.L; A.R = kConsumers; A.stages = p.stages; A.rows = p.n_outer; A.num_tiles = p.num_tiles;
            A.rows_per_cell = rpc; A.cell_coef = (const LineCoefT<double> *)coef; A.err = c->d_err;
            e = launch_contig_f64(m.in, m.out, A, p.grid, p.smem, c->stream);
        } else {
            ContigArgs<float> A{};
            A.L = p.L; A.R = kConsumers; A.stages = p.stages; A.rows = p.n_outer; A.num_tiles = p.num_tiles;
            A.rows_per_cell = rpc; A.cell_coef = (const LineCoefT<float> *)coef; A.err = c->d_err;
            e = launch_contig_f32(m.in, m.out, A, p.grid, p.smem, c->stream);
        }
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "velocity sweep launch");
    return VLASOV_OK;
}

static int prep_velocity(vlasov_ctx *c, const float *phi, double dt, int mask)
{
    if (!phi) return fail(c, VLASOV_EINVAL, "velocity sweeps need phi_dev");
    if (!isfinite(dt)) return fail(c, VLASOV_EINVAL, "dt must be finite");
    PartTimer t(c, VLASOV_T_COEF, 1);
    const cudaError_t e = launch_velocity_coef(c->gd, phi, dt, mask, c->d_coef[0], c->d_coef[1], c->d_coef[2],
                                               c->g.dtype == VLASOV_F64 ? 0 : 1, c->d_err, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "velocity coefficient launch");
    return VLASOV_OK;
}

extern "C" int vlasov_sweep(vlasov_ctx *c, int axis, double dt, double a, const float *phi_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    if (axis < 0 || axis > 5) return fail(c, VLASOV_EINVAL, "axis %d outside 0..5", axis);
    if (axis < 3) return run_position(c, axis, dt, a);
    int rc = prep_velocity(c, phi_dev, dt, 1 << (axis - 3));
    if (rc) return rc;
    return run_velocity(c, axis);
}

extern "C" int vlasov_moment(vlasov_ctx *c, double *rho_dev, double *mass_host)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    if (!rho_dev) return fail(c, VLASOV_EINVAL, "rho_dev is NULL");
    cudaError_t e;
    {
        PartTimer t(c, VLASOV_T_MOMENT, 1);
        if (c->scale)
            e = launch_moment_coded(c->gd, c->f, c->scale, c->g.dtype, rho_dev, c->stream, c->sm_count);
        else
            e = launch_moment(c->gd, c->f, c->g.dtype == VLASOV_F64 ? 0 : 1, rho_dev, c->stream, c->sm_count);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "moment launch");
    if (mass_host) {
        {
            PartTimer t(c, VLASOV_T_MASS, 1);
            e = launch_mass(c->gd, rho_dev, c->d_mass, c->stream);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "mass launch");
        VK_CUDA(c, cudaMemcpyAsync(mass_host, c->d_mass, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        VK_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return VLASOV_OK;
}

extern "C" int vlasov_moments(vlasov_ctx *c, double *rho_dev, double *umean_dev, double *sigma2_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    if (!rho_dev && !umean_dev && !sigma2_dev) return fail(c, VLASOV_EINVAL, "vlasov_moments: no output");
    PartTimer t(c, VLASOV_T_MOMENTS, 1);
    const cudaError_t e = launch_moments(c->gd, c->f, c->scale, c->g.dtype, rho_dev, umean_dev, sigma2_dev, c->stream,
                                         c->sm_count);
    if (e != cudaSuccess) return cuda_fail(c, e, "moments launch");
    return VLASOV_OK;
}

extern "C" int vlasov_poisson(vlasov_ctx *c, const double *rho_dev, const double *rho_bg_dev, double a,
                              double four_pi_G, float *phi_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    if (!rho_dev || !phi_dev) return fail(c, VLASOV_EINVAL, "vlasov_poisson: null rho or phi");
    if (!isfinite(a) || !isfinite(four_pi_G)) return fail(c, VLASOV_EINVAL, "vlasov_poisson: a and four_pi_G must be finite");
    PartTimer t(c, VLASOV_T_POISSON, 9);
    const cudaError_t e = launch_poisson(c->gd, c->ps, rho_dev, rho_bg_dev, a, four_pi_G, phi_dev, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "poisson launch");
    return VLASOV_OK;
}

// D_uz D_uy in one pass of the u_z line kernel (constants in d_coef[1], d_coef[2])
static int run_kick_tail(vlasov_ctx *c)
{
    c->sweeps += 2;
    ContigArgs<float> A{};
    A.L = c->g.nuz; A.R = line_sweep_rows_per_tile(); A.stages = 0; A.rows = c->lrows; A.num_tiles = c->ltiles;
    A.rows_per_cell = (long long)c->g.nux * c->g.nuy; A.err = c->d_err;
    A.cell_coef = (const LineCoefT<float> *)c->d_coef[2];
    A.cell_coef_y = (const LineCoefT<float> *)c->d_coef[1];
    A.scale = c->scale;
    A.seed = c->sweeps; // the stochastic-rounding stream of the D_uz encode (16-bit storage)
    line_slab(c, A);
    if (A.num_tiles <= 0) return VLASOV_OK;
    PartTimer t(c, VLASOV_T_SWEEP_UYUZ, 1);
    const cudaError_t e = launch_line_sweep(c->lmap, c->lmap, A, c->g.nuz, c->g.dtype,
                                            line_grid(c, c->lgrid_fused, A.num_tiles), c->stream, true);
    if (e != cudaSuccess) return cuda_fail(c, e, "fused kick launch");
    return VLASOV_OK;
}

// D_uz D_uy D_ux in one pass over each cell's velocity cube (constants in d_coef)
// D_uz D_uy (constants in d_coef[1], d_coef[2]) in one pass over staged planes
static int run_plane_tail(vlasov_ctx *c)
{
    c->sweeps += 2;
    PlaneTailArgs A{};
    A.nux = c->g.nux;
    A.plane0 = 0;
    A.nplanes = c->ncell * c->g.nux;
    if (c->slab_x1 > c->slab_x0) {
        const long long cpp = c->ncell / c->g.nx; // spatial cells per x-plane
        A.plane0 = c->slab_x0 * cpp * c->g.nux;
        A.nplanes = (c->slab_x1 - c->slab_x0) * cpp * c->g.nux;
    }
    A.coef_y = (const LineCoefT<float> *)c->d_coef[1];
    A.coef_z = (const LineCoefT<float> *)c->d_coef[2];
    A.err = c->d_err;
    A.scale = c->scale;
    A.seed = c->sweeps; // the stochastic-rounding stream of the D_uz encode (16-bit storage)
    if (A.nplanes <= 0) return VLASOV_OK;
    PartTimer t(c, VLASOV_T_SWEEP_UYUZ, 1);
    const cudaError_t e = launch_plane_tail(c->f, A, c->g.nuz, c->g.dtype, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "kick tail launch");
    return VLASOV_OK;
}

static int run_kick_cube(vlasov_ctx *c)
{
    KickArgs A{};
    A.seed_x = c->sweeps + 1; // the streams the separate u_x and fused u_y u_z kernels would draw
    A.seed_z = c->sweeps + 3;
    c->sweeps += 3;
    A.coef_x = (const LineCoefT<float> *)c->d_coef[0];
    A.coef_y = (const LineCoefT<float> *)c->d_coef[1];
    A.coef_z = (const LineCoefT<float> *)c->d_coef[2];
    A.err = c->d_err;
    A.cell0 = 0;
    A.ncells = c->ncell;
    if (c->slab_x1 > c->slab_x0) {
        const long long cpp = c->ncell / c->g.nx; // spatial cells per x-plane
        A.cell0 = c->slab_x0 * cpp;
        A.ncells = (c->slab_x1 - c->slab_x0) * cpp;
    }
    if (A.ncells <= 0) return VLASOV_OK;
    PartTimer t(c, VLASOV_T_KICK, 1);
    const int grid = int(A.ncells < c->kgrid ? A.ncells : c->kgrid);
    const cudaError_t e = launch_kick_cube(c->kmap, c->ksmap, A, c->g.nuz, c->g.dtype, grid, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "one-pass kick launch");
    return VLASOV_OK;
}

// one kick D_uz D_uy D_ux (constants already in d_coef), in place
static int run_kick(vlasov_ctx *c)
{
    int rc;
    if (c->can_kick_cube && c->fuse_kick >= 2) return run_kick_cube(c);
    if ((rc = run_velocity(c, 3))) return rc;
    if (c->can_fuse_kick && c->fuse_kick >= 1) return run_kick_tail(c);
    if (c->can_plane_tail && c->fuse_kick >= 1) return run_plane_tail(c);
    if ((rc = run_velocity(c, 4))) return rc;
    return run_velocity(c, 5);
}

extern "C" int vlasov_set_fused_kick(vlasov_ctx *c, int mode)
{
    if (!c) return VLASOV_EINVAL;
    if (mode < 0 || mode > 2) return fail(c, VLASOV_EINVAL, "vlasov_set_fused_kick: mode %d is not 0, 1 or 2", mode);
    c->fuse_kick = mode;
    return VLASOV_OK;
}

extern "C" int vlasov_kick(vlasov_ctx *c, double dt, const float *phi_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    int rc = prep_velocity(c, phi_dev, dt, 7);
    if (rc) return rc;
    return run_kick(c);
}

extern "C" int vlasov_set_position_tiles(vlasov_ctx *c, int on)
{
    if (!c) return VLASOV_EINVAL;
    c->use_tiles = on != 0;
    return VLASOV_OK;
}

extern "C" int vlasov_set_fused_moment(vlasov_ctx *c, int on)
{
    if (!c) return VLASOV_EINVAL;
    c->fuse_moment = on != 0;
    return VLASOV_OK;
}

extern "C" int vlasov_step(vlasov_ctx *c, double dt, double a_half, double a_full, const float *phi_n_dev,
                           const double *rho_bg_dev, double four_pi_G, float *phi_next_dev, double *rho_nu_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    if (!phi_n_dev) return fail(c, VLASOV_EINVAL, "vlasov_step: phi_n_dev is NULL");
    int rc;
    // kick D_uz D_uy D_ux (dt/2), D_ux first
    if ((rc = prep_velocity(c, phi_n_dev, 0.5 * dt, 7))) return rc;
    if ((rc = run_kick(c))) return rc;
    // drift D_x D_y D_z (dt), D_z first, at the mid-step scale factor; the x sweep
    // writes the moment when it can
    double *rho = rho_nu_dev ? rho_nu_dev : c->d_rho;
    const bool need_rho = rho_nu_dev || phi_next_dev;
    bool have_rho = false;
    for (int ax = 2; ax >= 0; --ax)
        if ((rc = run_position(c, ax, dt, a_half, nullptr, nullptr, ax == 0 && need_rho ? rho : nullptr, &have_rho)))
            return rc;
    if (need_rho && !have_rho)
        if ((rc = vlasov_moment(c, rho, nullptr))) return rc;
    if (phi_next_dev) {
        if ((rc = vlasov_poisson(c, rho, rho_bg_dev, a_full, four_pi_G, phi_next_dev))) return rc;
        if ((rc = prep_velocity(c, phi_next_dev, 0.5 * dt, 7))) return rc;
    }
    // second kick (the constants are unchanged when phi is)
    return run_kick(c);
}

// ----------------------------------------------------------------------------
// one step from and to a host buffer, transfers overlapped with the cell-local sweeps
// ----------------------------------------------------------------------------
// Largest |Courant number| of a position sweep (the streamed kernel needs < 1)
static double position_numax(const vlasov_ctx *c, int ax, double dt, double a)
{
    const int nvel = (&c->g.nux)[ax];
    const double du = 2.0 * c->g.V / nvel, dx = c->g.L / (&c->g.nx)[ax];
    double m = 0.0;
    for (int j = 0; j < nvel; ++j) m = fmax(m, fabs((-c->g.V + (j + 0.5) * du) * dt / (a * a * dx)));
    return m;
}

// x-slabs for the pipeline (0: the step cannot be split): every cell-local sweep
// (the kicks, D_z, D_y) must run on whole tiles of each slab
static int slab_count(const vlasov_ctx *c, double dt, double a_half)
{
    if (coded(c)) return 0; // the 16-bit encodes draw per-sweep random streams
    const bool cube = c->can_kick_cube && c->fuse_kick >= 2; // whole cubes: any x-slab
    const bool fused = c->can_fuse_kick && c->fuse_kick >= 1;
    const bool rows = rows_sweep_supported(int(c->g.nuz), c->g.dtype);
    if (!cube) {
        if (!rows && (!c->use_lines || c->ltpp <= 0)) return 0;
        if ((!use_reg_lines(c, 3) && c->splan_tpp[3] <= 0) || (!fused && !use_reg_lines(c, 4) && c->splan_tpp[4] <= 0))
            return 0;
    }
    for (int ax = 1; ax <= 2; ++ax)
        if (c->splan_tpp[ax] <= 0 || !(position_numax(c, ax, dt, a_half) < 1.0)) return 0;
    for (int sl = kMaxSlabs; sl >= 2; --sl)
        if (c->g.nx % sl == 0) return sl;
    return 0;
}

extern "C" int vlasov_step_host(vlasov_ctx *c, void *f_host, double dt, double a_half, double a_full,
                                const float *phi_n_dev, const double *rho_bg_dev, double four_pi_G,
                                float *phi_next_dev, double *rho_nu_dev)
{
    if (!c) return VLASOV_EINVAL;
    if (!f_host) return fail(c, VLASOV_EINVAL, "vlasov_step_host: null host buffer");
    if (!phi_n_dev) return fail(c, VLASOV_EINVAL, "vlasov_step_host: phi_n_dev is NULL");
    if (!(a_half > 0) || !isfinite(dt) || !isfinite(a_half)) return fail(c, VLASOV_EINVAL, "vlasov_step_host: need finite dt and a_half > 0");
    int rc;
    const int S = slab_count(c, dt, a_half);
    if (S == 0) {
        // not splittable: the three calls in sequence
        if ((rc = vlasov_upload(c, f_host))) return rc;
        if ((rc = vlasov_step(c, dt, a_half, a_full, phi_n_dev, rho_bg_dev, four_pi_G, phi_next_dev, rho_nu_dev))) return rc;
        return vlasov_download(c, f_host);
    }
    for (cudaStream_t *st : {&c->copy_stream, &c->down_stream}) {
        if (!*st && cudaStreamCreateWithFlags(st, cudaStreamNonBlocking) != cudaSuccess) {
            *st = nullptr;
            return fail(c, VLASOV_ECUDA, "vlasov_step_host: copy stream");
        }
    }
    if (!c->slab_ev_ok) {
        for (auto &e : c->slab_ev) VK_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (auto &e : c->down_ev) VK_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->slab_ev_ok = true;
    }
    cudaEvent_t *up = c->slab_ev, *ready = c->slab_ev + kMaxSlabs;
    cudaEvent_t start = c->slab_ev[2 * kMaxSlabs];
    const int planes = c->g.nx / S;
    const size_t plane_bytes = f_bytes(c) / c->g.nx, slab_bytes = plane_bytes * planes;
    unsigned char *fd = static_cast<unsigned char *>(c->f), *fh = static_cast<unsigned char *>(f_host);
    auto on_slab = [&](int sl) { c->slab_x0 = sl * planes; c->slab_x1 = (sl + 1) * planes; };
    auto all = [&]() { c->slab_x0 = c->slab_x1 = 0; };
    // Downloads of the previous call still in flight on the same slabs: each upload
    // waits for the download of its own slab only (the device slab it overwrites, the
    // host slab it reads), so this step's uploads run beside the previous step's
    // downloads, one direction each.  Otherwise the context stream waits for them all.
    // (The context stream reaches D_x only after every upload, so the later library
    // calls of this step, which wait for all of those downloads, wait for nothing.)
    const bool chain = c->pending_slabs == S && c->pending_slab_bytes == slab_bytes;
    if (!chain) VK_SETTLE(c);
    struct Reset { // whatever way this function returns, later calls see the whole grid
        vlasov_ctx *c;
        bool done;
        ~Reset()
        {
            c->slab_x0 = c->slab_x1 = 0;
            if (!done) settle(c); // an early return: later work waits for the previous downloads
        }
    } reset{c, false};
    // The uploads start once earlier work on f (queued on the context's stream) is done.
    // Chained, the library's own earlier work on each slab is behind that slab's
    // download, and the caller's work on f after the previous call would have come
    // after vlasov_host_wait (which ends the chain): the stream's tail (a read of rho,
    // say, queued behind the downloads on the copy engine) does not hold them up.
    if (!chain) {
        VK_CUDA(c, cudaEventRecord(start, c->stream));
        VK_CUDA(c, cudaStreamWaitEvent(c->copy_stream, start, 0));
    }
    for (int sl = 0; sl < S; ++sl) {
        if (chain) VK_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->down_ev[sl], 0));
        VK_CUDA(c, cudaMemcpyAsync(fd + sl * slab_bytes, fh + sl * slab_bytes, slab_bytes, cudaMemcpyHostToDevice,
                                   c->copy_stream));
        VK_CUDA(c, cudaEventRecord(up[sl], c->copy_stream));
    }
    // first kick, D_z, D_y: cell-local, one slab at a time as its upload lands
    if ((rc = prep_velocity(c, phi_n_dev, 0.5 * dt, 7))) return rc;
    for (int sl = 0; sl < S && !rc; ++sl) {
        VK_CUDA(c, cudaStreamWaitEvent(c->stream, up[sl], 0));
        on_slab(sl);
        if (!(rc = run_kick(c)) && !(rc = run_position(c, 2, dt, a_half))) rc = run_position(c, 1, dt, a_half);
    }
    all();
    if (rc) return rc;
    // D_x couples the slabs; it sums the moment when it can
    double *rho = rho_nu_dev ? rho_nu_dev : c->d_rho;
    const bool need_rho = rho_nu_dev || phi_next_dev;
    bool have_rho = false;
    if ((rc = run_position(c, 0, dt, a_half, nullptr, nullptr, need_rho ? rho : nullptr, &have_rho))) return rc;
    if (need_rho && !have_rho && (rc = vlasov_moment(c, rho, nullptr))) return rc;
    if (phi_next_dev) {
        if ((rc = vlasov_poisson(c, rho, rho_bg_dev, a_full, four_pi_G, phi_next_dev))) return rc;
        if ((rc = prep_velocity(c, phi_next_dev, 0.5 * dt, 7))) return rc;
    }
    // the previous downloads are behind every upload, so behind D_x: waiting for them
    // here costs nothing, and frees their events for this step's downloads
    VK_SETTLE(c);
    // second kick one slab at a time, each slab's download behind it on the download stream
    int queued = 0;
    for (int sl = 0; sl < S && !rc; ++sl) {
        on_slab(sl);
        if (!(rc = run_kick(c))) {
            VK_CUDA(c, cudaEventRecord(ready[sl], c->stream));
            VK_CUDA(c, cudaStreamWaitEvent(c->down_stream, ready[sl], 0));
            VK_CUDA(c, cudaMemcpyAsync(fh + sl * slab_bytes, fd + sl * slab_bytes, slab_bytes, cudaMemcpyDeviceToHost,
                                       c->down_stream));
            VK_CUDA(c, cudaEventRecord(c->down_ev[sl], c->down_stream));
            ++queued;
        }
    }
    all();
    VK_CUDA(c, cudaEventRecord(c->down_ev[kMaxSlabs], c->down_stream));
    if (rc || queued != S) {
        // later work waits for whatever was queued
        VK_CUDA(c, cudaStreamWaitEvent(c->stream, c->down_ev[kMaxSlabs], 0));
        return rc;
    }
    // later calls wait for the downloads (settle); the next vlasov_step_host per slab
    c->pending_slabs = S;
    c->pending_slab_bytes = slab_bytes;
    reset.done = true;
    return VLASOV_OK;
}

extern "C" int vlasov_host_wait(vlasov_ctx *c)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    return VLASOV_OK;
}

namespace {
// One thread waits, with the bounded wait of the TMA kernels, for an mbarrier phase that
// no thread completes (one arrival expected, none made): the wait runs out at its limit,
// the thread records ERR_TIMEOUT and the kernel returns.
__global__ void wait_selftest_kernel(unsigned *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_barrier_init();
    if (!mbar_wait_bounded(&bar, 0)) atomicOr(err, ERR_TIMEOUT);
}
} // namespace

extern "C" int vlasov_selftest_wait(vlasov_ctx *c)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    wait_selftest_kernel<<<1, 32, 0, c->stream>>>(c->d_err);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "wait self-test launch");
    return VLASOV_OK;
}

extern "C" int vlasov_status(vlasov_ctx *c)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    unsigned bits = 0;
    VK_CUDA(c, cudaStreamSynchronize(c->stream));
    VK_CUDA(c, cudaMemcpy(&bits, c->d_err, sizeof bits, cudaMemcpyDeviceToHost));
    VK_CUDA(c, cudaMemset(c->d_err, 0, sizeof bits));
    if (bits & ERR_TIMEOUT) return fail(c, VLASOV_ETIMEOUT, "a bounded device wait ran out (error bits 0x%x)", bits);
    if (bits & ERR_NAN) return fail(c, VLASOV_ENAN, "a sweep produced NaN/Inf or a negative line sum (error bits 0x%x)", bits);
    if (bits & ERR_CFL) return fail(c, VLASOV_ECFL, "a velocity-sweep Courant number reached 1 (error bits 0x%x)", bits);
    return VLASOV_OK;
}

extern "C" const char *vlasov_last_error(const vlasov_ctx *c) { return c ? c->msg : g_init_error; }

// ----------------------------------------------------------------------------
// adjoint (reverse mode) of the sweeps and of the step
// ----------------------------------------------------------------------------

static int ensure_buffer(vlasov_ctx *c, void **p, size_t bytes)
{
    if (*p) return VLASOV_OK;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, VLASOV_ENOMEM, "adjoint scratch allocation of %zu bytes failed", bytes);
    }
    return VLASOV_OK;
}

// lam <- (dD_axis/df)^T lam at the sweep input f_in.  Velocity sweeps read the
// constants in d_coef[axis - 3] (prepared for the same phi and dt) and add
// dL/dg to dLdg (ncell FP64, may be null).
template <typename C>
static int run_adjoint_t(vlasov_ctx *c, const void *f_in, void *lam, int ax, double dt, double a, double *dLdg)
{
    const long long d6[6] = {c->g.nx, c->g.ny, c->g.nz, c->g.nux, c->g.nuy, c->g.nuz};
    long long I = 1, O = 1;
    for (int k = ax + 1; k < 6; ++k) I *= d6[k];
    for (int k = 0; k < ax; ++k) O *= d6[k];
    AdjArgs<C> A{};
    A.L = int(d6[ax]);
    A.periodic = ax < 3;
    A.n_inner = I;
    A.n_outer = O;
    A.nlines = I * O;
    A.err = c->d_err;
    A.f_in = f_in;
    A.lam_in = lam;
    A.lam_out = lam;
    bool shifted = false;
    if (ax < 3) {
        if (!(a > 0) || !isfinite(dt) || !isfinite(a)) return fail(c, VLASOV_EINVAL, "adjoint sweep %d: need finite dt and a > 0", ax);
        const int nvel = (&c->g.nux)[ax];
        const double du = 2.0 * c->g.V / nvel;
        const double dx = c->g.L / (&c->g.nx)[ax];
        long long vstride = 1;
        for (int k = ax + 1; k < 3; ++k) vstride *= (&c->g.nux)[k];
        A.vstride = vstride;
        A.nvel = nvel;
        A.coef_mode = 0;
        A.outer_per_cell = 1;
        for (int j = 0; j < nvel; ++j) {
            const double nu = (-c->g.V + (j + 0.5) * du) * dt / (a * a * dx);
            A.table[j] = make_line_coef<C>(nu);
            shifted = shifted || fabs(nu) >= 1.0;
        }
        // z: group each block's threads by the sign of u_z (whole u_z lines per block)
        const int bt = adjoint_block(ax, false, int(d6[ax])), nuz = int(c->g.nuz);
        if (ax == 2 && nuz % 2 == 0 && bt % nuz == 0 && I % bt == 0) A.perm_line = nuz;
        if (shifted) {
            // lambda is read N cells on: write the result to scratch, then copy back
            int rc = ensure_buffer(c, &c->d_lam_tmp, f_bytes(c));
            if (rc) return rc;
            A.lam_out = c->d_lam_tmp;
        }
    } else {
        const long long opc = O / c->ncell;
        A.vstride = 1;
        A.nvel = 0;
        A.coef_mode = 1;
        A.outer_per_cell = opc;
        A.cell_coef = (const LineCoefT<C> *)c->d_coef[ax - 3];
        A.dLdg = dLdg;
        A.lines_per_cell = opc * I;
        A.dnu_dg = -dt / (2.0 * c->g.V / (&c->g.nux)[ax - 3]);
    }
    const bool rows = ax == 5 && adjoint_rows_supported(A.L, c->g.dtype);
    if (rows) A.outer_per_cell = A.lines_per_cell; // one row per line: cell = row / rows per cell
    // when a cell's lines fill whole blocks, each block writes its sum and a second pass adds
    // them per cell in a fixed order (reproducible); otherwise FP64 atomics
    const int bt = adjoint_block(ax, rows, A.L);
    const bool det = A.dLdg && A.lines_per_cell % bt == 0;
    if (det) {
        const size_t nblk = (size_t)(A.nlines / bt);
        if (c->part_len < nblk) {
            cudaFree(c->d_part);
            c->d_part = nullptr;
            c->part_len = 0;
            int rc = ensure_buffer(c, (void **)&c->d_part, sizeof(double) * nblk);
            if (rc) return rc;
            c->part_len = nblk;
        }
        A.block_part = c->d_part;
    }
    cudaError_t e;
    {
        PartTimer t(c, VLASOV_T_ADJ_X + ax, det ? 2 : 1);
        if constexpr (sizeof(C) == 8) e = launch_adjoint_f64(A, rows, c->stream);
        else e = launch_adjoint_f32(A, rows, c->stream);
        if (e == cudaSuccess && det)
            e = launch_cell_sum(c->ncell, int(A.lines_per_cell / bt), c->d_part, A.dnu_dg, A.dLdg, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint sweep launch");
    if (shifted) VK_CUDA(c, cudaMemcpyAsync(lam, c->d_lam_tmp, f_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
    return VLASOV_OK;
}

static int run_adjoint(vlasov_ctx *c, const void *f_in, void *lam, int ax, double dt, double a, double *dLdg)
{
    if (c->g.dtype == VLASOV_F64) return run_adjoint_t<double>(c, f_in, lam, ax, dt, a, dLdg);
    return run_adjoint_t<float>(c, f_in, lam, ax, dt, a, dLdg);
}

static int check_adjoint_args(vlasov_ctx *c, const void *f, const void *lam, const char *who)
{
    if (c->g.dtype != VLASOV_F32 && c->g.dtype != VLASOV_F64)
        return fail(c, VLASOV_EINVAL, "%s: FP32 or FP64 storage only", who);
    if (!f || !lam || reinterpret_cast<uintptr_t>(f) % 16 || reinterpret_cast<uintptr_t>(lam) % 16)
        return fail(c, VLASOV_EINVAL, "%s: f and lambda must be non-null and 16-byte aligned", who);
    if (f == lam) return fail(c, VLASOV_EINVAL, "%s: f and lambda must be different arrays", who);
    return VLASOV_OK;
}

extern "C" int vlasov_sweep_adjoint(vlasov_ctx *c, const void *f_in_dev, void *lam_dev, int axis, double dt, double a,
                                    const float *phi_dev, double *dLdg_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    if (axis < 0 || axis > 5) return fail(c, VLASOV_EINVAL, "axis %d outside 0..5", axis);
    int rc = check_adjoint_args(c, f_in_dev, lam_dev, "vlasov_sweep_adjoint");
    if (rc) return rc;
    if (axis >= 3 && (rc = prep_velocity(c, phi_dev, dt, 1 << (axis - 3)))) return rc;
    return run_adjoint(c, f_in_dev, lam_dev, axis, dt, a, axis >= 3 ? dLdg_dev : nullptr);
}

extern "C" int vlasov_moment_adjoint(vlasov_ctx *c, const double *dLdrho_dev, void *lam_dev, int accumulate)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    if (c->g.dtype != VLASOV_F32 && c->g.dtype != VLASOV_F64)
        return fail(c, VLASOV_EINVAL, "vlasov_moment_adjoint: FP32 or FP64 storage only");
    if (!dLdrho_dev || !lam_dev || reinterpret_cast<uintptr_t>(lam_dev) % 16)
        return fail(c, VLASOV_EINVAL, "vlasov_moment_adjoint: null dLdrho or null / misaligned lambda");
    PartTimer t(c, VLASOV_T_MOMENT_ADJ, 1);
    const cudaError_t e = launch_moment_adjoint(c->gd, dLdrho_dev, c->g.dtype == VLASOV_F64 ? 0 : 1, lam_dev,
                                                accumulate != 0, c->stream, c->sm_count);
    if (e != cudaSuccess) return cuda_fail(c, e, "moment adjoint launch");
    return VLASOV_OK;
}

// sweeps of one step, Eq. 5: kick u_x, u_y, u_z (dt/2), drift z, y, x (dt), kick (dt/2)
static const int kStepAxes[9] = {3, 4, 5, 2, 1, 0, 3, 4, 5};
static double step_dt(int k, double dt) { return (k >= 3 && k <= 5) ? dt : 0.5 * dt; }

static int check_records(vlasov_ctx *c, const void *const *rec, const char *who)
{
    if (!rec) return fail(c, VLASOV_EINVAL, "%s: rec_dev is NULL", who);
    for (int k = 0; k < 8; ++k)
        if (!rec[k] || reinterpret_cast<uintptr_t>(rec[k]) % 16)
            return fail(c, VLASOV_EINVAL, "%s: rec_dev[%d] must be a 16-byte aligned device array", who, k);
    return VLASOV_OK;
}

extern "C" int vlasov_step_record(vlasov_ctx *c, const void *f_n_dev, void *const *rec_dev, void *f_next_dev, double dt,
                                  double a_half, const float *phi_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    int rc = check_records(c, rec_dev, "vlasov_step_record");
    if (!rc) rc = check_adjoint_args(c, f_n_dev, rec_dev[0], "vlasov_step_record");
    if (rc) return rc;
    if (f_next_dev && reinterpret_cast<uintptr_t>(f_next_dev) % 16)
        return fail(c, VLASOV_EINVAL, "vlasov_step_record: f_next_dev must be 16-byte aligned");
    if ((rc = prep_velocity(c, phi_dev, 0.5 * dt, 7))) return rc;
    for (int k = 0; k < 9; ++k) {
        const void *src = k == 0 ? f_n_dev : rec_dev[k - 1];
        void *dst = k < 8 ? rec_dev[k] : f_next_dev;
        if (!dst) break;
        const int ax = kStepAxes[k];
        rc = ax >= 3 ? run_velocity(c, ax, src, dst) : run_position(c, ax, step_dt(k, dt), a_half, src, dst);
        if (rc) return rc;
    }
    return VLASOV_OK;
}

extern "C" int vlasov_step_adjoint_recorded(vlasov_ctx *c, const void *f_n_dev, const void *const *rec_dev, void *lam_dev,
                                            double dt, double a_half, const float *phi_dev, double *dLdphi_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    int rc = check_adjoint_args(c, f_n_dev, lam_dev, "vlasov_step_adjoint_recorded");
    if (!rc) rc = check_records(c, const_cast<void *const *>(rec_dev), "vlasov_step_adjoint_recorded");
    if (rc) return rc;
    for (int k = 0; k < 8; ++k)
        if (rec_dev[k] == lam_dev) return fail(c, VLASOV_EINVAL, "vlasov_step_adjoint_recorded: lambda aliases a record");
    if (dLdphi_dev && (rc = ensure_buffer(c, (void **)&c->d_dLdg, sizeof(double) * 3 * c->ncell))) return rc;
    // the kick constants (both kicks use phi and dt / 2)
    if ((rc = prep_velocity(c, phi_dev, 0.5 * dt, 7))) return rc;
    if (dLdphi_dev) VK_CUDA(c, cudaMemsetAsync(c->d_dLdg, 0, sizeof(double) * 3 * c->ncell, c->stream));
    // the nine adjoint sweeps, last sweep first
    for (int k = 8; k >= 0; --k) {
        const int ax = kStepAxes[k];
        const void *in = k == 0 ? f_n_dev : rec_dev[k - 1];
        double *dLdg = (ax >= 3 && dLdphi_dev) ? c->d_dLdg + (ax - 3) * c->ncell : nullptr;
        if ((rc = run_adjoint(c, in, lam_dev, ax, step_dt(k, dt), a_half, dLdg))) return rc;
    }
    if (dLdphi_dev) {
        PartTimer t(c, VLASOV_T_GRAD_ADJ, 3);
        for (int d = 0; d < 3; ++d) {
            const cudaError_t e = launch_gradient_adjoint(c->gd, c->d_dLdg + d * c->ncell, d, dLdphi_dev, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "gradient adjoint launch");
        }
    }
    return VLASOV_OK;
}

static int gradient_adjoint_all(vlasov_ctx *c, double *dLdphi);

// one sweep k of the external-potential step from src to dst (constants for the kicks in d_coef)
static int step_sweep(vlasov_ctx *c, int k, const void *src, void *dst, double dt, double a_half)
{
    const int ax = kStepAxes[k];
    return ax >= 3 ? run_velocity(c, ax, src, dst) : run_position(c, ax, step_dt(k, dt), a_half, src, dst);
}

// Step adjoint with four scratch arrays: keep the inputs of sweeps 3 and 6 and, for
// each group of three sweeps, rebuild the other two inputs just before their adjoints
// (12 forward sweeps instead of 8).
static int step_adjoint_low_memory(vlasov_ctx *c, const void *f_n, void *lam, double dt, double a_half,
                                   const float *phi, double *dLdphi)
{
    void *r3 = c->d_rec[0], *r6 = c->d_rec[1], *w1 = c->d_rec[2], *w2 = c->d_rec[3];
    int rc;
    if ((rc = prep_velocity(c, phi, 0.5 * dt, 7))) return rc;
    // inputs of sweeps 3 and 6, through the other two arrays
    if ((rc = step_sweep(c, 0, f_n, w1, dt, a_half)) || (rc = step_sweep(c, 1, w1, w2, dt, a_half)) ||
        (rc = step_sweep(c, 2, w2, r3, dt, a_half)) || (rc = step_sweep(c, 3, r3, w1, dt, a_half)) ||
        (rc = step_sweep(c, 4, w1, w2, dt, a_half)) || (rc = step_sweep(c, 5, w2, r6, dt, a_half)))
        return rc;
    if (dLdphi) VK_CUDA(c, cudaMemsetAsync(c->d_dLdg, 0, sizeof(double) * 3 * c->ncell, c->stream));
    const void *starts[3] = {f_n, r3, r6};
    for (int grp = 2; grp >= 0; --grp) {
        const int k0 = 3 * grp;
        // inputs of sweeps k0 + 1 and k0 + 2
        if ((rc = step_sweep(c, k0, starts[grp], w1, dt, a_half)) || (rc = step_sweep(c, k0 + 1, w1, w2, dt, a_half)))
            return rc;
        const void *in[3] = {starts[grp], w1, w2};
        for (int j = 2; j >= 0; --j) {
            const int ax = kStepAxes[k0 + j];
            double *dLdg = (ax >= 3 && dLdphi) ? c->d_dLdg + (ax - 3) * c->ncell : nullptr;
            if ((rc = run_adjoint(c, in[j], lam, ax, step_dt(k0 + j, dt), a_half, dLdg))) return rc;
        }
    }
    if (dLdphi && (rc = gradient_adjoint_all(c, dLdphi))) return rc;
    return VLASOV_OK;
}

extern "C" int vlasov_set_adjoint_arrays(vlasov_ctx *c, int arrays)
{
    if (!c) return VLASOV_EINVAL;
    if (arrays != 0 && arrays != 4 && arrays != 8) return fail(c, VLASOV_EINVAL, "adjoint arrays must be 0, 4 or 8");
    c->adj_arrays = arrays;
    return VLASOV_OK;
}

extern "C" int vlasov_step_adjoint(vlasov_ctx *c, const void *f_n_dev, void *lam_dev, double dt, double a_half,
                                   const float *phi_dev, double *dLdphi_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    int rc = check_adjoint_args(c, f_n_dev, lam_dev, "vlasov_step_adjoint");
    if (rc) return rc;
    if (!phi_dev) return fail(c, VLASOV_EINVAL, "vlasov_step_adjoint: phi_dev is NULL");
    const size_t bytes = f_bytes(c);
    if (dLdphi_dev && (rc = ensure_buffer(c, (void **)&c->d_dLdg, sizeof(double) * 3 * c->ncell))) return rc;
    // as many scratch arrays as the setting allows and the device holds: 8 (record every
    // input) or 4 (recompute within the step)
    int want = c->adj_arrays ? c->adj_arrays : 8;
    for (int k = 0; k < want && !rc; ++k) rc = ensure_buffer(c, &c->d_rec[k], bytes);
    if (rc && c->adj_arrays == 0) {
        for (int k = 4; k < 8; ++k) { cudaFree(c->d_rec[k]); c->d_rec[k] = nullptr; }
        rc = VLASOV_OK;
        want = 4;
        for (int k = 0; k < 4 && !rc; ++k) rc = ensure_buffer(c, &c->d_rec[k], bytes);
    }
    if (rc) return rc;
    bool all8 = want == 8;
    for (int k = 0; k < 8 && all8; ++k) all8 = c->d_rec[k] != nullptr;
    if (!all8) return step_adjoint_low_memory(c, f_n_dev, lam_dev, dt, a_half, phi_dev, dLdphi_dev);
    // run the step again from f_n, keeping the input of every sweep
    if ((rc = vlasov_step_record(c, f_n_dev, c->d_rec, nullptr, dt, a_half, phi_dev))) return rc;
    return vlasov_step_adjoint_recorded(c, f_n_dev, c->d_rec, lam_dev, dt, a_half, phi_dev, dLdphi_dev);
}

// ----------------------------------------------------------------------------
// self-consistent step: record and adjoint
// ----------------------------------------------------------------------------
extern "C" int vlasov_step_record_sc(vlasov_ctx *c, const void *f_n_dev, void *const *rec_dev, void *f_next_dev,
                                     double dt, double a_half, double a_full, const float *phi_n_dev,
                                     const double *rho_bg_dev, double four_pi_G, float *phi_next_dev,
                                     double *rho_nu_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    int rc = check_records(c, rec_dev, "vlasov_step_record_sc");
    if (!rc) rc = check_adjoint_args(c, f_n_dev, rec_dev[0], "vlasov_step_record_sc");
    if (rc) return rc;
    if (!phi_next_dev) return fail(c, VLASOV_EINVAL, "vlasov_step_record_sc: phi_next_dev is NULL");
    if (f_next_dev && reinterpret_cast<uintptr_t>(f_next_dev) % 16)
        return fail(c, VLASOV_EINVAL, "vlasov_step_record_sc: f_next_dev must be 16-byte aligned");
    if ((rc = prep_velocity(c, phi_n_dev, 0.5 * dt, 7))) return rc;
    double *rho = rho_nu_dev ? rho_nu_dev : c->d_rho;
    bool have_rho = false; // the x sweep (k = 5) writes the moment when it can, as in vlasov_step
    for (int k = 0; k < 9; ++k) {
        if (k == 6) {
            // after the drift (rec[5] = input of sweep 6): moment, Poisson, the second kick's constants
            if (!have_rho) {
                cudaError_t e;
                {
                    PartTimer t(c, VLASOV_T_MOMENT, 1);
                    e = launch_moment(c->gd, rec_dev[5], c->g.dtype == VLASOV_F64 ? 0 : 1, rho, c->stream, c->sm_count);
                }
                if (e != cudaSuccess) return cuda_fail(c, e, "moment launch");
            }
            if ((rc = vlasov_poisson(c, rho, rho_bg_dev, a_full, four_pi_G, phi_next_dev))) return rc;
            if ((rc = prep_velocity(c, phi_next_dev, 0.5 * dt, 7))) return rc;
        }
        const void *src = k == 0 ? f_n_dev : rec_dev[k - 1];
        void *dst = k < 8 ? rec_dev[k] : f_next_dev;
        if (!dst) break;
        const int ax = kStepAxes[k];
        rc = ax >= 3 ? run_velocity(c, ax, src, dst)
                     : run_position(c, ax, step_dt(k, dt), a_half, src, dst, k == 5 ? rho : nullptr, &have_rho);
        if (rc) return rc;
    }
    return VLASOV_OK;
}

static int gradient_adjoint_all(vlasov_ctx *c, double *dLdphi)
{
    PartTimer t(c, VLASOV_T_GRAD_ADJ, 3);
    for (int d = 0; d < 3; ++d) {
        const cudaError_t e = launch_gradient_adjoint(c->gd, c->d_dLdg + d * c->ncell, d, dLdphi, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "gradient adjoint launch");
    }
    return VLASOV_OK;
}

extern "C" int vlasov_step_adjoint_recorded_sc(vlasov_ctx *c, const void *f_n_dev, const void *const *rec_dev,
                                               void *lam_dev, double dt, double a_half, double a_full,
                                               const float *phi_n_dev, const float *phi_next_dev, double four_pi_G,
                                               const double *lam_phi_next_dev, double *dLdphi_n_dev,
                                               double *dLdrho_bg_dev)
{
    if (!c) return VLASOV_EINVAL;
    VK_SETTLE(c);
    int rc = check_adjoint_args(c, f_n_dev, lam_dev, "vlasov_step_adjoint_recorded_sc");
    if (!rc) rc = check_records(c, const_cast<void *const *>(rec_dev), "vlasov_step_adjoint_recorded_sc");
    if (rc) return rc;
    for (int k = 0; k < 8; ++k)
        if (rec_dev[k] == lam_dev) return fail(c, VLASOV_EINVAL, "vlasov_step_adjoint_recorded_sc: lambda aliases a record");
    if (!phi_next_dev) return fail(c, VLASOV_EINVAL, "vlasov_step_adjoint_recorded_sc: phi_next_dev is NULL");
    if ((rc = ensure_buffer(c, (void **)&c->d_dLdg, sizeof(double) * 3 * c->ncell))) return rc;
    if ((rc = ensure_buffer(c, (void **)&c->d_sc, sizeof(double) * 2 * c->ncell))) return rc;
    const long long nc = c->ncell;
    double *dphi1 = c->d_sc, *drho = c->d_sc + nc;
    // second kick, with phi^{n+1}
    if ((rc = prep_velocity(c, phi_next_dev, 0.5 * dt, 7))) return rc;
    VK_CUDA(c, cudaMemsetAsync(c->d_dLdg, 0, sizeof(double) * 3 * nc, c->stream));
    for (int k = 8; k >= 6; --k) {
        const int ax = kStepAxes[k];
        if ((rc = run_adjoint(c, rec_dev[k - 1], lam_dev, ax, step_dt(k, dt), a_half, c->d_dLdg + (ax - 3) * nc))) return rc;
    }
    // dL/dphi^{n+1}: from later steps plus the second kick's G^T dL/dg
    if (lam_phi_next_dev) VK_CUDA(c, cudaMemcpyAsync(dphi1, lam_phi_next_dev, sizeof(double) * nc, cudaMemcpyDeviceToDevice, c->stream));
    else VK_CUDA(c, cudaMemsetAsync(dphi1, 0, sizeof(double) * nc, c->stream));
    if ((rc = gradient_adjoint_all(c, dphi1))) return rc;
    // Poisson (its own transpose) and the moment
    cudaError_t e;
    {
        PartTimer t(c, VLASOV_T_POISSON, 9);
        e = launch_poisson(c->gd, c->ps, dphi1, nullptr, a_full, four_pi_G, nullptr, c->stream, drho);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "poisson adjoint launch");
    if (dLdrho_bg_dev && (e = launch_add(nc, drho, dLdrho_bg_dev, false, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "rho_bg gradient launch");
    {
        PartTimer t(c, VLASOV_T_MOMENT_ADJ, 1);
        e = launch_moment_adjoint(c->gd, drho, c->g.dtype == VLASOV_F64 ? 0 : 1, lam_dev, 1, c->stream, c->sm_count);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "moment adjoint launch");
    // drift
    for (int k = 5; k >= 3; --k)
        if ((rc = run_adjoint(c, rec_dev[k - 1], lam_dev, kStepAxes[k], step_dt(k, dt), a_half, nullptr))) return rc;
    // first kick, with phi_n
    if ((rc = prep_velocity(c, phi_n_dev, 0.5 * dt, 7))) return rc;
    VK_CUDA(c, cudaMemsetAsync(c->d_dLdg, 0, sizeof(double) * 3 * nc, c->stream));
    for (int k = 2; k >= 0; --k) {
        const int ax = kStepAxes[k];
        const void *in = k == 0 ? f_n_dev : rec_dev[k - 1];
        if ((rc = run_adjoint(c, in, lam_dev, ax, step_dt(k, dt), a_half, c->d_dLdg + (ax - 3) * nc))) return rc;
    }
    if (dLdphi_n_dev && (rc = gradient_adjoint_all(c, dLdphi_n_dev))) return rc;
    return VLASOV_OK;
}

// ----------------------------------------------------------------------------
// velocity sweep without allocation (vlasov_sweep_velocity_static)
// ----------------------------------------------------------------------------
// Scratch of the allocation-free entry point: 256 B of header (the error word
// used when the caller passes no status word) followed by the per-cell sweep
// constants of up to VLASOV_STATIC_MAX_CELLS spatial cells.  Device code could
// name the array directly; host code must use the address that
// cudaGetSymbolAddress returns for the current device.
constexpr size_t kStaticHeader = 256;
constexpr size_t kStaticBytes = kStaticHeader + (size_t)VLASOV_STATIC_MAX_CELLS * sizeof(LineCoefT<float>);
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Device address of g_static_scratch in the current device's context.  It is looked up
// on every call (a table lookup once the module is loaded): an address kept from an
// earlier call would be stale after a cudaDeviceReset, which unloads the module.
static cudaError_t static_scratch_address(unsigned char **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}

extern "C" int vlasov_sweep_velocity_static(const vlasov_grid *g, float *f_dev, int axis, double dt,
                                            const float *phi_dev, unsigned int *status_dev, void *stream)
{
    if (!g || !f_dev || !phi_dev) return fail(nullptr, VLASOV_EINVAL, "vlasov_sweep_velocity_static: null argument");
    if (axis < 3 || axis > 5) return fail(nullptr, VLASOV_EINVAL, "vlasov_sweep_velocity_static: axis %d is not 3..5", axis);
    if (g->dtype != VLASOV_F32) return fail(nullptr, VLASOV_EINVAL, "vlasov_sweep_velocity_static: FP32 storage only");
    if (!isfinite(dt)) return fail(nullptr, VLASOV_EINVAL, "vlasov_sweep_velocity_static: dt must be finite");
    const int dims[6] = {g->nx, g->ny, g->nz, g->nux, g->nuy, g->nuz};
    for (int k = 0; k < 3; ++k)
        if (dims[k] < 4 || dims[k] > 256) return fail(nullptr, VLASOV_EINVAL, "spatial size %d outside [4, 256]", dims[k]);
    for (int k = 3; k < 6; ++k)
        if (dims[k] < 4 || dims[k] > kMaxVel || dims[k] % 4)
            return fail(nullptr, VLASOV_EINVAL, "velocity size %d must be a multiple of 4 in [4, %d]", dims[k], kMaxVel);
    if (!(g->L > 0) || !(g->V > 0)) return fail(nullptr, VLASOV_EINVAL, "L and V must be positive");
    if (reinterpret_cast<uintptr_t>(f_dev) % 16) return fail(nullptr, VLASOV_EINVAL, "f_dev must be 16-byte aligned");
    const long long ncell = (long long)g->nx * g->ny * g->nz;
    if (ncell > VLASOV_STATIC_MAX_CELLS)
        return fail(nullptr, VLASOV_EINVAL,
                    "vlasov_sweep_velocity_static: %lld spatial cells exceed the static scratch (%d cells)", ncell,
                    VLASOV_STATIC_MAX_CELLS);
    if (ncell * g->nux * g->nuy >= (1ll << 31)) return fail(nullptr, VLASOV_EINVAL, "too many u_z lines for 32-bit TMA coordinates");
    if (ncell * ((long long)g->nux * g->nuy * g->nuz) / g->nx >= (1ll << 32))
        return fail(nullptr, VLASOV_EINVAL, "grid too large for 32-bit TMA extents");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    unsigned char *scratch = nullptr;
    if (e == cudaSuccess) e = static_scratch_address(&scratch);
    if (e != cudaSuccess) return fail(nullptr, VLASOV_ECUDA, "static scratch lookup: %s", cudaGetErrorString(e));

    // A context on the stack: the plan and the launch helpers need no allocation.
    vlasov_ctx c{};
    c.g = *g;
    c.f = f_dev;
    c.stream = (cudaStream_t)stream;
    c.es = 4;
    c.ncell = ncell;
    c.gd.n[0] = g->nx; c.gd.n[1] = g->ny; c.gd.n[2] = g->nz;
    c.gd.nu[0] = g->nux; c.gd.nu[1] = g->nuy; c.gd.nu[2] = g->nuz;
    c.gd.L = g->L;
    c.gd.V = g->V;
    e = cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(nullptr, VLASOV_ECUDA, "device query: %s", cudaGetErrorString(e));
    int rc = plan_axes(&c, 1 << axis); // the swept axis only
    if (rc != VLASOV_OK) return fail(nullptr, rc, "%s", c.msg);

    unsigned *err = status_dev;
    if (!err) {
        // the shared error word starts every call at zero
        err = reinterpret_cast<unsigned *>(scratch);
        e = cudaMemsetAsync(err, 0, sizeof(unsigned), c.stream);
        if (e != cudaSuccess) return fail(nullptr, VLASOV_ECUDA, "clearing the static error word: %s", cudaGetErrorString(e));
    }
    void *coef = scratch + kStaticHeader;
    c.d_err = err;
    c.d_coef[axis - 3] = coef;
    rc = prep_velocity(&c, phi_dev, dt, 1 << (axis - 3));
    if (rc == VLASOV_OK) rc = run_velocity(&c, axis);
    if (rc != VLASOV_OK) return fail(nullptr, rc, "%s", c.msg);
    return VLASOV_OK;
}

// ----------------------------------------------------------------------------
// 16-bit storage codec (vlasov_encode / vlasov_decode)
// ----------------------------------------------------------------------------

static int codec_args(long long nlines, int nuz, const void *vals, int vdtype, const void *codes, int cdtype,
                      const float *scale, const char *who)
{
    if (nlines < 0 || nuz < 1 || nuz > kMaxVel)
        return fail(nullptr, VLASOV_EINVAL, "%s: need nlines >= 0 and 1 <= nuz <= %d", who, kMaxVel);
    if (vdtype != VLASOV_F64 && vdtype != VLASOV_F32)
        return fail(nullptr, VLASOV_EINVAL, "%s: values must be VLASOV_F64 or VLASOV_F32", who);
    if (cdtype != VLASOV_BF16 && cdtype != VLASOV_F16)
        return fail(nullptr, VLASOV_EINVAL, "%s: codes must be VLASOV_BF16 or VLASOV_F16", who);
    if (nlines == 0) return VLASOV_OK;
    if (!vals || !codes || !scale) return fail(nullptr, VLASOV_EINVAL, "%s: null pointer", who);
    const uintptr_t va = reinterpret_cast<uintptr_t>(vals), ca = reinterpret_cast<uintptr_t>(codes),
                    sa = reinterpret_cast<uintptr_t>(scale);
    if (va % (vdtype == VLASOV_F64 ? 8 : 4) || ca % 2 || sa % 4)
        return fail(nullptr, VLASOV_EINVAL, "%s: a pointer is not aligned to its element size", who);
    return VLASOV_OK;
}

static int current_sm_count(int *sm)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(nullptr, VLASOV_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    return VLASOV_OK;
}

extern "C" int vlasov_encode(long long nlines, int nuz, const void *src_dev, int src_dtype, void *codes_dev,
                             int code_dtype, float *scale_dev, void *stream)
{
    int rc = codec_args(nlines, nuz, src_dev, src_dtype, codes_dev, code_dtype, scale_dev, "vlasov_encode");
    if (rc != VLASOV_OK || nlines == 0) return rc;
    int sm = 0;
    if ((rc = current_sm_count(&sm))) return rc;
    const cudaError_t e = launch_encode(nlines, nuz, src_dev, src_dtype == VLASOV_F64 ? 0 : 1, codes_dev, code_dtype,
                                        scale_dev, (cudaStream_t)stream, sm);
    if (e != cudaSuccess) return fail(nullptr, VLASOV_ECUDA, "encode launch: %s", cudaGetErrorString(e));
    return VLASOV_OK;
}

extern "C" int vlasov_decode(long long nlines, int nuz, const void *codes_dev, int code_dtype, const float *scale_dev,
                             void *dst_dev, int dst_dtype, void *stream)
{
    int rc = codec_args(nlines, nuz, dst_dev, dst_dtype, codes_dev, code_dtype, scale_dev, "vlasov_decode");
    if (rc != VLASOV_OK || nlines == 0) return rc;
    int sm = 0;
    if ((rc = current_sm_count(&sm))) return rc;
    const cudaError_t e = launch_decode(nlines, nuz, codes_dev, code_dtype, scale_dev, dst_dev,
                                        dst_dtype == VLASOV_F64 ? 0 : 1, (cudaStream_t)stream, sm);
    if (e != cudaSuccess) return fail(nullptr, VLASOV_ECUDA, "decode launch: %s", cudaGetErrorString(e));
    return VLASOV_OK;
}
