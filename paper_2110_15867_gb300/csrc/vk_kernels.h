// vk_kernels.h -- internal interface between the C ABI (vlasov_api.cu) and the
// kernel translation units of libvlasov.  Not installed; not part of the ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace vk {

// sticky error bits of the device error word
enum : unsigned { ERR_CFL = 1u, ERR_NAN = 2u, ERR_TIMEOUT = 4u };

// Division of 32-bit unsigned integers by an invariant divisor d >= 1: one multiply-high,
// a subtract, an add and two shifts instead of a division routine (the round-up method
// of Granlund & Montgomery, "Division by invariant integers using multiplication",
// PLDI 1994): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0), t = mulhi(m, n), for every n < 2^32.
struct FastDivU32 {
    unsigned m, s1, s2;
};
inline FastDivU32 make_fastdiv(unsigned d)
{
    unsigned l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    return FastDivU32{unsigned(m), l ? 1u : 0u, l ? l - 1 : 0u};
}
#ifdef __CUDACC__
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDivU32 &f)
{
    const unsigned t = __umulhi(n, f.m);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}
#endif

constexpr int kMaxVel = 128;       // largest velocity-axis length a position table holds
constexpr int kConsumers = 256;    // consumer threads per CTA (8 warps)
constexpr int kProducer = 32;      // one producer warp (lane 0 drives the TMA engine)

// Per-line SL-MPP5 constants, see LineCoef in the kernels.  C = float for
// FP32 / 16-bit storage, double for FP64 storage.
// nd = 2 N + (dir < 0), or -1: leave the line untouched (Courant number out of range).
template <typename C> struct LineCoefT {
    C w[5];
    C s;
    C alpha;
    int nd;
    int pad;
};

// Weights of the mean over the departure interval, fbar = sum_m W_m(s) c_{j-2+m},
// W_m(s) = K1_m + K2_m s + K3_m s^2 + K4_m s^3 + K5_m s^4.  They come from
// expanding, in powers of s, the exact integral over [x_{j+1/2} - s dx,
// x_{j+1/2}] of the quintic that interpolates the primitive function at the six
// faces j-5/2 .. j+5/2, divided by s (K1 is the classic fifth-order face value).
__host__ __device__ inline void sl5_weights(double s, double w[5])
{
    const double K1[5] = {1.0 / 30, -13.0 / 60, 47.0 / 60, 9.0 / 20, -1.0 / 20};
    const double K2[5] = {0.0, -1.0 / 24, 5.0 / 8, -5.0 / 8, 1.0 / 24};
    const double K3[5] = {-1.0 / 24, 1.0 / 4, -1.0 / 3, 1.0 / 12, 1.0 / 24};
    const double K4[5] = {0.0, 1.0 / 24, -1.0 / 8, 1.0 / 8, -1.0 / 24};
    const double K5[5] = {1.0 / 120, -1.0 / 30, 1.0 / 20, -1.0 / 30, 1.0 / 120};
    for (int m = 0; m < 5; ++m) w[m] = K1[m] + s * (K2[m] + s * (K3[m] + s * (K4[m] + s * K5[m])));
}

// Constants of a line with signed Courant number nu.
template <typename C> __host__ __device__ inline LineCoefT<C> make_line_coef(double nu)
{
    LineCoefT<C> k;
    const int neg = nu < 0.0;
    const double a = neg ? -nu : nu;
    const double Nf = floor(a);
    const double s = a - Nf;
    double w[5];
    sl5_weights(s, w);
    for (int m = 0; m < 5; ++m) k.w[m] = (C)w[m];
    k.s = (C)s;
    // Suresh-Huynh alpha tied to the departure fraction: a monotone update needs
    // s (1 + alpha) <= 1; capped where s -> 0 (the flux then vanishes anyway).
    const double alpha = s > 0.0 ? (1.0 - s) / s : 1e6;
    k.alpha = (C)(alpha > 1e6 ? 1e6 : alpha);
    k.nd = (int)(2.0 * Nf) + neg;
    k.pad = 0;
    return k;
}

// ----------------------------------------------------------------------------
// strided sweep (axes x, y, z, u_x, u_y)
// ----------------------------------------------------------------------------
// f viewed as [O][L][I] (outer, swept, inner).  A tile is the TMA box
// {W inner, L swept, P outer}; each consumer thread owns one (inner, outer)
// column and marches it along the swept axis.
template <typename C> struct StridedArgs {
    int L, W, P, stages;
    int tiles_inner;
    int periodic;
    long long n_inner, n_outer;
    long long num_tiles;
    // position sweeps: j = (inner / vstride) % nvel indexes table
    long long vstride;
    int nvel;
    int coef_mode; // 0 = position table, 1 = per-cell array
    // velocity sweeps: cell = outer / outer_per_cell indexes cell_coef
    long long outer_per_cell;
    const LineCoefT<C> *cell_coef;
    unsigned *err;
    LineCoefT<C> table[kMaxVel];
};

// ----------------------------------------------------------------------------
// streamed strided sweep (axes x, y, z, u_x, u_y with |nu| < 1): a block of
// columns {W inner} x {P outer} walks down the swept axis in chunks of R rows
// (TMA box {W, R, P}); each consumer thread owns Lane<T>::V columns.
// ----------------------------------------------------------------------------
constexpr int kStreamConsumers = 128;
constexpr int kStreamRows = 4;  // rows per chunk (power of two, >= 3 for the periodic prologue)
constexpr int kStreamRing = 8;  // chunk slots in the ring (power of two)

template <typename C> struct StreamArgs {
    int L, W, P, R, stages;
    int tiles_inner;
    int periodic;
    int perm_line; // > 0: group the threads by the sign of u along lines of this length
    long long n_inner, n_outer;
    long long num_blocks;
    long long tile0; // first tile of this launch (num_blocks tiles from there)
    long long vstride;
    int nvel;
    int coef_mode;
    long long outer_per_cell;
    const LineCoefT<C> *cell_coef;
    unsigned *err;
    const float *scale; // 16-bit storage: one FP32 scale per u_z line (else null)
    long long nuz;
    unsigned seed;      // 16-bit storage: stochastic-rounding stream of this sweep
    int scale_rank;     // 16-bit storage: rank of the scale tensor map (3, or 2 for the u_y sweep)
    int swidth;         // 16-bit storage: inner extent of the scale box (a multiple of 4); a block at
                        // inner offset c0 loads the scales of u_z lines (c0 / nuz) & ~3 onward
    // x sweep with the velocity moment fused (FP32 / FP64 storage, P = 1, W x the element
    // size = 1024 bytes, W divides the velocity cube): a moment warp sums every output row;
    // row x of the block at inner offset c0 adds to spatial cell x (n_inner / cube) +
    // c0 / cube as partial k = (c0 % cube) / W of nparts = cube / W, stored in the
    // storage type at mpart[((c0 / cube) nparts + k) L + x] (null: no moment)
    void *mpart;
    long long cube;
    int nparts;
    // set by the launchers: fast32 = 1 when tile indices, inner and outer offsets all stay
    // below 2^32, so that the per-block index arithmetic takes these dividers
    int fast32;
    FastDivU32 div_tiles, div_vstride, div_nvel, div_opc;
    LineCoefT<C> table[kMaxVel];
};

// 16-bit storage: smap views the scale array like map views f, with the u_z line collapsed
cudaError_t launch_stream_bf16(const CUtensorMap &map, const CUtensorMap &smap, const StreamArgs<float> &a, int grid,
                               size_t smem, cudaStream_t st);
cudaError_t launch_stream_f16(const CUtensorMap &map, const CUtensorMap &smap, const StreamArgs<float> &a, int grid,
                              size_t smem, cudaStream_t st);
// FP32 / FP64: load through map, store through dmap (the same map for an in-place sweep)
cudaError_t launch_stream_f32(const CUtensorMap &map, const CUtensorMap &dmap, const StreamArgs<float> &a, int grid,
                              size_t smem, cudaStream_t st);
cudaError_t launch_stream_f64(const CUtensorMap &map, const CUtensorMap &dmap, const StreamArgs<double> &a, int grid,
                              size_t smem, cudaStream_t st);
int occupancy_stream(int dtype, int periodic, size_t smem); // dtype: 0 f64, 1 f32, 2 bf16, 3 f16
// rho[x cells_per_row + c] = du3 * sum over k of mpart[(c nparts + k) nx + x] (FP32 or FP64
// partials: dtype 1 / 0), in FP64 in a fixed order
cudaError_t launch_moment_finish(const void *mpart, int dtype, int nparts, int nx, long long cells_per_row, double du3,
                                 double *rho, cudaStream_t st, int sm_count);
int stream_columns_per_thread(int dtype); // V: the streamed block is V * stream_consumers columns
int stream_consumers(int dtype);

// ----------------------------------------------------------------------------
// contiguous sweep (axis u_z): rows of nuz cells
// ----------------------------------------------------------------------------
template <typename C> struct ContigArgs {
    int L;      // nuz
    int R;      // rows per tile (= consumer threads)
    int stages;
    long long rows;
    long long num_tiles;
    long long rows_per_cell;
    const LineCoefT<C> *cell_coef;
    unsigned *err;
    float *scale; // 16-bit storage: one FP32 scale per row (u_z line), updated in place
    unsigned seed;
    const LineCoefT<C> *cell_coef_y; // fused kick tail: the u_y sweep's per-cell constants
    long long tile0;                 // first tile of this launch (num_tiles tiles from there)
    FastDivU32 div_rpc;              // set by launch_line_sweep: division by rows_per_cell
};

// u_z sweep with whole lines in registers (FP32, n_uz 16 or 32): TMA box
// {n_uz, 256 rows} with the 64/128-byte swizzle
bool line_sweep_supported(int nu, long long rows_per_cell);
size_t line_sweep_smem(int nu, int es, bool fuse_y = false);
bool line_sweep_fused_supported(int dtype); // the fused kick tail for this storage type (1 f32, 2 bf16, 3 f16)
int line_sweep_rows_per_tile();
// fuse_y: D_uy on the tile's (cell, j_x) planes first (FP32, n_uy = n_uz)
int occupancy_line_sweep(int nu, int dtype, bool fuse_y = false); // dtype: 1 f32, 2 bf16, 3 f16

// ----------------------------------------------------------------------------
// one kick D_uz D_uy D_ux in a single pass (kick_cube.cu): n_ux = n_uy = n_uz = 16 or 32,
// FP32 / BF16 / FP16 storage.  fmap views f as rows of NU values (the u_z lines) with box
// {NU, kick_cube_box_rows(NU)} and the 32/64/128-byte swizzle of the row size; smap (16-bit)
// views the scales as [ncell NU][NU] with box {NU, NU / 2}.
// ----------------------------------------------------------------------------
struct KickArgs {
    long long cell0, ncells; // the cubes of spatial cells [cell0, cell0 + ncells)
    const LineCoefT<float> *coef_x, *coef_y, *coef_z;
    unsigned *err;
    unsigned seed_x, seed_z; // 16-bit: stochastic-rounding streams of the D_ux and D_uz encodes
};
bool kick_cube_supported(int nux, int nuy, int nuz, int dtype); // dtype 1 f32, 2 bf16, 3 f16
int kick_cube_box_rows(int nu);
size_t kick_cube_smem(int nu, int dtype);
int occupancy_kick_cube(int nu, int dtype);
cudaError_t launch_kick_cube(const CUtensorMap &fmap, const CUtensorMap &smap, const KickArgs &a, int nu, int dtype,
                             int grid, cudaStream_t st);

// ----------------------------------------------------------------------------
// the kick tail D_uz D_uy in one pass over (cell, j_x) planes (plane_tail.cu): FP32 or
// 16-bit codes (dtype 1, 2, 3), n_uy = n_uz = 48, n_ux a multiple of 4; planes [plane0,
// plane0 + nplanes) with plane p in spatial cell p / nux, both multiples of 4
// ----------------------------------------------------------------------------
struct PlaneTailArgs {
    long long plane0, nplanes;
    long long nux;
    const LineCoefT<float> *coef_y, *coef_z;
    unsigned *err;
    float *scale;  // 16-bit storage: one scale per u_z line (row of a plane), refreshed
    unsigned seed; // 16-bit storage: the stochastic-rounding streams of the D_uz encode
};
bool plane_tail_supported(int nuy, int nuz, int nux, int dtype);
cudaError_t launch_plane_tail(void *f, const PlaneTailArgs &a, int nu, int dtype, cudaStream_t st);

// ----------------------------------------------------------------------------
// position sweeps with whole lines staged per tile (sweep_tile.cu): FP32, periodic,
// |nu| < 1, L = 16, 24, 32, 48 or 64 cells, n_inner a multiple of 256.  map views f as
// [n_outer][L][n_inner / 32][32] with box {32, 8, L, 1} and the 128-byte swizzle.
// ----------------------------------------------------------------------------
struct TileArgs {
    int L;
    long long n_inner, n_outer, tiles_inner; // tiles_inner = n_inner / 256
    long long tile0, num_tiles;              // tiles [tile0, tile0 + num_tiles), t = outer tiles_inner + block
    long long vstride;                       // column j takes table[(inner / vstride) % nvel]
    int nvel;
    int nuz;                                 // 16-bit storage: n_uz (32 or 48), the length of a scale's line
    int zperm;                               // z sweep with n_uz = 32: warps grouped by the sign of u_z
    int tile_sign;                           // 1: every warp's columns have one sign of u (else per column)
    unsigned seed;                           // 16-bit storage: the stochastic-rounding streams of this sweep
    unsigned *err;
    // u_x sweep (zero-flux lines): the Courant numbers per outer index (a cell); null for
    // the position sweeps, which take table[] per column
    const LineCoefT<float> *cell_coef;
    // x sweep with the moment: per-cell partial sums as in StreamArgs (null: no moment)
    void *mpart;
    long long cube;
    int nparts;
    LineCoefT<float> table[kMaxVel];
};
// dtype 1 (FP32), 2 (BF16), 3 (FP16; n_uz = 32 with L up to 96, or n_uz = 48 with L = 48;
// one scale per u_z line)
bool tile_sweep_supported(int L, long long n_inner, int dtype, int nuz);
// the u_x sweep on the same tiles ([cell][u_x][u_y u_z]): lines of 48 cells (16-bit: n_uz = 48)
bool tile_sweep_zf_supported(int L, long long n_inner, int dtype, int nuz);
int occupancy_tile_sweep(int L, int dtype, bool moment, int nuz);
// FP32: tiles loaded through map and stored through dmap (the same map in place).  16-bit:
// in place through map (codes, box {32, 8, L, 1}, no swizzle) with the scales through smap
// ([n_outer][L][n_inner / n_uz] floats, box {8, L, 1} for n_uz = 32, {12, L, 1} for 48)
cudaError_t launch_tile_sweep(const CUtensorMap &map, const CUtensorMap &dmap, const CUtensorMap &smap,
                              const TileArgs &a, int dtype, int grid, cudaStream_t st);

// host launchers (return cudaGetLastError() of the launch); tiles are loaded
// through map and stored through dmap (the same map for an in-place sweep)
cudaError_t launch_strided_f32(const CUtensorMap &map, const CUtensorMap &dmap, const StridedArgs<float> &a, int grid,
                               size_t smem, cudaStream_t st);
cudaError_t launch_strided_f64(const CUtensorMap &map, const CUtensorMap &dmap, const StridedArgs<double> &a, int grid,
                               size_t smem, cudaStream_t st);
cudaError_t launch_contig_f32(const CUtensorMap &map, const CUtensorMap &dmap, const ContigArgs<float> &a, int grid,
                              size_t smem, cudaStream_t st);
cudaError_t launch_contig_f64(const CUtensorMap &map, const CUtensorMap &dmap, const ContigArgs<double> &a, int grid,
                              size_t smem, cudaStream_t st);
// largest resident CTAs per SM for a launcher's kernel with this dynamic smem
// Zero-flux velocity lines of L = 16 or 32 FP32 cells strided by n_inner (u_x, u_y):
// one line per thread, loaded whole into registers (coalesced along the contiguous
// axis), marched, stored.  Lines [line0, line0 + nlines) of f viewed as
// [n_outer][L][n_inner]; constants per spatial cell (cell = outer / outer_per_cell).
// 16-bit storage: element e's value is code * scale[e / nuz] (its u_z line), and the
// line's codes are re-encoded with stochastic rounding (stream seeded per line and sweep).
struct RegLineArgs {
    int L;
    long long n_inner, n_outer, line0, nlines, outer_per_cell;
    const LineCoefT<float> *cell_coef;
    unsigned *err;
    const float *scale; // 16-bit storage only
    int nuz;
    unsigned seed;
    // set by launch_reg_lines: line indices below 2^32 take these dividers
    FastDivU32 div_inner, div_opc, div_nuz;
};
// u_z lines (rows of n_uz contiguous FP32 cells) of lengths the TMA line kernel does not
// take (n_uz = 24, 40, 48): each warp stages 32 rows through shared memory with coalesced
// 16-byte loads (padded pitch), each lane marches its row in registers, and the warp
// writes the rows back the same way.  Rows [row0, row0 + nrows).
struct RowsArgs {
    int L;
    long long row0, nrows, rows_per_cell;
    const void *cell_coef; // LineCoefT<double> for FP64 storage, else LineCoefT<float>
    unsigned *err;
    float *scale;  // 16-bit storage: the FP32 scale of each row, refreshed by the sweep (else null)
    unsigned seed; // 16-bit storage: stochastic-rounding stream of this sweep
    FastDivU32 div_rpc; // set by launch_rows_sweep: division by rows_per_cell
};
// u_z rows of L = 24, 40 or 48 cells (dtype 0 f64, 1 f32, 2 bf16, 3 f16), in place or src -> dst
bool rows_sweep_supported(int L, int dtype);
cudaError_t launch_rows_sweep(const void *src, void *dst, const RowsArgs &a, int dtype, cudaStream_t st);
bool reg_lines_supported(int L);
// dtype: 1 f32, 2 bf16, 3 f16
cudaError_t launch_reg_lines(const void *src, void *dst, const RegLineArgs &a, int dtype, cudaStream_t st);
int occupancy_strided(int dtype, int periodic, size_t smem);
int occupancy_contig(int dtype, size_t smem);
cudaError_t launch_line_sweep(const CUtensorMap &map, const CUtensorMap &dmap, const ContigArgs<float> &a, int nu,
                              int dtype, int grid, cudaStream_t st, bool fuse_y = false);

// ----------------------------------------------------------------------------
// fields: velocity-sweep coefficients, moment, Poisson
// ----------------------------------------------------------------------------
struct GridDims {
    int n[3];
    int nu[3];
    double L, V;
};

// ----------------------------------------------------------------------------
// adjoint sweep (reverse mode, FP32 / FP64 storage): one thread per line
// ----------------------------------------------------------------------------
// f viewed as [O][L][I]; line t = (outer t / I, inner t % I).  Constants as in
// the forward sweep: coef_mode 0 = table[(inner / vstride) % nvel] (position),
// 1 = cell_coef[outer / outer_per_cell] (velocity).  lam_in = dL/df_out and
// lam_out = dL/df_in (the same array unless a position line shifts whole cells).
template <typename C> struct AdjArgs {
    int L;
    int periodic;
    long long n_inner, n_outer, nlines;
    long long vstride;
    int nvel;
    int coef_mode;
    long long outer_per_cell;
    const LineCoefT<C> *cell_coef;
    unsigned *err;
    const void *f_in;
    const void *lam_in;
    void *lam_out;
    double *dLdg;             // velocity sweeps: dL/dg per spatial cell (may be null)
    long long lines_per_cell; // velocity sweeps: cell = t / lines_per_cell
    double dnu_dg;            // -dt / du
    double *block_part;       // non-null: every block lies in one cell; block sums go here (no atomics)
    int perm_line;            // > 0 (z sweep): the Courant number changes sign in the middle of each u_z
                              // line of this length; a block's first half of threads takes the u_z < 0
                              // halves of its lines and the second half the rest (whole warps of one sign)
    // set by the launchers: fast32 = 1 when line indices and divisors fit 32 bits
    int fast32;
    FastDivU32 div_inner, div_vstride, div_nvel, div_opc, div_lpc;
    LineCoefT<C> table[kMaxVel];
};

// rows = true: u_z lines of 8, 16 or 32 cells, one row per thread in registers (FP32: dtype 1)
bool adjoint_rows_supported(int L, int dtype);
cudaError_t launch_adjoint_f32(const AdjArgs<float> &a, bool rows, cudaStream_t st);
cudaError_t launch_adjoint_f64(const AdjArgs<double> &a, bool rows, cudaStream_t st);
// lines (threads) per block of the adjoint kernel of axis (rows: the u_z row kernels; L: line length)
int adjoint_block(int axis, bool rows, int L);
// dLdg[c] += fac * sum_q part[c * blocks_per_cell + q] in order
cudaError_t launch_cell_sum(long long ncell, int blocks_per_cell, const double *part, double fac, double *dLdg,
                            cudaStream_t st);
// dL/dphi += G_d^T dL/dg (FP64, nx*ny*nz)
cudaError_t launch_gradient_adjoint(const GridDims &g, const double *dLdg, int d, double *dLdphi, cudaStream_t st);

// For each axis d with bit d set in mask: coef[d][cell] for a velocity sweep
// of length dt from the 4th-order gradient of phi (FP32, nx*ny*nz).
cudaError_t launch_velocity_coef(const GridDims &g, const float *phi, double dt, int mask,
                                 void *coef_x, void *coef_y, void *coef_z, int dtype, unsigned *err,
                                 cudaStream_t st);

cudaError_t launch_moment(const GridDims &g, const void *f, int dtype, double *rho, cudaStream_t st,
                          int sm_count);
// 16-bit storage (dtype 2 bf16, 3 f16) with one scale per u_z line
cudaError_t launch_moment_coded(const GridDims &g, const void *f, const float *scale, int dtype, double *rho,
                                cudaStream_t st, int sm_count);
// density, mean velocity [3][ncell] and dispersion tensor [6][ncell] (xx, yy, zz, xy,
// xz, yz) per spatial cell; any output may be null; scale: 16-bit storage only
cudaError_t launch_moments(const GridDims &g, const void *f, const float *scale, int dtype, double *rho,
                           double *umean, double *sigma2, cudaStream_t st, int sm_count);
// lam (+)= du^3 dLdrho(x) over each velocity cube (FP64 or FP32 lam: dtype 0 / 1)
cudaError_t launch_moment_adjoint(const GridDims &g, const double *dLdrho, int dtype, void *lam, int accumulate,
                                  cudaStream_t st, int sm_count);
// y += x (or y = x when assign), FP64, n values
cudaError_t launch_add(long long n, const double *x, double *y, bool assign, cudaStream_t st);
// 16-bit storage codec over nlines u_z lines of nuz values (codec.cu): src / dst FP64 or
// FP32 (dtype 0 / 1), codes BF16 or FP16 (code_dtype 2 / 3), one FP32 scale per line
cudaError_t launch_encode(long long nlines, int nuz, const void *src, int src_dtype, void *codes, int code_dtype,
                          float *scale, cudaStream_t st, int sm_count);
cudaError_t launch_decode(long long nlines, int nuz, const void *codes, int code_dtype, const float *scale, void *dst,
                          int dst_dtype, cudaStream_t st, int sm_count);
// mass = dx dy dz * sum rho (FP64, compensated) written to out (device)
cudaError_t launch_mass(const GridDims &g, const double *rho, double *out, cudaStream_t st);

// scratch of the spectral solve: 2 complex buffers of nx*ny*nz and twiddles
struct PoissonScratch {
    double2 *z0, *z1;
    double2 *tw[3]; // tw[d][q] = (cos, sin)(2 pi q / n_d)
};
// phi (FP32) and / or phi64 (FP64) receive the solution (either may be null)
cudaError_t launch_poisson(const GridDims &g, const PoissonScratch &ps, const double *rho,
                           const double *rho_bg, double a, double four_pi_G, float *phi,
                           cudaStream_t st, double *phi64 = nullptr);

} // namespace vk
