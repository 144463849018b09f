/*
 * vlasov.h -- C ABI of libvlasov, the GB300 (sm_103a) hot path of the split 6D
 * Vlasov solver for relic neutrinos (Yoshikawa, Tanaka & Yoshida, SC'21).
 *
 * The library advances the neutrino distribution function f(x, u) on a
 * uniform 6D grid with the directionally split scheme of Eq. (5): three 1D
 * position advections, Eq. (3), and three 1D velocity advections, Eq. (4),
 * each done by SL-MPP5 (Sec. 4.2: conservative semi-Lagrangian flux, one
 * flux evaluation per step, monotonicity- and positivity-preserving
 * constraints), and reduces f to the density rho_nu(x) = int f d^3u that feeds
 * the Poisson equation, Eq. (2).
 *
 * Conventions for every entry point
 *   - Pointers named *_dev are CUDA device pointers; *_host are host pointers.
 *   - The caller owns every buffer it passes (f, scale, phi, rho, lambda).
 *     The library owns only its scratch, allocated in vlasov_init and freed by
 *     vlasov_destroy.
 *   - All GPU work is queued on the context's stream and is asynchronous
 *     unless the entry point says it synchronises.
 *   - Return value 0 = success, a negative VLASOV_E* code on failure; the
 *     message is available from vlasov_last_error().  No C++ exception and
 *     no device trap crosses this boundary.  Errors detected on the device
 *     (a velocity Courant number >= 1, a NaN, a bounded wait that ran out)
 *     are sticky in a device word and are returned by vlasov_status().
 *
 * Grid and layout
 *   f is one array f[ix][iy][iz][jx][jy][jz] with jz fastest (Listing 1 keeps
 *   each spatial cell's velocity cube contiguous with u_z innermost).
 *   Spatial cell centres x_i = (i + 1/2) L / n, periodic on 0 <= x < L
 *   (Sec. 4.1.3).  Velocity cell centres u_j = -V + (j + 1/2) du, du = 2V/n_u,
 *   on -V <= u < V; the outer velocity faces carry no flux.
 */
#ifndef VLASOV_H
#define VLASOV_H

#ifdef __cplusplus
extern "C" {
#endif

#define VLASOV_OK 0
#define VLASOV_EINVAL (-1)   /* bad argument: axis, size, null or misaligned pointer */
#define VLASOV_ECFL (-2)     /* a velocity-sweep Courant number |nu| >= 1           */
#define VLASOV_ECUDA (-3)    /* a CUDA runtime call failed                            */
#define VLASOV_ENAN (-4)     /* a sweep produced a NaN/Inf or a negative line sum     */
#define VLASOV_ETIMEOUT (-5) /* a bounded device wait ran out (kernel returned early) */
#define VLASOV_ENOMEM (-6)   /* scratch allocation failed                             */

/* storage type of f */
#define VLASOV_F64 0
#define VLASOV_F32 1
#define VLASOV_BF16 2
#define VLASOV_F16 3

typedef struct vlasov_ctx vlasov_ctx; /* opaque, owned by the library */

typedef struct {
    int nx, ny, nz;    /* spatial cells (each >= 4, <= 256)                    */
    int nux, nuy, nuz; /* velocity cells (each >= 4, <= 128, multiple of 4)    */
    double L;          /* box side                                              */
    double V;          /* velocity half-extent: -V <= u < V                     */
    int dtype;         /* VLASOV_F64 / F32 / BF16 / F16 (storage type of f)     */
} vlasov_grid;

/*
 * Create a context for the grid g and the caller's distribution function
 * f_dev (nx*ny*nz*nux*nuy*nuz elements of g->dtype, 16-byte aligned).
 * scale_dev must be NULL for F64/F32.  BF16 / F16 storage (the 16-bit codec):
 * f holds codes, value = code x the FP32 scale of its u_z line; scale_dev holds
 * nx*ny*nz*nux*nuy floats (16-byte aligned, caller-owned), refreshed by every
 * u_z sweep to the line's largest value (BF16: at least 2^-64); nuz must be 16
 * or 32 with nux*nuy a multiple of 256, or 24, 40 or 48; arithmetic is FP32 and
 * every encode rounds stochastically.  stream is a cudaStream_t (NULL = the
 * legacy default stream).  Allocates the library's scratch on the current
 * device.  On success *out receives the context.  Errors: VLASOV_EINVAL for a
 * grid outside these limits or a misaligned / missing / unexpected pointer.
 */
int vlasov_init(vlasov_ctx **out, const vlasov_grid *g, void *f_dev, float *scale_dev,
                void *stream);

/* Free the scratch and the context (synchronises the stream).  NULL is a no-op. */
void vlasov_destroy(vlasov_ctx *ctx);

/* Queue all later work of ctx on this cudaStream_t. */
int vlasov_set_stream(vlasov_ctx *ctx, void *stream);

/*
 * Point ctx at another distribution function of the same grid and storage type
 * (and, for 16-bit storage, its scale array); later calls read and update that
 * array.  The caller keeps ownership of both arrays.  Host work only.
 */
int vlasov_set_f(vlasov_ctx *ctx, void *f_dev, float *scale_dev);

/*
 * One directional sweep D_axis(dt) of f in place (Eq. 3 for axis 0..2 =
 * x, y, z; Eq. 4 for axis 3..5 = u_x, u_y, u_z).
 *   Position sweep i: Courant number nu_j = u_j dt / (a^2 dx_i) for each
 *   velocity column j (any magnitude: whole-cell shifts are exact);
 *   phi_dev is ignored.
 *   Velocity sweep i: nu(x) = -g_i(x) dt / du_i, g_i the periodic 4th-order
 *   central difference of phi_dev (nx*ny*nz FP32, C order).  |nu| must be < 1
 *   in every cell; a cell that breaks it is left unchanged and VLASOV_ECFL is
 *   raised through vlasov_status().  a is ignored.
 */
int vlasov_sweep(vlasov_ctx *ctx, int axis, double dt, double a, const float *phi_dev);

/*
 * The 16-bit storage codec, for getting a distribution function into and out of
 * BF16 / FP16 storage (vlasov_init with VLASOV_BF16 or VLASOV_F16).  The paper
 * keeps f in FP32 (Sec. 5.1); this storage and its codec are the library's own.
 * Both calls work on nlines u_z lines of nuz values each (1 <= nuz <= 128), laid
 * out one line after another (a whole grid is nx*ny*nz*nux*nuy lines of nuz; a
 * slab of x-planes is a contiguous part of it); they need no context, allocate
 * nothing and queue one kernel on stream (a cudaStream_t, NULL = legacy default).
 *
 * vlasov_encode: src_dev holds the values (src_dtype VLASOV_F64 or VLASOV_F32).
 * For each line, with w_k = v_k rounded to FP32 (to nearest even):
 *   scale_dev[line] = s = max(max_k w_k, 0), for BF16 codes at least 2^-64 (the
 *                     floor the sweeps keep on every scale refresh),
 *   codes_dev[line * nuz + k] = w_k / s (IEEE FP32 quotient) rounded to nearest
 *                     even in code_dtype (VLASOV_BF16 or VLASOV_F16); 0 where s = 0.
 * The values of a distribution function are non-negative, so codes lie in [0, 1].
 * vlasov_decode: dst_dev[line * nuz + k] = code x scale, exact for
 * dst_dtype = VLASOV_F64, rounded to nearest even for VLASOV_F32.
 * Every pointer is a device pointer aligned to its element size; the caller owns
 * all of them.  Errors (VLASOV_EINVAL for sizes, types, null or misaligned
 * pointers; VLASOV_ECUDA for a failed launch) are returned with the message in
 * vlasov_last_error(NULL).
 */
int vlasov_encode(long long nlines, int nuz, const void *src_dev, int src_dtype, void *codes_dev, int code_dtype,
                  float *scale_dev, void *stream);
int vlasov_decode(long long nlines, int nuz, const void *codes_dev, int code_dtype, const float *scale_dev,
                  void *dst_dev, int dst_dtype, void *stream);

/*
 * How the kicks of vlasov_step and vlasov_kick (D_uz D_uy D_ux, Eq. 5) run.
 *   mode 2 (the default): with n_ux = n_uy = n_uz = 16 or 32 (FP32, BF16 or FP16
 *     storage) the whole kick runs in one pass over f: each spatial cell's velocity
 *     cube goes through shared memory once and the three sweeps run on it there
 *     (a kick never leaves the cell, Sec. 4.1.3).  The result equals the separate
 *     sweeps bit for bit, for 16-bit storage too (the same rounding points and
 *     stochastic-rounding streams: D_ux encodes with the line scales it kept, D_uy
 *     stays FP32, D_uz refreshes the scales and encodes).  Other shapes fall back
 *     to mode 1.
 *   mode 1: D_ux alone, then D_uy and D_uz in one pass over f where n_uy = n_uz =
 *     16 or 32: each u_z tile of 256 rows holds whole (cell, j_x) planes, whose
 *     columns are the u_y lines, so D_uy runs on the staged tile before D_uz (FP32:
 *     the separate sweeps bit for bit; 16-bit storage: D_uy's result stays FP32 in
 *     shared memory and only D_uz's is encoded); and with n_uy = n_uz = 48 (n_ux a
 *     multiple of 4), over four staged (cell, j_x) planes per block (FP32: the
 *     separate sweeps bit for bit; 16-bit: decoded as staged, encoded once after
 *     D_uz with refreshed line scales).
 *   mode 0: three separate sweeps.
 * FP64 storage always runs the sweeps separately.  Errors: VLASOV_EINVAL for
 * another mode.
 */
int vlasov_set_fused_kick(vlasov_ctx *ctx, int mode);

/*
 * One kick of Eq. (5): D_uz D_uy D_ux (dt), D_ux first, with the acceleration
 * -grad phi (phi_dev: FP32 potential on the device, nx*ny*nz, as for
 * vlasov_sweep).  vlasov_step runs it with dt/2 before and after the drift; it runs
 * as vlasov_set_fused_kick selects.  Same errors as vlasov_sweep.
 */
int vlasov_kick(vlasov_ctx *ctx, double dt, const float *phi_dev);

/*
 * Staged tiles.  Position sweeps (Eq. 3, |nu| < 1) with lines of 16, 24, 32, 48 or
 * 64 cells (FP32) or of 16-96 cells with n_uz = 32 and of 48 cells with n_uz = 48
 * (BF16 / FP16), and a multiple of 256 cells on the faster axes, run with whole
 * lines staged in shared memory: each tile of 256 lines x all their cells is
 * loaded once, every line is marched by one thread and the tile is stored once.
 * The u_x sweep (Eq. 4) with n_ux = 48 (FP32; 16-bit with n_uz = 48) and n_uy n_uz
 * a multiple of 256 runs on the same tiles of [cell][u_x][u_y u_z] when the kick
 * does not take the one-pass kernel.  FP32 results equal the streamed and
 * register-line sweeps bit for bit; 16-bit results draw their own rounding
 * streams.  On by default; on = 0 runs the streamed / register-line sweeps, which
 * FP64 storage and other shapes always use.
 */
int vlasov_set_position_tiles(vlasov_ctx *ctx, int on);

/*
 * The moment rho_nu that vlasov_step and vlasov_step_record_sc take after the
 * drift (Eq. 5, Sec. 4.1.3) is summed by the x sweep itself when that sweep is
 * streamed (|nu| < 1 in every velocity column) on FP32 or FP64 storage and the
 * velocity cube is a multiple of 256 (FP32) or 128 (FP64) cells: a moment warp in
 * each block adds up every output row the block writes (pairwise, FP32 for FP32
 * storage, at most 8 roundings deep) and a second kernel adds each cell's partials
 * in FP64 in a fixed order, so f is read once less per step.  The result equals
 * vlasov_moment's to rounding (within 10 units in the last place of FP32;
 * reproducible run to run).  Needs ncell x cube / 64 bytes of device memory (FP32
 * and FP64), allocated on first use (without it the separate moment kernel runs).
 * On by default; on = 0 always runs the separate moment kernel.
 */
int vlasov_set_fused_moment(vlasov_ctx *ctx, int on);

/*
 * rho_nu(x) = du_x du_y du_z * sum over the velocity cube of f (Sec. 4.1.3),
 * written to rho_dev (nx*ny*nz FP64).  Each cell sum is formed from
 * compensated FP32 partial sums combined in FP64.  If mass_host is non-NULL
 * the call synchronises and stores dx dy dz * sum_x rho_nu there.
 */
int vlasov_moment(vlasov_ctx *ctx, double *rho_dev, double *mass_host);

/*
 * The velocity moments the paper keeps per spatial cell (Sec. 4.1.3, Listing 1:
 * mass density, mean velocity, velocity dispersion tensor), as sums over the
 * velocity cell centres u_j: S0 = sum f, S1_i = sum u_i f, S2_ij = sum u_i u_j f.
 *   rho_dev    nx*ny*nz FP64: du_x du_y du_z S0
 *   umean_dev  3*nx*ny*nz FP64, component-major [3][nx][ny][nz]: S1_i / S0
 *   sigma2_dev 6*nx*ny*nz FP64, [6][nx][ny][nz] in the order xx, yy, zz, xy, xz,
 *              yz: S2_ij / S0 - umean_i umean_j
 * (umean and sigma2 are 0 where S0 = 0).  Any output may be NULL (not all).
 * One pass over f, per-thread FP32 compensated sums (FP64 for FP64 storage)
 * combined in FP64 in a fixed order; any storage type.
 */
int vlasov_moments(vlasov_ctx *ctx, double *rho_dev, double *umean_dev, double *sigma2_dev);

/*
 * Eq. (2): solve nabla^2 phi = four_pi_G a^2 (rho - mean rho) on the periodic
 * spatial grid by a discrete Fourier transform (continuous |k|^2 =
 * (2 pi n / L)^2, the k = 0 mode set to zero).  rho = rho_dev + rho_bg_dev
 * (rho_bg_dev may be NULL), both nx*ny*nz FP64.  phi_dev receives FP32.
 */
int vlasov_poisson(vlasov_ctx *ctx, const double *rho_dev, const double *rho_bg_dev, double a,
                   double four_pi_G, float *phi_dev);

/*
 * One time step of Eq. (5), operators applied right to left:
 *   kick  D_ux, D_uy, D_uz (dt/2) with phi_n,
 *   drift D_z, D_y, D_x (dt) at scale factor a_half,
 *   kick  D_ux, D_uy, D_uz (dt/2) with phi_next if non-NULL, else phi_n.
 * If phi_next_dev is non-NULL the step is self-consistent: after the drift
 * rho_nu + rho_bg_dev (FP64, may be NULL) is turned into phi_next by
 * vlasov_poisson at a_full.  rho_nu_dev (FP64, may be NULL) receives the
 * post-drift moment.
 */
int vlasov_step(vlasov_ctx *ctx, double dt, double a_half, double a_full, const float *phi_n_dev,
                const double *rho_bg_dev, double four_pi_G, float *phi_next_dev,
                double *rho_nu_dev);

/*
 * Copy the whole distribution function between a caller's host buffer
 * (nx*ny*nz*nux*nuy*nuz elements of the storage type; pinned memory makes the
 * copy asynchronous) and the context's device array f, on the context stream.
 * The host buffer must stay valid until the stream reaches the copy.
 */
int vlasov_upload(vlasov_ctx *ctx, const void *f_host);
int vlasov_download(vlasov_ctx *ctx, void *f_host);

/*
 * One Eq. (5) step of a distribution function held in host memory: f_host is
 * read, stepped and written back in place (the same result as vlasov_upload,
 * vlasov_step, vlasov_download; the other arguments as for vlasov_step).  The
 * velocity sweeps and D_z, D_y are local to planes of constant x, so f moves in
 * up to 16 x-slabs on a second stream: each slab's first kick and D_z, D_y start
 * as soon as it has arrived, and each slab goes back as soon as its second kick
 * is done; only D_x, the moment and the Poisson solve wait for the whole grid.
 * Without pinned host memory the copies do not overlap.  Falls back to the
 * three calls in sequence for 16-bit storage, a whole-cell shift in D_z or D_y,
 * or a grid whose tiles do not fall on x-planes.
 *
 * Ordering.  The uploads run on a stream of the library's own after the work
 * queued on the context stream before the call; the downloads on another, and
 * the call returns with them queued, not waited for.  The next vlasov_step_host
 * on the same slabs starts each slab's upload once the download of that slab is
 * done, and nothing else (so one step's downloads and the next step's uploads
 * share the link, one direction each); every other call of this library on the
 * context, and vlasov_host_wait, first makes the context stream wait for all of
 * them.  Work the caller queues on the stream itself after vlasov_step_host that
 * reads the host buffer or reads or writes f on the device comes after
 * vlasov_host_wait (or vlasov_status, which synchronises); other work (reading
 * rho_nu or phi^{n+1}, say) need not.  f_host must stay valid until then.
 */
int vlasov_step_host(vlasov_ctx *ctx, void *f_host, double dt, double a_half, double a_full,
                     const float *phi_n_dev, const double *rho_bg_dev, double four_pi_G, float *phi_next_dev,
                     double *rho_nu_dev);

/*
 * Make the context stream wait for the downloads of the last vlasov_step_host
 * (a no-op when none are outstanding).  Queues the wait and returns; the
 * paper has no counterpart (it keeps f in memory).  VLASOV_EINVAL for a null
 * context.
 */
int vlasov_host_wait(vlasov_ctx *ctx);

/*
 * Failure-path self-test (no counterpart in the paper).  Queues one kernel whose
 * thread waits, with the library's bounded device wait (the wait of every TMA
 * kernel for a copy or a peer; 2 s at most), for an mbarrier phase that nothing
 * completes: the wait runs out, the kernel records the timeout in the context's
 * error word and returns, with nothing left in flight.  The next vlasov_status
 * returns VLASOV_ETIMEOUT and clears the word; the context stays usable.  No fault,
 * trap or endless loop is involved.  VLASOV_EINVAL for a null context.
 */
int vlasov_selftest_wait(vlasov_ctx *ctx);

/*
 * Per-part timers (the paper times each part of a step, Sec. 5.1).  While
 * enabled, every kernel the library queues is bracketed by two CUDA events on
 * the context stream.  vlasov_read_timers synchronises the stream and, for each
 * kind k < nkinds, writes the summed event time in ms to ms[k] (may be NULL)
 * and the number of kernel launches to launches[k] (counted whether or not
 * timers are enabled), then resets both.
 */
#define VLASOV_T_SWEEP_X 0 /* kinds 0..5: sweeps along x, y, z, u_x, u_y, u_z */
#define VLASOV_T_MOMENT 6
#define VLASOV_T_POISSON 7
#define VLASOV_T_COEF 8 /* velocity-sweep constants (potential gradient)      */
#define VLASOV_T_MASS 9
#define VLASOV_T_ADJ_X 10     /* kinds 10..15: adjoint sweeps along x, y, z, u_x, u_y, u_z */
#define VLASOV_T_GRAD_ADJ 16  /* transposed potential gradient of the step adjoint   */
#define VLASOV_T_MOMENT_ADJ 17 /* moment adjoint                                      */
#define VLASOV_T_SWEEP_UYUZ 18 /* fused kick tail D_uz D_uy (see vlasov_set_fused_kick) */
#define VLASOV_T_MOMENTS 19    /* vlasov_moments                                      */
#define VLASOV_T_KICK 20       /* one-pass kick D_uz D_uy D_ux (see vlasov_set_fused_kick) */
#define VLASOV_T_KINDS 21
int vlasov_enable_timers(vlasov_ctx *ctx, int on);
int vlasov_read_timers(vlasov_ctx *ctx, double *ms, long long *launches, int nkinds);

/*
 * Velocity sweep for callers that must not allocate device memory: code that
 * runs under a fixed memory budget reserved up front, an allocator that is
 * closed after start-up, or a host framework that owns every allocation and
 * forbids the library from calling cudaMalloc.  The paper has no counterpart;
 * this is a deployment variant of vlasov_sweep for axis 3..5 (u_x, u_y, u_z)
 * on FP32 storage, with the same arithmetic and the same kernels.
 *
 * It creates no context and calls no cudaMalloc / cudaFree or any allocating
 * routine.  Its scratch (the per-cell sweep constants and an error word) is a
 * static device array built into the library, VLASOV_STATIC_MAX_CELLS spatial
 * cells in size (about 1.2 MB, held on every GPU that loads the library until
 * the process exits).  Grids with more spatial cells are rejected with
 * VLASOV_EINVAL.  Every call looks up the array's device address on the
 * current device (cudaGetSymbolAddress), so the address stays right after a
 * cudaDeviceReset; the first call on a device loads the library's kernels
 * there, so make that first call before any stream capture.  All calls share
 * the one array, which keeps the last call's contents: calls that may overlap
 * on the GPU (different streams, different host threads) race and must be
 * serialised by the caller.
 *
 *   g        grid (dtype must be VLASOV_F32); f_dev as for vlasov_init
 *   axis     3, 4 or 5; dt, phi_dev as for vlasov_sweep
 *   status_dev  device word (may be NULL) into which the sweep ORs its
 *            device-side error bits: 1 = a cell's |nu| >= 1 (that cell is
 *            left unchanged), 2 = NaN/Inf or negative line sum, 4 = a bounded
 *            wait ran out.  With NULL those bits are dropped.
 *   stream   cudaStream_t the work is queued on (asynchronous).
 * Host-side failures return a negative code; the message is
 * vlasov_last_error(NULL).
 */
#define VLASOV_STATIC_MAX_CELLS 32768
int vlasov_sweep_velocity_static(const vlasov_grid *g, float *f_dev, int axis, double dt,
                                 const float *phi_dev, unsigned int *status_dev, void *stream);

/*
 * Adjoint (reverse mode) of one sweep, for gradients of a loss L through the
 * solver.  The paper has no counterpart: it is the transpose of the sweep's
 * Jacobian at the sweep input, with every limiter choice (min / max / clamp of
 * Sec. 4.2's monotonicity and positivity constraints) frozen at the branch
 * the forward evaluation takes there.
 *   f_in_dev  the sweep's input (same grid and storage type as ctx; FP32 or
 *             FP64 only), read only;
 *   lam_dev   on entry dL/df_out, on exit dL/df_in (same layout as f; must not
 *             be f_in_dev; 16-byte aligned), updated in place;
 *   axis, dt, a, phi_dev  as for vlasov_sweep;
 *   dLdg_dev  velocity sweeps only (else ignored, may be NULL): nx*ny*nz FP64
 *             to which dL/dg_i(x) is ADDED, g_i the potential gradient that
 *             sets the Courant number nu(x) = -g_i(x) dt / du_i.
 * A whole-cell shift of a position sweep (|nu| >= 1) uses a scratch copy of
 * lambda allocated on first use.
 */
int vlasov_sweep_adjoint(vlasov_ctx *ctx, const void *f_in_dev, void *lam_dev, int axis, double dt,
                         double a, const float *phi_dev, double *dLdg_dev);

/*
 * Adjoint of vlasov_moment: rho_nu(x) = du_x du_y du_z sum_u f(x, u), so
 * lam_dev(x, u) receives du_x du_y du_z * dLdrho_dev(x) for every u (added
 * to its contents when accumulate != 0, else written).  dLdrho_dev is
 * nx*ny*nz FP64; lam_dev has f's layout and storage type (FP32 / FP64 only).
 */
int vlasov_moment_adjoint(vlasov_ctx *ctx, const double *dLdrho_dev, void *lam_dev, int accumulate);

/*
 * One vlasov_step with an external potential (both kicks use phi_dev, the
 * drift uses a_half), run out of place so that the input of every sweep is
 * kept: rec_dev is a HOST array of 8 device arrays the size of f, and
 * rec_dev[k] receives the input of sweep k + 1 (sweep 0 reads f_n_dev, which
 * is not changed).  f_next_dev (may be NULL) receives the step's result.
 * ctx's own array f is neither read nor changed.  Each sweep reads one array
 * and writes the next, so recording costs no copies.
 */
int vlasov_step_record(vlasov_ctx *ctx, const void *f_n_dev, void *const *rec_dev, void *f_next_dev,
                       double dt, double a_half, const float *phi_dev);

/*
 * Adjoint of one vlasov_step with an external potential (phi_next_dev NULL:
 * both kicks use phi_dev, the drift uses a_half), from the sweep inputs that
 * vlasov_step_record kept (rec_dev as there, read only).  f_n_dev is the state
 * at the start of the step (read only); lam_dev holds dL/df^{n+1} on entry
 * and dL/df^n on exit.  The nine adjoint sweeps run last to first.  If
 * dLdphi_dev (nx*ny*nz FP64) is non-NULL, dL/dphi is ADDED to it: each
 * velocity sweep's dL/dg_i goes through the transposed 4th-order gradient.
 */
int vlasov_step_adjoint_recorded(vlasov_ctx *ctx, const void *f_n_dev, const void *const *rec_dev,
                                 void *lam_dev, double dt, double a_half, const float *phi_dev,
                                 double *dLdphi_dev);

/*
 * Self-consistent versions (Eq. 5 with phi^{n+1} from the post-drift moment,
 * as vlasov_step with phi_next_dev): the state is (f, phi).
 *
 * vlasov_step_record_sc: one step from f_n_dev and phi_n_dev, out of place,
 * keeping the input of every sweep in rec_dev (as vlasov_step_record);
 * phi_next_dev (FP32, required) receives phi^{n+1}, rho_nu_dev (FP64, may be
 * NULL) the post-drift moment; rho_bg_dev, four_pi_G, a_full as vlasov_step.
 *
 * vlasov_step_adjoint_recorded_sc: from those records and both potentials,
 * lam_dev <- dL/df^n (in: dL/df^{n+1}).  lam_phi_next_dev (FP64, may be NULL)
 * is dL/dphi^{n+1} from later steps; dL/dphi_n and dL/drho_bg are ADDED to
 * dLdphi_n_dev and dLdrho_bg_dev (FP64, either may be NULL).  Order: second
 * kick (whose dL/dg adds to dL/dphi^{n+1}), the Poisson solve (a real
 * circulant with an even multiplier: its own transpose, applied in FP64),
 * the moment (dL/df += du^3 dL/drho), drift, first kick.  The FP32 rounding
 * of phi^{n+1} passes gradients unchanged.  The paper has no counterpart.
 */
int vlasov_step_record_sc(vlasov_ctx *ctx, const void *f_n_dev, void *const *rec_dev, void *f_next_dev,
                          double dt, double a_half, double a_full, const float *phi_n_dev,
                          const double *rho_bg_dev, double four_pi_G, float *phi_next_dev,
                          double *rho_nu_dev);
int vlasov_step_adjoint_recorded_sc(vlasov_ctx *ctx, const void *f_n_dev, const void *const *rec_dev,
                                    void *lam_dev, double dt, double a_half, double a_full,
                                    const float *phi_n_dev, const float *phi_next_dev, double four_pi_G,
                                    const double *lam_phi_next_dev, double *dLdphi_n_dev,
                                    double *dLdrho_bg_dev);

/*
 * vlasov_step_record into eight scratch arrays the size of f (allocated on
 * the first call, kept until vlasov_destroy) followed by
 * vlasov_step_adjoint_recorded.  Arguments as there.  When eight arrays do not
 * fit on the device (or vlasov_set_adjoint_arrays(ctx, 4) asked for it) it uses
 * four: it keeps the inputs of sweeps 3 and 6 and rebuilds the other inputs of
 * each group of three sweeps before their adjoints (12 forward sweeps instead of
 * 8, the same results).
 */
int vlasov_step_adjoint(vlasov_ctx *ctx, const void *f_n_dev, void *lam_dev, double dt, double a_half,
                        const float *phi_dev, double *dLdphi_dev);

/* Scratch arrays the size of f that vlasov_step_adjoint may hold: 8, 4, or 0 =
 * 8 when they fit, else 4 (the default).  Arrays already held are kept. */
int vlasov_set_adjoint_arrays(vlasov_ctx *ctx, int arrays);

/*
 * Synchronise the stream, read and clear the device error word.  Returns 0 or
 * the first of VLASOV_ETIMEOUT, VLASOV_ENAN, VLASOV_ECFL that was raised.
 */
int vlasov_status(vlasov_ctx *ctx);

/* Message of the last failure on ctx (or of the last failed vlasov_init when ctx is NULL). */
const char *vlasov_last_error(const vlasov_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* VLASOV_H */
