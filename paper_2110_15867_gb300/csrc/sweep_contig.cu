// sweep_contig.cu -- SL-MPP5 sweep along the contiguous axis u_z.
//
// Eq. (4) for i = 3 (Yoshikawa, Tanaka & Yoshida, SC'21).  A u_z line is a
// row of nuz contiguous cells.  A thread marching a row of a dense
// [rows][nuz] tile would hit one shared-memory bank with all 32 lanes, so the
// tile goes through a transpose in shared memory first: the GPU counterpart of
// the paper's "load and transpose" (LAT, Sec. 4.3), which loads contiguous
// rows and transposes them so that one SIMD lane walks one line.
//
// Per tile of R rows (R = consumer threads):
//   TMA-load the dense box {nuz, R} -> transpose into B[nuz][R + 1]
//   (compute type; the odd row pitch makes both transposes conflict-free)
//   -> thread r marches column r of B -> transpose back -> TMA-store.
// The producer / consumer pipeline and the bounded waits are those of the
// strided sweep.
#include "vk_common.cuh"

namespace vk {

// all consumer threads agree on a failure flag (named barrier 1, reduction)
__device__ __forceinline__ bool consumer_any(bool v, int nthreads)
{
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(int(v)), "r"(nthreads)
        : "memory");
    return r != 0;
}

template <typename T>
__global__ void __launch_bounds__(kConsumers + kProducer)
    contig_sweep_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap dmap,
                        const __grid_constant__ ContigArgs<typename Compute<T>::type> args)
{
    using C = typename Compute<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = args.stages;
    const int L = args.L, R = args.R;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *done = full + S;
    const int tile_elems = L * R;
    const unsigned tile_bytes = unsigned(tile_elems * sizeof(T));
    T *stage0 = reinterpret_cast<T *>(smem + 128);
    const size_t stage_bytes = (size_t(tile_bytes) + 127) & ~size_t(127);
    C *B = reinterpret_cast<C *>(smem + 128 + stage_bytes * S);
    const int pitch = R + 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&done[s], kConsumers);
        }
        fence_barrier_init();
    }
    __syncthreads();

    const long long G = gridDim.x, b = blockIdx.x;
    const long long n_my = (args.num_tiles > b) ? (args.num_tiles - b + G - 1) / G : 0;
    auto stage_ptr = [&](int st) { return reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(stage0) + stage_bytes * st); };

    if (threadIdx.x < kProducer) {
        if (threadIdx.x != 0) return;
        bool ok = true;
        long long issued = 0;
        for (long long k = 0; k < n_my; ++k) {
            const int st = int(k % S);
            if (k >= S) {
                const long long kp = k - S;
                if (!mbar_wait_bounded(&done[st], unsigned((kp / S) & 1))) { ok = false; break; }
                tma_store_2d(&dmap, stage_ptr(st), 0, int((b + kp * G) * R));
                bulk_commit();
                bulk_wait_read_all();
            }
            mbar_arrive_expect_tx(&full[st], tile_bytes);
            tma_load_2d(stage_ptr(st), &map, &full[st], 0, int((b + k * G) * R));
            ++issued;
        }
        if (ok) {
            for (long long kp = (n_my > S ? n_my - S : 0); kp < n_my; ++kp) {
                const int st = int(kp % S);
                if (!mbar_wait_bounded(&done[st], unsigned((kp / S) & 1))) { ok = false; break; }
                tma_store_2d(&dmap, stage_ptr(st), 0, int((b + kp * G) * R));
                bulk_commit();
            }
        }
        bulk_wait_all();
        if (!ok) {
            atomicOr(args.err, ERR_TIMEOUT);
            for (long long t = (issued > S ? issued - S : 0); t < issued; ++t)
                mbar_wait_bounded(&full[t % S], unsigned((t / S) & 1));
        }
        return;
    }

    const int tid = threadIdx.x - kProducer;
    const int r0 = tid / L, j0 = tid - (tid / L) * L;
    const int dr = kConsumers / L, dj = kConsumers - (kConsumers / L) * L;
    for (long long k = 0; k < n_my; ++k) {
        const int st = int(k % S);
        const bool ok = mbar_wait_bounded(&full[st], unsigned((k / S) & 1));
        // the barrier also orders the previous tile's reads of B before the writes below
        if (consumer_any(!ok, kConsumers)) {
            if (tid == 0) atomicOr(args.err, ERR_TIMEOUT);
            break;
        }
        T *A = stage_ptr(st);
        // element e = r L + j of A visits B[j][r]; e advances by kConsumers per pass
        for (int e = tid, r = r0, j = j0; e < tile_elems; e += kConsumers) {
            B[j * pitch + r] = to_c(A[e]);
            r += dr;
            j += dj;
            if (j >= L) { j -= L; ++r; }
        }
        consumer_sync(kConsumers);
        const long long row = (b + k * G) * R + tid;
        if (tid < R && row < args.rows) {
            const LineCoefT<C> kc = args.cell_coef[row / args.rows_per_cell];
            if (kc.nd >= 0) {
                const bool neg = kc.nd & 1;
                C *col = B + tid;
                C *base = neg ? col + size_t(L - 1) * pitch : col;
                const long step = neg ? -long(pitch) : long(pitch);
                const C sum = march_line<C, false, C>(base, step, L, to_lim(kc));
                if (!(sum >= C(0)) || isinf(sum)) atomicOr(args.err, ERR_NAN);
            }
        }
        consumer_sync(kConsumers);
        for (int e = tid, r = r0, j = j0; e < tile_elems; e += kConsumers) {
            A[e] = from_c<T>(B[j * pitch + r]);
            r += dr;
            j += dj;
            if (j >= L) { j -= L; ++r; }
        }
        fence_proxy_async();
        mbar_arrive(&done[st]);
    }
}

template <typename T>
static cudaError_t launch_contig_t(const CUtensorMap &map, const CUtensorMap &dmap, const ContigArgs<typename Compute<T>::type> &a,
                                   int grid, size_t smem, cudaStream_t st)
{
    auto kern = contig_sweep_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, kConsumers + kProducer, smem, st>>>(map, dmap, a);
    return cudaGetLastError();
}

cudaError_t launch_contig_f32(const CUtensorMap &map, const CUtensorMap &dmap, const ContigArgs<float> &a, int grid, size_t smem,
                              cudaStream_t st)
{
    return launch_contig_t<float>(map, dmap, a, grid, smem, st);
}

cudaError_t launch_contig_f64(const CUtensorMap &map, const CUtensorMap &dmap, const ContigArgs<double> &a, int grid, size_t smem,
                              cudaStream_t st)
{
    return launch_contig_t<double>(map, dmap, a, grid, smem, st);
}

int occupancy_contig(int dtype, size_t smem)
{
    const void *k = dtype == 0 ? (const void *)contig_sweep_kernel<double> : (const void *)contig_sweep_kernel<float>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kConsumers + kProducer, smem) != cudaSuccess) return 0;
    return n;
}

} // namespace vk
