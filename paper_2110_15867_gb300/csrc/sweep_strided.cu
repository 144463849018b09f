// sweep_strided.cu -- SL-MPP5 sweeps along a strided axis (x, y, z, u_x, u_y).
//
// Eq. (3) (position advection, periodic) and Eq. (4) (velocity advection,
// zero-flux faces) of Yoshikawa, Tanaka & Yoshida, SC'21, one directional
// sweep at a time as in the split step of Eq. (5).
//
// f is viewed as a 3D tensor [O][L][I]: the swept axis (length L, stride I
// elements) between all slower axes (O) and all faster axes (I).  The GPU
// analogue of the paper's "SIMD over the second innermost loop" (Sec. 4.3):
// threads run over the contiguous inner index, each marching one whole line
// held in shared memory.
//
// Pipeline (one persistent CTA per SM slot):
//   warp 0, lane 0 (producer): TMA-loads box {W, L, P} tiles into a ring of
//     `stages` shared-memory buffers (mbarrier full[s] with transaction
//     bytes), and TMA-stores each finished tile back in place once the
//     consumers release it (mbarrier done[s]); a buffer is reloaded only after
//     the store has read it out.
//   warps 1..8 (consumers): one column each, sliding-window SL-MPP5 update in
//     shared memory, in place.
// Every wait is bounded: on expiry the kernel raises ERR_TIMEOUT in the error
// word and returns.
#include "vk_common.cuh"

namespace vk {

template <typename T, bool PERIODIC>
__global__ void __launch_bounds__(kConsumers + kProducer)
    strided_sweep_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap dmap,
                         const __grid_constant__ StridedArgs<typename Compute<T>::type> args)
{
    using C = typename Compute<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = args.stages;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *done = full + S;
    LineCoefT<C> *tab = reinterpret_cast<LineCoefT<C> *>(smem + 128);
    const size_t tab_bytes = (args.coef_mode == 0) ? ((sizeof(LineCoefT<C>) * args.nvel + 127) & ~size_t(127)) : 0;
    T *stage0 = reinterpret_cast<T *>(smem + 128 + tab_bytes);
    const int L = args.L, W = args.W, P = args.P;
    const int tile_elems = W * L * P;
    const unsigned tile_bytes = unsigned(tile_elems * sizeof(T));
    // stage pitch in elements: each stage starts on a 128-byte boundary
    const size_t stage_elems = ((size_t(tile_bytes) + 127) & ~size_t(127)) / sizeof(T);

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&done[s], kConsumers);
        }
        fence_barrier_init();
    }
    if (args.coef_mode == 0)
        for (int j = threadIdx.x; j < args.nvel; j += blockDim.x) tab[j] = args.table[j];
    __syncthreads();

    const long long G = gridDim.x, b = blockIdx.x;
    const long long n_my = (args.num_tiles > b) ? (args.num_tiles - b + G - 1) / G : 0;
    auto tile_coords = [&](long long t, int &ci, int &co) {
        const long long ti = t % args.tiles_inner;
        const long long to = t / args.tiles_inner;
        ci = int(ti * W);
        co = int(to * P);
    };

    if (threadIdx.x < kProducer) {
        if (threadIdx.x != 0) return;
        bool ok = true;
        long long issued = 0;
        for (long long k = 0; k < n_my; ++k) {
            const int st = int(k % S);
            if (k >= S) {
                const long long kp = k - S;
                if (!mbar_wait_bounded(&done[st], unsigned((kp / S) & 1))) { ok = false; break; }
                int ci, co;
                tile_coords(b + kp * G, ci, co);
                tma_store_3d(&dmap, stage0 + size_t(st) * stage_elems, ci, 0, co);
                bulk_commit();
                bulk_wait_read_all();
            }
            int ci, co;
            tile_coords(b + k * G, ci, co);
            mbar_arrive_expect_tx(&full[st], tile_bytes);
            tma_load_3d(stage0 + size_t(st) * stage_elems, &map, &full[st], ci, 0, co);
            ++issued;
        }
        if (ok) {
            for (long long kp = (n_my > S ? n_my - S : 0); kp < n_my; ++kp) {
                const int st = int(kp % S);
                if (!mbar_wait_bounded(&done[st], unsigned((kp / S) & 1))) { ok = false; break; }
                int ci, co;
                tile_coords(b + kp * G, ci, co);
                tma_store_3d(&dmap, stage0 + size_t(st) * stage_elems, ci, 0, co);
                bulk_commit();
            }
        }
        bulk_wait_all();
        if (!ok) {
            atomicOr(args.err, ERR_TIMEOUT);
            // let the loads still in flight land before the CTA's shared memory goes away
            for (long long t = (issued > S ? issued - S : 0); t < issued; ++t)
                mbar_wait_bounded(&full[t % S], unsigned((t / S) & 1));
        }
        return;
    }

    // consumers
    const int tid = threadIdx.x - kProducer;
    const int w = tid % W, p = tid / W;
    const bool has_col = tid < W * P;
    for (long long k = 0; k < n_my; ++k) {
        const int st = int(k % S);
        if (!mbar_wait_bounded(&full[st], unsigned((k / S) & 1))) {
            atomicOr(args.err, ERR_TIMEOUT);
            break;
        }
        const long long t = b + k * G;
        const long long inner = (t % args.tiles_inner) * W + w;
        const long long outer = (t / args.tiles_inner) * P + p;
        if (has_col && inner < args.n_inner && outer < args.n_outer) {
            LineCoefT<C> kc;
            if (args.coef_mode == 0)
                kc = tab[(inner / args.vstride) % args.nvel];
            else
                kc = args.cell_coef[outer / args.outer_per_cell];
            if (kc.nd >= 0) {
                const int N = kc.nd >> 1;
                const bool neg = kc.nd & 1;
                T *col = stage0 + size_t(st) * stage_elems + size_t(p) * L * W + w;
                T *base = neg ? col + size_t(L - 1) * W : col;
                const long step = neg ? -long(W) : long(W);
                const C sum = march_line<T, PERIODIC, C>(base, step, L, to_lim(kc));
                if (PERIODIC && N != 0) rotate_line(base, step, L, N % L);
                if (!(sum >= C(0)) || isinf(sum)) atomicOr(args.err, ERR_NAN);
            }
        }
        fence_proxy_async();
        mbar_arrive(&done[st]);
    }
}

template <typename T>
static cudaError_t launch_strided_t(const CUtensorMap &map, const CUtensorMap &dmap, const StridedArgs<typename Compute<T>::type> &a,
                                    int grid, size_t smem, cudaStream_t st)
{
    auto kern = a.periodic ? strided_sweep_kernel<T, true> : strided_sweep_kernel<T, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, kConsumers + kProducer, smem, st>>>(map, dmap, a);
    return cudaGetLastError();
}

cudaError_t launch_strided_f32(const CUtensorMap &map, const CUtensorMap &dmap, const StridedArgs<float> &a, int grid, size_t smem,
                               cudaStream_t st)
{
    return launch_strided_t<float>(map, dmap, a, grid, smem, st);
}

cudaError_t launch_strided_f64(const CUtensorMap &map, const CUtensorMap &dmap, const StridedArgs<double> &a, int grid, size_t smem,
                               cudaStream_t st)
{
    return launch_strided_t<double>(map, dmap, a, grid, smem, st);
}

int occupancy_strided(int dtype, int periodic, size_t smem)
{
    const void *k;
    if (dtype == 0)
        k = periodic ? (const void *)strided_sweep_kernel<double, true> : (const void *)strided_sweep_kernel<double, false>;
    else
        k = periodic ? (const void *)strided_sweep_kernel<float, true> : (const void *)strided_sweep_kernel<float, false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kConsumers + kProducer, smem) != cudaSuccess) return 0;
    return n;
}

} // namespace vk
