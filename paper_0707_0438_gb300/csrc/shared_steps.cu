// Shared-step Hermite runs of small systems in one cooperative launch
// (Sect. 3: predictor, direct sum, corrector; Sect. 3.1 split over host and
// accelerator, here all on the device).
//
// A system of a few thousand particles is latency-bound: each of the
// predictor, force, split-reduction and corrector kernels of a step waits
// microseconds on its launch and on memory for well under a microsecond of
// arithmetic.  Here one CTA per SM stays resident for the whole run:
//  * CTA b owns particles [b n / P, (b + 1) n / P) of P CTAs.  It corrects
//    them (the step kernels' corrector) and at once predicts them to the
//    next step (the step kernels' predictor), into the global j image of
//    the step's parity;
//  * one grid barrier per step publishes the image.  Two images alternate, so
//    a CTA that is still summing step s never sees step s + 1's records;
//  * every CTA copies the whole image into its shared memory (a 1-D bulk copy
//    and an mbarrier per tile) and sums its own particles against it with the
//    pair body of the force kernels: two i per thread, j-groups of threads
//    over the j of each tile, partial sums folded in double-single, the
//    groups of a warp combined by shuffles and the warps in warp order.
// FP64 work stays on the owning thread (FP64 is the scarce pipe here); the
// step's only grid-wide dependency is the barrier.
#include <cuda_runtime.h>

#include "kirin_internal.cuh"
#include "loop_internal.cuh"
#include "pair_mixed.cuh"
#include "step_math.cuh"
#include "tma.cuh"

namespace kirin {
namespace {

constexpr int SH_THREADS = 512;
constexpr int SH_WARPS = SH_THREADS / 32;
constexpr int SH_FLUSH_J = 256;  // j per FP32 partial sum and thread, as in the force kernels
constexpr int SH_MAX_TILES = SH_MAX_N / TILE_J;
constexpr int SH_BAR_BYTES = 256;  // the tiles' mbarriers, ahead of the image
constexpr uint32_t SH_TILE_BYTES = TILE_J * sizeof(JMixed);
static_assert(SH_MAX_N % TILE_J == 0 && SH_MAX_TILES * 8 <= SH_BAR_BYTES, "mbarrier area");
static_assert(SH_TILE_BYTES % 16 == 0 && SH_BAR_BYTES % 16 == 0, "bulk copies want 16-byte multiples");

// GT threads of a j-group hold up to 2 GT particles, two per thread (packed FP32x2 lanes); the
// SH_THREADS / GT groups share out the j of every tile.
template <int GT>
__host__ __device__ constexpr size_t sh_red_bytes() { return (size_t)SH_WARPS * 7 * 2 * GT * sizeof(float2); }

template <int GT>
__host__ __device__ constexpr size_t sh_smem_bytes(int n_pad)
{
    return SH_BAR_BYTES + (size_t)n_pad * sizeof(JMixed) + sh_red_bytes<GT>();
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Order this thread's earlier global accesses (made visible to it by the grid barrier) before its
// later bulk copies, which read global memory through the async proxy.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Grid-wide barrier of a cooperative launch, bounded: bar[0] counts the CTAs that arrived, bar[1] is
// the generation.  The last CTA to arrive zeroes the count and advances the generation; the others
// wait for it at most WAIT_LIMIT_NS, then flag ERR_TIMEOUT and return false (the host zeroes the
// barrier after a failed run).  Every thread of the CTA calls it.
__device__ bool grid_sync(unsigned *bar, unsigned *err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire_gpu(bar + 1);
        __threadfence();  // the CTA's writes (ordered before by the CTA barrier) before the arrival
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            st_release_gpu(bar + 1, gen + 1);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_gpu(bar + 1) == gen) {
                if (global_ns() - t0 > WAIT_LIMIT_NS) {
                    atomicOr(err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <int GT, bool GUARD>
__global__ void __launch_bounds__(SH_THREADS, 1) k_shared_steps(const SharedStepArgs A)
{
    constexpr int GROUPS = SH_THREADS / GT;
    constexpr int I_CTA = 2 * GT;
    constexpr int JG = TILE_J / GROUPS;  // j per group and tile
    static_assert(32 % GT == 0 && JG >= 1, "groups tile the warps and the j tile");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);                     // [n_tiles]
    JMixed *img = reinterpret_cast<JMixed *>(smem_raw + SH_BAR_BYTES);           // [n_pad]
    float2 *red = reinterpret_cast<float2 *>(smem_raw + SH_BAR_BYTES + (size_t)A.n_pad * sizeof(JMixed));
    const int n = A.n, n_pad = A.n_pad, n_tiles = n_pad / TILE_J;
    const int P = (int)gridDim.x, b = (int)blockIdx.x;
    const int lo = (int)((long long)n * b / P), hi = (int)((long long)n * (b + 1) / P);
    const int own = hi - lo;  // at most I_CTA (the launch checks)
    const int tid = (int)threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = tid / GT, s = tid - g * GT;
    const float eps2f = (float)A.eps2, rmin2f = (float)A.rmin2;
    const bool need_mask = eps2f != 0.f;  // with eps = 0 the guard zeroes the self pair anyway
    if (tid == 0) {
        for (int q = 0; q < n_tiles; ++q)
            mbar_init(&bars[q], 1);
        mbar_fence_init();
    }
    // step 0's image: own particles predicted to t0 + dt; the last CTA writes both images' padding
    if (tid < own)
        predict_one(lo + tid, n, A.t0 + A.dt, 1, A.m, A.x, A.v, A.a, A.jerk_b, A.t_b, A.xp, A.vp, A.img, nullptr,
                    A.err);
    if (b == P - 1)
        for (int k = n + tid; k < n_pad; k += SH_THREADS) {
            predict_one(k, n, 0.0, 0, A.m, A.x, A.v, A.a, A.jerk_b, A.t_b, nullptr, nullptr, A.img, nullptr, A.err);
            predict_one(k, n, 0.0, 0, A.m, A.x, A.v, A.a, A.jerk_b, A.t_b, nullptr, nullptr, A.img + n_pad, nullptr,
                        A.err);
        }
    fence_proxy_async_global();  // the image records written above are read by bulk copies
    if (!grid_sync(A.bar, A.err))
        return;
    double t = A.t0;
    for (int step = 0; step < A.n_steps; ++step) {
        const double tn = t + A.dt;
        const uint32_t parity = (uint32_t)(step & 1);
        // 1. the whole image of this step into shared memory, a tile per mbarrier
        if (tid == 0) {
            fence_proxy_async_global();
            const JMixed *src = A.img + (size_t)(step & 1) * n_pad;
            for (int q = 0; q < n_tiles; ++q) {
                mbar_arrive_expect_tx(&bars[q], SH_TILE_BYTES);
                bulk_g2s(img + (size_t)q * TILE_J, src + (size_t)q * TILE_J, SH_TILE_BYTES, &bars[q]);
            }
        }
        // 2. own particles (thread s of group g holds slots s and s + GT) against every j
        //    (a failed wait is made warp-uniform, so no lane leaves its warp's votes behind)
        bool failed = !__all_sync(0xffffffffu, mbar_wait_bounded(&bars[lo / TILE_J], parity) &&
                                                   mbar_wait_bounded(&bars[(hi - 1) / TILE_J], parity));
        int idx[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k = lo + s + q * GT;
            idx[q] = k < hi ? k : -1;
        }
        Lane7 acc0, acc1;
        acc0.zero();
        acc1.zero();
        if (!failed) {
            const IPair I = load_ipair(img + (idx[0] >= 0 ? idx[0] : lo), img + (idx[1] >= 0 ? idx[1] : lo), eps2f,
                                       rmin2f);
            Tile7 tt;
            tt.zero();
            int since = 0;
            for (int q = 0; q < n_tiles; ++q) {
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[q], parity))) {
                    failed = true;
                    break;
                }
                const int j0 = q * TILE_J + g * JG;
                const JMixed *T = img + j0;
                const bool mine =
                    (unsigned)(idx[0] - j0) < (unsigned)JG || (unsigned)(idx[1] - j0) < (unsigned)JG;
                if (need_mask && __any_sync(0xffffffffu, mine)) {
                    for (int jj = 0; jj < JG; ++jj)
                        pair<GUARD, MODE_ACC_JERK_POT, true>(T[jj], I, tt, j0 + jj, idx[0], idx[1]);
                } else {
#pragma unroll
                    for (int jj = 0; jj < JG; ++jj)
                        pair<GUARD, MODE_ACC_JERK_POT>(T[jj], I, tt);
                }
                since += JG;
                if (since >= SH_FLUSH_J) {
                    fold<MODE_ACC_JERK_POT>(tt, acc0, acc1);
                    since = 0;
                }
            }
            fold<MODE_ACC_JERK_POT>(tt, acc0, acc1);
        }
        fence_proxy_async_smem();  // this step's reads of the image before the next step's copies
        if (__syncthreads_or(failed)) {
            if (tid == 0) {  // no copy of this CTA may still be landing when it leaves
                atomicOr(A.err, ERR_TIMEOUT);
                for (int q = 0; q < n_tiles; ++q)
                    if (!mbar_wait_bounded(&bars[q], parity)) {
                        atomicOr(A.err, ERR_DRAIN);
                        break;
                    }
            }
            return;  // the other CTAs give up at their next grid barrier
        }
        // 3. the groups of a warp combined by shuffles (a fixed tree), then the warps in warp order
#pragma unroll
        for (int q7 = 0; q7 < 7; ++q7) {
#pragma unroll
            for (int off = GT; off < 32; off <<= 1) {
                float oh = __shfl_xor_sync(0xffffffffu, acc0.h[q7], off);
                float ol = __shfl_xor_sync(0xffffffffu, acc0.l[q7], off);
                two_sum(acc0.h[q7], acc0.l[q7], oh);
                acc0.l[q7] = __fadd_rn(acc0.l[q7], ol);
                oh = __shfl_xor_sync(0xffffffffu, acc1.h[q7], off);
                ol = __shfl_xor_sync(0xffffffffu, acc1.l[q7], off);
                two_sum(acc1.h[q7], acc1.l[q7], oh);
                acc1.l[q7] = __fadd_rn(acc1.l[q7], ol);
            }
            if (lane < GT) {
                red[(warp * 7 + q7) * I_CTA + s] = make_float2(acc0.h[q7], acc0.l[q7]);
                red[(warp * 7 + q7) * I_CTA + s + GT] = make_float2(acc1.h[q7], acc1.l[q7]);
            }
        }
        __syncthreads();
        for (int o = tid; o < 7 * own; o += SH_THREADS) {
            const int q7 = o / own, slot = o - q7 * own;
            float2 v = red[q7 * I_CTA + slot];
            float h = v.x, l = v.y;
#pragma unroll
            for (int w = 1; w < SH_WARPS; ++w) {
                v = red[(w * 7 + q7) * I_CTA + slot];
                two_sum(h, l, v.x);
                l = __fadd_rn(l, v.y);
            }
            const double val = (double)h + (double)l;
            const int p = lo + slot;
            if (q7 < 3)
                A.f_acc[3 * (size_t)p + q7] = A.G * val;
            else if (q7 < 6)
                A.f_jerk[3 * (size_t)p + (q7 - 3)] = A.G * val;
            else if (A.f_pot)
                A.f_pot[p] = -A.G * val;
        }
        __syncthreads();  // the rows are read back by the corrector
        // 4. own particles corrected (shared step: the step size stays), then predicted to the next
        //    step into the other image
        if (tid < own) {
            const int k = lo + tid;
            correct_at((size_t)k, k, tn, A.eta, A.dt_min, A.dt_max, 0, A.xp, A.vp, A.f_acc, A.f_jerk, A.x, A.v,
                       A.a, A.jerk_b, A.t_b, A.dt_b);
            if (step + 1 < A.n_steps)
                predict_one(k, n, tn + A.dt, 1, A.m, A.x, A.v, A.a, A.jerk_b, A.t_b, A.xp, A.vp,
                            A.img + (size_t)((step + 1) & 1) * n_pad, nullptr, A.err);
            fence_proxy_async_global();
        }
        if (step + 1 < A.n_steps && !grid_sync(A.bar, A.err))
            return;
        t = tn;
    }
}

template <int GT, bool GUARD>
cudaError_t sh_launch(const SharedStepArgs &a, bool query_only, int *grid, cudaStream_t st)
{
    const auto kern = k_shared_steps<GT, GUARD>;
    if (query_only) {
        // opt in once for the largest image, so a smaller context cannot lower a larger one's limit
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sh_smem_bytes<GT>(SH_MAX_N));
        if (e != cudaSuccess)
            return e;
        int dev = 0, nsm = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SH_THREADS, sh_smem_bytes<GT>(a.n_pad))) !=
                cudaSuccess)
            return e;
        const int ctas = nsm * (per_sm > 0 ? 1 : 0);  // one CTA per SM
        *grid = ctas < a.n ? ctas : a.n;
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(a.ctas);
    cfg.blockDim = dim3(SH_THREADS);
    cfg.dynamicSmemBytes = sh_smem_bytes<GT>(a.n_pad);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// Narrowest j-group that holds a CTA's share of the particles.
template <bool GUARD>
cudaError_t sh_dispatch(const SharedStepArgs &a, int own_max, bool query_only, int *grid, cudaStream_t st)
{
    if (own_max <= 16)
        return sh_launch<8, GUARD>(a, query_only, grid, st);
    if (own_max <= 32)
        return sh_launch<16, GUARD>(a, query_only, grid, st);
    if (own_max <= 64)
        return sh_launch<32, GUARD>(a, query_only, grid, st);
    return cudaErrorInvalidValue;
}

int own_max_of(int n, int ctas) { return (n + ctas - 1) / ctas; }

}  // namespace

int shared_steps_grid(int n, bool guard)
{
    if (n < 1 || n > SH_MAX_N)
        return 0;
    SharedStepArgs a{};
    a.n = n;
    a.n_pad = (n + TILE_J - 1) / TILE_J * TILE_J;
    // the grid does not depend on the group width (one CTA per SM): ask the widest, then check the
    // share against the width that will run
    int grid = 0;
    cudaError_t e = guard ? sh_dispatch<true>(a, 64, true, &grid, nullptr) : sh_dispatch<false>(a, 64, true, &grid, nullptr);
    if (e != cudaSuccess || grid < 1 || own_max_of(n, grid) > 64) {
        cudaGetLastError();
        return 0;
    }
    int g2 = 0;
    const int own = own_max_of(n, grid);
    e = guard ? sh_dispatch<true>(a, own, true, &g2, nullptr) : sh_dispatch<false>(a, own, true, &g2, nullptr);
    if (e != cudaSuccess || g2 < grid) {
        cudaGetLastError();
        return 0;
    }
    return grid;
}

cudaError_t launch_shared_steps(const SharedStepArgs &a, bool guard, cudaStream_t st)
{
    if (a.n < 1 || a.n > SH_MAX_N || a.n_pad % TILE_J != 0 || a.n_pad < a.n || a.n_pad > SH_MAX_N ||
        a.n_steps < 0 || a.ctas < 1 || a.ctas > a.n || own_max_of(a.n, a.ctas) > 64 || !a.img || !a.bar)
        return cudaErrorInvalidValue;
    if (a.n_steps == 0)
        return cudaSuccess;
    const int own = own_max_of(a.n, a.ctas);
    return guard ? sh_dispatch<true>(a, own, false, nullptr, st) : sh_dispatch<false>(a, own, false, nullptr, st);
}

}  // namespace kirin
