// Mixed-precision direct-summation kernel: acceleration, jerk and potential
// of the active i-particles against every j-particle (Sect. 3, Sect. 3.1,
// Sect. 3.2), for sm_103a.
//
// Design (GB300 rather than the G80 of the paper):
//  * j-particles stream through shared memory in tiles of TILE_J, fetched by
//    one thread with 1-D bulk (TMA) copies into a STAGES-deep ring guarded by
//    mbarriers; the paper's "each thread caches one particle" loop (Sect. 3.1
//    steps 1-3) becomes an asynchronous copy overlapped with compute.
//  * Every thread owns two i-particles held in the two lanes of packed FP32x2
//    registers, so each pair-interaction instruction is one FADD2/FMUL2/FFMA2
//    for two pairs; j data are stored twice per record so that the broadcast
//    shared-memory loads deliver {v, v} operands directly.
//  * Positions are double-single; the separation is formed from the hi and lo
//    parts before it is rounded to FP32.  The reciprocal square root is the
//    MUFU instruction.
//  * Per-thread FP32 partial sums cover at most FLUSH_J j-particles, then are
//    folded into double-single (hi, lo) accumulators with an error-free
//    two-sum; jerk is carried as two sums (w/s^3 and (d.w) d/s^5) combined at
//    each fold.
//  * The self pair (j = i) never enters a sum: only on the tile that holds a
//    thread's own i (a warp-uniform branch, a few tiles per warp) does the
//    loop compare j with i and zero that pair, so the large m_i/eps potential
//    term cannot round the FP32 partial sums.  With eps = 0 the guarded
//    variant zeroes every pair at zero separation anyway (Sect. 3.3.1).
//  * Small active blocks: GROUPS > 1 splits each tile over thread groups with
//    a shared-memory reduction, and grid.y > 1 splits the j range over CTAs
//    whose partial sums are reduced on the device (Sect. 3.2 does this last
//    sum on the host).
//  * MODE_ACC_POT drops the jerk (the force-only evaluation of Sect. 4.3).
//    MODE_ADJOINT is the reverse-mode derivative (no counterpart in the
//    paper): the velocity slots of each record carry g = dL/da and the same
//    seven sums become dL/dx_k = G sum_j [w/s^3 - 3 (d.w) d/s^5] with
//    w = m_k g_j - m_j g_k (jerk slots) and dL/dm_k = -G sum_j g_j.d/s^3
//    (potential slot).
#include <cuda_runtime.h>

#include "kirin_internal.cuh"
#include "pair_mixed.cuh"
#include "tma.cuh"

namespace kirin {
namespace {

// j-particles per FP32 partial sum and thread; the adjoint's terms cancel
// across j (tidal sums), so its partial sums are kept shorter
#ifndef KIRIN_FLUSH_J
#define KIRIN_FLUSH_J 256
#endif
#ifndef KIRIN_MIX_UNROLL
#define KIRIN_MIX_UNROLL 4
#endif
#ifndef KIRIN_MIX_MINB
#define KIRIN_MIX_MINB 2
#endif
constexpr int FLUSH_J = KIRIN_FLUSH_J;
constexpr int FLUSH_J_ADJOINT = 64;
constexpr int MIX_UNROLL = KIRIN_MIX_UNROLL;

__device__ __forceinline__ void write_out(const ForceArgs &A, int n_i, int q, int k, double val)
{
    if (k >= n_i)
        return;
    if (A.n_split > 1)
        A.partial[((size_t)blockIdx.y * A.nq + q) * A.n_i_pad + k] = val;
    else
        store_final(A, q, k, val);
}

// Nearest-neighbour result of slot k: to the split partials, or final.
__device__ __forceinline__ void write_nn(const ForceArgs &A, int n_i, int k, double r2, double j)
{
    if (k >= n_i)
        return;
    if (A.n_split > 1) {
        A.partial[((size_t)blockIdx.y * A.nq + 7) * A.n_i_pad + k] = r2;
        A.partial[((size_t)blockIdx.y * A.nq + 8) * A.n_i_pad + k] = j;
    } else {
        store_nn(A, k, r2, j);
    }
}

// Dynamic shared memory of one CTA: the tile ring, reused after the loop as
// the [GROUPS][nq][I_CTA] doubles of the cross-group reduction (up to 9 x
// MIX_I_PER_THREAD x 256 doubles whatever GROUPS is), so the larger of the two.
constexpr size_t MIX_RING_BYTES = (size_t)STAGES * TILE_J * sizeof(JMixed);
constexpr size_t MIX_RED_BYTES = (size_t)9 * MIX_I_PER_THREAD * FORCE_THREADS * sizeof(double);
constexpr size_t MIX_SMEM_BYTES = MIX_RING_BYTES > MIX_RED_BYTES ? MIX_RING_BYTES : MIX_RED_BYTES;

// DEVN: the block size is read from A.n_i_dev (device-driven loops); the grid
// then covers an upper bound and the CTAs beyond the block return at once.
template <int GROUPS, bool GUARD, int MODE, bool DEVN>
__global__ void __launch_bounds__(FORCE_THREADS, KIRIN_MIX_MINB) k_force_mixed(const ForceArgs A)
{
    const int n_i = DEVN ? *A.n_i_dev : A.n_i;
    constexpr bool ADJ = MODE == MODE_ADJOINT;
    constexpr bool NN = MODE == MODE_NN;
    constexpr int NQ = NN ? 9 : 7;              // reduced quantities per i
    constexpr int NP = MIX_IPAIRS;              // packed i-pairs per thread
    constexpr int NI = 2 * NP;                  // i-particles per thread
    constexpr int GT = FORCE_THREADS / GROUPS;  // threads per j-group
    constexpr int I_CTA = NI * GT;              // i-particles per CTA
    constexpr int JG = TILE_J / GROUPS;         // j per group and tile
    constexpr uint32_t TILE_BYTES = TILE_J * sizeof(JMixed);
    static_assert(GT >= 32, "a warp must read one j at a time (broadcast loads)");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    JMixed *tiles = reinterpret_cast<JMixed *>(smem_raw);
    __shared__ __align__(8) uint64_t bars[STAGES];
    if (DEVN && (long long)blockIdx.x * I_CTA >= n_i)
        return;  // beyond the block (uniform over the CTA)

    const int tid = threadIdx.x;
    const int g = tid / GT;
    const int s = tid - g * GT;
    const JMixed *__restrict__ J = static_cast<const JMixed *>(A.jimg);

    // ---- the i-particles of this thread: slot s + q * GT of the CTA's block,
    //      lanes (x, y) of pair p holding q = 2p and 2p + 1 ----
    int idx[NI];
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int k = blockIdx.x * I_CTA + s + q * GT;
        int i = -1;
        if (k < n_i) {
            i = A.ilist ? A.ilist[k] : k;
            if (i < 0 || i >= A.n_j) {
                atomicOr(A.err, ERR_INDEX);
                i = -1;
            }
        }
        idx[q] = i;
    }
    const float eps2f = (float)A.eps2;
    const float rmin2f = (float)A.rmin2;
    IPair I[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
        I[p] = load_ipair(J + (idx[2 * p] >= 0 ? idx[2 * p] : 0), J + (idx[2 * p + 1] >= 0 ? idx[2 * p + 1] : 0),
                          eps2f, rmin2f);
    // the self pair is masked unless eps = 0 zeroes it anyway (in the adjoint,
    // w = m_k g_j - m_j g_k is formed with a multiply-add, which leaves ~u m g
    // for j = k instead of zero, times 1/eps^3)
    // (the neighbour search always excludes j = i by index)
    const bool need_mask = eps2f != 0.f || NN;

    // ---- j range of this CTA (grid.y splits the tiles) ----
    const int y = blockIdx.y;
    const int tb = A.tile0 + (int)(((long long)A.ntiles * y) / A.n_split);
    const int te = A.tile0 + (int)(((long long)A.ntiles * (y + 1)) / A.n_split);
    const int nt = te - tb;

    if (tid == 0) {
#pragma unroll
        for (int st = 0; st < STAGES; ++st)
            mbar_init(&bars[st], 1);
        mbar_fence_init();
    }
    const uint64_t pol = l2_policy_evict_last();
    __syncthreads();
    if (tid == 0) {
        for (int st = 0; st < STAGES && st < nt; ++st) {
            mbar_arrive_expect_tx(&bars[st], TILE_BYTES);
            bulk_g2s_hint(tiles + st * TILE_J, J + (size_t)(tb + st) * TILE_J, TILE_BYTES, &bars[st], pol);
        }
    }

    Tile7 t[NP];
    Lane7 acc[NI];
    NNPair nnp[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        t[p].zero();
        nnp[p].reset();
    }
#pragma unroll
    for (int q = 0; q < NI; ++q)
        acc[q].zero();

    int since = 0;
    int k = 0;
    bool aborted = false;
    for (; k < nt; ++k) {
        const int st = k % STAGES;
        const uint32_t par = (uint32_t)(k / STAGES) & 1u;
        const bool ok = mbar_wait_bounded(&bars[st], par);
        if (ok) {
            const JMixed *__restrict__ T = tiles + st * TILE_J + g * JG;
            const int j0 = (tb + k) * TILE_J + g * JG;  // index of T[0]
            bool mine = false;
#pragma unroll
            for (int q = 0; q < NI; ++q)
                mine = mine || (unsigned)(idx[q] - j0) < (unsigned)JG;
            if (need_mask && __any_sync(0xffffffffu, mine)) {
#pragma unroll 2
                for (int jj = 0; jj < JG; ++jj) {
#pragma unroll
                    for (int p = 0; p < NP; ++p)
                        pair<GUARD, MODE, true>(T[jj], I[p], t[p], j0 + jj, idx[2 * p], idx[2 * p + 1], &nnp[p],
                                                A.n_j);
                }
            } else {
#pragma unroll MIX_UNROLL
                for (int jj = 0; jj < JG; ++jj) {
#pragma unroll
                    for (int p = 0; p < NP; ++p)
                        pair<GUARD, MODE>(T[jj], I[p], t[p], j0 + jj, -1, -1, &nnp[p], A.n_j);
                }
            }
            since += JG;
            if (since >= (ADJ ? FLUSH_J_ADJOINT : FLUSH_J)) {
#pragma unroll
                for (int p = 0; p < NP; ++p)
                    fold<MODE>(t[p], acc[2 * p], acc[2 * p + 1]);
                since = 0;
            }
        }
        // every thread learns whether any wait in the CTA timed out
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        if (tid == 0 && k + STAGES < nt) {
            mbar_arrive_expect_tx(&bars[st], TILE_BYTES);
            bulk_g2s_hint(tiles + st * TILE_J, J + (size_t)(tb + k + STAGES) * TILE_J, TILE_BYTES, &bars[st], pol);
        }
    }
    if (aborted) {
        // let every copy already issued land before the CTA's shared memory goes away
        if (tid == 0) {
            const int last = min(nt, k + STAGES);
            for (int kk = k; kk < last; ++kk) {
                if (!mbar_wait_bounded(&bars[kk % STAGES], (uint32_t)(kk / STAGES) & 1u)) {
                    atomicOr(A.err, ERR_DRAIN);
                    break;
                }
            }
            atomicOr(A.err, ERR_TIMEOUT);
        }
        return;
    }
#pragma unroll
    for (int p = 0; p < NP; ++p)
        fold<MODE>(t[p], acc[2 * p], acc[2 * p + 1]);

    // neighbour of slot q: lane (q & 1) of pair q / 2
    auto nn_r = [&](int q) { return (double)((q & 1) ? nnp[q >> 1].r1 : nnp[q >> 1].r0); };
    auto nn_j = [&](int q) { return (double)((q & 1) ? nnp[q >> 1].j1 : nnp[q >> 1].j0); };
    if (GROUPS == 1) {
#pragma unroll
        for (int q = 0; q < NI; ++q) {
            const int slot = blockIdx.x * I_CTA + s + q * GT;
#pragma unroll
            for (int c = 0; c < 7; ++c)
                write_out(A, n_i, c, slot, (double)acc[q].h[c] + (double)acc[q].l[c]);
            if (NN)
                write_nn(A, n_i, slot, nn_r(q), nn_j(q));
        }
    } else {
        // Cross-group sum in double-single (FP32 two-sums): FP64 is the scarce
        // pipe on this part, so each output is converted to FP64 once, after
        // the groups are summed, instead of every group's partial.
        __syncthreads();  // all tiles consumed: reuse the ring as reduction space
        static_assert((size_t)GROUPS * NQ * I_CTA * sizeof(float2) <= MIX_SMEM_BYTES, "reduction space");
        float2 *red = reinterpret_cast<float2 *>(smem_raw);  // [GROUPS][NQ][I_CTA] of (hi, lo)
#pragma unroll
        for (int q = 0; q < NI; ++q) {
#pragma unroll
            for (int c = 0; c < 7; ++c)
                red[(g * NQ + c) * I_CTA + s + q * GT] = make_float2(acc[q].h[c], acc[q].l[c]);
            if (NN) {  // (nearest r2, its index as bits)
                const NNPair &np = nnp[q >> 1];
                red[(g * NQ + 7) * I_CTA + s + q * GT] =
                    make_float2((q & 1) ? np.r1 : np.r0, __int_as_float((q & 1) ? np.j1 : np.j0));
            }
        }
        __syncthreads();
        for (int o = tid; o < 7 * I_CTA; o += FORCE_THREADS) {
            const int c = o / I_CTA;
            const int slot = o - c * I_CTA;
            float2 v = red[c * I_CTA + slot];
            float hi = v.x, lo = v.y;
#pragma unroll
            for (int gg = 1; gg < GROUPS; ++gg) {
                v = red[(gg * NQ + c) * I_CTA + slot];
                two_sum(hi, lo, v.x);
                lo = __fadd_rn(lo, v.y);
            }
            write_out(A, n_i, c, blockIdx.x * I_CTA + slot, (double)hi + (double)lo);
        }
        if (NN) {
            for (int slot = tid; slot < I_CTA; slot += FORCE_THREADS) {
                double r2 = INFINITY, j = -1.0;
#pragma unroll
                for (int gg = 0; gg < GROUPS; ++gg) {
                    const float2 v = red[(gg * NQ + 7) * I_CTA + slot];
                    nn_min(r2, j, (double)v.x, (double)__float_as_int(v.y));
                }
                write_nn(A, n_i, blockIdx.x * I_CTA + slot, r2, j);
            }
        }
    }
}

// Tiny blocks (n_i <= TINY_MAX): CTA (x, y) stages the j range x of the
// padded image (at most TINY_JCHUNK records) in shared memory, and its warp
// w takes i-particle k = 8 y + w, lane l the records l, l + 32 of each 64 in
// the two float2 lanes of the pair body (the i duplicated in both; the self
// pair gets zero mass).  Lane sums meet across the warp in double-single;
// lanes 0..6 convert one output each to FP64 and write the CTA's partial
// (n_split = gridDim.x), which the split reduction sums.
constexpr int TINY_THREADS = 256;
constexpr int TINY_WARPS = TINY_THREADS / 32;

template <bool GUARD, bool DEVN>
__global__ void __launch_bounds__(TINY_THREADS) k_force_tiny(const ForceArgs A)
{
    __shared__ __align__(16) JMixed js[TINY_JCHUNK];
    const int n_i = DEVN ? *A.n_i_dev : A.n_i;
    if ((int)blockIdx.y * TINY_WARPS >= n_i)
        return;  // no i-particle for this CTA (uniform)
    const JMixed *__restrict__ J = static_cast<const JMixed *>(A.jimg);
    const int n_pad = A.ntiles * TILE_J;  // the records summed: [jb, jb + n_pad) of the padded image
    const int jb = A.tile0 * TILE_J;
    const int chunk = (n_pad + (int)gridDim.x - 1) / (int)gridDim.x;
    if (chunk > TINY_JCHUNK) {  // the host sizes the grid so that this cannot happen
        if (threadIdx.x == 0)
            atomicOr(A.err, ERR_INDEX);
        return;
    }
    const int j0 = jb + min(n_pad, (int)blockIdx.x * chunk);
    const int len = min(jb + n_pad, j0 + chunk) - j0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = (int)blockIdx.y * TINY_WARPS + warp;
    int i = -1;
    JMixed rec;
    if (k < n_i) {
        i = A.ilist ? A.ilist[k] : k;
        if (i < 0 || i >= A.n_j) {
            if (lane == 0)
                atomicOr(A.err, ERR_INDEX);
            i = -1;
        } else {
            rec = J[i];
        }
    }
    for (int r = threadIdx.x; r < len; r += TINY_THREADS)
        js[r] = J[j0 + r];
    __syncthreads();
    if (k >= n_i)
        return;
    Tile7 t;
    t.zero();
    if (i >= 0) {
        const IPair I = load_ipair(&rec, &rec, (float)A.eps2, (float)A.rmin2);
        for (int b0 = 0; b0 < len; b0 += 64) {
            const int ra = b0 + lane, rb = ra + 32;
            float4 a[5], b[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                a[c] = ra < len ? js[ra].q[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                b[c] = rb < len ? js[rb].q[c] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            JMixed r;
            r.q[0] = make_float4(a[0].x, b[0].x, a[0].z, b[0].z);
            r.q[1] = make_float4(a[1].x, b[1].x, j0 + ra == i ? 0.f : a[1].z, j0 + rb == i ? 0.f : b[1].z);
            r.q[2] = make_float4(a[2].x, b[2].x, a[2].z, b[2].z);
            r.q[3] = make_float4(a[3].x, b[3].x, a[3].z, b[3].z);
            r.q[4] = make_float4(a[4].x, b[4].x, a[4].z, b[4].z);
            pair<GUARD, MODE_ACC_JERK_POT>(r, I, t);
        }
    }
    float hi[7], lo[7];
    hi[0] = t.ax.x + t.ax.y;
    hi[1] = t.ay.x + t.ay.y;
    hi[2] = t.az.x + t.az.y;
    hi[3] = __fmaf_rn(-3.f, t.j2x.x, t.j1x.x) + __fmaf_rn(-3.f, t.j2x.y, t.j1x.y);
    hi[4] = __fmaf_rn(-3.f, t.j2y.x, t.j1y.x) + __fmaf_rn(-3.f, t.j2y.y, t.j1y.y);
    hi[5] = __fmaf_rn(-3.f, t.j2z.x, t.j1z.x) + __fmaf_rn(-3.f, t.j2z.y, t.j1z.y);
    hi[6] = t.pt.x + t.pt.y;
#pragma unroll
    for (int q = 0; q < 7; ++q)
        lo[q] = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi[q], o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo[q], o);
            two_sum(hi[q], lo[q], h2);
            lo[q] = __fadd_rn(lo[q], l2);
        }
    }
    float h = hi[0], l = lo[0];
#pragma unroll
    for (int q = 1; q < 7; ++q)
        if (lane == q) {
            h = hi[q];
            l = lo[q];
        }
    if (lane < 7)
        A.partial[((size_t)blockIdx.x * A.nq + lane) * A.n_i_pad + k] = (double)h + (double)l;
}

template <bool GUARD>
cudaError_t launch_tiny(const ForceArgs &a, int ctas, cudaStream_t st)
{
    if (a.n_i > TINY_MAX || a.n_split != ctas || a.nq != 7 || !a.partial || a.n_i_pad < TINY_MAX || ctas < 1 ||
        (a.ntiles * TILE_J + ctas - 1) / ctas > TINY_JCHUNK)
        return cudaErrorInvalidValue;
    const dim3 grid(ctas, (a.n_i + TINY_WARPS - 1) / TINY_WARPS);
    if (a.n_i_dev)
        k_force_tiny<GUARD, true><<<grid, TINY_THREADS, 0, st>>>(a);
    else
        k_force_tiny<GUARD, false><<<grid, TINY_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

template <int GROUPS, bool GUARD, int MODE, bool DEVN>
cudaError_t launch_v(const ForceArgs &a, int iblocks, int n_split, cudaStream_t st)
{
    const size_t smem = MIX_SMEM_BYTES;
    if (smem > 48 * 1024) {
        static bool opted = false;  // per template instance
        if (!opted) {
            cudaFuncSetAttribute(k_force_mixed<GROUPS, GUARD, MODE, DEVN>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            opted = true;
        }
    }
    dim3 grid(iblocks, n_split);
    k_force_mixed<GROUPS, GUARD, MODE, DEVN><<<grid, FORCE_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <int GROUPS, bool GUARD, int MODE>
cudaError_t launch_t(const ForceArgs &a, int n_split, cudaStream_t st)
{
    constexpr int I_CTA = MIX_I_PER_THREAD * FORCE_THREADS / GROUPS;
    const int iblocks = (a.n_i + I_CTA - 1) / I_CTA;
    if (iblocks == 0)
        return cudaSuccess;
    if (a.n_i_dev) {  // only the block-step force of the device-driven loop reads n_i on the device
        if constexpr (MODE == MODE_ACC_JERK_POT)
            return launch_v<GROUPS, GUARD, MODE, true>(a, iblocks, n_split, st);
        else
            return cudaErrorInvalidValue;
    }
    return launch_v<GROUPS, GUARD, MODE, false>(a, iblocks, n_split, st);
}

template <int GROUPS, bool GUARD, int MODE>
int occ_t()
{
    int n = 0;
    const size_t smem = MIX_SMEM_BYTES;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_force_mixed<GROUPS, GUARD, MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_force_mixed<GROUPS, GUARD, MODE, false>,
                                                  FORCE_THREADS, smem);
    return n;
}

template <bool GUARD, int MODE>
cudaError_t launch_g(const ForceArgs &a, Shape s, cudaStream_t st)
{
    switch (s.groups) {
    case 1: return launch_t<1, GUARD, MODE>(a, s.n_split, st);
    case 2: return launch_t<2, GUARD, MODE>(a, s.n_split, st);
    case 4: return launch_t<4, GUARD, MODE>(a, s.n_split, st);
    case 8: return launch_t<8, GUARD, MODE>(a, s.n_split, st);
    default: return cudaErrorInvalidValue;
    }
}

template <bool GUARD, int MODE>
int occ_g(int groups)
{
    switch (groups) {
    case 1: return occ_t<1, GUARD, MODE>();
    case 2: return occ_t<2, GUARD, MODE>();
    case 4: return occ_t<4, GUARD, MODE>();
    case 8: return occ_t<8, GUARD, MODE>();
    default: return 0;
    }
}

template <int MODE>
cudaError_t launch_m(const ForceArgs &a, Shape s, bool guard, cudaStream_t st)
{
    return guard ? launch_g<true, MODE>(a, s, st) : launch_g<false, MODE>(a, s, st);
}

}  // namespace

cudaError_t launch_force_mixed(const ForceArgs &a, Shape s, bool guard, int mode, cudaStream_t st)
{
    if (s.groups == 0) {  // tiny-block kernel
        if (mode != MODE_ACC_JERK_POT)
            return cudaErrorInvalidValue;
        if (a.n_i == 0)
            return cudaSuccess;
        return guard ? launch_tiny<true>(a, s.n_split, st) : launch_tiny<false>(a, s.n_split, st);
    }
    switch (mode) {
    case MODE_ACC_JERK_POT: return launch_m<MODE_ACC_JERK_POT>(a, s, guard, st);
    case MODE_ACC_POT: return launch_m<MODE_ACC_POT>(a, s, guard, st);
    case MODE_ADJOINT: return launch_m<MODE_ADJOINT>(a, s, guard, st);
    case MODE_NN: return launch_m<MODE_NN>(a, s, guard, st);
    default: return cudaErrorInvalidValue;
    }
}

int force_mixed_ctas_per_sm(int groups, bool guard, int mode)
{
    switch (mode) {
    case MODE_ACC_JERK_POT: return guard ? occ_g<true, MODE_ACC_JERK_POT>(groups) : occ_g<false, MODE_ACC_JERK_POT>(groups);
    case MODE_ACC_POT: return guard ? occ_g<true, MODE_ACC_POT>(groups) : occ_g<false, MODE_ACC_POT>(groups);
    case MODE_ADJOINT: return guard ? occ_g<true, MODE_ADJOINT>(groups) : occ_g<false, MODE_ADJOINT>(groups);
    case MODE_NN: return guard ? occ_g<true, MODE_NN>(groups) : occ_g<false, MODE_NN>(groups);
    default: return 0;
    }
}

}  // namespace kirin
