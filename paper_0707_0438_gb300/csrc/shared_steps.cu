// Shared-step Hermite runs of small systems in one cooperative launch
// (Sect. 3: predictor, direct sum, corrector; Sect. 3.1 split over host and
// accelerator, here all on the device).
//
// A system of a few thousand particles is latency-bound: each of the
// predictor, force, split-reduction and corrector kernels of a step waits
// microseconds on its launch and on memory for well under a microsecond of
// arithmetic.  Here one CTA per SM stays resident for the whole run:
//  * CTA b owns particles [b n / P, (b + 1) n / P) of P CTAs and keeps their
//    FP64 state in shared memory for the launch (written through to the
//    context's arrays every step).  Warps 0, 1 and 2 (and 3, 4, 5 for a
//    slice of more than 32) correct the x, y and z components of the slice
//    and predict them at once to the next step, with the step kernels'
//    arithmetic: FP64 is the scarce pipe on this part and a warp instruction
//    costs the same with 1 or 32 lanes, so three short chains on three SM
//    sub-partitions beat one long chain;
//  * the predicted records go to the global j image of the next step's
//    parity (two images alternate), and the CTA adds 1 to an arrival counter
//    that only grows (a fire-and-forget release add).  Before step s each CTA
//    waits until the counter holds (s + 1) arrivals per CTA (one thread polls,
//    bounded), which also proves that nobody still reads the image it is
//    about to overwrite: no CTA can arrive a (s + 2)-th time before that;
//  * every CTA copies the whole image into its shared memory (a 1-D bulk copy
//    and an mbarrier per tile) and sums its own particles against it with the
//    pair body of the force kernels: two i per thread; each warp takes a
//    contiguous sixteenth of the j, its groups of threads interleaved record
//    by record (consecutive 80-byte records fall on disjoint banks); partial
//    sums folded in double-single, the groups of a warp combined by shuffles
//    and the warps in warp order.  Above 2048 records the image streams
//    through a ring of tiles instead, in two halves (the CTA sums one while
//    the other fills, one CTA barrier per half), each warp taking its
//    sixteenth of every tile.
// With init set, the launch instead evaluates the particles as they are at t0
// and initialises the integrator (a, jerk, t and the first block step, the
// initialisation kernel's arithmetic): one launch for kirin_hermite_init.
#include <cuda_runtime.h>

#include "kirin_internal.cuh"
#include "loop_internal.cuh"
#include "pair_mixed.cuh"
#include "grid_sync.cuh"
#include "step_math.cuh"
#include "tma.cuh"

namespace kirin {
namespace {

constexpr int SH_THREADS = 512;
constexpr int SH_WARPS = SH_THREADS / 32;
constexpr int SH_MAX_OWN = 64;  // particles per CTA (groups of up to 32 threads, two i each)
// Images of more than SH_RESIDENT_N records stream through a ring of SH_RING tiles in two halves of
// SH_CH: the CTA sums one half while the other fills, one CTA barrier per half.
constexpr int SH_RESIDENT_N = 2048;
constexpr int SH_CH = 6;
constexpr int SH_RING = 2 * SH_CH;
constexpr int SH_FLUSH_J = 256;  // j per FP32 partial sum and thread, as in the force kernels
constexpr int SH_MAX_TILES = SH_RESIDENT_N / TILE_J;
constexpr int SH_BAR_BYTES = 256;  // the tiles' mbarriers, ahead of the image
constexpr uint32_t SH_TILE_BYTES = TILE_J * sizeof(JMixed);
static_assert(SH_RESIDENT_N % TILE_J == 0 && SH_MAX_N % TILE_J == 0, "whole tiles");
static_assert(SH_MAX_TILES * 8 <= SH_BAR_BYTES && SH_RING * 8 <= SH_BAR_BYTES, "mbarrier area");
static_assert(SH_TILE_BYTES % 16 == 0 && SH_BAR_BYTES % 16 == 0, "bulk copies want 16-byte multiples");
static_assert(SH_RESIDENT_N * 16 / SH_THREADS <= SH_FLUSH_J, "one fold per step holds a resident group's j");
static_assert(TILE_J % SH_WARPS == 0 && (TILE_J / SH_WARPS) % 2 == 0, "a warp's records of a streamed tile");

// Own-state rows in shared memory, doubles [row][I_CTA]: per component c the
// rows 6c + (x, v, a, jerk, x_p, v_p), the 7 force rows of the step, then the
// step's corrector and predictor intervals and powers (computed while the CTA
// waits for the others).
constexpr int ST_ROWS = 3 * 6 + 7 + 7 + 3;
__device__ __forceinline__ int st_row(int c, int f) { return 6 * c + f; }
__device__ __forceinline__ int force_row(int q7) { return 18 + q7; }
constexpr int CORR_ROW = 25, PRED_ROW = 32;

template <int GT>
__host__ __device__ constexpr size_t sh_red_bytes() { return (size_t)SH_WARPS * 7 * 2 * GT * sizeof(float2); }

// Resident: the whole image.  Streamed: the ring, then the CTA's own records.
template <int GT, bool STREAM>
__host__ __device__ constexpr size_t sh_smem_bytes(int n_pad)
{
    return SH_BAR_BYTES + (size_t)(STREAM ? SH_RING * TILE_J + 2 * GT : n_pad) * sizeof(JMixed) + sh_red_bytes<GT>() +
           (size_t)ST_ROWS * 2 * GT * sizeof(double);
}

// Component c of particle k predicted to X, V: the FP64 rows x_p, v_p, and the c-parts of its j
// image record (the layout write_images gives, written here a float2 at a time).
__device__ __forceinline__ void emit_component(const SharedStepArgs &A, JMixed *img, int c, int k, double X, double V,
                                               double M)
{
    A.xp[3 * (size_t)k + c] = X;
    A.vp[3 * (size_t)k + c] = V;
    float h, l;
    split_ds(X, h, l);
    const float vf = f32pack::to_f32(V);
    float2 *rec = reinterpret_cast<float2 *>(img + k);
    rec[c] = make_float2(h, h);           // q[0].xy, q[0].zw, q[1].xy: x, y, z high words
    rec[4 + c] = make_float2(l, l);       // q[2].xy, q[2].zw, q[3].xy: low words
    rec[7 + c] = make_float2(vf, vf);     // q[3].zw, q[4].xy, q[4].zw: velocity
    bool bad = !(f32pack::finite(X) && f32pack::finite(V));
    if (c == 0) {
        const float mf = f32pack::to_f32(M);
        rec[3] = make_float2(mf, mf);     // q[1].zw: mass
        bad = bad || !f32pack::finite(M);
    }
    if (bad)
        atomicOr(A.err, ERR_NONFINITE);
    fence_proxy_async_global();
}

template <int GT, bool GUARD, bool STREAM>
__global__ void __launch_bounds__(SH_THREADS, 1) k_shared_steps(const SharedStepArgs A)
{
    constexpr int GROUPS = SH_THREADS / GT;
    constexpr int I_CTA = 2 * GT;
    static_assert(32 % GT == 0 && I_CTA <= SH_MAX_OWN, "groups tile the warps");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int n = A.n, n_pad = A.n_pad, n_tiles = n_pad / TILE_J;
    constexpr int IMG = STREAM ? SH_RING * TILE_J + I_CTA : 0;  // streamed: ring and own records
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);                     // [n_tiles] or [SH_RING]
    JMixed *img = reinterpret_cast<JMixed *>(smem_raw + SH_BAR_BYTES);           // [n_pad] or the ring
    JMixed *orec = img + SH_RING * TILE_J;                                        // streamed: [I_CTA]
    float2 *red = reinterpret_cast<float2 *>(img + (STREAM ? IMG : n_pad));       // [SH_WARPS][7][I_CTA]
    double *st = reinterpret_cast<double *>(red + SH_WARPS * 7 * I_CTA);          // [ST_ROWS][I_CTA]
    const int P = (int)gridDim.x, b = (int)blockIdx.x;
    const int lo = (int)((long long)n * b / P), hi = (int)((long long)n * (b + 1) / P);
    const int own = hi - lo;  // 1 .. I_CTA (the launch checks)
    const int tid = (int)threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = tid / GT, s = tid - g * GT;
    // warp w's j: [wb, wb + n_pad / SH_WARPS); group gw of the warp reads wb + gw + W jj, jj < L
    constexpr int W = 32 / GT;
    const int L = n_pad / GROUPS, wb = warp * (n_pad / SH_WARPS), gw = g - warp * W;
    const float eps2f = (float)A.eps2, rmin2f = (float)A.rmin2;
    const bool need_mask = eps2f != 0.f;  // with eps = 0 the guard zeroes the self pair anyway
    const unsigned count0 = A.arrivals0, per_step = (unsigned)P;
    // the component lanes: warp w < 3 CW (CW warps per component), component c = w % 3, particle
    // slot sl = lane + 32 (w / 3)
    constexpr int CW = I_CTA > 32 ? 2 : 1;
    const int c = warp % 3, sl = lane + 32 * (warp / 3);
    const bool comp = warp < 3 * CW && sl < own;
    const int kc = lo + sl;
    if (tid == 0 && !STREAM) {  // (streamed: the ring's barriers are set up at every step)
        for (int q = 0; q < n_tiles; ++q)
            mbar_init(&bars[q], 1);
        mbar_fence_init();
    }
    for (int o = tid; o < 12 * own; o += SH_THREADS) {
        const int slot = o / 12, r = o - 12 * slot, f = r / 3, cc = r - 3 * f;
        const double *src = f == 0 ? A.x : f == 1 ? A.v : f == 2 ? A.a : A.jerk_b;
        st[st_row(cc, f) * I_CTA + slot] = src[3 * (size_t)(lo + slot) + cc];
    }
    double tb = 0.0, M = 0.0;  // the component lane's particle time and mass
    if (comp) {
        tb = A.t_b[kc];
        M = A.m[kc];
    }
    __syncthreads();
    // the first image: own particles predicted to t0 + dt (or, to initialise, as they are); the last
    // CTA writes both images' padding
    if (comp) {
        double X = st[st_row(c, 0) * I_CTA + sl], V = st[st_row(c, 1) * I_CTA + sl];
        if (!A.init)
            predict_xv(predict_dt((A.t0 + A.dt) - tb), X, V, st[st_row(c, 2) * I_CTA + sl],
                       st[st_row(c, 3) * I_CTA + sl], X, V);
        st[st_row(c, 4) * I_CTA + sl] = X;
        st[st_row(c, 5) * I_CTA + sl] = V;
        emit_component(A, A.img, c, kc, X, V, M);
    }
    if (b == P - 1) {
        for (int k = n + tid; k < n_pad; k += SH_THREADS) {
            write_images(k, PAD_POS, PAD_POS, PAD_POS, 0.0, 0.0, 0.0, 0.0, A.img, nullptr);
            write_images(k, PAD_POS, PAD_POS, PAD_POS, 0.0, 0.0, 0.0, 0.0, A.img + n_pad, nullptr);
        }
        fence_proxy_async_global();
    }
    arrive(A.arrivals);
    double t = A.t0;
    const int n_iter = A.init ? 1 : A.n_steps;
    for (int step = 0; step < n_iter; ++step) {
        const double tn = A.init ? A.t0 : t + A.dt;
        const uint32_t parity = (uint32_t)(step & 1);
        // 0. while thread 0 waits: the corrector's interval and powers (warp 1, from the particle's
        //    own time) and the predictor's for the next step (warp 2), into shared memory
        if (A.init) {
        } else if (comp && c == 1) {
            const CorrectDt S = correct_dt(tn - tb);
            const double r[7] = {S.dt, S.idt2, S.idt3, S.c3, S.c4, S.c5, S.dt6};
#pragma unroll
            for (int q = 0; q < 7; ++q)
                st[(CORR_ROW + q) * I_CTA + sl] = r[q];
        } else if (comp && c == 2) {
            const PredictDt Pd = predict_dt((tn + A.dt) - tn);
            st[PRED_ROW * I_CTA + sl] = Pd.dt;
            st[(PRED_ROW + 1) * I_CTA + sl] = Pd.dt2;
            st[(PRED_ROW + 2) * I_CTA + sl] = Pd.dt3;
        }
        // 1. every CTA's records of this step are out: the whole image into shared memory
        if (!wait_arrivals(A.arrivals, count0 + ((unsigned)step + 1u) * per_step, A.err))
            return;  // no copy of this step was issued yet
        int idx[2];  // thread s of group g holds slots s and s + GT
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k = lo + s + q * GT;
            idx[q] = k < hi ? k : -1;
        }
        Lane7 acc0, acc1;
        acc0.zero();
        acc1.zero();
        const JMixed *src = A.img + (size_t)(step & 1) * n_pad;
        if constexpr (!STREAM) {
            if (tid == 0) {
                fence_proxy_async_global();
                for (int q = 0; q < n_tiles; ++q) {
                    mbar_arrive_expect_tx(&bars[q], SH_TILE_BYTES);
                    bulk_g2s(img + (size_t)q * TILE_J, src + (size_t)q * TILE_J, SH_TILE_BYTES, &bars[q]);
                }
            }
            // 2. own particles against the group's j; wait for the tiles this thread reads (a failed wait is
            //    made warp-uniform, so no lane leaves its warp's votes behind)
            const bool failed = !__all_sync(0xffffffffu, mbar_wait_bounded(&bars[lo / TILE_J], parity) &&
                                                             mbar_wait_bounded(&bars[(hi - 1) / TILE_J], parity) &&
                                                             mbar_wait_bounded(&bars[wb / TILE_J], parity) &&
                                                             mbar_wait_bounded(&bars[(wb + W * L - 1) / TILE_J], parity));
            if (!failed) {
                const IPair I = load_ipair(img + (idx[0] >= 0 ? idx[0] : lo), img + (idx[1] >= 0 ? idx[1] : lo),
                                           eps2f, rmin2f);
                Tile7 tt;
                tt.zero();
                const JMixed *T = img + wb + gw;
                const bool mine =
                    (unsigned)(idx[0] - wb) < (unsigned)(W * L) || (unsigned)(idx[1] - wb) < (unsigned)(W * L);
                if (need_mask && __any_sync(0xffffffffu, mine)) {
                    for (int jj = 0; jj < L; ++jj)
                        pair<GUARD, MODE_ACC_JERK_POT, true>(T[W * jj], I, tt, wb + gw + W * jj, idx[0], idx[1]);
                } else {
#pragma unroll 4
                    for (int jj = 0; jj < L; ++jj)
                        pair<GUARD, MODE_ACC_JERK_POT>(T[W * jj], I, tt);
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
                return;  // the other CTAs give up waiting for this one's arrival
            }
        } else {
            // 2 streamed: the CTA's own records from the global image (its own writes), and the image
            // tile by tile through the ring.  The ring's barriers are set up afresh every step, so tile q
            // (slot q % SH_RING) completes phase (q / SH_RING) & 1 of its slot's barrier.  Warp w sums
            // records [w JW, (w + 1) JW) of each tile, its groups interleaved record by record.
            constexpr int JW = TILE_J / SH_WARPS;
            for (int q = tid; q < 5 * own; q += SH_THREADS) {
                const int k = q / 5, w5 = q - 5 * k;
                orec[k].q[w5] = __ldcg(reinterpret_cast<const float4 *>(src + lo + k) + w5);
            }
            auto issue = [&](int q) {
                const int slot = q % SH_RING;
                mbar_arrive_expect_tx(&bars[slot], SH_TILE_BYTES);
                bulk_g2s(img + (size_t)slot * TILE_J, src + (size_t)q * TILE_J, SH_TILE_BYTES, &bars[slot]);
            };
            if (tid == 0) {
                for (int q = 0; q < SH_RING; ++q)
                    mbar_init(&bars[q], 1);
                mbar_fence_init();
                fence_proxy_async_global();
                for (int q = 0; q < n_tiles && q < SH_RING; ++q)
                    issue(q);
            }
            __syncthreads();  // own records and barriers ready
            const IPair I = load_ipair(orec + (idx[0] >= 0 ? idx[0] - lo : 0), orec + (idx[1] >= 0 ? idx[1] - lo : 0),
                                       eps2f, rmin2f);
            Tile7 tt;
            tt.zero();
            int since = 0;
            bool failed = false;
            const int n_chunks = (n_tiles + SH_CH - 1) / SH_CH;
            int cch = 0;
            for (; cch < n_chunks; ++cch) {
                const int q1 = min(n_tiles, (cch + 1) * SH_CH);
                for (int q = cch * SH_CH; q < q1; ++q) {
                    const int slot = q % SH_RING;
                    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[slot], (uint32_t)(q / SH_RING) & 1u))) {
                        failed = true;
                        break;
                    }
                    const int j0 = q * TILE_J + warp * JW;
                    const JMixed *T = img + (size_t)slot * TILE_J + warp * JW + gw;
                    const bool mine =
                        (unsigned)(idx[0] - j0) < (unsigned)JW || (unsigned)(idx[1] - j0) < (unsigned)JW;
                    if (need_mask && __any_sync(0xffffffffu, mine)) {
                        for (int jj = 0; jj < JW / W; ++jj)
                            pair<GUARD, MODE_ACC_JERK_POT, true>(T[W * jj], I, tt, j0 + gw + W * jj, idx[0], idx[1]);
                    } else {
#pragma unroll
                        for (int jj = 0; jj < JW / W; ++jj)
                            pair<GUARD, MODE_ACC_JERK_POT>(T[W * jj], I, tt);
                    }
                    since += JW / W;
                    if (since >= SH_FLUSH_J) {
                        fold<MODE_ACC_JERK_POT>(tt, acc0, acc1);
                        since = 0;
                    }
                }
                fence_proxy_async_smem();  // this half's reads before its refill
                if (__syncthreads_or(failed)) {
                    failed = true;
                    break;
                }
                if (tid == 0)  // the half just summed takes the chunk after next
                    for (int q = (cch + 2) * SH_CH; q < n_tiles && q < (cch + 3) * SH_CH; ++q)
                        issue(q);
            }
            if (failed) {
                if (tid == 0) {  // every copy issued and not yet consumed lands first (chunks cch, cch + 1)
                    atomicOr(A.err, ERR_TIMEOUT);
                    for (int q = cch * SH_CH; q < n_tiles && q < (cch + 2) * SH_CH; ++q)
                        if (!mbar_wait_bounded(&bars[q % SH_RING], (uint32_t)(q / SH_RING) & 1u)) {
                            atomicOr(A.err, ERR_DRAIN);
                            break;
                        }
                }
                return;
            }
            fold<MODE_ACC_JERK_POT>(tt, acc0, acc1);
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
            const double row = q7 < 6 ? A.G * val : -A.G * val;
            st[force_row(q7) * I_CTA + slot] = row;
            const int p = lo + slot;
            if (q7 < 3)
                A.f_acc[3 * (size_t)p + q7] = row;
            else if (q7 < 6)
                A.f_jerk[3 * (size_t)p + (q7 - 3)] = row;
            else if (A.f_pot)
                A.f_pot[p] = row;
        }
        __syncthreads();
        // 4. initialisation: a, jerk and t of each own particle, and its first block step
        if (A.init) {
            if (comp && c == 0) {
                double a0[3], j0[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    a0[q] = st[force_row(q) * I_CTA + sl];
                    j0[q] = st[force_row(3 + q) * I_CTA + sl];
                    A.a[3 * (size_t)kc + q] = a0[q];
                    A.jerk_b[3 * (size_t)kc + q] = j0[q];
                }
                A.t_b[kc] = A.t0;
                A.dt_b[kc] = initial_step(a0, j0, A.dt_min, A.dt_max);
            }
            break;
        }
        // 4. component c of each own particle corrected (shared step: the step size stays), then
        //    predicted to the next step into the other image
        if (comp) {
            CorrectDt S;
            S.dt = st[CORR_ROW * I_CTA + sl];
            S.idt2 = st[(CORR_ROW + 1) * I_CTA + sl];
            S.idt3 = st[(CORR_ROW + 2) * I_CTA + sl];
            S.c3 = st[(CORR_ROW + 3) * I_CTA + sl];
            S.c4 = st[(CORR_ROW + 4) * I_CTA + sl];
            S.c5 = st[(CORR_ROW + 5) * I_CTA + sl];
            S.dt6 = st[(CORR_ROW + 6) * I_CTA + sl];
            const double a1 = st[force_row(c) * I_CTA + sl], j1 = st[force_row(3 + c) * I_CTA + sl];
            double x1, v1, a2, a3;
            correct_xv(S, st[st_row(c, 2) * I_CTA + sl], st[st_row(c, 3) * I_CTA + sl], a1, j1,
                       st[st_row(c, 4) * I_CTA + sl], st[st_row(c, 5) * I_CTA + sl], x1, v1, a2, a3);
            tb = tn;
            st[st_row(c, 0) * I_CTA + sl] = x1;
            st[st_row(c, 1) * I_CTA + sl] = v1;
            st[st_row(c, 2) * I_CTA + sl] = a1;
            st[st_row(c, 3) * I_CTA + sl] = j1;
            const size_t o = 3 * (size_t)kc + c;
            A.x[o] = x1;
            A.v[o] = v1;
            A.a[o] = a1;
            A.jerk_b[o] = j1;
            if (c == 0)
                A.t_b[kc] = tn;
            if (step + 1 < A.n_steps) {
                PredictDt Pd;
                Pd.dt = st[PRED_ROW * I_CTA + sl];
                Pd.dt2 = st[(PRED_ROW + 1) * I_CTA + sl];
                Pd.dt3 = st[(PRED_ROW + 2) * I_CTA + sl];
                double X, V;
                predict_xv(Pd, x1, v1, a1, j1, X, V);
                st[st_row(c, 4) * I_CTA + sl] = X;
                st[st_row(c, 5) * I_CTA + sl] = V;
                emit_component(A, A.img + (size_t)((step + 1) & 1) * n_pad, c, kc, X, V, M);
            }
        }
        if (step + 1 < A.n_steps)
            arrive(A.arrivals);
        t = tn;
    }
}

// Self-test of the bounded arrival wait: one CTA waits for an arrival on a word that nothing
// increments and gives up after limit_ns, as a shared-step CTA does when another never arrives.
__device__ unsigned g_never_arrives = 0u;

__global__ void k_arrival_selftest(unsigned long long limit_ns, unsigned *err)
{
    wait_arrivals(&g_never_arrives, 1u, err, limit_ns);
}

template <int GT, bool GUARD, bool STREAM>
cudaError_t sh_launch(const SharedStepArgs &a, bool query_only, int *grid, cudaStream_t st)
{
    const auto kern = k_shared_steps<GT, GUARD, STREAM>;
    if (query_only) {
        // opt in once for the largest image, so a smaller context cannot lower a larger one's limit
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sh_smem_bytes<GT, STREAM>(SH_RESIDENT_N));
        if (e != cudaSuccess)
            return e;
        int dev = 0, nsm = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SH_THREADS,
                                                               sh_smem_bytes<GT, STREAM>(a.n_pad))) != cudaSuccess)
            return e;
        const int ctas = per_sm > 0 ? nsm : 0;  // one CTA per SM
        *grid = ctas < a.n ? ctas : a.n;
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(a.ctas);
    cfg.blockDim = dim3(SH_THREADS);
    cfg.dynamicSmemBytes = sh_smem_bytes<GT, STREAM>(a.n_pad);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// Narrowest j-group that holds a CTA's share of the particles; the image resident in shared memory up
// to SH_RESIDENT_N records, streamed above.
template <bool GUARD>
cudaError_t sh_dispatch(const SharedStepArgs &a, int own_max, bool query_only, int *grid, cudaStream_t st)
{
    if (a.n_pad <= SH_RESIDENT_N) {
        if (own_max <= 8)
            return sh_launch<4, GUARD, false>(a, query_only, grid, st);
        if (own_max <= 16)
            return sh_launch<8, GUARD, false>(a, query_only, grid, st);
        if (own_max <= 32)
            return sh_launch<16, GUARD, false>(a, query_only, grid, st);
        return cudaErrorInvalidValue;
    }
    if (own_max <= 16)
        return sh_launch<8, GUARD, true>(a, query_only, grid, st);
    if (own_max <= 32)
        return sh_launch<16, GUARD, true>(a, query_only, grid, st);
    if (own_max <= SH_MAX_OWN)
        return sh_launch<32, GUARD, true>(a, query_only, grid, st);
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
    // the grid does not depend on the group width (one CTA per SM): ask the widest of the path (resident
    // or streamed), then check the share against the width that will run
    const int widest = a.n_pad <= SH_RESIDENT_N ? 32 : SH_MAX_OWN;
    int grid = 0;
    cudaError_t e = guard ? sh_dispatch<true>(a, widest, true, &grid, nullptr)
                          : sh_dispatch<false>(a, widest, true, &grid, nullptr);
    if (e != cudaSuccess || grid < 1 || own_max_of(n, grid) > widest) {
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

cudaError_t launch_arrival_selftest(unsigned long long limit_ns, unsigned *err, cudaStream_t st)
{
    k_arrival_selftest<<<1, 64, 0, st>>>(limit_ns, err);
    return cudaGetLastError();
}

cudaError_t launch_shared_steps(const SharedStepArgs &a, bool guard, cudaStream_t st)
{
    if (a.n < 1 || a.n > SH_MAX_N || a.n_pad % TILE_J != 0 || a.n_pad < a.n || a.n_pad > SH_MAX_N ||
        a.n_steps < 0 || a.ctas < 1 || a.ctas > a.n || own_max_of(a.n, a.ctas) > SH_MAX_OWN || !a.img ||
        !a.arrivals)
        return cudaErrorInvalidValue;
    if (a.n_steps == 0 && !a.init)
        return cudaSuccess;
    const int own = own_max_of(a.n, a.ctas);
    return guard ? sh_dispatch<true>(a, own, false, nullptr, st) : sh_dispatch<false>(a, own, false, nullptr, st);
}

}  // namespace kirin
