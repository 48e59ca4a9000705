// O(N) kernels around the direct sum: the j-split reduction (Sect. 3.2), the
// predictor that builds the j-particle images (Sect. 3.1, done on the device
// instead of the host), energy sums (Eq. 2), and the Hermite corrector and
// block-step scheduler (Sect. 3, Sect. 3.1).  All FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "kirin_internal.cuh"
#include "loop_internal.cuh"
#include "step_math.cuh"
#include "tma.cuh"

namespace kirin {
namespace {

constexpr int AUX_THREADS = 256;
constexpr int CORR_THREADS = 32;     // one warp per CTA: FP64-bound, spread over SMs
constexpr int CORR_MAX_CTAS = 1024;  // the corrector loops beyond this

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

// Sum the n_split partial results of every (i, quantity) and write the
// scaled outputs (acc, jerk: G * sum; pot: -G * sum); with the neighbour
// search also the nearest (r2, j) over the splits.  L lanes share one output:
// lane l sums splits l, l + L, ... in order, then the L partial sums meet in
// a fixed xor tree, so the result does not depend on timing.  Threads are
// ordered quantity-major, i fastest, so L = 1 reads are coalesced.
template <int L>
__global__ void k_reduce_splits(const ForceArgs Ain)
{
    ForceArgs A = Ain;
    if (Ain.n_i_dev)
        A.n_i = *Ain.n_i_dev;
    const int nout = A.nq > 7 ? 8 : 7;  // the neighbour pair (r2, j) is output 7
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long g = t / L;
    const int lane = (int)(t % L);
    if (g >= (long long)nout * A.n_i)
        return;  // whole groups leave together (L divides the warp)
    const int q = (int)(g / A.n_i);
    const int k = (int)(g - (long long)q * A.n_i);
    const unsigned wl = threadIdx.x & 31u;
    const unsigned mask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << (wl & ~(unsigned)(L - 1)));
    if (q < 7) {
        double sum = 0.0;
        for (int y = lane; y < A.n_split; y += L)
            sum += A.partial[((size_t)y * A.nq + q) * A.n_i_pad + k];
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1)
            sum += __shfl_xor_sync(mask, sum, o, L);
        if (lane == 0)
            store_final(A, q, k, sum);
    } else {  // nearest neighbour: lexicographic minimum over the splits
        double r2 = INFINITY, j = -1.0;
        for (int y = lane; y < A.n_split; y += L)
            nn_min(r2, j, A.partial[((size_t)y * A.nq + 7) * A.n_i_pad + k],
                   A.partial[((size_t)y * A.nq + 8) * A.n_i_pad + k]);
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            const double r2b = __shfl_xor_sync(mask, r2, o, L);
            const double jb = __shfl_xor_sync(mask, j, o, L);
            nn_min(r2, j, r2b, jb);
        }
        if (lane == 0)
            store_nn(A, k, r2, j);
    }
}

__global__ void k_predict_pack(int n, int n_pad, double t, int predict, const double *__restrict__ m,
                               const double *__restrict__ x, const double *__restrict__ v,
                               const double *__restrict__ a, const double *__restrict__ jk,
                               const double *__restrict__ t0, double *xp, double *vp, JMixed *jm,
                               JF64 *jd, unsigned *err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_pad)
        predict_one(k, n, t, predict, m, x, v, a, jk, t0, xp, vp, jm, jd, err);
}

// Images from (m, x) only (velocities zero), for acceleration-only clients.
__global__ void k_pack_xm(int n, int n_pad, const double *__restrict__ m, const double *__restrict__ x,
                          JMixed *jm, JF64 *jd, unsigned *err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pad)
        return;
    if (k >= n) {
        write_images(k, PAD_POS, PAD_POS, PAD_POS, 0.0, 0.0, 0.0, 0.0, jm, jd);
        return;
    }
    const double X = x[3 * (size_t)k], Y = x[3 * (size_t)k + 1], Z = x[3 * (size_t)k + 2];
    if (!(isfinite(X) && isfinite(Y) && isfinite(Z) && isfinite(m[k])))
        atomicOr(err, ERR_NONFINITE);
    write_images(k, X, Y, Z, m[k], 0.0, 0.0, 0.0, jm, jd);
}

// Device-to-device upload of particles [first, first + n) into the base state.
__global__ void k_scatter_state(int first, int n, const double *m, const double *x, const double *v,
                                const double *a, const double *jk, const double *t0, double *bm,
                                double *bx, double *bv, double *ba, double *bj, double *bt0,
                                unsigned *err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n)
        return;
    const size_t d = (size_t)first + k;
    bool fin = isfinite(m[k]);
    bm[d] = m[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double xc = x[3 * (size_t)k + c], vc = v[3 * (size_t)k + c];
        const double ac = a ? a[3 * (size_t)k + c] : 0.0;
        const double jc = jk ? jk[3 * (size_t)k + c] : 0.0;
        fin = fin && isfinite(xc) && isfinite(vc) && isfinite(ac) && isfinite(jc);
        bx[3 * d + c] = xc;
        bv[3 * d + c] = vc;
        ba[3 * d + c] = ac;
        bj[3 * d + c] = jc;
    }
    const double tt = t0 ? t0[k] : 0.0;
    bt0[d] = tt;
    if (!(fin && isfinite(tt)))
        atomicOr(err, ERR_NONFINITE);
}

// One CTA: K = sum 1/2 m |v|^2 and W = 1/2 sum m phi, fixed order (deterministic).
__global__ void __launch_bounds__(1024) k_energy(int n, const double *__restrict__ m,
                                                 const double *__restrict__ v,
                                                 const double *__restrict__ pot, double *out)
{
    __shared__ double sk[1024], sw[1024];
    double kk = 0.0, ww = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double vx = v[3 * (size_t)i], vy = v[3 * (size_t)i + 1], vz = v[3 * (size_t)i + 2];
        kk += 0.5 * m[i] * (vx * vx + vy * vy + vz * vz);
        ww += 0.5 * m[i] * pot[i];
    }
    sk[threadIdx.x] = kk;
    sw[threadIdx.x] = ww;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sk[threadIdx.x] += sk[threadIdx.x + w];
            sw[threadIdx.x] += sw[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sk[0];
        out[1] = sw[0];
    }
}

__global__ void k_hermite_init(int n, double t, const double *acc, const double *jerk, double dt_min,
                               double dt_max, double *ba, double *bj, double *bt, double *bdt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n)
        return;
    double a[3], j[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a[c] = acc[3 * (size_t)k + c];
        j[c] = jerk[3 * (size_t)k + c];
        ba[3 * (size_t)k + c] = a[c];
        bj[3 * (size_t)k + c] = j[c];
    }
    bt[k] = t;
    bdt[k] = initial_step(a, j, dt_min, dt_max);
}

// Order-preserving map of doubles to unsigned keys (the sign bit set for
// non-negative values, every bit flipped for negative ones; NaN the largest
// key), so an unsigned atomic minimum finds the smallest end time whatever
// its sign.  ~0 (the start value of a minimum) maps back to NaN: no block.
__device__ __forceinline__ unsigned long long time_key(double d)
{
    if (d != d)
        return ~0ull;
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_time(unsigned long long k)
{
    if (k == ~0ull)
        return __longlong_as_double(0x7ff8000000000000ll);
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// Block selection: t_next = min_i (t_i + dt_i) and the ordered list of the
// i with t_i + dt_i == t_next (Sect. 3.1 block time-steps).  Three passes
// over the particles, each fully parallel: an atomic minimum over the keys
// (time_key) of the end times, per-CTA counts, then ordered writes at
// offsets summed from the counts, so the list is in index order.
constexpr int SEL_THREADS = 256;
constexpr int SEL_ITEMS = 4;  // particles per thread, SEL_THREADS apart
constexpr int SEL_PER_CTA = SEL_THREADS * SEL_ITEMS;

__global__ void __launch_bounds__(SEL_THREADS) k_sel_min(int n, const double *__restrict__ bt,
                                                         const double *__restrict__ bdt,
                                                         unsigned long long *minw)
{
    unsigned long long mn = ~0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        mn = min(mn, time_key(bt[i] + bdt[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0)
        atomicMin(minw, mn);
}

__global__ void __launch_bounds__(SEL_THREADS) k_sel_count(int n, const double *__restrict__ bt,
                                                           const double *__restrict__ bdt,
                                                           const unsigned long long *minw, int32_t *counts)
{
    const double tn = key_time(*minw);
    int total = 0;
#pragma unroll
    for (int j = 0; j < SEL_ITEMS; ++j) {
        const int i = blockIdx.x * SEL_PER_CTA + j * SEL_THREADS + threadIdx.x;
        total += __syncthreads_count(i < n && bt[i] + bdt[i] == tn);
    }
    if (threadIdx.x == 0)
        counts[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SEL_THREADS) k_sel_write(int n, const double *__restrict__ bt,
                                                           const double *__restrict__ bdt,
                                                           const unsigned long long *minw,
                                                           const int32_t *__restrict__ counts, double t_end,
                                                           int32_t *ilist, double *t_next_out,
                                                           int32_t *count_out, double *t_next_host,
                                                           int32_t *count_host)
{
    __shared__ int warp_tot[SEL_THREADS / 32];
    __shared__ int red[SEL_THREADS];
    const double tn = key_time(*minw);
    const bool due = tn <= t_end;
    // offset of this CTA: sum of the counts of the CTAs before it
    int part = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += SEL_THREADS)
        part += counts[b];
    red[threadIdx.x] = part;
    __syncthreads();
    for (int w = SEL_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    int base = red[0];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < SEL_ITEMS; ++j) {
        const int i = blockIdx.x * SEL_PER_CTA + j * SEL_THREADS + threadIdx.x;
        const bool flag = due && i < n && bt[i] + bdt[i] == tn;
        const unsigned ballot = __ballot_sync(0xffffffffu, flag);
        if (lane == 0)
            warp_tot[warp] = __popc(ballot);
        __syncthreads();
        int before = 0, all = 0;
#pragma unroll
        for (int w = 0; w < SEL_THREADS / 32; ++w) {
            before += w < warp ? warp_tot[w] : 0;
            all += warp_tot[w];
        }
        if (flag)
            ilist[base + before + __popc(ballot & ((1u << lane) - 1u))] = i;
        base += all;
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        *count_out = due ? base : 0;
        *t_next_out = tn;
        if (count_host) {  // mapped host copies: the host reads them once the stream has synchronised
            *count_host = due ? base : 0;
            *t_next_host = tn;
        }
    }
}

__device__ __forceinline__ void correct_one(int k, const int32_t *ilist, double t_next, double eta, double dt_min,
                                            double dt_max, int update_dt, const double *xp, const double *vp,
                                            const double *acc, const double *jerk, double *bx, double *bv,
                                            double *ba, double *bj, double *bt, double *bdt)
{
    correct_at(ilist ? (size_t)ilist[k] : (size_t)k, k, t_next, eta, dt_min, dt_max, update_dt, xp, vp, acc, jerk,
               bx, bv, ba, bj, bt, bdt);
}

// One warp per CTA, and member k on CTA k mod gridDim (lane k / gridDim):
// a short block puts one member on each of many SMs, since an FP64 warp
// instruction costs the same with one active lane as with 32.
__global__ void __launch_bounds__(CORR_THREADS) k_hermite_correct(
    int n_act, const int32_t *__restrict__ ilist, double t_next, double eta, double dt_min, double dt_max,
    int update_dt, const double *__restrict__ xp, const double *__restrict__ vp, const double *__restrict__ acc,
    const double *__restrict__ jerk, double *bx, double *bv, double *ba, double *bj, double *bt, double *bdt)
{
    for (long long k = blockIdx.x + (long long)threadIdx.x * gridDim.x; k < n_act;
         k += (long long)CORR_THREADS * gridDim.x)
        correct_one((int)k, ilist, t_next, eta, dt_min, dt_max, update_dt, xp, vp, acc, jerk, bx, bv, ba, bj, bt,
                    bdt);
}

// ---- block step of the device-driven loop -------------------------------------

constexpr int STEP_THREADS = 256;
constexpr int STEP_WARPS = STEP_THREADS / 32;

__device__ __forceinline__ unsigned long long cta_min_u64(unsigned long long v)
{
    __shared__ unsigned long long part[STEP_WARPS];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0)
        part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < STEP_WARPS; ++w)
            v = min(v, part[w]);
    return v;  // valid in thread 0
}

__device__ __forceinline__ int cta_sum(int v)
{
    __shared__ int part[STEP_WARPS];
    __shared__ int total;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0)
        part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < STEP_WARPS; ++w)
            t += part[w];
        total = t;
    }
    __syncthreads();
    return total;
}

__device__ __forceinline__ void chunk_of(int n, int &c0, int &c1)
{
    const int chunk = (n + (int)gridDim.x - 1) / (int)gridDim.x;
    c0 = min(n, (int)blockIdx.x * chunk);
    c1 = min(n, c0 + chunk);
}

// Rank of this thread's flag among the CTA's flags of one pass (index order),
// and the pass's total; uniform call over the CTA.
__device__ __forceinline__ int cta_rank(bool flag, int &all)
{
    __shared__ int warp_tot[STEP_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned ballot = __ballot_sync(0xffffffffu, flag);
    if (lane == 0)
        warp_tot[warp] = __popc(ballot);
    __syncthreads();
    int ahead = 0;
    all = 0;
#pragma unroll
    for (int w = 0; w < STEP_WARPS; ++w) {
        ahead += w < warp ? warp_tot[w] : 0;
        all += warp_tot[w];
    }
    __syncthreads();
    return ahead + __popc(ballot & ((1u << lane) - 1u));
}

// Correct the pending block and take min (t_i + dt_i).  Thread t of CTA b
// owns particles c0 + t, c0 + t + 256, ... of its chunk.  A member of the
// pending block is recognised by t_i + dt_i == the block time; the select
// kernel listed the chunk's members in index order from chunk_off[b], so a
// member's rank among them gives its row of the force results.  Members add
// their new end time to the minimum, the others their unchanged one.
//
// A pass with at most SPLIT_MEMBERS members (every pass of a small block)
// corrects each member on three warps, one per component, and then runs
// Aarseth's criterion on one thread: an FP64 warp instruction costs the same
// whatever its active lanes, so the latency of a member's corrector is its
// instruction chain, and the components' share of it runs side by side.  The
// operations are correct_at's, in its order, so the bits are the same.
constexpr int SPLIT_MEMBERS = 64;

__global__ void __launch_bounds__(STEP_THREADS) k_step_correct(const StepArgs A)
{
    static_assert(STEP_WARPS >= 3 * (SPLIT_MEMBERS / 32), "three component warps per 32 members");
    __shared__ int mem_i[SPLIT_MEMBERS];                 // the pass's members by rank
    __shared__ double comp_v[4][3][SPLIT_MEMBERS];       // a1, j1, a2e, a3 per component
    __shared__ double step_v[3][SPLIT_MEMBERS];          // dt, dt^2, 1/dt of each member's step
    __shared__ bool step_p2[SPLIT_MEMBERS];
    RunState *R = A.run;
    const int par = (int)(R->steps & 1);
    const bool any = R->pending > 0;
    const double t_prev = R->t_last;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    int c0, c1;
    chunk_of(A.n, c0, c1);
    int base = any ? A.chunk_off[blockIdx.x] : 0;
    unsigned long long mn = ~0ull;
    for (int i0 = c0; i0 < c1; i0 += STEP_THREADS) {
        const int i = i0 + threadIdx.x;
        double end = 0.0;
        bool member = false;
        if (i < c1) {
            end = A.bt[i] + A.bdt[i];
            member = any && end == t_prev;
        }
        int all;
        const int rank = cta_rank(member, all);
        if (all == 0 || all > SPLIT_MEMBERS) {
            if (member)
                end = correct_at((size_t)i, base + rank, t_prev, A.eta, A.dt_min, A.dt_max, 1, A.xp, A.vp, A.acc,
                                 A.jerk, A.bx, A.bv, A.ba, A.bj, A.bt, A.bdt);
            if (i < c1)
                mn = min(mn, time_key(end));
        } else {
            if (member)
                mem_i[rank] = i;
            else if (i < c1)
                mn = min(mn, time_key(end));
            __syncthreads();
            const int c = warp % 3, sl = lane + 32 * (warp / 3);
            if (warp < 3 * (SPLIT_MEMBERS / 32) && sl < all) {
                const size_t im = (size_t)mem_i[sl];
                const CorrectDt S = correct_dt(t_prev - A.bt[im]);
                double a1, j1, a2e, a3;
                correct_component(S, c, im, base + sl, A.xp, A.vp, A.acc, A.jerk, A.bx, A.bv, A.ba, A.bj, a1, j1,
                                  a2e, a3);
                comp_v[0][c][sl] = a1;
                comp_v[1][c][sl] = j1;
                comp_v[2][c][sl] = a2e;
                comp_v[3][c][sl] = a3;
                if (c == 0) {
                    step_v[0][sl] = S.dt;
                    step_v[1][sl] = S.dt2;
                    step_v[2][sl] = S.idt;
                    step_p2[sl] = S.p2;
                }
            }
            __syncthreads();
            const int m = (int)threadIdx.x;
            if (m < all) {
                double A2 = 0.0, J = 0.0, N2 = 0.0, N3 = 0.0;
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    A2 = fma(comp_v[0][cc][m], comp_v[0][cc][m], A2);
                    J = fma(comp_v[1][cc][m], comp_v[1][cc][m], J);
                    N2 = fma(comp_v[2][cc][m], comp_v[2][cc][m], N2);
                    N3 = fma(comp_v[3][cc][m], comp_v[3][cc][m], N3);
                }
                const size_t im = (size_t)mem_i[m];
                const double q = aarseth_step(A2, J, N2, N3, step_v[0][m], step_v[1][m], step_p2[m], step_v[2][m],
                                              t_prev, A.eta, A.dt_min, A.dt_max);
                A.bt[im] = t_prev;
                A.bdt[im] = q;
                mn = min(mn, time_key(t_prev + q));
            }
        }
        base += all;
    }
    mn = cta_min_u64(mn);
    if (threadIdx.x == 0) {
        atomicMin(&R->minw[par], mn);
        if (blockIdx.x == 0) {  // fresh words for the select kernel and the next step
            R->minw[par ^ 1] = ~0ull;
            R->list_done = 0ull;
        }
    }
}

// Predict every j to t_next and list the next block.  One 64-bit atomic per
// CTA reserves its range of the list (low word) and counts finished CTAs
// (high word); the CTA that reserves last publishes the block at once (the
// list itself is read only by later kernels).
__global__ void __launch_bounds__(STEP_THREADS) k_step_select(const StepArgs A)
{
    RunState *R = A.run;
    const long long steps0 = R->steps;
    const double tn = key_time(R->minw[steps0 & 1]);
    const long long lim = R->max_steps;
    bool due = tn <= R->t_end && (lim <= 0 || steps0 < lim);
    const bool stall = due && steps0 > 0 && !(tn > R->t_last);
    if (stall)
        due = false;
    if (!due) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (stall)
                atomicOr(A.err, ERR_STALL);  // the block time stopped advancing: stop rather than loop forever
            *A.count_out = 0;
            R->pending = 0;
            cudaGraphSetConditional(A.branch, (unsigned)A.n_classes);
            cudaGraphSetConditional(A.loop, 0u);
        }
        return;
    }
    int c0, c1;
    chunk_of(A.n, c0, c1);
    int c = 0;
    for (int k = c0 + threadIdx.x; k < c1; k += STEP_THREADS) {
        predict_one(k, A.n, tn, 1, A.bm, A.bx, A.bv, A.ba, A.bj, A.bt, A.xp, A.vp, A.jm, A.jd, A.err);
        c += A.bt[k] + A.bdt[k] == tn;
    }
    for (int k = A.n + blockIdx.x * STEP_THREADS + threadIdx.x; k < A.n_pad; k += gridDim.x * STEP_THREADS)
        predict_one(k, A.n, tn, 1, A.bm, A.bx, A.bv, A.ba, A.bj, A.bt, A.xp, A.vp, A.jm, A.jd, A.err);  // padding
    const int cnt = cta_sum(c);
    __shared__ int base_s;
    if (threadIdx.x == 0) {
        const unsigned long long prev = atomicAdd(&R->list_done, (1ull << 32) | (unsigned long long)cnt);
        const int off = (int)(prev & 0xffffffffull);
        base_s = off;
        A.chunk_off[blockIdx.x] = off;
        if ((unsigned)(prev >> 32) == gridDim.x - 1) {  // the last reservation: the block is complete
            const int count = off + cnt;
            unsigned cls = (unsigned)A.n_classes - 1;
            for (int q = A.n_classes - 1; q >= 0; --q)
                if (count <= A.class_max[q])
                    cls = (unsigned)q;
            *A.count_out = count;
            *A.t_next_out = tn;
            R->steps = steps0 + 1;
            R->pairs += (double)count * (double)A.n_j;
            R->t_last = tn;
            R->pending = count;
            cudaGraphSetConditional(A.branch, cls);
            cudaGraphSetConditional(A.loop, 1u);
        }
    }
    __syncthreads();
    if (cnt) {
        int base = base_s;
        for (int i0 = c0; i0 < c1; i0 += STEP_THREADS) {
            const int i = i0 + threadIdx.x;
            const bool flag = i < c1 && A.bt[i] + A.bdt[i] == tn;
            int all;
            const int rank = cta_rank(flag, all);
            if (flag)
                A.ilist[base + rank] = i;
            base += all;
        }
    }
}

// Leapfrog pieces (Sect. 4.3 integrator): v_h = v + h a; x' = x + dt v_h
// (optionally recorded into hist); and the closing kick v' = v_h + h a'.
__global__ void k_lf_kick_drift(int n, double h, double dt, const double *__restrict__ a, double *v, double *x,
                                double *hist)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * n)
        return;
    const double vh = v[k] + h * a[k];
    const double xn = x[k] + dt * vh;
    v[k] = vh;
    x[k] = xn;
    if (hist)
        hist[k] = xn;
}

__global__ void k_axpy(int n, double alpha, const double *__restrict__ xv, double *y)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n)
        y[k] += alpha * xv[k];
}

__global__ void k_copy(int n, const double *__restrict__ src, double *dst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n)
        dst[k] = src[k];
}

// Images of (m, x) with c * lv in the velocity slots: the g = dL/da of one
// adjoint force call of the leapfrog's reverse sweep.
__global__ void k_pack_adjoint(int n, int n_pad, const double *__restrict__ m, const double *__restrict__ x,
                               const double *__restrict__ lv, double c, JMixed *jm, JF64 *jd, unsigned *err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pad)
        return;
    if (k >= n) {
        write_images(k, PAD_POS, PAD_POS, PAD_POS, 0.0, 0.0, 0.0, 0.0, jm, jd);
        return;
    }
    const size_t o = 3 * (size_t)k;
    const double gx = c * lv[o], gy = c * lv[o + 1], gz = c * lv[o + 2];
    if (!(isfinite(x[o]) && isfinite(x[o + 1]) && isfinite(x[o + 2]) && isfinite(gx) && isfinite(gy) &&
          isfinite(gz)))
        atomicOr(err, ERR_NONFINITE);
    write_images(k, x[o], x[o + 1], x[o + 2], m[k], gx, gy, gz, jm, jd);
}

// Self-test of the bounded waits: one thread waits on an mbarrier phase that
// nothing completes (the barrier expects two arrivals and gets one) and gives
// up after limit_ns; the CTA then reports ERR_TIMEOUT like a stalled copy would.
__global__ void k_wait_selftest(unsigned long long limit_ns, unsigned *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
        if (!mbar_wait_bounded(&bar, 0, limit_ns))
            atomicOr(err, ERR_TIMEOUT);
    }
}

}  // namespace

cudaError_t launch_reduce_splits(const ForceArgs &a, cudaStream_t st)
{
    if (a.n_i == 0)
        return cudaSuccess;
    // lanes per output: the smallest power of two that leaves each lane at most 8 splits
    int lanes = 1;
    while (lanes < 32 && lanes * 8 < a.n_split)
        lanes *= 2;
    const long long threads = (long long)(a.nq > 7 ? 8 : 7) * a.n_i * lanes;
    const int grid = (int)((threads + AUX_THREADS - 1) / AUX_THREADS);
    switch (lanes) {
    case 1: k_reduce_splits<1><<<grid, AUX_THREADS, 0, st>>>(a); break;
    case 2: k_reduce_splits<2><<<grid, AUX_THREADS, 0, st>>>(a); break;
    case 4: k_reduce_splits<4><<<grid, AUX_THREADS, 0, st>>>(a); break;
    case 8: k_reduce_splits<8><<<grid, AUX_THREADS, 0, st>>>(a); break;
    case 16: k_reduce_splits<16><<<grid, AUX_THREADS, 0, st>>>(a); break;
    default: k_reduce_splits<32><<<grid, AUX_THREADS, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_predict_pack(int n, int n_pad, double t, int predict, const double *m,
                                const double *x, const double *v, const double *a,
                                const double *jk, const double *t0, double *xp, double *vp,
                                JMixed *jm, JF64 *jd, unsigned *err, cudaStream_t st)
{
    if (n_pad == 0)
        return cudaSuccess;
    k_predict_pack<<<blocks_for(n_pad, AUX_THREADS), AUX_THREADS, 0, st>>>(
        n, n_pad, t, predict, m, x, v, a, jk, t0, xp, vp, jm, jd, err);
    return cudaGetLastError();
}

cudaError_t launch_pack_xm(int n, int n_pad, const double *m, const double *x, JMixed *jm,
                           JF64 *jd, unsigned *err, cudaStream_t st)
{
    if (n_pad == 0)
        return cudaSuccess;
    k_pack_xm<<<blocks_for(n_pad, AUX_THREADS), AUX_THREADS, 0, st>>>(n, n_pad, m, x, jm, jd, err);
    return cudaGetLastError();
}

cudaError_t launch_scatter_state(int first, int n, const double *m, const double *x,
                                 const double *v, const double *a, const double *jk,
                                 const double *t0, double *bm, double *bx, double *bv,
                                 double *ba, double *bj, double *bt0, unsigned *err,
                                 cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    k_scatter_state<<<blocks_for(n, AUX_THREADS), AUX_THREADS, 0, st>>>(first, n, m, x, v, a, jk, t0,
                                                                       bm, bx, bv, ba, bj, bt0, err);
    return cudaGetLastError();
}

cudaError_t launch_energy(int n, const double *m, const double *v, const double *pot,
                          double *out2, cudaStream_t st)
{
    k_energy<<<1, 1024, 0, st>>>(n, m, v, pot, out2);
    return cudaGetLastError();
}

cudaError_t launch_hermite_init(int n, double t, const double *acc, const double *jerk,
                                double dt_min, double dt_max, double *ba, double *bj,
                                double *bt, double *bdt, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    k_hermite_init<<<blocks_for(n, AUX_THREADS), AUX_THREADS, 0, st>>>(n, t, acc, jerk, dt_min,
                                                                      dt_max, ba, bj, bt, bdt);
    return cudaGetLastError();
}

cudaError_t launch_block_select(int n, const double *bt, const double *bdt, double t_end, int32_t *ilist,
                                double *t_next_out, int32_t *count_out, unsigned long long *minw,
                                int32_t *counts, cudaStream_t st, double *t_next_host, int32_t *count_host)
{
    const int nblk = blocks_for(n, SEL_PER_CTA);
    cudaError_t e = cudaMemsetAsync(minw, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess)
        return e;
    k_sel_min<<<std::min(nblk * SEL_ITEMS, 1024), SEL_THREADS, 0, st>>>(n, bt, bdt, minw);
    k_sel_count<<<nblk, SEL_THREADS, 0, st>>>(n, bt, bdt, minw, counts);
    k_sel_write<<<nblk, SEL_THREADS, 0, st>>>(n, bt, bdt, minw, counts, t_end, ilist, t_next_out, count_out,
                                              t_next_host, count_host);
    return cudaGetLastError();
}


cudaError_t launch_hermite_correct(int n_act, const int32_t *ilist, double t_next, double eta,
                                   double dt_min, double dt_max, int update_dt,
                                   const double *xp, const double *vp, const double *acc,
                                   const double *jerk, double *bx, double *bv, double *ba,
                                   double *bj, double *bt, double *bdt, cudaStream_t st)
{
    if (n_act == 0)
        return cudaSuccess;
    k_hermite_correct<<<std::min(n_act, CORR_MAX_CTAS), CORR_THREADS, 0, st>>>(
        n_act, ilist, t_next, eta, dt_min, dt_max, update_dt, xp, vp, acc, jerk, bx, bv, ba, bj, bt, bdt);
    return cudaGetLastError();
}

}  // namespace kirin

namespace kirin {

cudaError_t launch_lf_kick_drift(int n, double h, double dt, const double *a, double *v, double *x,
                                 double *hist, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    k_lf_kick_drift<<<blocks_for(3LL * n, AUX_THREADS), AUX_THREADS, 0, st>>>(n, h, dt, a, v, x, hist);
    return cudaGetLastError();
}

cudaError_t launch_axpy(int n, double alpha, const double *x, double *y, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    k_axpy<<<blocks_for(n, AUX_THREADS), AUX_THREADS, 0, st>>>(n, alpha, x, y);
    return cudaGetLastError();
}

cudaError_t launch_copy(int n, const double *src, double *dst, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    k_copy<<<blocks_for(n, AUX_THREADS), AUX_THREADS, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_pack_adjoint(int n, int n_pad, const double *m, const double *x, const double *lv, double c,
                                JMixed *jm, JF64 *jd, unsigned *err, cudaStream_t st)
{
    if (n_pad == 0)
        return cudaSuccess;
    k_pack_adjoint<<<blocks_for(n_pad, AUX_THREADS), AUX_THREADS, 0, st>>>(n, n_pad, m, x, lv, c, jm, jd, err);
    return cudaGetLastError();
}

}  // namespace kirin

namespace kirin {

// j partition: output k of the seven per-i quantities is the sum of the
// parts' partial values in part order, the same on every rank.
__global__ void k_sum_parts(int n_parts, long long n_i, const double *__restrict__ parts, double *acc,
                            double *jerk, double *pot)
{
    const long long count = 7 * n_i;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count)
        return;
    double s = 0.0;
    for (int r = 0; r < n_parts; ++r)
        s += __ldcg(parts + (size_t)r * count + k);
    if (k < 3 * n_i) {
        if (acc)
            acc[k] = s;
    } else if (k < 6 * n_i) {
        if (jerk)
            jerk[k - 3 * n_i] = s;
    } else if (pot) {
        pot[k - 6 * n_i] = s;
    }
}

cudaError_t launch_sum_parts(int n_parts, int64_t n_i, const double *parts, double *acc, double *jerk,
                             double *pot, cudaStream_t st)
{
    if (n_i <= 0)
        return cudaSuccess;
    const long long count = 7 * (long long)n_i;
    k_sum_parts<<<(unsigned)((count + AUX_THREADS - 1) / AUX_THREADS), AUX_THREADS, 0, st>>>(n_parts, n_i, parts,
                                                                                              acc, jerk, pot);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned long long limit_ns, unsigned *err, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(limit_ns, err);
    return cudaGetLastError();
}

cudaError_t launch_block_step(const StepArgs &a, int ctas, cudaStream_t st)
{
    k_step_correct<<<ctas, STEP_THREADS, 0, st>>>(a);
    k_step_select<<<ctas, STEP_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace kirin
