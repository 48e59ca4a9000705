// Batched ensembles: hundreds of independent clusters of uneven size advanced
// by the kick-drift-kick leapfrog (the shared-step integrator the paper uses
// for its treecode client, Sect. 4.3), with every force evaluation of every
// cluster done by one persistent launch.
//
//  * Work items are (cluster, block of i-particles, range of j tiles); they
//    are sorted by cost so that the largest go first, and CTAs (one or two
//    per SM) take them from an atomic counter until none are left; no CTA
//    ever waits for another.  The i-block size (512, 256 or 128: one, two or
//    four j-groups per CTA) and the longest j range (whole clusters by
//    default) are set per context; the autotuner times the choices.  When a
//    cluster's j range is split, each item leaves its sums in a partial
//    buffer and the item that completes the group adds the splits in order,
//    so results do not depend on scheduling.
//  * Each cluster's j image is padded to whole tiles with zero-mass records,
//    so a work item streams exactly its own cluster through the same
//    bulk-copy ring and the same pair arithmetic (acceleration and
//    potential, FP32 pair math on double-single positions) as the
//    single-system kernel.
//  * A leapfrog step is four device operations (kick-drift + image pack,
//    counter reset, force, kick); n_steps of them can be captured once into a
//    CUDA graph and replayed.
#include <cuda_runtime.h>

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "f32_pack.cuh"
#include "kirin_internal.cuh"
#include "pair_mixed.cuh"
#include "tma.cuh"

using namespace kirin;

namespace {

constexpr int BATCH_FLUSH_J = 256;
constexpr int BATCH_NQ = 4;  // sums per i: acceleration (3) and potential

// One unit of the work queue: j tiles [jt0, jt1) of a cluster against one
// block of its i-particles.  group >= 0 when the cluster's j range is split
// over several items: their sums meet in the partial buffer and the item
// that finishes last adds them up (in split order, so the result does not
// depend on which CTA comes last).
struct Item {
    int32_t cluster;
    int32_t iblock;
    int32_t jt0, jt1;
    int32_t group;
    int32_t split;
};

struct Group {
    int32_t nsplit;
    int32_t slot0;  // first partial slot (one per split)
};

struct BatchArgs {
    const JMixed *jimg;
    const Item *items;
    int n_items;
    const int32_t *off;   // particle offsets, n_clusters + 1
    const int32_t *poff;  // image offsets (each cluster padded to TILE_J)
    const float *eps2;    // per cluster
    double G;
    double *acc;          // n_total x 3
    double *pot;          // n_total or null
    const Group *groups;
    unsigned *gcount;     // per group: items finished (set back to 0 by the last)
    double *partial;      // [slot][BATCH_NQ][i per item]
    unsigned *counter;
    unsigned *err;
};

// Final value of sum q (0-2: acceleration, 3: potential) of particle p.
__device__ __forceinline__ void batch_store(const BatchArgs &A, size_t p, int q, double sum)
{
    if (q < 3)
        A.acc[3 * p + q] = A.G * sum;
    else if (A.pot)
        A.pot[p] = -A.G * sum;
}

// GROUPS j-groups per CTA: an item holds 2 * 256 / GROUPS i-particles (two
// per thread, as in the single-system kernel) and each tile of TILE_J j is
// shared out among the groups, whose sums meet in shared memory at the end of
// the item.
template <int GROUPS, bool GUARD>
__global__ void __launch_bounds__(FORCE_THREADS, 2) k_batch_accel(const BatchArgs A)
{
    constexpr int GT = FORCE_THREADS / GROUPS;  // threads per j-group
    constexpr int I_ITEM = 2 * GT;              // i-particles per item
    constexpr int JG = TILE_J / GROUPS;         // j per group and tile
    constexpr uint32_t TILE_BYTES = TILE_J * sizeof(JMixed);
    static_assert(GT >= 32, "a warp must read one j at a time (broadcast loads)");
    static_assert((size_t)GROUPS * BATCH_NQ * I_ITEM * sizeof(float2) <= (size_t)STAGES * TILE_J * sizeof(JMixed),
                  "cross-group reduction space");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    JMixed *tiles = reinterpret_cast<JMixed *>(smem_raw);
    __shared__ __align__(8) uint64_t bars[STAGES];
    __shared__ int item_s;
    __shared__ int last_s;

    const int tid = threadIdx.x;
    const int g = tid / GT;
    const int s = tid - g * GT;
    if (tid == 0) {
#pragma unroll
        for (int st = 0; st < STAGES; ++st)
            mbar_init(&bars[st], 1);
        mbar_fence_init();
    }
    const uint64_t pol = l2_policy_evict_last();
    int kt = 0;  // tiles consumed so far by this CTA (stage / phase bookkeeping)
    while (true) {
        if (tid == 0)
            item_s = (int)atomicAdd(A.counter, 1u);
        __syncthreads();
        const int it = item_s;
        if (it >= A.n_items)
            return;
        const Item W = A.items[it];
        const int off = A.off[W.cluster];
        const int n_c = A.off[W.cluster + 1] - off;
        const int nt = W.jt1 - W.jt0;
        const JMixed *__restrict__ J = A.jimg + A.poff[W.cluster];
        const float eps2f = A.eps2[W.cluster];

        const int k0 = W.iblock * I_ITEM + s, k1 = k0 + GT;
        const bool v0 = k0 < n_c, v1 = k1 < n_c;
        const IPair I = load_ipair(J + (v0 ? k0 : 0), J + (v1 ? k1 : 0), eps2f, 0.0f);

        if (tid == 0) {
            for (int st = 0; st < STAGES && st < nt; ++st) {
                const int slot = (kt + st) % STAGES;
                mbar_arrive_expect_tx(&bars[slot], TILE_BYTES);
                bulk_g2s_hint(tiles + slot * TILE_J, J + (size_t)(W.jt0 + st) * TILE_J, TILE_BYTES, &bars[slot],
                              pol);
            }
        }
        Tile7 t;
        t.zero();
        Lane7 acc0, acc1;
        acc0.zero();
        acc1.zero();
        int since = 0;
        int k = 0;
        bool aborted = false;
        for (; k < nt; ++k) {
            const int slot = (kt + k) % STAGES;
            const uint32_t par = (uint32_t)((kt + k) / STAGES) & 1u;
            const bool ok = mbar_wait_bounded(&bars[slot], par);
            if (ok) {
                const JMixed *__restrict__ T = tiles + slot * TILE_J + g * JG;
                const int j0 = (W.jt0 + k) * TILE_J + g * JG;  // cluster-local index of T[0]
                const bool mine = (v0 && (unsigned)(k0 - j0) < (unsigned)JG) ||
                                  (v1 && (unsigned)(k1 - j0) < (unsigned)JG);
                if (eps2f != 0.f && __any_sync(0xffffffffu, mine)) {
#pragma unroll 2
                    for (int jj = 0; jj < JG; ++jj)
                        pair<GUARD, MODE_ACC_POT, true>(T[jj], I, t, j0 + jj, v0 ? k0 : -1, v1 ? k1 : -1);
                } else {
#pragma unroll 4
                    for (int jj = 0; jj < JG; ++jj)
                        pair<GUARD, MODE_ACC_POT>(T[jj], I, t);
                }
                since += JG;
                if (since >= BATCH_FLUSH_J) {
                    fold<MODE_ACC_POT>(t, acc0, acc1);
                    since = 0;
                }
            }
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
            if (tid == 0 && k + STAGES < nt) {
                mbar_arrive_expect_tx(&bars[slot], TILE_BYTES);
                bulk_g2s_hint(tiles + slot * TILE_J, J + (size_t)(W.jt0 + k + STAGES) * TILE_J, TILE_BYTES,
                              &bars[slot], pol);
            }
        }
        if (aborted) {
            if (tid == 0) {
                const int last = min(nt, k + STAGES);
                for (int kk = k; kk < last; ++kk) {
                    if (!mbar_wait_bounded(&bars[(kt + kk) % STAGES], (uint32_t)((kt + kk) / STAGES) & 1u)) {
                        atomicOr(A.err, ERR_DRAIN);
                        break;
                    }
                }
                atomicOr(A.err, ERR_TIMEOUT);
            }
            return;
        }
        kt += nt;
        fold<MODE_ACC_POT>(t, acc0, acc1);

        // this item's sums: final values, or the partial slot of its split
        double *part = nullptr;
        Group grp{1, 0};
        if (W.group >= 0) {
            grp = A.groups[W.group];
            part = A.partial + (size_t)(grp.slot0 + W.split) * BATCH_NQ * I_ITEM;
        }
        auto emit = [&](int slot, int q, double sum) {
            const int kk = W.iblock * I_ITEM + slot;
            if (part)
                part[q * I_ITEM + slot] = sum;
            else if (kk < n_c)
                batch_store(A, (size_t)off + kk, q, sum);
        };
        if (GROUPS == 1) {
#pragma unroll
            for (int q = 0; q < BATCH_NQ; ++q) {
                const int c = q < 3 ? q : 6;
                emit(s, q, (double)acc0.h[c] + (double)acc0.l[c]);
                emit(s + GT, q, (double)acc1.h[c] + (double)acc1.l[c]);
            }
        } else {
            // every tile is consumed and no copy is in flight: the ring is free
            float2 *red = reinterpret_cast<float2 *>(smem_raw);  // [GROUPS][BATCH_NQ][I_ITEM] of (hi, lo)
#pragma unroll
            for (int q = 0; q < BATCH_NQ; ++q) {
                const int c = q < 3 ? q : 6;
                red[(g * BATCH_NQ + q) * I_ITEM + s] = make_float2(acc0.h[c], acc0.l[c]);
                red[(g * BATCH_NQ + q) * I_ITEM + s + GT] = make_float2(acc1.h[c], acc1.l[c]);
            }
            __syncthreads();
            for (int o = tid; o < BATCH_NQ * I_ITEM; o += FORCE_THREADS) {
                const int q = o / I_ITEM;
                const int slot = o - q * I_ITEM;
                float2 v = red[q * I_ITEM + slot];
                float hi = v.x, lo = v.y;
#pragma unroll
                for (int gg = 1; gg < GROUPS; ++gg) {
                    v = red[(gg * BATCH_NQ + q) * I_ITEM + slot];
                    two_sum(hi, lo, v.x);
                    lo = __fadd_rn(lo, v.y);
                }
                emit(slot, q, (double)hi + (double)lo);
            }
            // the next item's copies refill this space after the barrier below
            fence_proxy_async_smem();
        }
        if (part) {
            // publish this split's sums; the last split of the group adds them all up
            __threadfence();
            __syncthreads();
            if (tid == 0)
                last_s = atomicAdd(&A.gcount[W.group], 1u) + 1u == (unsigned)grp.nsplit;
            __syncthreads();
            if (last_s) {
                __threadfence();
                const double *base = A.partial + (size_t)grp.slot0 * BATCH_NQ * I_ITEM;
                for (int o = tid; o < BATCH_NQ * I_ITEM; o += FORCE_THREADS) {
                    const int q = o / I_ITEM;
                    const int slot = o - q * I_ITEM;
                    const int kk = W.iblock * I_ITEM + slot;
                    if (kk >= n_c)
                        continue;
                    double sum = 0.0;
                    for (int sp = 0; sp < grp.nsplit; ++sp)
                        sum += __ldcg(base + ((size_t)sp * BATCH_NQ + q) * I_ITEM + slot);
                    batch_store(A, (size_t)off + kk, q, sum);
                }
                if (tid == 0)
                    A.gcount[W.group] = 0u;
            }
        }
        // item_s, last_s and the reduction space are rewritten only after every thread passed this barrier
        __syncthreads();
    }
}

__device__ __forceinline__ void pack_record(JMixed *dst, double X, double Y, double Z, double M)
{
    float xh, xl, yh, yl, zh, zl;
    f32pack::split(X, xh, xl);
    f32pack::split(Y, yh, yl);
    f32pack::split(Z, zh, zl);
    const float m = f32pack::to_f32(M);
    JMixed r;
    r.q[0] = make_float4(xh, xh, yh, yh);
    r.q[1] = make_float4(zh, zh, m, m);
    r.q[2] = make_float4(xl, xl, yl, yl);
    r.q[3] = make_float4(zl, zl, 0.f, 0.f);
    r.q[4] = make_float4(0.f, 0.f, 0.f, 0.f);
    *dst = r;
}

// v_h = v + h a;  x' = x + dt v_h;  image of x'  (h = dt = 0: image only)
__global__ void k_kick_drift(int n, double h, double dt, const double *__restrict__ a, double *v, double *x,
                             const double *__restrict__ m, const int32_t *__restrict__ img_idx, JMixed *jm,
                             unsigned *err)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    double X[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const size_t o = 3 * (size_t)p + c;
        const double vh = v[o] + h * a[o];
        X[c] = x[o] + dt * vh;
        v[o] = vh;
        x[o] = X[c];
    }
    if (!(f32pack::finite(X[0]) && f32pack::finite(X[1]) && f32pack::finite(X[2])))
        atomicOr(err, ERR_NONFINITE);
    pack_record(jm + img_idx[p], X[0], X[1], X[2], m[p]);
}

__global__ void k_kick(int n, double h, const double *__restrict__ a, double *v)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 3 * n)
        return;
    v[p] += h * a[p];
}

// Device-to-device state upload with the finiteness check of the host path.
__global__ void k_batch_scatter(int n, const double *__restrict__ m, const double *__restrict__ x,
                                const double *__restrict__ v, double *bm, double *bx, double *bv, unsigned *err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n)
        return;
    bool fin = isfinite(m[k]);
    bm[k] = m[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double xc = x[3 * (size_t)k + c], vc = v[3 * (size_t)k + c];
        fin = fin && isfinite(xc) && isfinite(vc);
        bx[3 * (size_t)k + c] = xc;
        bv[3 * (size_t)k + c] = vc;
    }
    if (!fin)
        atomicOr(err, ERR_NONFINITE);
}

__global__ void k_fill_pad(int n_img, JMixed *jm)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_img)
        return;
    pack_record(jm + p, PAD_POS, PAD_POS, PAD_POS, 0.0);
}

}  // namespace

struct kirin_batch {
    int device = 0;
    int nsm = 0;
    int ctas = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nc = 0;
    int64_t n_total = 0, n_img = 0;
    double G = 1.0;
    bool guard = false;
    int32_t *d_off = nullptr, *d_poff = nullptr, *d_img_idx = nullptr;
    float *d_eps2 = nullptr;
    double *m = nullptr, *x = nullptr, *v = nullptr, *a = nullptr;
    JMixed *jm = nullptr;
    std::vector<int64_t> sizes;  // particles per cluster
    // work decomposition (kirin_batch_set_launch): j-groups per CTA and the
    // longest j range of an item in tiles (0: whole clusters)
    int groups = 1;
    int j_tiles = 0;
    Item *d_items = nullptr;
    int n_items = 0;
    Group *d_groups = nullptr;
    unsigned *d_gcount = nullptr;
    double *d_partial = nullptr;
    int n_groups = 0;
    unsigned *d_counter = nullptr, *d_err = nullptr, *h_err = nullptr;
    bool a_valid = false;
    bool have_state = false;
    cudaGraphExec_t gexec = nullptr;
    double g_dt = 0;
    int g_steps = 0;
};

namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != d)
            cudaSetDevice(d);
    }
    ~DevGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

void batch_free(kirin_batch *b)
{
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    void *ptrs[] = {b->d_off, b->d_poff, b->d_img_idx, b->d_eps2, b->m, b->x, b->v, b->a, b->jm,
                    b->d_items, b->d_groups, b->d_gcount, b->d_partial, b->d_counter, b->d_err};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    if (b->h_err)
        cudaFreeHost(b->h_err);
    if (b->own_stream && b->stream)
        cudaStreamDestroy(b->stream);
}

template <int GROUPS, bool GUARD>
void launch_batch(const kirin_batch *b, const BatchArgs &A)
{
    const size_t smem = (size_t)STAGES * TILE_J * sizeof(JMixed);
    k_batch_accel<GROUPS, GUARD><<<b->ctas, FORCE_THREADS, smem, b->stream>>>(A);
}

// The kernel instance of a decomposition, and its resident CTAs per SM.
template <bool GUARD>
int batch_occupancy(int groups)
{
    const size_t smem = (size_t)STAGES * TILE_J * sizeof(JMixed);
    int occ = 0;
    auto occ_of = [&](auto kern) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, FORCE_THREADS, smem);
    };
    if (groups == 4)
        occ_of(k_batch_accel<4, GUARD>);
    else if (groups == 2)
        occ_of(k_batch_accel<2, GUARD>);
    else
        occ_of(k_batch_accel<1, GUARD>);
    return occ;
}

cudaError_t enqueue_force(kirin_batch *b)
{
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), b->stream);
    if (e != cudaSuccess)
        return e;
    BatchArgs A{};
    A.jimg = b->jm;
    A.items = b->d_items;
    A.n_items = b->n_items;
    A.off = b->d_off;
    A.poff = b->d_poff;
    A.eps2 = b->d_eps2;
    A.G = b->G;
    A.acc = b->a;
    A.pot = nullptr;
    A.groups = b->d_groups;
    A.gcount = b->d_gcount;
    A.partial = b->d_partial;
    A.counter = b->d_counter;
    A.err = b->d_err;
    switch (b->groups * 2 + (b->guard ? 1 : 0)) {
    case 2: launch_batch<1, false>(b, A); break;
    case 3: launch_batch<1, true>(b, A); break;
    case 4: launch_batch<2, false>(b, A); break;
    case 5: launch_batch<2, true>(b, A); break;
    case 8: launch_batch<4, false>(b, A); break;
    case 9: launch_batch<4, true>(b, A); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Work items of a decomposition: i-blocks of 2 * 256 / groups particles
// against j ranges of at most j_tiles tiles (0: the whole cluster), the
// costliest first (longest j range, then largest cluster) so that the atomic
// queue ends on short items.
struct Plan {
    std::vector<Item> items;
    std::vector<Group> groups;
    int64_t slots = 0;
};

Plan make_plan(const std::vector<int64_t> &nc, int groups, int j_tiles)
{
    Plan P;
    const int i_item = 2 * FORCE_THREADS / groups;
    for (int c = 0; c < (int)nc.size(); ++c) {
        const int64_t nt = (nc[c] + TILE_J - 1) / TILE_J;
        const int64_t S = (j_tiles > 0 && nt > j_tiles) ? (nt + j_tiles - 1) / j_tiles : 1;
        for (int64_t ib = 0; ib * i_item < nc[c]; ++ib) {
            int32_t grp = -1;
            if (S > 1) {
                grp = (int32_t)P.groups.size();
                P.groups.push_back(Group{(int32_t)S, (int32_t)P.slots});
                P.slots += S;
            }
            for (int64_t sp = 0; sp < S; ++sp)
                P.items.push_back(Item{c, (int32_t)ib, (int32_t)(nt * sp / S), (int32_t)(nt * (sp + 1) / S), grp,
                                       (int32_t)sp});
        }
    }
    std::stable_sort(P.items.begin(), P.items.end(), [&](const Item &p, const Item &q) {
        const int lp = p.jt1 - p.jt0, lq = q.jt1 - q.jt0;
        if (lp != lq)
            return lp > lq;
        return nc[p.cluster] > nc[q.cluster];
    });
    return P;
}

// Partial sums of split clusters are capped at this many bytes.
constexpr size_t BATCH_PARTIAL_MAX = (size_t)1 << 30;

// Build and upload the work items of (groups, j_tiles); on failure the
// context keeps its previous decomposition.
int install_plan(kirin_batch *b, int groups, int j_tiles)
{
    const Plan P = make_plan(b->sizes, groups, j_tiles);
    const int i_item = 2 * FORCE_THREADS / groups;
    const size_t partial_bytes = (size_t)P.slots * BATCH_NQ * i_item * sizeof(double);
    if (P.items.size() > (size_t)INT32_MAX || partial_bytes > BATCH_PARTIAL_MAX)
        return KIRIN_EINVAL;
    Item *items = nullptr;
    Group *grps = nullptr;
    unsigned *gcount = nullptr;
    double *partial = nullptr;
    bool ok = cudaMalloc((void **)&items, std::max<size_t>(P.items.size() * sizeof(Item), 16)) == cudaSuccess &&
              cudaMalloc((void **)&grps, std::max<size_t>(P.groups.size() * sizeof(Group), 16)) == cudaSuccess &&
              cudaMalloc((void **)&gcount, std::max<size_t>(P.groups.size() * sizeof(unsigned), 16)) == cudaSuccess &&
              cudaMalloc((void **)&partial, std::max<size_t>(partial_bytes, 16)) == cudaSuccess;
    if (ok && !P.items.empty())
        ok = cudaMemcpy(items, P.items.data(), P.items.size() * sizeof(Item), cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && !P.groups.empty())
        ok = cudaMemcpy(grps, P.groups.data(), P.groups.size() * sizeof(Group), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemset(gcount, 0, std::max<size_t>(P.groups.size() * sizeof(unsigned), 16)) == cudaSuccess;
    const int occ = b->guard ? batch_occupancy<true>(groups) : batch_occupancy<false>(groups);
    if (!ok || occ < 1) {
        cudaFree(items);
        cudaFree(grps);
        cudaFree(gcount);
        cudaFree(partial);
        cudaGetLastError();
        return ok ? KIRIN_ECUDA : KIRIN_ENOMEM;
    }
    cudaFree(b->d_items);
    cudaFree(b->d_groups);
    cudaFree(b->d_gcount);
    cudaFree(b->d_partial);
    b->d_items = items;
    b->d_groups = grps;
    b->d_gcount = gcount;
    b->d_partial = partial;
    b->n_items = (int)P.items.size();
    b->n_groups = (int)P.groups.size();
    b->groups = groups;
    b->j_tiles = j_tiles;
    b->ctas = occ * b->nsm;
    if (b->gexec) {  // the captured launches carry the old items
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return KIRIN_OK;
}

cudaError_t enqueue_pack(kirin_batch *b)
{
    const int n = (int)b->n_total;
    k_kick_drift<<<(n + 255) / 256, 256, 0, b->stream>>>(n, 0.0, 0.0, b->a, b->v, b->x, b->m, b->d_img_idx,
                                                         b->jm, b->d_err);
    return cudaGetLastError();
}

cudaError_t enqueue_steps(kirin_batch *b, double dt, int n_steps)
{
    const int n = (int)b->n_total;
    const double h = 0.5 * dt;
    for (int s = 0; s < n_steps; ++s) {
        k_kick_drift<<<(n + 255) / 256, 256, 0, b->stream>>>(n, h, dt, b->a, b->v, b->x, b->m, b->d_img_idx,
                                                             b->jm, b->d_err);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
        e = enqueue_force(b);
        if (e != cudaSuccess)
            return e;
        k_kick<<<(3 * n + 255) / 256, 256, 0, b->stream>>>(n, h, b->a, b->v);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

int batch_errors(kirin_batch *b)
{
    if (cudaMemcpyAsync(b->h_err, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        return KIRIN_ECUDA;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess)
        return KIRIN_ECUDA;
    const unsigned e = *b->h_err;
    if (!e)
        return KIRIN_OK;
    cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), b->stream);
    if (b->n_groups)  // an aborted item never counted itself in
        cudaMemsetAsync(b->d_gcount, 0, b->n_groups * sizeof(unsigned), b->stream);
    if (e & (ERR_TIMEOUT | ERR_DRAIN))
        return KIRIN_ETIMEOUT;
    if (e & ERR_NONFINITE)
        return KIRIN_ENONFINITE;
    return KIRIN_ECUDA;
}

}  // namespace

extern "C" {

int kirin_batch_create(kirin_batch **out, int32_t n_clusters, const int64_t *offsets, const double *eps,
                       double G, int32_t device, void *stream)
{
    if (!out || !offsets || !eps || n_clusters < 1 || !isfinite(G))
        return KIRIN_EINVAL;
    *out = nullptr;
    if (offsets[0] != 0)
        return KIRIN_EINVAL;
    for (int c = 0; c < n_clusters; ++c) {
        if (offsets[c + 1] < offsets[c] || !(eps[c] >= 0.0) || !isfinite(eps[c]))
            return KIRIN_EINVAL;
    }
    const int64_t n_total = offsets[n_clusters];
    if (n_total < 1 || n_total > (int64_t)INT32_MAX / 2)
        return KIRIN_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return KIRIN_ECUDA;
    }
    DevGuard dg(device);
    kirin_batch *b = new (std::nothrow) kirin_batch();
    if (!b)
        return KIRIN_ENOMEM;
    b->device = device;
    b->nc = n_clusters;
    b->n_total = n_total;
    b->G = G;
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, device);

    std::vector<int32_t> off(n_clusters + 1), poff(n_clusters + 1), img_idx((size_t)n_total);
    std::vector<float> eps2(n_clusters);
    b->sizes.resize(n_clusters);
    poff[0] = 0;
    for (int c = 0; c < n_clusters; ++c) {
        off[c] = (int32_t)offsets[c];
        const int64_t nc = offsets[c + 1] - offsets[c];
        poff[c + 1] = poff[c] + (int32_t)((nc + TILE_J - 1) / TILE_J * TILE_J);
        eps2[c] = (float)(eps[c] * eps[c]);
        if (eps[c] == 0.0)
            b->guard = true;
        for (int64_t k = 0; k < nc; ++k)
            img_idx[(size_t)(offsets[c] + k)] = poff[c] + (int32_t)k;
        b->sizes[c] = nc;
    }
    off[n_clusters] = (int32_t)n_total;
    b->n_img = std::max<int32_t>(poff[n_clusters], TILE_J);

    bool ok = true;
    auto dalloc = [&](void **p, size_t bytes) {
        if (ok && cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess)
            ok = false;
    };
    const size_t n = (size_t)n_total;
    dalloc((void **)&b->d_off, (n_clusters + 1) * sizeof(int32_t));
    dalloc((void **)&b->d_poff, (n_clusters + 1) * sizeof(int32_t));
    dalloc((void **)&b->d_img_idx, n * sizeof(int32_t));
    dalloc((void **)&b->d_eps2, n_clusters * sizeof(float));
    dalloc((void **)&b->m, n * sizeof(double));
    dalloc((void **)&b->x, 3 * n * sizeof(double));
    dalloc((void **)&b->v, 3 * n * sizeof(double));
    dalloc((void **)&b->a, 3 * n * sizeof(double));
    dalloc((void **)&b->jm, (size_t)b->n_img * sizeof(JMixed));
    dalloc((void **)&b->d_counter, sizeof(unsigned));
    dalloc((void **)&b->d_err, sizeof(unsigned));
    if (ok && cudaMallocHost((void **)&b->h_err, sizeof(unsigned)) != cudaSuccess)
        ok = false;
    if (ok) {
        if (stream) {
            b->stream = (cudaStream_t)stream;
        } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
            b->own_stream = true;
        } else {
            ok = false;
        }
    }
    if (ok) {
        ok = cudaMemcpy(b->d_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(b->d_poff, poff.data(), poff.size() * sizeof(int32_t), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(b->d_img_idx, img_idx.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(b->d_eps2, eps2.data(), eps2.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(b->d_err, 0, sizeof(unsigned)) == cudaSuccess;
    }
    if (ok) {
        k_fill_pad<<<(int)((b->n_img + 255) / 256), 256, 0, b->stream>>>((int)b->n_img, b->jm);
        ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(b->stream) == cudaSuccess;
    }
    if (ok)  // default decomposition: blocks of 512 i against whole clusters
        ok = install_plan(b, 1, 0) == KIRIN_OK;
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        delete b;
        return KIRIN_ENOMEM;
    }
    *out = b;
    return KIRIN_OK;
}

int kirin_batch_destroy(kirin_batch *b)
{
    if (!b)
        return KIRIN_OK;
    DevGuard dg(b->device);
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
    return KIRIN_OK;
}

int kirin_batch_set_state(kirin_batch *b, const double *m, const double *x, const double *v)
{
    if (!b || !m || !x || !v)
        return KIRIN_EINVAL;
    const size_t n = (size_t)b->n_total;
    for (size_t k = 0; k < n; ++k)
        if (!isfinite(m[k]))
            return KIRIN_ENONFINITE;
    for (size_t k = 0; k < 3 * n; ++k)
        if (!isfinite(x[k]) || !isfinite(v[k]))
            return KIRIN_ENONFINITE;
    DevGuard dg(b->device);
    if (cudaMemcpyAsync(b->m, m, n * sizeof(double), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->x, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->v, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return KIRIN_ECUDA;
    b->a_valid = false;
    b->have_state = true;
    return KIRIN_OK;
}

int kirin_batch_get_state(kirin_batch *b, double *x, double *v)
{
    if (!b)
        return KIRIN_EINVAL;
    DevGuard dg(b->device);
    const size_t n = (size_t)b->n_total;
    if (x && cudaMemcpyAsync(x, b->x, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        return KIRIN_ECUDA;
    if (v && cudaMemcpyAsync(v, b->v, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        return KIRIN_ECUDA;
    return batch_errors(b);
}

int kirin_batch_accel(kirin_batch *b, double *acc)
{
    if (!b || !acc)
        return KIRIN_EINVAL;
    if (!b->have_state)
        return KIRIN_ESTATE;
    DevGuard dg(b->device);
    if (enqueue_pack(b) != cudaSuccess || enqueue_force(b) != cudaSuccess)
        return KIRIN_ECUDA;
    b->a_valid = true;
    if (cudaMemcpyAsync(acc, b->a, 3 * (size_t)b->n_total * sizeof(double), cudaMemcpyDeviceToHost, b->stream) !=
        cudaSuccess)
        return KIRIN_ECUDA;
    return batch_errors(b);
}

int kirin_batch_set_state_dev(kirin_batch *b, const double *m, const double *x, const double *v)
{
    if (!b || !m || !x || !v)
        return KIRIN_EINVAL;
    DevGuard dg(b->device);
    const int n = (int)b->n_total;
    k_batch_scatter<<<(n + 255) / 256, 256, 0, b->stream>>>(n, m, x, v, b->m, b->x, b->v, b->d_err);
    if (cudaGetLastError() != cudaSuccess)
        return KIRIN_ECUDA;
    b->a_valid = false;
    b->have_state = true;
    return KIRIN_OK;
}

int kirin_batch_get_state_dev(kirin_batch *b, double *x, double *v)
{
    if (!b)
        return KIRIN_EINVAL;
    DevGuard dg(b->device);
    const size_t bytes = 3 * (size_t)b->n_total * sizeof(double);
    if (x && cudaMemcpyAsync(x, b->x, bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
        return KIRIN_ECUDA;
    if (v && cudaMemcpyAsync(v, b->v, bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
        return KIRIN_ECUDA;
    return KIRIN_OK;
}

int kirin_batch_accel_dev(kirin_batch *b, double *acc)
{
    if (!b || !acc)
        return KIRIN_EINVAL;
    if (!b->have_state)
        return KIRIN_ESTATE;
    DevGuard dg(b->device);
    if (enqueue_pack(b) != cudaSuccess || enqueue_force(b) != cudaSuccess)
        return KIRIN_ECUDA;
    b->a_valid = true;
    if (cudaMemcpyAsync(acc, b->a, 3 * (size_t)b->n_total * sizeof(double), cudaMemcpyDeviceToDevice,
                        b->stream) != cudaSuccess)
        return KIRIN_ECUDA;
    return KIRIN_OK;
}

int kirin_batch_leapfrog(kirin_batch *b, double dt, int32_t n_steps, int32_t use_graph)
{
    if (!b || !isfinite(dt) || n_steps < 0)
        return KIRIN_EINVAL;
    if (!b->have_state)
        return KIRIN_ESTATE;
    if (n_steps == 0)
        return KIRIN_OK;
    DevGuard dg(b->device);
    if (!b->a_valid) {
        if (enqueue_pack(b) != cudaSuccess || enqueue_force(b) != cudaSuccess)
            return KIRIN_ECUDA;
        b->a_valid = true;
    }
    if (!use_graph)
        return enqueue_steps(b, dt, n_steps) == cudaSuccess ? KIRIN_OK : KIRIN_ECUDA;
    if (!b->gexec || b->g_dt != dt || b->g_steps != n_steps) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return KIRIN_ECUDA;
        const cudaError_t e = enqueue_steps(b, dt, n_steps);
        const cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph)
                cudaGraphDestroy(graph);
            cudaGetLastError();
            return KIRIN_ECUDA;
        }
        const cudaError_t e3 = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) {
            b->gexec = nullptr;
            return KIRIN_ECUDA;
        }
        b->g_dt = dt;
        b->g_steps = n_steps;
    }
    return cudaGraphLaunch(b->gexec, b->stream) == cudaSuccess ? KIRIN_OK : KIRIN_ECUDA;
}

int kirin_batch_sync(kirin_batch *b)
{
    if (!b)
        return KIRIN_EINVAL;
    DevGuard dg(b->device);
    return batch_errors(b);
}

int kirin_batch_set_launch(kirin_batch *b, int32_t groups, int32_t j_tiles)
{
    if (!b || (groups != 1 && groups != 2 && groups != 4) || j_tiles < 0)
        return KIRIN_EINVAL;
    DevGuard dg(b->device);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess)
        return KIRIN_ECUDA;
    return install_plan(b, groups, j_tiles);
}

int kirin_batch_get_launch(const kirin_batch *b, int32_t *groups, int32_t *j_tiles, int32_t *n_items)
{
    if (!b)
        return KIRIN_EINVAL;
    if (groups)
        *groups = b->groups;
    if (j_tiles)
        *j_tiles = b->j_tiles;
    if (n_items)
        *n_items = b->n_items;
    return KIRIN_OK;
}

}  // extern "C"
