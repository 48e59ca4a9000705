// Batched ensembles: hundreds of independent clusters of uneven size advanced
// by the kick-drift-kick leapfrog (the shared-step integrator the paper uses
// for its treecode client, Sect. 4.3), with every force evaluation of every
// cluster done by one persistent launch.
//
//  * Work items are (cluster, block of 512 i-particles); they are sorted by
//    cost (cluster size) so that the largest go first, and CTAs (one or two
//    per SM) take them from an atomic counter until none are left; no CTA
//    ever waits for another.
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

#include "kirin_internal.cuh"
#include "pair_mixed.cuh"
#include "tma.cuh"

using namespace kirin;

namespace {

constexpr int BATCH_I = 2 * FORCE_THREADS;  // i-particles per work item
constexpr int BATCH_FLUSH_J = 256;

struct Item {
    int32_t cluster;
    int32_t iblock;
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
    unsigned *counter;
    unsigned *err;
};

template <bool GUARD>
__global__ void __launch_bounds__(FORCE_THREADS, 2) k_batch_accel(const BatchArgs A)
{
    constexpr uint32_t TILE_BYTES = TILE_J * sizeof(JMixed);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    JMixed *tiles = reinterpret_cast<JMixed *>(smem_raw);
    __shared__ __align__(8) uint64_t bars[STAGES];
    __shared__ int item_s;

    const int tid = threadIdx.x;
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
        const int c = A.items[it].cluster;
        const int b = A.items[it].iblock;
        const int off = A.off[c];
        const int n_c = A.off[c + 1] - off;
        const int poff = A.poff[c];
        const int nt = (n_c + TILE_J - 1) / TILE_J;
        const JMixed *__restrict__ J = A.jimg + poff;
        const float eps2f = A.eps2[c];

        const int k0 = b * BATCH_I + tid, k1 = k0 + FORCE_THREADS;
        const bool v0 = k0 < n_c, v1 = k1 < n_c;
        const IPair I = load_ipair(J + (v0 ? k0 : 0), J + (v1 ? k1 : 0), eps2f, 0.0f);

        if (tid == 0) {
            for (int st = 0; st < STAGES && st < nt; ++st) {
                const int slot = (kt + st) % STAGES;
                mbar_arrive_expect_tx(&bars[slot], TILE_BYTES);
                bulk_g2s_hint(tiles + slot * TILE_J, J + (size_t)st * TILE_J, TILE_BYTES, &bars[slot], pol);
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
                const JMixed *__restrict__ T = tiles + slot * TILE_J;
                const int j0 = k * TILE_J;  // cluster-local index of T[0]
                const bool mine = (v0 && (unsigned)(k0 - j0) < (unsigned)TILE_J) ||
                                  (v1 && (unsigned)(k1 - j0) < (unsigned)TILE_J);
                if (eps2f != 0.f && __any_sync(0xffffffffu, mine)) {
#pragma unroll 2
                    for (int jj = 0; jj < TILE_J; ++jj)
                        pair<GUARD, MODE_ACC_POT, true>(T[jj], I, t, j0 + jj, v0 ? k0 : -1, v1 ? k1 : -1);
                } else {
#pragma unroll 4
                    for (int jj = 0; jj < TILE_J; ++jj)
                        pair<GUARD, MODE_ACC_POT>(T[jj], I, t);
                }
                since += TILE_J;
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
                bulk_g2s_hint(tiles + slot * TILE_J, J + (size_t)(k + STAGES) * TILE_J, TILE_BYTES, &bars[slot], pol);
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
        if (v0) {
            const size_t p = (size_t)off + k0;
#pragma unroll
            for (int q = 0; q < 3; ++q)
                A.acc[3 * p + q] = A.G * ((double)acc0.h[q] + (double)acc0.l[q]);
            if (A.pot)
                A.pot[p] = -A.G * ((double)acc0.h[6] + (double)acc0.l[6]);
        }
        if (v1) {
            const size_t p = (size_t)off + k1;
#pragma unroll
            for (int q = 0; q < 3; ++q)
                A.acc[3 * p + q] = A.G * ((double)acc1.h[q] + (double)acc1.l[q]);
            if (A.pot)
                A.pot[p] = -A.G * ((double)acc1.h[6] + (double)acc1.l[6]);
        }
        // item_s is rewritten only after every thread passed this barrier
        __syncthreads();
    }
}

__device__ __forceinline__ void pack_record(JMixed *dst, double X, double Y, double Z, double M)
{
    const float xh = __double2float_rn(X), yh = __double2float_rn(Y), zh = __double2float_rn(Z);
    const float xl = __double2float_rn(X - (double)xh), yl = __double2float_rn(Y - (double)yh),
                zl = __double2float_rn(Z - (double)zh);
    const float m = __double2float_rn(M);
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
    if (!(isfinite(X[0]) && isfinite(X[1]) && isfinite(X[2])))
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
    Item *d_items = nullptr;
    int n_items = 0;
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
                    b->d_items, b->d_counter, b->d_err};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    if (b->h_err)
        cudaFreeHost(b->h_err);
    if (b->own_stream && b->stream)
        cudaStreamDestroy(b->stream);
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
    A.counter = b->d_counter;
    A.err = b->d_err;
    const size_t smem = (size_t)STAGES * TILE_J * sizeof(JMixed);
    if (b->guard)
        k_batch_accel<true><<<b->ctas, FORCE_THREADS, smem, b->stream>>>(A);
    else
        k_batch_accel<false><<<b->ctas, FORCE_THREADS, smem, b->stream>>>(A);
    return cudaGetLastError();
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
    std::vector<Item> items;
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
        for (int64_t ib = 0; ib * BATCH_I < nc; ++ib)
            items.push_back(Item{c, (int32_t)ib});
    }
    off[n_clusters] = (int32_t)n_total;
    b->n_img = std::max<int32_t>(poff[n_clusters], TILE_J);
    // largest clusters first: their items cost the most (n_c pairs per i)
    std::stable_sort(items.begin(), items.end(), [&](const Item &p, const Item &q) {
        return offsets[p.cluster + 1] - offsets[p.cluster] > offsets[q.cluster + 1] - offsets[q.cluster];
    });
    b->n_items = (int)items.size();

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
    dalloc((void **)&b->d_items, items.size() * sizeof(Item));
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
             cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(b->d_err, 0, sizeof(unsigned)) == cudaSuccess;
    }
    if (ok) {
        k_fill_pad<<<(int)((b->n_img + 255) / 256), 256, 0, b->stream>>>((int)b->n_img, b->jm);
        ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(b->stream) == cudaSuccess;
    }
    if (ok) {
        int occ = 0;
        const size_t smem = (size_t)STAGES * TILE_J * sizeof(JMixed);
        if (smem > 48 * 1024) {
            cudaFuncSetAttribute(k_batch_accel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(k_batch_accel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        }
        if (b->guard)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_accel<true>, FORCE_THREADS, smem);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_accel<false>, FORCE_THREADS, smem);
        b->ctas = std::max(1, occ) * b->nsm;
    }
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

}  // extern "C"
