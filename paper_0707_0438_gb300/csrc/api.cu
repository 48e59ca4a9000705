// libkirin host runtime: the C ABI of include/kirin.h.
//
// A context owns, for up to n_max particles, the FP64 base state (m, x, v, a,
// jerk, t_i, dt_i), the predicted positions and velocities, the two j images
// (mixed and FP64) that the force kernels stream, the i-list, result and
// split-partial buffers, and one CUDA stream.  Host <-> device traffic per
// call is only what the caller passes in or asks for; the j-particles stay
// resident between calls (the paper re-sends every particle each block step,
// Sect. 3.1).
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "kirin_internal.cuh"
#include "loop_internal.cuh"

using namespace kirin;

// Everything the instantiated graph bakes in: sizes, parameters, shapes and
// the addresses of buffers that can be re-allocated.  Compared byte for byte
// (the struct is zero-filled first, padding included).
struct RunKey {
    double par[6];
    int64_t n_j, prec;
    const void *partial;
    int32_t n_classes;
    int32_t class_max[MAX_SEL_CLASSES];
    Shape shape[MAX_SEL_CLASSES];
};

struct kirin_ctx {
    int device = 0;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t n_max = 0;
    int64_t n_img = 0;   // image capacity (multiple of TILE_J)
    int64_t n_hi = 0;    // highest particle index ever set + 1
    int64_t n_j = 0;     // j-particles in use
    double eps = 0, G = 1, r_min = 0;
    int prec = KIRIN_MIXED;

    // FP64 base state
    double *bm = nullptr, *bx = nullptr, *bv = nullptr, *ba = nullptr, *bj = nullptr;
    double *bt = nullptr, *bdt = nullptr;
    // current (possibly predicted) positions / velocities and the images
    double *xp = nullptr, *vp = nullptr;
    JMixed *jm = nullptr;
    JF64 *jd = nullptr;
    bool images_dirty = true;
    int pred_mode = 0;  // 0: base x, v; 1: predicted to pred_t
    double pred_t = 0;

    int32_t *d_ilist = nullptr;
    int32_t *h_ilist = nullptr;  // pinned staging
    double *d_acc = nullptr, *d_jerk = nullptr, *d_pot = nullptr;
    double *d_partial = nullptr;
    size_t partial_cap = 0;  // doubles
    unsigned *d_err = nullptr;
    double *d_scal = nullptr;  // [0] t_next, [1..2] energies, [3] block-selection minimum (bits)
    int32_t *d_count = nullptr;  // [0] block size
    int32_t *d_sel_counts = nullptr;  // per-CTA counts of the block selection
    double *h_scal = nullptr;  // pinned mirrors
    int32_t *h_count = nullptr;
    unsigned *h_err = nullptr;
    // a host word the kernels report their errors to directly (mapped pinned memory: read after the
    // stream synchronises, no copy), or null where mapping is unavailable (then d_err)
    unsigned *h_err_map = nullptr, *d_err_map = nullptr;
    // mapped host copies of a host-driven block step's time and size (same condition), or null
    double *h_sel_t = nullptr, *d_sel_t = nullptr;
    int32_t *h_sel_n = nullptr, *d_sel_n = nullptr;

    bool pending = false;
    int64_t pending_n = 0;

    // Hermite integrator
    bool hermite_ready = false;
    double eta = 0.01, dt_min = 1.0 / (1 << 20), dt_max = 0.125, t_shared = 0;

    // Device-driven block steps: one graph whose WHILE node repeats select ->
    // predict -> force (a SWITCH over block-size classes) -> correct, so a
    // run to t_end is one graph launch and one read-back.
    bool device_loop = true;
    cudaGraphExec_t run_exec = nullptr;
    RunKey run_key = {};          // what the graph was built for
    RunState *d_run = nullptr;      // run parameters, counters and barrier words (device)
    RunState *h_run = nullptr;      // pinned mirror
    int32_t *d_step_counts = nullptr;  // per-CTA list offsets and counts of the step kernels
    int step_ctas = 0;

    // launch-shape override (0 = automatic), tuned table and occupancy cache
    int fix_groups = 0, fix_split = 0;
    static constexpr int MAX_TABLE = 64;
    static constexpr int N_KINDS = 3;   // kirin_call_kind: acc+jerk+pot, acc+pot, adjoint
    int table_n[N_KINDS] = {};
    int64_t table_ni[N_KINDS][MAX_TABLE] = {};   // entry k covers n_i <= table_ni[k] (ascending)
    int32_t table_groups[N_KINDS][MAX_TABLE] = {};
    int32_t table_split[N_KINDS][MAX_TABLE] = {};
    int table_prec[N_KINDS] = {-1, -1, -1};      // each table applies to the precision it was set for
    int occ[2][N_MODES][2][4] = {};  // [prec][mode][guard][log2 groups]

    // j partition over several contexts (usually one per GPU): this context sums
    // tiles [part T / n_parts, (part + 1) T / n_parts) of the T j tiles, and the
    // exchange callback gathers every part's 7 n_i partial sums, which
    // k_sum_parts adds in part order
    int part = 0, n_parts = 1;
    kirin_allgather_fn allgather = nullptr;
    void *allgather_user = nullptr;
    double *d_send = nullptr, *d_recv = nullptr;
    size_t send_cap = 0, recv_cap = 0;  // doubles

    // shared-step runs of small systems in one cooperative launch (shared_steps.cu)
    bool shared_persistent = true;
    int sh_grid = 0;  // CTAs of that launch for sh_fit_n particles; 0: it does not fit
    int64_t sh_fit_n = -1;
    int sh_fit_guard = -1;
    JMixed *sh_img = nullptr;  // [2][sh_img_pad]: the even and odd steps' j images
    int64_t sh_img_pad = 0;
    unsigned *sh_arrivals = nullptr;  // the launch's arrival counter
    uint32_t sh_count = 0;            // its value between launches

    // nearest-neighbour search of the host-pointer path (GRAPE's neighbour list)
    bool want_nn = false;
    bool nn_valid = false;
    int32_t *d_nn = nullptr;
    double *d_nn_r2 = nullptr;

    // tracing (kirin_set_tracing): event pairs around the stream work of traced calls, folded into
    // the totals when read or when many are pending
    bool tracing = false;
    int trace_depth = 0;  // nested traced calls record once, at the outermost
    int64_t trace_calls = 0;
    double trace_ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> trace_pending, trace_free;

    char msg[256] = {0};
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

int set_msg(kirin_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(ctx, call)                                                                           \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return set_msg(ctx, KIRIN_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));          \
    } while (0)

int64_t round_up(int64_t n, int64_t m) { return (n + m - 1) / m * m; }

// Tiles [*tile0, *tile0 + return) of a j partition's part among the
// ceil(n_j / TILE_J) tiles of the padded image (every tile when n_parts = 1).
int part_tiles(int64_t n_j, int part, int n_parts, int *tile0)
{
    const int64_t total = (std::max<int64_t>(n_j, 1) + TILE_J - 1) / TILE_J;
    const int64_t b = total * part / n_parts, e = total * (part + 1) / n_parts;
    if (tile0)
        *tile0 = (int)b;
    return (int)(e - b);
}

int ilog2(int g) { return g == 1 ? 0 : g == 2 ? 1 : g == 4 ? 2 : 3; }

bool guard_on(const kirin_ctx *c) { return c->eps == 0.0 || c->r_min > 0.0; }

// The launch-table kind of a force mode (kirin_call_kind), -1 for none.
int call_kind(int mode)
{
    switch (mode) {
    case MODE_ACC_JERK_POT: return KIRIN_CALL_FORCES;
    case MODE_ACC_POT: return KIRIN_CALL_ACC_POT;
    case MODE_ADJOINT: return KIRIN_CALL_ADJOINT;
    default: return -1;
    }
}

int mode_of_kind(int kind)
{
    return kind == KIRIN_CALL_ACC_POT ? MODE_ACC_POT : kind == KIRIN_CALL_ADJOINT ? MODE_ADJOINT : MODE_ACC_JERK_POT;
}

// The j image the context's precision reads; packs write only that one.
JMixed *img_m(const kirin_ctx *c) { return c->prec == KIRIN_MIXED ? c->jm : nullptr; }
JF64 *img_d(const kirin_ctx *c) { return c->prec == KIRIN_MIXED ? nullptr : c->jd; }

int ctas_per_sm(kirin_ctx *c, int prec, int mode, bool guard, int groups)
{
    int &slot = c->occ[prec == KIRIN_MIXED][mode][guard][ilog2(groups)];
    if (slot == 0) {
        slot = prec == KIRIN_MIXED ? force_mixed_ctas_per_sm(groups, guard, mode)
                                   : force_fp64_ctas_per_sm(groups, mode);
        if (slot <= 0)
            slot = 1;
    }
    return slot;
}

// Launch shape for n_i i-particles against ntiles j tiles: minimise a simple
// cost model, (waves of CTAs) x (pair slots per CTA) + per-CTA overhead +
// split-partial traffic, over j-groups {1,2,4,8} and n_split.
Shape choose_shape(kirin_ctx *c, int64_t n_i, int ntiles, int prec, int mode, bool guard)
{
    if (c->fix_groups > 0 && c->fix_split > 0) {
        Shape s{c->fix_groups, std::min(c->fix_split, std::max(1, ntiles))};
        return s;
    }
    if (prec == KIRIN_MIXED && mode == MODE_ACC_JERK_POT && n_i <= TINY_MAX &&
        (int64_t)ntiles * TILE_J <= (int64_t)TINY_JCHUNK * 2 * c->nsm) {
        // tiny block: j ranges of 64..TINY_JCHUNK records, about two CTAs per SM
        const int ctas = std::max(1, std::min(2 * c->nsm, ntiles * TILE_J / 64));
        return Shape{0, ctas};
    }
    const int kind = call_kind(mode);
    if (kind >= 0 && c->table_n[kind] > 0 && prec == c->table_prec[kind]) {
        for (int k = 0; k < c->table_n[kind]; ++k)
            if (n_i <= c->table_ni[kind][k])
                return Shape{c->table_groups[kind][k], std::min<int>(c->table_split[kind][k], std::max(1, ntiles))};
    }
    const int per_thread = prec == KIRIN_MIXED ? MIX_I_PER_THREAD : 1;
    // a split's partial write and reduction launch in pair slots of this precision: an FP64 pair
    // takes about 64 times a mixed one (1.6e10 against 1e12 pairs/s), so the same time is worth
    // 64 times fewer FP64 slots
    const double split_scale = prec == KIRIN_MIXED ? 1.0 : 1.0 / 64.0;
    Shape best{1, 1};
    double best_cost = 1e300;
    const size_t cap_entries = (size_t)1 << 27;  // bound on n_split * 7 * n_i_pad doubles (1 GiB)
    for (int groups = 1; groups <= 8; groups *= 2) {
        const int i_cta = per_thread * FORCE_THREADS / groups;
        const int64_t iblocks = (n_i + i_cta - 1) / i_cta;
        const double slots = (double)c->nsm * ctas_per_sm(c, prec, mode, guard, groups);
        const int max_split = std::min(ntiles, MAX_SPLIT);
        for (int ns = 1; ns <= max_split; ns = ns < 64 ? ns + 1 : ns * 5 / 4) {
            if (ns > 1 && (size_t)ns * 9 * iblocks * i_cta > cap_entries)
                break;
            const double ctas = (double)iblocks * ns;
            const double waves = ceil(ctas / slots);
            const double tiles_per = ceil((double)ntiles / ns);
            // one CTA: tiles_per tiles of TILE_J x i_cta pair slots, plus ~2 tiles of set-up
            const double cta_cost = (tiles_per + 2.0) * TILE_J * (double)i_cta;
            double cost = waves * cta_cost;
            if (ns > 1)  // partial write + reduction, in pair-slot units
                cost += split_scale * ((double)ns * 7 * iblocks * i_cta * 4.0 / slots + 5.0e3 * TILE_J);
            if (cost < best_cost * 0.999) {
                best_cost = cost;
                best = Shape{groups, ns};
            }
        }
    }
    return best;
}

int ensure_partial(kirin_ctx *c, size_t doubles)
{
    if (doubles <= c->partial_cap)
        return KIRIN_OK;
    if (c->d_partial) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->d_partial);
        c->d_partial = nullptr;
        c->partial_cap = 0;
    }
    if (cudaMalloc(&c->d_partial, doubles * sizeof(double)) != cudaSuccess)
        return set_msg(c, KIRIN_ENOMEM, "split-partial buffer of %zu doubles", doubles);
    c->partial_cap = doubles;
    return KIRIN_OK;
}

// The word the context's kernels report errors to: the mapped host word where there is one (read
// after a synchronisation without a copy), else a device word copied back.
unsigned *err_word(const kirin_ctx *c) { return c->d_err_map ? c->d_err_map : c->d_err; }

int ensure_images(kirin_ctx *c)
{
    if (!c->images_dirty)
        return KIRIN_OK;
    const int64_t n_pad = round_up(std::max<int64_t>(c->n_j, 1), TILE_J);
    CK(c, launch_predict_pack((int)c->n_j, (int)n_pad, c->pred_t, c->pred_mode, c->bm, c->bx, c->bv,
                              c->ba, c->bj, c->bt, c->xp, c->vp, img_m(c), img_d(c), err_word(c), c->stream));
    c->images_dirty = false;
    return KIRIN_OK;
}

// Enqueue one force launch (plus split reduction) over the current images,
// with a given shape, on stream st.  n_i bounds the grid; with n_i_dev set the
// kernels read the actual count from there (device-driven loops).  The split
// partial buffer must already hold the launch.
int enqueue_force(kirin_ctx *c, cudaStream_t st, Shape s, int64_t n_i, const int32_t *n_i_dev,
                  const int32_t *d_ilist, int n_j, int mode, double *acc, double *jerk, double *pot,
                  int accumulate = 0, int32_t *nn = nullptr, double *nn_r2 = nullptr)
{
    if (n_i == 0)
        return KIRIN_OK;
    int tile0 = 0;
    const int ntiles = part_tiles(n_j, c->part, c->n_parts, &tile0);
    ForceArgs a{};
    a.jimg = c->prec == KIRIN_MIXED ? (const void *)c->jm : (const void *)c->jd;
    a.ilist = d_ilist;
    a.n_i = (int)n_i;
    a.n_i_dev = n_i_dev;
    a.n_j = n_j;
    a.ntiles = ntiles;
    a.tile0 = tile0;
    a.n_split = s.n_split;
    a.eps2 = c->eps * c->eps;
    a.rmin2 = c->r_min * c->r_min;
    a.G = c->G;
    a.acc = acc;
    a.jerk = jerk;
    a.pot = pot;
    a.accumulate = accumulate;
    a.err = err_word(c);
    a.nn = nn;
    a.nn_r2 = nn_r2;
    a.nq = mode == MODE_NN ? 9 : 7;
    a.n_i_pad = (int)round_up(n_i, shape_i_cta(s, c->prec == KIRIN_MIXED));
    if (s.n_split > 1) {
        if ((size_t)s.n_split * a.nq * a.n_i_pad > c->partial_cap)
            return set_msg(c, KIRIN_ESTATE, "split-partial buffer too small for the launch");
        a.partial = c->d_partial;
    }
    if (c->prec == KIRIN_MIXED)
        CK(c, launch_force_mixed(a, s, guard_on(c), mode, st));
    else
        CK(c, launch_force_fp64(a, s, mode, st));
    if (s.n_split > 1)
        CK(c, launch_reduce_splits(a, st));
    return KIRIN_OK;
}

// Doubles of split partials a launch of n_i i-particles with shape s needs.
size_t partial_doubles(const kirin_ctx *c, Shape s, int64_t n_i, int mode)
{
    if (s.n_split <= 1)
        return 0;
    return (size_t)s.n_split * (mode == MODE_NN ? 9 : 7) * (size_t)round_up(n_i, shape_i_cta(s, c->prec == KIRIN_MIXED));
}

// Enqueue one force launch (plus split reduction) over the current images on
// the context's stream, with the shape of choose_shape.
int run_force(kirin_ctx *c, int64_t n_i, const int32_t *d_ilist, int n_j, int mode, double *acc,
              double *jerk, double *pot, int accumulate = 0, int32_t *nn = nullptr, double *nn_r2 = nullptr)
{
    if (n_i == 0)
        return KIRIN_OK;
    const bool parted = c->n_parts > 1;
    if (parted && (accumulate || (mode != MODE_ACC_JERK_POT && mode != MODE_ACC_POT)))
        return set_msg(c, KIRIN_ESTATE, "this call does not support a j partition (kirin_set_j_partition)");
    const int ntiles = part_tiles(n_j, c->part, c->n_parts, nullptr);
    const Shape s = choose_shape(c, n_i, ntiles, c->prec, mode, guard_on(c));
    int rc = ensure_partial(c, partial_doubles(c, s, n_i, mode));
    if (rc)
        return rc;
    if (!parted || !c->allgather)  // whole sums, or this part's partial sums for the caller to combine
        return enqueue_force(c, c->stream, s, n_i, nullptr, d_ilist, n_j, mode, acc, jerk, pot, accumulate, nn,
                             nn_r2);
    // this part's sums into the send buffer [acc 3 n_i | jerk 3 n_i | pot n_i], every part's gathered by
    // the caller's exchange, then their sum in part order
    const int64_t count = 7 * n_i;
    if ((size_t)count > c->send_cap || (size_t)count * c->n_parts > c->recv_cap)
        return set_msg(c, KIRIN_EINVAL, "j partition: %lld i-particles exceed the exchange buffers",
                       (long long)n_i);
    double *sd = c->d_send;
    rc = enqueue_force(c, c->stream, s, n_i, nullptr, d_ilist, n_j, mode, sd, sd + 3 * n_i, sd + 6 * n_i);
    if (rc)
        return rc;
    const int ex = c->allgather(c->allgather_user, sd, c->d_recv, count, (void *)c->stream);
    if (ex != 0)
        return set_msg(c, KIRIN_EEXCHANGE, "j partition: the all-gather callback returned %d", ex);
    CK(c, launch_sum_parts(c->n_parts, n_i, c->d_recv, acc, jerk, pot, c->stream));
    return KIRIN_OK;
}

// The return code of a set of device error bits.
int error_code(kirin_ctx *c, unsigned e)
{
    if (e == 0)
        return KIRIN_OK;
    if (e & (ERR_TIMEOUT | ERR_DRAIN))
        return set_msg(c, KIRIN_ETIMEOUT, "a bounded device wait gave up (flags 0x%x)", e);
    if (e & ERR_NONFINITE)
        return set_msg(c, KIRIN_ENONFINITE, "non-finite particle data on the device");
    if (e & ERR_STALL)
        return set_msg(c, KIRIN_ESTATE, "block time stopped advancing (t + dt == t in FP64)");
    if (e & ERR_INDEX)
        return set_msg(c, KIRIN_EINVAL, "i index outside [0, n_j) on the device");
    return set_msg(c, KIRIN_ECUDA, "device error flags 0x%x", e);
}

// Synchronise the stream and report (and clear) the kernels' error bits.
int read_device_errors(kirin_ctx *c)
{
    if (c->h_err_map) {
        CK(c, cudaStreamSynchronize(c->stream));
        volatile unsigned *w = c->h_err_map;
        const unsigned e = *w;
        if (e)
            *w = 0u;  // written before the next launch, which therefore sees it
        return error_code(c, e);
    }
    CK(c, cudaMemcpyAsync(c->h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const unsigned e = *c->h_err;
    if (e == 0)
        return KIRIN_OK;
    CK(c, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream));
    return error_code(c, e);
}

bool all_finite(const double *p, int64_t n)
{
    for (int64_t k = 0; k < n; ++k)
        if (!isfinite(p[k]))
            return false;
    return true;
}

void free_all(kirin_ctx *c)
{
    void *ptrs[] = {c->bm, c->bx, c->bv, c->ba, c->bj, c->bt, c->bdt, c->xp, c->vp, c->jm, c->jd,
                    c->d_ilist, c->d_acc, c->d_jerk, c->d_pot, c->d_partial, c->d_err, c->d_scal,
                    c->d_count, c->d_sel_counts, c->d_nn, c->d_nn_r2, c->d_step_counts, c->d_send, c->d_recv,
                    c->sh_img, c->sh_arrivals};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    if (c->h_ilist)
        cudaFreeHost(c->h_ilist);
    if (c->h_scal)
        cudaFreeHost(c->h_scal);
    if (c->h_count)
        cudaFreeHost(c->h_count);
    if (c->h_err)
        cudaFreeHost(c->h_err);
    if (c->h_err_map)
        cudaFreeHost(c->h_err_map);
    if (c->h_sel_t)
        cudaFreeHost(c->h_sel_t);
    if (c->h_run)
        cudaFreeHost(c->h_run);
    if (c->d_run)
        cudaFree(c->d_run);
    if (c->run_exec)
        cudaGraphExecDestroy(c->run_exec);
    for (auto *v : {&c->trace_pending, &c->trace_free})
        for (auto &e : *v) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    if (c->own_stream && c->stream)
        cudaStreamDestroy(c->stream);
}

// Add every pending event pair's elapsed time to the totals (waiting for the last of them) and
// keep the events for reuse; with count false (a reset) the pairs are only waited for.
cudaError_t trace_fold(kirin_ctx *c, bool count)
{
    cudaError_t err = cudaSuccess;
    for (auto &e : c->trace_pending) {
        float ms = 0.f;
        cudaError_t r = cudaEventSynchronize(e.second);
        if (r == cudaSuccess)
            r = cudaEventElapsedTime(&ms, e.first, e.second);
        if (r != cudaSuccess && err == cudaSuccess)
            err = r;
        if (count && r == cudaSuccess) {
            c->trace_calls += 1;
            c->trace_ms += (double)ms;
        }
        c->trace_free.push_back(e);
    }
    c->trace_pending.clear();
    return err;
}

// One traced API call: with tracing on, an NVTX range named after the call (seen by an attached
// profiler) and two CUDA events around the stream work it enqueues, unless the stream is being
// captured into a graph (events there become graph nodes and time nothing).  Declared after the
// call's argument checks and DeviceGuard; the outermost of nested traced calls records.
struct TraceScope {
    kirin_ctx *c;
    bool on = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TraceScope(kirin_ctx *ctx, const char *name) : c(ctx)
    {
        if (!c->tracing || c->trace_depth++ > 0)
            return;
        on = true;
        nvtxRangePushA(name);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return;
        }
        if (!c->trace_free.empty()) {
            e0 = c->trace_free.back().first;
            e1 = c->trace_free.back().second;
            c->trace_free.pop_back();
        } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            if (e0)
                cudaEventDestroy(e0);
            cudaGetLastError();
            e0 = e1 = nullptr;
            return;
        }
        if (cudaEventRecord(e0, c->stream) != cudaSuccess)
            cudaGetLastError();  // the pair is then not counted; the call's own checks stay clean
    }
    ~TraceScope()
    {
        if (!c->tracing && !on)
            return;
        if (c->trace_depth > 0)
            --c->trace_depth;
        if (!on)
            return;
        if (e0) {
            if (cudaEventRecord(e1, c->stream) != cudaSuccess)
                cudaGetLastError();
            c->trace_pending.emplace_back(e0, e1);
            if (c->trace_pending.size() >= 1024 && trace_fold(c, true) != cudaSuccess)
                cudaGetLastError();  // an unreadable pair is dropped, as kirin_get_trace would report
        }
        nvtxRangePop();
    }
};

int check_params(double eps, double G, double r_min, int prec)
{
    if (!(eps >= 0.0) || !isfinite(eps) || !isfinite(G) || !(r_min >= 0.0) || !isfinite(r_min))
        return KIRIN_EINVAL;
    if (prec != KIRIN_FP64 && prec != KIRIN_MIXED)
        return KIRIN_EINVAL;
    return KIRIN_OK;
}


// ---- device-driven block steps ---------------------------------------------
//
// The graph:  WHILE(loop) { correct + minimum; select + predict; SWITCH(branch)
// { force launch for block-size class 0 | 1 | ... } }.  The step kernels
// correct the block forced in the previous iteration, select and predict the
// next one and set both conditions; the iteration that selects nothing ends
// the loop, so every block of a run is corrected before the graph returns.
// (Two plain kernels: a dependent kernel node costs about 0.8 us on this
// part, a grid-wide barrier inside one kernel about 2.4 us.)  Each
// class c covers block sizes (class_max[c-1], class_max[c]]; its force launch
// has a grid for class_max[c] and the shape chosen for a block of about
// 0.7 class_max[c], and its CTAs beyond the actual block return at once.

// Block steps per iteration of the WHILE node: one iteration costs about
// 3.4 us on its own, so the body holds several steps.
constexpr int RUN_UNROLL = 4;

struct RunPlan {
    int n_classes = 0;
    int32_t class_max[MAX_SEL_CLASSES] = {};
    Shape shape[MAX_SEL_CLASSES] = {};
};

RunPlan plan_run(kirin_ctx *c)
{
    RunPlan p;
    const int64_t n = c->n_j;
    int64_t hi = n;
    int32_t desc[MAX_SEL_CLASSES];
    int k = 0;
    while (hi > TINY_MAX && k < MAX_SEL_CLASSES - 1) {
        desc[k++] = (int32_t)hi;
        hi = (hi + 1) / 2;
    }
    desc[k++] = (int32_t)hi;
    p.n_classes = k;
    const int ntiles = (int)((std::max<int64_t>(n, 1) + TILE_J - 1) / TILE_J);
    for (int q = 0; q < k; ++q) {
        p.class_max[q] = desc[k - 1 - q];
        // a class above the tiny-block bound needs a regular shape (its grid covers class_max)
        const int64_t floor_rep = p.class_max[q] > TINY_MAX ? TINY_MAX + 1 : 1;
        const int64_t rep = std::max<int64_t>(floor_rep, (int64_t)(0.7 * p.class_max[q]));
        p.shape[q] = choose_shape(c, rep, ntiles, c->prec, MODE_ACC_JERK_POT, guard_on(c));
    }
    return p;
}

// Whether shared-step runs take the single-launch kernel: mixed precision, at most SH_MAX_N
// particles, no fixed launch shape (which names the per-kernel path) and no j partition, enabled, and
// its cooperative launch fitting on this GPU.
bool shared_steps_on(kirin_ctx *c)
{
    if (!c->shared_persistent || c->prec != KIRIN_MIXED || c->n_j < 1 || c->n_j > SH_MAX_N || c->n_parts > 1 ||
        (c->fix_groups > 0 && c->fix_split > 0))
        return false;
    const bool guard = guard_on(c);
    if (c->sh_fit_n != c->n_j || c->sh_fit_guard != (int)guard) {
        c->sh_grid = shared_steps_grid((int)c->n_j, guard);
        cudaGetLastError();
        c->sh_fit_n = c->n_j;
        c->sh_fit_guard = (int)guard;
    }
    return c->sh_grid > 0;
}

// One launch of the shared-step kernel (shared_steps_on(c) holds): n_steps shared steps of dt from
// t0, or with init the evaluation at t0 and the initialisation of the integrator.  Allocates the two
// j images and the arrival counter on first use.
int shared_launch(kirin_ctx *c, double t0, double dt, int64_t n_steps, int init, double dt_min, double dt_max)
{
    const int n = (int)c->n_j;
    const int64_t n_pad = round_up(n, TILE_J);
    if (c->sh_img_pad < n_pad) {
        if (c->sh_img)
            cudaFree(c->sh_img);
        c->sh_img = nullptr;
        c->sh_img_pad = 0;
        if (cudaMalloc(&c->sh_img, 2 * (size_t)n_pad * sizeof(JMixed)) != cudaSuccess) {
            c->sh_img = nullptr;
            cudaGetLastError();
            return set_msg(c, KIRIN_ENOMEM, "shared steps: no room for the two j images");
        }
        c->sh_img_pad = n_pad;
    }
    if (!c->sh_arrivals) {
        if (cudaMalloc(&c->sh_arrivals, sizeof(unsigned)) != cudaSuccess) {
            c->sh_arrivals = nullptr;
            cudaGetLastError();
            return set_msg(c, KIRIN_ENOMEM, "shared steps: no room for the arrival counter");
        }
        CK(c, cudaMemsetAsync(c->sh_arrivals, 0, sizeof(unsigned), c->stream));
        c->sh_count = 0;
    }
    SharedStepArgs a{};
    a.n = n;
    a.n_pad = (int)n_pad;
    a.img = c->sh_img;
    a.arrivals = c->sh_arrivals;
    a.arrivals0 = c->sh_count;
    a.ctas = c->sh_grid;
    a.m = c->bm;
    a.x = c->bx;
    a.v = c->bv;
    a.a = c->ba;
    a.jerk_b = c->bj;
    a.t_b = c->bt;
    a.dt_b = c->bdt;
    a.xp = c->xp;
    a.vp = c->vp;
    a.f_acc = c->d_acc;
    a.f_jerk = c->d_jerk;
    a.f_pot = c->d_pot;
    a.eps2 = c->eps * c->eps;
    a.rmin2 = c->r_min * c->r_min;
    a.G = c->G;
    a.eta = c->eta;
    a.dt_min = dt_min;
    a.dt_max = dt_max;
    a.t0 = t0;
    a.dt = dt;
    a.n_steps = init ? 0 : (int)n_steps;
    a.init = init;
    a.err = err_word(c);
    CK(c, launch_shared_steps(a, guard_on(c), c->stream));
    // every CTA arrives once per step (once when initialising)
    c->sh_count += (uint32_t)c->sh_grid * (uint32_t)(init ? 1 : n_steps);
    return KIRIN_OK;
}

// The errors of a shared-step launch (read_device_errors); after a timeout (CTAs left mid-run) the
// arrival counter starts from zero again.
int read_shared_errors(kirin_ctx *c)
{
    const int rc = read_device_errors(c);
    if (rc == KIRIN_ETIMEOUT && c->sh_arrivals) {
        CK(c, cudaMemsetAsync(c->sh_arrivals, 0, sizeof(unsigned), c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        c->sh_count = 0;
    }
    return rc;
}

RunKey run_key(const kirin_ctx *c, const RunPlan &p)
{
    RunKey k;
    memset(&k, 0, sizeof(k));
    const double par[6] = {c->eps, c->G, c->r_min, c->eta, c->dt_min, c->dt_max};
    memcpy(k.par, par, sizeof(par));
    k.n_j = c->n_j;
    k.prec = c->prec;
    k.partial = c->d_partial;
    k.n_classes = p.n_classes;
    for (int q = 0; q < p.n_classes; ++q) {
        k.class_max[q] = p.class_max[q];
        k.shape[q] = p.shape[q];
    }
    return k;
}

// Capture onto the body graph with stream cs.
#define CKG(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            rc = set_msg(c, KIRIN_ECUDA, "device loop: %s: %s", #call, cudaGetErrorString(e_)); \
            goto done;                                                                         \
        }                                                                                      \
    } while (0)

int build_run_graph(kirin_ctx *c, const RunPlan &p, cudaGraphExec_t *exec_out)
{
    int rc = KIRIN_OK;
    cudaGraph_t top = nullptr;
    cudaStream_t cs = nullptr;
    bool capturing = false;
    cudaGraphConditionalHandle h_loop, h_branch[RUN_UNROLL];
    cudaGraphNodeParams wp{}, sp[RUN_UNROLL] = {};
    cudaGraphNode_t wnode, snode;
    cudaGraph_t body, cap_graph;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus status;
    StepArgs a{};
    const int n = (int)c->n_j;

    CKG(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CKG(cudaGraphCreate(&top, 0));
    CKG(cudaGraphConditionalHandleCreate(&h_loop, top, 1, cudaGraphCondAssignDefault));
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    CKG(cudaGraphAddNode(&wnode, top, nullptr, nullptr, 0, &wp));
    body = wp.conditional.phGraph_out[0];
    for (int u = 0; u < RUN_UNROLL; ++u)
        CKG(cudaGraphConditionalHandleCreate(&h_branch[u], body, 0, cudaGraphCondAssignDefault));

    a.n = n;
    a.n_pad = (int)round_up(std::max<int64_t>(n, 1), TILE_J);
    a.bm = c->bm;
    a.bx = c->bx;
    a.bv = c->bv;
    a.ba = c->ba;
    a.bj = c->bj;
    a.bt = c->bt;
    a.bdt = c->bdt;
    a.xp = c->xp;
    a.vp = c->vp;
    a.jm = img_m(c);
    a.jd = img_d(c);
    a.acc = c->d_acc;
    a.jerk = c->d_jerk;
    a.ilist = c->d_ilist;
    a.chunk_off = c->d_step_counts;
    a.eta = c->eta;
    a.dt_min = c->dt_min;
    a.dt_max = c->dt_max;
    a.run = c->d_run;
    a.count_out = c->d_count;
    a.t_next_out = c->d_scal;
    a.err = err_word(c);
    a.loop = h_loop;
    a.n_classes = p.n_classes;
    for (int q = 0; q < p.n_classes; ++q)
        a.class_max[q] = p.class_max[q];
    a.n_j = n;

    // loop body: RUN_UNROLL block steps, each the two step kernels and a SWITCH
    // over force launches (a step after the one that ended the run finds nothing
    // pending and nothing due, and does nothing)
    CKG(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    capturing = true;
    for (int u = 0; u < RUN_UNROLL; ++u) {
        a.branch = h_branch[u];
        CKG(launch_block_step(a, c->step_ctas, cs));
        CKG(cudaStreamGetCaptureInfo(cs, &status, nullptr, &cap_graph, &deps, nullptr, &ndeps));
        sp[u].type = cudaGraphNodeTypeConditional;
        sp[u].conditional.handle = h_branch[u];
        sp[u].conditional.type = cudaGraphCondTypeSwitch;
        sp[u].conditional.size = (unsigned)p.n_classes;
        CKG(cudaGraphAddNode(&snode, cap_graph, deps, nullptr, ndeps, &sp[u]));
        CKG(cudaStreamUpdateCaptureDependencies(cs, &snode, nullptr, 1, cudaStreamSetCaptureDependencies));
    }
    capturing = false;
    CKG(cudaStreamEndCapture(cs, &cap_graph));

    // the force branches
    for (int u = 0; u < RUN_UNROLL; ++u)
        for (int q = 0; q < p.n_classes; ++q) {
            CKG(cudaStreamBeginCaptureToGraph(cs, sp[u].conditional.phGraph_out[q], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
            capturing = true;
            rc = enqueue_force(c, cs, p.shape[q], p.class_max[q], c->d_count, c->d_ilist, n, MODE_ACC_JERK_POT,
                               c->d_acc, c->d_jerk, c->d_pot);
            if (rc)
                goto done;
            capturing = false;
            CKG(cudaStreamEndCapture(cs, &cap_graph));
        }
    CKG(cudaGraphInstantiate(exec_out, top, 0));

done:
    if (capturing) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(cs, &junk);
        cudaGetLastError();
    }
    if (top)
        cudaGraphDestroy(top);
    if (cs)
        cudaStreamDestroy(cs);
    return rc;
}
#undef CKG

int hermite_run_device(kirin_ctx *c, double t_end, int64_t max_steps, int64_t *n_steps, double *n_pairs)
{
    DeviceGuard dg(c->device);
    const RunPlan p = plan_run(c);
    size_t need = 0;
    for (int q = 0; q < p.n_classes; ++q)
        need = std::max(need, partial_doubles(c, p.shape[q], p.class_max[q], MODE_ACC_JERK_POT));
    int rc = ensure_partial(c, need);
    if (rc)
        return rc;
    const RunKey key = run_key(c, p);
    if (!c->run_exec || memcmp(&key, &c->run_key, sizeof(key)) != 0) {
        if (c->run_exec) {
            CK(c, cudaStreamSynchronize(c->stream));
            cudaGraphExecDestroy(c->run_exec);
            c->run_exec = nullptr;
        }
        rc = build_run_graph(c, p, &c->run_exec);
        if (rc) {
            c->run_exec = nullptr;
            return rc;
        }
        memcpy(&c->run_key, &key, sizeof(key));
    }
    // the pinned mirror may still be the source or target of the last run's copies
    CK(c, cudaStreamSynchronize(c->stream));
    RunState init{};
    init.t_end = t_end;
    init.max_steps = (long long)std::max<int64_t>(max_steps, 0);
    init.minw[0] = init.minw[1] = ~0ull;
    *c->h_run = init;
    CK(c, cudaMemcpyAsync(c->d_run, c->h_run, sizeof(RunState), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaGraphLaunch(c->run_exec, c->stream));
    CK(c, cudaMemcpyAsync(c->h_run, c->d_run, sizeof(RunState), cudaMemcpyDeviceToHost, c->stream));
    rc = read_device_errors(c);  // synchronises the stream
    if (rc)
        return rc;
    const RunState out = *c->h_run;
    if (n_steps)
        *n_steps = out.steps;
    if (n_pairs)
        *n_pairs = out.pairs;
    if (out.steps > 0) {
        c->pred_mode = 1;
        c->pred_t = out.t_last;
    }
    c->images_dirty = true;  // base state moved
    c->pending = false;
    return KIRIN_OK;
}

}  // namespace

extern "C" {

const char *kirin_strerror(int code)
{
    switch (code) {
    case KIRIN_OK: return "success";
    case KIRIN_EINVAL: return "invalid argument";
    case KIRIN_ENOMEM: return "out of memory";
    case KIRIN_ECUDA: return "CUDA runtime error";
    case KIRIN_ENONFINITE: return "non-finite particle data";
    case KIRIN_ETIMEOUT: return "device wait timed out";
    case KIRIN_ESTATE: return "call out of order";
    case KIRIN_EEXCHANGE: return "j-partition exchange failed";
    default: return "unknown error";
    }
}

const char *kirin_last_error(const kirin_ctx *ctx) { return ctx ? ctx->msg : "no context"; }

int kirin_init(kirin_ctx **out, int64_t n_max, const kirin_config *cfg)
{
    if (!out || !cfg)
        return KIRIN_EINVAL;
    *out = nullptr;
    if (n_max < 1 || n_max > (int64_t)INT32_MAX - 256)
        return KIRIN_EINVAL;
    if (check_params(cfg->eps, cfg->G, cfg->r_min, cfg->prec))
        return KIRIN_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return KIRIN_ECUDA;
    }
    DeviceGuard dg(cfg->device);
    if (!dg.ok)
        return KIRIN_ECUDA;
    kirin_ctx *c = new (std::nothrow) kirin_ctx();
    if (!c)
        return KIRIN_ENOMEM;
    c->device = cfg->device;
    c->n_max = n_max;
    c->n_img = round_up(n_max, TILE_J);
    c->eps = cfg->eps;
    c->G = cfg->G;
    c->r_min = cfg->r_min;
    c->prec = cfg->prec;
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (cfg->stream) {
        c->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return KIRIN_ECUDA;
        }
        c->own_stream = true;
    }
    const size_t n = (size_t)n_max;
    bool ok = true;
    auto dalloc = [&](void **p, size_t bytes) {
        if (ok && cudaMalloc(p, bytes) != cudaSuccess)
            ok = false;
    };
    dalloc((void **)&c->bm, n * sizeof(double));
    dalloc((void **)&c->bx, 3 * n * sizeof(double));
    dalloc((void **)&c->bv, 3 * n * sizeof(double));
    dalloc((void **)&c->ba, 3 * n * sizeof(double));
    dalloc((void **)&c->bj, 3 * n * sizeof(double));
    dalloc((void **)&c->bt, n * sizeof(double));
    dalloc((void **)&c->bdt, n * sizeof(double));
    dalloc((void **)&c->xp, 3 * n * sizeof(double));
    dalloc((void **)&c->vp, 3 * n * sizeof(double));
    dalloc((void **)&c->jm, (size_t)c->n_img * sizeof(JMixed));
    dalloc((void **)&c->jd, (size_t)c->n_img * sizeof(JF64));
    dalloc((void **)&c->d_ilist, n * sizeof(int32_t));
    dalloc((void **)&c->d_acc, 3 * n * sizeof(double));
    dalloc((void **)&c->d_jerk, 3 * n * sizeof(double));
    dalloc((void **)&c->d_pot, n * sizeof(double));
    dalloc((void **)&c->d_err, sizeof(unsigned));
    dalloc((void **)&c->d_scal, 4 * sizeof(double));
    dalloc((void **)&c->d_count, sizeof(int32_t));
    dalloc((void **)&c->d_sel_counts, ((n + 1023) / 1024 + 1) * sizeof(int32_t));
    dalloc((void **)&c->d_nn, n * sizeof(int32_t));
    dalloc((void **)&c->d_nn_r2, n * sizeof(double));
    if (ok && cudaMallocHost((void **)&c->h_ilist, n * sizeof(int32_t)) != cudaSuccess)
        ok = false;
    if (ok && cudaMallocHost((void **)&c->h_scal, 4 * sizeof(double)) != cudaSuccess)
        ok = false;
    if (ok && cudaMallocHost((void **)&c->h_count, sizeof(int32_t)) != cudaSuccess)
        ok = false;
    if (ok && cudaMallocHost((void **)&c->h_err, sizeof(unsigned)) != cudaSuccess)
        ok = false;
    int host_atomics = 0;  // the kernels' atomicOr on the mapped word needs native host atomics
    cudaDeviceGetAttribute(&host_atomics, cudaDevAttrHostNativeAtomicSupported, c->device);
    if (ok && host_atomics) {  // optional: without it the kernels report through d_err
        if (cudaHostAlloc((void **)&c->h_err_map, sizeof(unsigned), cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer((void **)&c->d_err_map, c->h_err_map, 0) == cudaSuccess) {
            *(volatile unsigned *)c->h_err_map = 0u;
            // the block step's time and size, in one mapped allocation (a double, then an int32)
            if (cudaHostAlloc((void **)&c->h_sel_t, 16, cudaHostAllocMapped) == cudaSuccess &&
                cudaHostGetDevicePointer((void **)&c->d_sel_t, c->h_sel_t, 0) == cudaSuccess) {
                c->h_sel_n = reinterpret_cast<int32_t *>(c->h_sel_t + 1);
                c->d_sel_n = reinterpret_cast<int32_t *>(c->d_sel_t + 1);
            } else {
                cudaGetLastError();
                if (c->h_sel_t)
                    cudaFreeHost(c->h_sel_t);
                c->h_sel_t = nullptr;
                c->d_sel_t = nullptr;
            }
        } else {
            cudaGetLastError();
            if (c->h_err_map)
                cudaFreeHost(c->h_err_map);
            c->h_err_map = nullptr;
            c->d_err_map = nullptr;
        }
    }
    dalloc((void **)&c->d_run, sizeof(RunState));
    if (ok && cudaMallocHost((void **)&c->h_run, sizeof(RunState)) != cudaSuccess)
        ok = false;
    c->step_ctas = std::max(c->nsm, 1) * STEP_CTAS_PER_SM;
    dalloc((void **)&c->d_step_counts, 2 * (size_t)c->step_ctas * sizeof(int32_t));
    if (ok && cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream) != cudaSuccess)
        ok = false;
    if (ok && cudaMemsetAsync(c->bt, 0, n * sizeof(double), c->stream) != cudaSuccess)
        ok = false;
    if (ok && cudaStreamSynchronize(c->stream) != cudaSuccess)
        ok = false;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return KIRIN_ENOMEM;
    }
    *out = c;
    return KIRIN_OK;
}

int kirin_finalize(kirin_ctx *ctx)
{
    if (!ctx)
        return KIRIN_OK;
    DeviceGuard dg(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
    return KIRIN_OK;
}

int kirin_query(const kirin_ctx *ctx, int64_t *n_max, int32_t *tile_i, int32_t *tile_j)
{
    if (!ctx)
        return KIRIN_EINVAL;
    if (n_max)
        *n_max = ctx->n_max;
    if (tile_i)
        *tile_i = (ctx->prec == KIRIN_MIXED ? MIX_I_PER_THREAD : 1) * FORCE_THREADS;
    if (tile_j)
        *tile_j = TILE_J;
    return KIRIN_OK;
}

int kirin_set_params(kirin_ctx *ctx, double eps, double G, double r_min, int32_t prec)
{
    if (!ctx || check_params(eps, G, r_min, prec))
        return KIRIN_EINVAL;
    ctx->eps = eps;
    ctx->G = G;
    ctx->r_min = r_min;
    if (prec != ctx->prec)
        ctx->images_dirty = true;  // only the image of the old precision is current
    ctx->prec = prec;
    return KIRIN_OK;
}

int kirin_set_stream(kirin_ctx *ctx, void *stream)
{
    if (!ctx)
        return KIRIN_EINVAL;
    DeviceGuard dg(ctx->device);
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->own_stream) {
        cudaStreamDestroy(ctx->stream);
        ctx->own_stream = false;
    }
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        CK(ctx, cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    return KIRIN_OK;
}

int kirin_set_launch(kirin_ctx *ctx, int32_t groups, int32_t n_split)
{
    if (!ctx)
        return KIRIN_EINVAL;
    if (groups == 0 && n_split == 0) {
        ctx->fix_groups = ctx->fix_split = 0;
        return KIRIN_OK;
    }
    if ((groups != 1 && groups != 2 && groups != 4 && groups != 8) || n_split < 1 || n_split > MAX_SPLIT)
        return KIRIN_EINVAL;
    ctx->fix_groups = groups;
    ctx->fix_split = n_split;
    return KIRIN_OK;
}

int kirin_set_launch_table_for(kirin_ctx *ctx, int32_t kind, int32_t n_entries, const int64_t *n_i_max,
                               const int32_t *groups, const int32_t *n_split)
{
    if (!ctx || kind < 0 || kind >= kirin_ctx::N_KINDS || n_entries < 0 || n_entries > kirin_ctx::MAX_TABLE)
        return KIRIN_EINVAL;
    if (n_entries > 0 && (!n_i_max || !groups || !n_split))
        return KIRIN_EINVAL;
    for (int k = 0; k < n_entries; ++k) {
        const int g = groups[k];
        if ((g != 1 && g != 2 && g != 4 && g != 8) || n_split[k] < 1 || n_split[k] > MAX_SPLIT || n_i_max[k] < 0 ||
            (k > 0 && n_i_max[k] <= n_i_max[k - 1]))
            return KIRIN_EINVAL;
    }
    for (int k = 0; k < n_entries; ++k) {
        ctx->table_ni[kind][k] = n_i_max[k];
        ctx->table_groups[kind][k] = groups[k];
        ctx->table_split[kind][k] = n_split[k];
    }
    ctx->table_n[kind] = n_entries;
    ctx->table_prec[kind] = ctx->prec;
    return KIRIN_OK;
}

int kirin_set_launch_table(kirin_ctx *ctx, int32_t n_entries, const int64_t *n_i_max, const int32_t *groups,
                           const int32_t *n_split)
{
    return kirin_set_launch_table_for(ctx, KIRIN_CALL_FORCES, n_entries, n_i_max, groups, n_split);
}

int kirin_get_launch_for(kirin_ctx *ctx, int32_t kind, int64_t n_i, int32_t *groups, int32_t *n_split)
{
    if (!ctx || n_i < 0 || kind < 0 || kind >= kirin_ctx::N_KINDS)
        return KIRIN_EINVAL;
    DeviceGuard dg(ctx->device);
    const int ntiles = part_tiles(ctx->n_j, ctx->part, ctx->n_parts, nullptr);
    const Shape s = choose_shape(ctx, n_i, ntiles, ctx->prec, mode_of_kind(kind), guard_on(ctx));
    if (groups)
        *groups = s.groups;
    if (n_split)
        *n_split = s.n_split;
    return KIRIN_OK;
}

int kirin_get_launch(kirin_ctx *ctx, int64_t n_i, int32_t *groups, int32_t *n_split)
{
    return kirin_get_launch_for(ctx, KIRIN_CALL_FORCES, n_i, groups, n_split);
}

int kirin_set_j_particles(kirin_ctx *ctx, int64_t first, int64_t n, const double *m, const double *x,
                          const double *v, const double *a, const double *jerk, const double *t0)
{
    if (!ctx || !m || !x || !v || first < 0 || n < 0 || first + n > ctx->n_max)
        return set_msg(ctx, KIRIN_EINVAL, "set_j_particles: bad range or NULL array");
    if (n == 0)
        return KIRIN_OK;
    if (!all_finite(m, n) || !all_finite(x, 3 * n) || !all_finite(v, 3 * n) ||
        (a && !all_finite(a, 3 * n)) || (jerk && !all_finite(jerk, 3 * n)) || (t0 && !all_finite(t0, n)))
        return set_msg(ctx, KIRIN_ENONFINITE, "set_j_particles: NaN or Inf in input");
    DeviceGuard dg(ctx->device);
    const size_t f = (size_t)first, nn = (size_t)n;
    cudaStream_t s = ctx->stream;
    CK(ctx, cudaMemcpyAsync(ctx->bm + f, m, nn * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(ctx, cudaMemcpyAsync(ctx->bx + 3 * f, x, 3 * nn * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(ctx, cudaMemcpyAsync(ctx->bv + 3 * f, v, 3 * nn * sizeof(double), cudaMemcpyHostToDevice, s));
    if (a)
        CK(ctx, cudaMemcpyAsync(ctx->ba + 3 * f, a, 3 * nn * sizeof(double), cudaMemcpyHostToDevice, s));
    else
        CK(ctx, cudaMemsetAsync(ctx->ba + 3 * f, 0, 3 * nn * sizeof(double), s));
    if (jerk)
        CK(ctx, cudaMemcpyAsync(ctx->bj + 3 * f, jerk, 3 * nn * sizeof(double), cudaMemcpyHostToDevice, s));
    else
        CK(ctx, cudaMemsetAsync(ctx->bj + 3 * f, 0, 3 * nn * sizeof(double), s));
    if (t0)
        CK(ctx, cudaMemcpyAsync(ctx->bt + f, t0, nn * sizeof(double), cudaMemcpyHostToDevice, s));
    else
        CK(ctx, cudaMemsetAsync(ctx->bt + f, 0, nn * sizeof(double), s));
    // host sources may be reused as soon as we return
    CK(ctx, cudaStreamSynchronize(s));
    ctx->n_hi = std::max(ctx->n_hi, first + n);
    ctx->n_j = std::max(ctx->n_j, first + n);
    ctx->pred_mode = 0;
    ctx->images_dirty = true;
    ctx->hermite_ready = false;
    return KIRIN_OK;
}

int kirin_set_j_particles_dev(kirin_ctx *ctx, int64_t first, int64_t n, const double *m,
                              const double *x, const double *v, const double *a, const double *jerk,
                              const double *t0)
{
    if (!ctx || !m || !x || !v || first < 0 || n < 0 || first + n > ctx->n_max)
        return set_msg(ctx, KIRIN_EINVAL, "set_j_particles_dev: bad range or NULL array");
    if (n == 0)
        return KIRIN_OK;
    DeviceGuard dg(ctx->device);
    CK(ctx, launch_scatter_state((int)first, (int)n, m, x, v, a, jerk, t0, ctx->bm, ctx->bx, ctx->bv,
                                 ctx->ba, ctx->bj, ctx->bt, err_word(ctx), ctx->stream));
    ctx->n_hi = std::max(ctx->n_hi, first + n);
    ctx->n_j = std::max(ctx->n_j, first + n);
    ctx->pred_mode = 0;
    ctx->images_dirty = true;
    ctx->hermite_ready = false;
    return KIRIN_OK;
}

int kirin_set_nj(kirin_ctx *ctx, int64_t n_j)
{
    if (!ctx || n_j < 0 || n_j > ctx->n_hi)
        return set_msg(ctx, KIRIN_EINVAL, "set_nj: n_j outside [0, highest index set]");
    ctx->n_j = n_j;
    ctx->images_dirty = true;
    return KIRIN_OK;
}

int kirin_predict(kirin_ctx *ctx, double t)
{
    if (!ctx || !isfinite(t))
        return KIRIN_EINVAL;
    if (ctx->n_j == 0)
        return set_msg(ctx, KIRIN_ESTATE, "predict: no particles");
    ctx->pred_mode = 1;
    ctx->pred_t = t;
    ctx->images_dirty = true;
    return KIRIN_OK;
}

int kirin_compute_forces(kirin_ctx *ctx, int64_t n_i, const int32_t *i_list)
{
    if (!ctx)
        return KIRIN_EINVAL;
    if (ctx->n_j == 0)
        return set_msg(ctx, KIRIN_ESTATE, "compute_forces: no particles");
    if (!i_list)
        n_i = ctx->n_j;
    if (n_i < 0 || n_i > ctx->n_max)
        return set_msg(ctx, KIRIN_EINVAL, "compute_forces: n_i out of range");
    if (i_list)
        for (int64_t k = 0; k < n_i; ++k)
            if (i_list[k] < 0 || i_list[k] >= ctx->n_j)
                return set_msg(ctx, KIRIN_EINVAL, "compute_forces: i_list[%lld] = %d outside [0, %lld)",
                               (long long)k, i_list[k], (long long)ctx->n_j);
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_compute_forces");
    const int32_t *d_list = nullptr;
    if (i_list) {
        // the previous upload may still be in flight from the pinned buffer
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        memcpy(ctx->h_ilist, i_list, (size_t)n_i * sizeof(int32_t));
        CK(ctx, cudaMemcpyAsync(ctx->d_ilist, ctx->h_ilist, (size_t)n_i * sizeof(int32_t),
                                cudaMemcpyHostToDevice, ctx->stream));
        d_list = ctx->d_ilist;
    }
    int rc = ensure_images(ctx);
    if (rc)
        return rc;
    const int mode = ctx->want_nn ? MODE_NN : MODE_ACC_JERK_POT;
    rc = run_force(ctx, n_i, d_list, (int)ctx->n_j, mode, ctx->d_acc, ctx->d_jerk, ctx->d_pot, 0, ctx->d_nn,
                   ctx->d_nn_r2);
    if (rc)
        return rc;
    ctx->pending = true;
    ctx->pending_n = n_i;
    ctx->nn_valid = ctx->want_nn;
    return KIRIN_OK;
}

int kirin_j_partition_range(int64_t n_j, int32_t part, int32_t n_parts, int64_t *j_begin, int64_t *j_end)
{
    if (n_j < 0 || n_parts < 1 || n_parts > KIRIN_MAX_PARTS || part < 0 || part >= n_parts || !j_begin || !j_end)
        return KIRIN_EINVAL;
    int tile0 = 0;
    const int nt = part_tiles(n_j, part, n_parts, &tile0);
    *j_begin = std::min<int64_t>(n_j, (int64_t)tile0 * TILE_J);
    *j_end = std::min<int64_t>(n_j, (int64_t)(tile0 + nt) * TILE_J);
    return KIRIN_OK;
}

int kirin_set_j_partition(kirin_ctx *ctx, int32_t part, int32_t n_parts, kirin_allgather_fn allgather, void *user)
{
    if (!ctx || n_parts < 1 || n_parts > KIRIN_MAX_PARTS || part < 0 || part >= n_parts)
        return set_msg(ctx, KIRIN_EINVAL, "set_j_partition: part %d of %d", part, n_parts);
    DeviceGuard dg(ctx->device);
    CK(ctx, cudaStreamSynchronize(ctx->stream));  // no launch still reads the old buffers
    if (n_parts > 1 && allgather) {
        const size_t send = 7 * (size_t)std::max<int64_t>(ctx->n_max, 1);
        const size_t recv = send * (size_t)n_parts;
        if (send > ctx->send_cap || recv > ctx->recv_cap) {
            if (ctx->d_send)
                cudaFree(ctx->d_send);
            if (ctx->d_recv)
                cudaFree(ctx->d_recv);
            ctx->d_send = ctx->d_recv = nullptr;
            ctx->send_cap = ctx->recv_cap = 0;
            if (cudaMalloc(&ctx->d_send, send * sizeof(double)) != cudaSuccess ||
                cudaMalloc(&ctx->d_recv, recv * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                if (ctx->d_send)
                    cudaFree(ctx->d_send);
                ctx->d_send = nullptr;
                ctx->part = 0;
                ctx->n_parts = 1;
                ctx->allgather = nullptr;
                return set_msg(ctx, KIRIN_ENOMEM, "set_j_partition: exchange buffers of %zu doubles", send + recv);
            }
            ctx->send_cap = send;
            ctx->recv_cap = recv;
        }
    }
    ctx->part = part;
    ctx->n_parts = n_parts;
    ctx->allgather = n_parts > 1 ? allgather : nullptr;
    ctx->allgather_user = n_parts > 1 ? user : nullptr;
    ctx->pending = false;
    return KIRIN_OK;
}

int kirin_set_nn(kirin_ctx *ctx, int32_t enable)
{
    if (!ctx)
        return KIRIN_EINVAL;
    ctx->want_nn = enable != 0;
    return KIRIN_OK;
}

int kirin_get_nn(kirin_ctx *ctx, int32_t *nn, double *nn_r2)
{
    if (!ctx)
        return KIRIN_EINVAL;
    if (!ctx->nn_valid)
        return set_msg(ctx, KIRIN_ESTATE, "get_nn: the last compute_forces did not search neighbours");
    DeviceGuard dg(ctx->device);
    const size_t n = (size_t)ctx->pending_n;
    if (nn)
        CK(ctx, cudaMemcpyAsync(nn, ctx->d_nn, n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    if (nn_r2)
        CK(ctx, cudaMemcpyAsync(nn_r2, ctx->d_nn_r2, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return read_device_errors(ctx);
}

int kirin_compute_forces_nn_dev(kirin_ctx *ctx, int64_t n_i, const int32_t *i_list, double *acc, double *jerk,
                                double *pot, int32_t *nn, double *nn_r2)
{
    if (!ctx)
        return KIRIN_EINVAL;
    if (ctx->n_j == 0)
        return set_msg(ctx, KIRIN_ESTATE, "compute_forces_nn_dev: no particles");
    if (!i_list)
        n_i = ctx->n_j;
    if (n_i < 0 || n_i > ctx->n_max)
        return set_msg(ctx, KIRIN_EINVAL, "compute_forces_nn_dev: n_i out of range");
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_compute_forces_nn_dev");
    int rc = ensure_images(ctx);
    if (rc)
        return rc;
    return run_force(ctx, n_i, i_list, (int)ctx->n_j, MODE_NN, acc, jerk, pot, 0, nn, nn_r2);
}

int kirin_get_acc_jerk_pot(kirin_ctx *ctx, double *acc, double *jerk, double *pot)
{
    if (!ctx)
        return KIRIN_EINVAL;
    if (!ctx->pending)
        return set_msg(ctx, KIRIN_ESTATE, "get_acc_jerk_pot: no pending compute_forces");
    DeviceGuard dg(ctx->device);
    const size_t n = (size_t)ctx->pending_n;
    if (acc)
        CK(ctx, cudaMemcpyAsync(acc, ctx->d_acc, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (jerk)
        CK(ctx, cudaMemcpyAsync(jerk, ctx->d_jerk, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (pot)
        CK(ctx, cudaMemcpyAsync(pot, ctx->d_pot, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    const int rc = read_device_errors(ctx);
    ctx->pending = false;
    return rc;
}

int kirin_compute_forces_dev(kirin_ctx *ctx, int64_t n_i, const int32_t *i_list, double *acc,
                             double *jerk, double *pot)
{
    if (!ctx)
        return KIRIN_EINVAL;
    if (ctx->n_j == 0)
        return set_msg(ctx, KIRIN_ESTATE, "compute_forces_dev: no particles");
    if (!i_list)
        n_i = ctx->n_j;
    if (n_i < 0 || n_i > ctx->n_max)
        return set_msg(ctx, KIRIN_EINVAL, "compute_forces_dev: n_i out of range");
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_compute_forces_dev");
    int rc = ensure_images(ctx);
    if (rc)
        return rc;
    return run_force(ctx, n_i, i_list, (int)ctx->n_j, MODE_ACC_JERK_POT, acc, jerk, pot);
}

int kirin_sync(kirin_ctx *ctx)
{
    if (!ctx)
        return KIRIN_EINVAL;
    DeviceGuard dg(ctx->device);
    return read_device_errors(ctx);
}

int kirin_energy(kirin_ctx *ctx, const double *v, double *kin, double *pot)
{
    if (!ctx)
        return KIRIN_EINVAL;
    if (ctx->n_j == 0)
        return set_msg(ctx, KIRIN_ESTATE, "energy: no particles");
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_energy");
    int rc = ensure_images(ctx);
    if (rc)
        return rc;
    const int n = (int)ctx->n_j;
    rc = run_force(ctx, n, nullptr, n, MODE_ACC_POT, ctx->d_acc, nullptr, ctx->d_pot);
    if (rc)
        return rc;
    const double *dv = ctx->vp;
    if (v) {
        if (!all_finite(v, 3 * (int64_t)n))
            return set_msg(ctx, KIRIN_ENONFINITE, "energy: NaN or Inf in v");
        CK(ctx, cudaMemcpyAsync(ctx->d_jerk, v, 3 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice,
                                ctx->stream));
        dv = ctx->d_jerk;
    }
    CK(ctx, launch_energy(n, ctx->bm, dv, ctx->d_pot, ctx->d_scal + 1, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->h_scal + 1, ctx->d_scal + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream));
    rc = read_device_errors(ctx);
    if (rc)
        return rc;
    if (kin)
        *kin = ctx->h_scal[1];
    if (pot)
        *pot = ctx->h_scal[2];
    ctx->pending = false;
    return KIRIN_OK;
}

// ---- Hermite integrator -----------------------------------------------------

int kirin_hermite_init(kirin_ctx *ctx, double t, double eta, double dt_min, double dt_max)
{
    if (!ctx || !isfinite(t) || !(eta > 0) || !(dt_min > 0) || !(dt_max >= dt_min))
        return KIRIN_EINVAL;
    if (ctx->n_j == 0)
        return set_msg(ctx, KIRIN_ESTATE, "hermite_init: no particles");
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_hermite_init");
    ctx->pred_mode = 0;
    ctx->images_dirty = true;
    int rc;
    if (shared_steps_on(ctx)) {
        // small systems: evaluation and initialisation in one launch of the shared-step kernel
        rc = shared_launch(ctx, t, 0.0, 0, 1, dt_min, dt_max);
        if (rc)
            return rc;
        rc = read_shared_errors(ctx);
    } else {
        rc = ensure_images(ctx);
        if (rc)
            return rc;
        const int n = (int)ctx->n_j;
        rc = run_force(ctx, n, nullptr, n, MODE_ACC_JERK_POT, ctx->d_acc, ctx->d_jerk, ctx->d_pot);
        if (rc)
            return rc;
        CK(ctx, launch_hermite_init(n, t, ctx->d_acc, ctx->d_jerk, dt_min, dt_max, ctx->ba, ctx->bj, ctx->bt,
                                    ctx->bdt, ctx->stream));
        rc = read_device_errors(ctx);
    }
    if (rc)
        return rc;
    ctx->eta = eta;
    ctx->dt_min = dt_min;
    ctx->dt_max = dt_max;
    ctx->t_shared = t;
    ctx->hermite_ready = true;
    ctx->pending = false;
    return KIRIN_OK;
}

int kirin_hermite_block_step(kirin_ctx *ctx, double t_end, double *t_now, int64_t *n_active)
{
    if (!ctx)
        return KIRIN_EINVAL;
    if (!ctx->hermite_ready)
        return set_msg(ctx, KIRIN_ESTATE, "hermite_block_step: call kirin_hermite_init first");
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_hermite_block_step");
    const int n = (int)ctx->n_j;
    CK(ctx, launch_block_select(n, ctx->bt, ctx->bdt, t_end, ctx->d_ilist, ctx->d_scal, ctx->d_count,
                                reinterpret_cast<unsigned long long *>(ctx->d_scal + 3), ctx->d_sel_counts,
                                ctx->stream, ctx->d_sel_t, ctx->d_sel_n));
    double t_next;
    int n_act;
    if (ctx->h_sel_t) {  // the selection wrote its mapped copies: read them once the stream is done
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        t_next = *(volatile double *)ctx->h_sel_t;
        n_act = *(volatile int32_t *)ctx->h_sel_n;
    } else {
        CK(ctx, cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaMemcpyAsync(ctx->h_count, ctx->d_count, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        t_next = ctx->h_scal[0];
        n_act = *ctx->h_count;
    }
    if (t_now)
        *t_now = t_next;
    if (n_active)
        *n_active = n_act;
    if (n_act == 0)
        return KIRIN_OK;
    ctx->pred_mode = 1;
    ctx->pred_t = t_next;
    ctx->images_dirty = true;
    int rc = ensure_images(ctx);
    if (rc)
        return rc;
    rc = run_force(ctx, n_act, ctx->d_ilist, n, MODE_ACC_JERK_POT, ctx->d_acc, ctx->d_jerk, ctx->d_pot);
    if (rc)
        return rc;
    CK(ctx, launch_hermite_correct(n_act, ctx->d_ilist, t_next, ctx->eta, ctx->dt_min, ctx->dt_max, 1,
                                   ctx->xp, ctx->vp, ctx->d_acc, ctx->d_jerk, ctx->bx, ctx->bv, ctx->ba,
                                   ctx->bj, ctx->bt, ctx->bdt, ctx->stream));
    ctx->images_dirty = true;  // base state moved
    ctx->pending = false;
    return KIRIN_OK;
}

int kirin_hermite_run(kirin_ctx *ctx, double t_end, int64_t max_steps, int64_t *n_steps, double *n_pairs)
{
    if (!ctx || !isfinite(t_end))
        return KIRIN_EINVAL;
    if (!ctx->hermite_ready)
        return set_msg(ctx, KIRIN_ESTATE, "hermite_run: call kirin_hermite_init first");
    DeviceGuard dg0(ctx->device);
    TraceScope ts(ctx, "kirin_hermite_run");
    if (ctx->device_loop && ctx->n_parts == 1)  // a partitioned context exchanges from the host each step
        return hermite_run_device(ctx, t_end, max_steps, n_steps, n_pairs);
    int64_t steps = 0;
    double pairs = 0.0, t_last = 0.0;
    while (max_steps <= 0 || steps < max_steps) {
        double t_now = 0;
        int64_t n_act = 0;
        const int rc = kirin_hermite_block_step(ctx, t_end, &t_now, &n_act);
        if (rc)
            return rc;
        if (n_act == 0)
            break;
        if (steps > 0 && !(t_now > t_last))
            return set_msg(ctx, KIRIN_ESTATE, "block time stopped advancing (t + dt == t in FP64)");
        t_last = t_now;
        ++steps;
        pairs += (double)n_act * (double)ctx->n_j;
    }
    if (n_steps)
        *n_steps = steps;
    if (n_pairs)
        *n_pairs = pairs;
    DeviceGuard dg(ctx->device);
    return read_device_errors(ctx);
}

int kirin_set_tracing(kirin_ctx *ctx, int32_t enable)
{
    if (!ctx)
        return KIRIN_EINVAL;
    DeviceGuard dg(ctx->device);
    const cudaError_t err = trace_fold(ctx, false);  // pending pairs of the old setting are dropped
    ctx->trace_calls = 0;
    ctx->trace_ms = 0.0;
    ctx->tracing = enable != 0;
    if (err != cudaSuccess) {
        cudaGetLastError();
        return set_msg(ctx, KIRIN_ECUDA, "set_tracing: %s", cudaGetErrorString(err));
    }
    return KIRIN_OK;
}

int kirin_get_trace(kirin_ctx *ctx, int64_t *n_calls, double *device_ms)
{
    if (!ctx || !n_calls || !device_ms)
        return KIRIN_EINVAL;
    DeviceGuard dg(ctx->device);
    const cudaError_t err = trace_fold(ctx, true);
    *n_calls = ctx->trace_calls;
    *device_ms = ctx->trace_ms;
    if (err != cudaSuccess) {
        cudaGetLastError();
        return set_msg(ctx, KIRIN_ECUDA, "get_trace: %s", cudaGetErrorString(err));
    }
    return KIRIN_OK;
}

int kirin_set_shared_persistent(kirin_ctx *ctx, int32_t enable)
{
    if (!ctx)
        return KIRIN_EINVAL;
    ctx->shared_persistent = enable != 0;
    return KIRIN_OK;
}

int kirin_get_shared_persistent(kirin_ctx *ctx, int32_t *active)
{
    if (!ctx || !active)
        return KIRIN_EINVAL;
    DeviceGuard dg(ctx->device);
    *active = shared_steps_on(ctx) ? 1 : 0;
    return KIRIN_OK;
}

int kirin_set_device_loop(kirin_ctx *ctx, int32_t enable)
{
    if (!ctx)
        return KIRIN_EINVAL;
    ctx->device_loop = enable != 0;
    return KIRIN_OK;
}

int kirin_hermite_shared_step(kirin_ctx *ctx, double dt) { return kirin_hermite_shared_run(ctx, dt, 1); }

int kirin_hermite_shared_run(kirin_ctx *ctx, double dt, int64_t n_steps)
{
    if (!ctx || !(dt > 0) || !isfinite(dt) || n_steps < 0)
        return KIRIN_EINVAL;
    if (!ctx->hermite_ready)
        return set_msg(ctx, KIRIN_ESTATE, "hermite_shared_run: call kirin_hermite_init first");
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_hermite_shared_run");
    const int n = (int)ctx->n_j;
    if (shared_steps_on(ctx) && n_steps > 0 && n_steps <= INT32_MAX) {
        // the whole run in one cooperative launch (small systems, mixed precision)
        const int rc = shared_launch(ctx, ctx->t_shared, dt, n_steps, 0, ctx->dt_min, ctx->dt_max);
        if (rc != KIRIN_OK)
            return rc;
        double t = ctx->t_shared;
        for (int64_t s = 0; s < n_steps; ++s)  // the kernel's time arithmetic, step by step
            t = t + dt;
        ctx->t_shared = t;
        ctx->pred_mode = 1;
        ctx->pred_t = t;
        ctx->images_dirty = true;
        ctx->pending = false;
        return read_shared_errors(ctx);
    }
    for (int64_t s = 0; s < n_steps; ++s) {  // enqueued back to back; one synchronisation at the end
        const double t_next = ctx->t_shared + dt;
        ctx->pred_mode = 1;
        ctx->pred_t = t_next;
        ctx->images_dirty = true;
        int rc = ensure_images(ctx);
        if (rc)
            return rc;
        rc = run_force(ctx, n, nullptr, n, MODE_ACC_JERK_POT, ctx->d_acc, ctx->d_jerk, ctx->d_pot);
        if (rc)
            return rc;
        CK(ctx, launch_hermite_correct(n, nullptr, t_next, ctx->eta, ctx->dt_min, ctx->dt_max, 0, ctx->xp,
                                       ctx->vp, ctx->d_acc, ctx->d_jerk, ctx->bx, ctx->bv, ctx->ba, ctx->bj,
                                       ctx->bt, ctx->bdt, ctx->stream));
        ctx->t_shared = t_next;
        ctx->images_dirty = true;
    }
    ctx->pending = false;
    return read_device_errors(ctx);
}

int kirin_get_state(kirin_ctx *ctx, double *x, double *v, double *a, double *jerk, double *t, double *dt)
{
    if (!ctx)
        return KIRIN_EINVAL;
    DeviceGuard dg(ctx->device);
    const size_t n = (size_t)ctx->n_j;
    cudaStream_t s = ctx->stream;
    if (x)
        CK(ctx, cudaMemcpyAsync(x, ctx->bx, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (v)
        CK(ctx, cudaMemcpyAsync(v, ctx->bv, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (a)
        CK(ctx, cudaMemcpyAsync(a, ctx->ba, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (jerk)
        CK(ctx, cudaMemcpyAsync(jerk, ctx->bj, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (t)
        CK(ctx, cudaMemcpyAsync(t, ctx->bt, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (dt)
        CK(ctx, cudaMemcpyAsync(dt, ctx->bdt, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    return read_device_errors(ctx);
}

int kirin_set_state(kirin_ctx *ctx, int64_t n, const double *m, const double *x, const double *v, const double *a,
                    const double *jerk, const double *t, const double *dt, double eta, double dt_min, double dt_max)
{
    if (!ctx || !m || !x || !v || !a || !jerk || !t || !dt || n < 1 || n > ctx->n_max || !(eta > 0) ||
        !(dt_min > 0) || !(dt_max >= dt_min))
        return set_msg(ctx, KIRIN_EINVAL, "set_state: bad argument");
    if (!all_finite(dt, n))
        return set_msg(ctx, KIRIN_ENONFINITE, "set_state: NaN or Inf in dt");
    int rc = kirin_set_j_particles(ctx, 0, n, m, x, v, a, jerk, t);
    if (rc)
        return rc;
    DeviceGuard dg(ctx->device);
    CK(ctx, cudaMemcpyAsync(ctx->bdt, dt, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->n_j = n;
    ctx->eta = eta;
    ctx->dt_min = dt_min;
    ctx->dt_max = dt_max;
    ctx->t_shared = t[0];
    ctx->hermite_ready = true;
    return KIRIN_OK;
}

int kirin_selftest_wait_timeout(kirin_ctx *ctx, int64_t limit_ns)
{
    if (!ctx || limit_ns < 0)
        return KIRIN_EINVAL;
    DeviceGuard dg(ctx->device);
    CK(ctx, launch_wait_selftest((unsigned long long)limit_ns, err_word(ctx), ctx->stream));
    return read_device_errors(ctx);
}

int kirin_selftest_arrival_timeout(kirin_ctx *ctx, int64_t limit_ns)
{
    if (!ctx || limit_ns < 0)
        return KIRIN_EINVAL;
    DeviceGuard dg(ctx->device);
    CK(ctx, launch_arrival_selftest((unsigned long long)limit_ns, err_word(ctx), ctx->stream));
    return read_device_errors(ctx);
}

// ---- device particle sets -------------------------------------------------------

int kirin_accel_dev(kirin_ctx *ctx, int64_t n, const double *m, const double *x, double *acc, double *pot)
{
    if (!ctx || !m || !x || n < 0 || n > ctx->n_max)
        return set_msg(ctx, KIRIN_EINVAL, "accel_dev: bad size or NULL array");
    if (n == 0)
        return KIRIN_OK;
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_accel_dev");
    const int64_t n_pad = round_up(n, TILE_J);
    CK(ctx, launch_pack_xm((int)n, (int)n_pad, m, x, img_m(ctx), img_d(ctx), err_word(ctx), ctx->stream));
    ctx->images_dirty = true;  // the images no longer show the context's particles
    return run_force(ctx, n, nullptr, (int)n, MODE_ACC_POT, acc, nullptr, pot);
}

int kirin_accel_adjoint_dev(kirin_ctx *ctx, int64_t n, const double *m, const double *x, const double *g,
                            double *gx, double *gm)
{
    if (!ctx || !m || !x || !g || n < 0 || n > ctx->n_max)
        return set_msg(ctx, KIRIN_EINVAL, "accel_adjoint_dev: bad size or NULL array");
    if (n == 0)
        return KIRIN_OK;
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_accel_adjoint_dev");
    const int64_t n_pad = round_up(n, TILE_J);
    // images of (x, m) with g in the velocity slots
    CK(ctx, launch_predict_pack((int)n, (int)n_pad, 0.0, 0, m, x, g, nullptr, nullptr, nullptr, nullptr,
                                nullptr, img_m(ctx), img_d(ctx), err_word(ctx), ctx->stream));
    ctx->images_dirty = true;
    return run_force(ctx, n, nullptr, (int)n, MODE_ADJOINT, nullptr, gx, gm);
}

// ---- leapfrog on device arrays and its discrete adjoint -------------------------

int kirin_leapfrog_dev(kirin_ctx *ctx, int64_t n, const double *m, double *x, double *v, double *acc, double dt,
                       int32_t n_steps, int32_t acc_valid, double *x_hist)
{
    if (!ctx || !m || !x || !v || !acc || n < 0 || n > ctx->n_max || n_steps < 0 || !isfinite(dt))
        return set_msg(ctx, KIRIN_EINVAL, "leapfrog_dev: bad argument");
    if (n == 0)
        return KIRIN_OK;
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_leapfrog_dev");
    const int nn = (int)n;
    const int64_t n_pad = round_up(n, TILE_J);
    const double h = 0.5 * dt;
    auto accel = [&]() -> int {
        CK(ctx, launch_pack_xm(nn, (int)n_pad, m, x, img_m(ctx), img_d(ctx), err_word(ctx), ctx->stream));
        return run_force(ctx, n, nullptr, nn, MODE_ACC_POT, acc, nullptr, nullptr);
    };
    ctx->images_dirty = true;
    if (!acc_valid) {
        const int rc = accel();
        if (rc)
            return rc;
    }
    if (x_hist)
        CK(ctx, launch_copy(3 * nn, x, x_hist, ctx->stream));
    for (int s = 0; s < n_steps; ++s) {
        CK(ctx, launch_lf_kick_drift(nn, h, dt, acc, v, x, x_hist ? x_hist + 3 * (size_t)n * (s + 1) : nullptr,
                                     ctx->stream));
        const int rc = accel();
        if (rc)
            return rc;
        CK(ctx, launch_axpy(3 * nn, h, acc, v, ctx->stream));
    }
    return KIRIN_OK;
}

int kirin_leapfrog_adjoint_dev(kirin_ctx *ctx, int64_t n, const double *m, const double *x_hist, int32_t n_steps,
                               double dt, double *lx, double *lv, double *lm, int32_t flags)
{
    if (!ctx || !m || !x_hist || !lx || !lv || !lm || n < 0 || n > ctx->n_max || n_steps < 0 || !isfinite(dt))
        return set_msg(ctx, KIRIN_EINVAL, "leapfrog_adjoint_dev: bad argument");
    if (n == 0)
        return KIRIN_OK;
    DeviceGuard dg(ctx->device);
    TraceScope ts(ctx, "kirin_leapfrog_adjoint_dev");
    const int nn = (int)n;
    const int64_t n_pad = round_up(n, TILE_J);
    const double h = 0.5 * dt;
    const bool at_end = flags & 1, at_start = flags & 2;
    ctx->images_dirty = true;
    // lx += J(x)^T (c lv), lm += M(x)^T (c lv)
    auto adjoint_at = [&](const double *xk, double c) -> int {
        CK(ctx, launch_pack_adjoint(nn, (int)n_pad, m, xk, lv, c, img_m(ctx), img_d(ctx), err_word(ctx), ctx->stream));
        return run_force(ctx, n, nullptr, nn, MODE_ADJOINT, nullptr, lx, lm, 1);
    };
    for (int k = n_steps - 1; k >= 0; --k) {
        // the closing half-kick of step k and the opening half-kick of step k + 1
        // both act at x_{k+1}: one call with the summed weight
        const double c = (k == n_steps - 1 && at_end) ? h : dt;
        int rc = adjoint_at(x_hist + 3 * (size_t)n * (k + 1), c);
        if (rc)
            return rc;
        CK(ctx, launch_axpy(3 * nn, dt, lx, lv, ctx->stream));  // drift: lv_h += dt lx
    }
    if (at_start)
        return adjoint_at(x_hist, h);
    return KIRIN_OK;
}

}  // extern "C"
