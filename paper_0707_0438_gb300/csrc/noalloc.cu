// Allocation-free force evaluation: kirin_forces_noalloc.
//
// Some callers cannot allocate GPU memory at the moment they need forces:
// code running inside another framework's memory pool that has reserved the
// whole device, callbacks that must not call cudaMalloc/cudaFree (they
// synchronise the device and can deadlock against the caller's own streams),
// or embedded hosts that forbid allocation after start-up.  A libkirin
// context allocates its buffers in kirin_init, so this entry point does the
// same mixed-precision evaluation as kirin_compute_forces_dev without any
// context: the j image and the j-split partial sums live in one fixed,
// file-scope device array that every GPU loading the library holds until the
// process exits.
//
// The paper has no counterpart; its kernel and sums are those of
// force_mixed.cu, only the scratch memory differs.
#include <cuda_runtime.h>

#include <math.h>

#include <algorithm>
#include <mutex>

#include "kirin_internal.cuh"

using namespace kirin;

namespace {

// Limits of the static scratch (documented in kirin.h).
constexpr int64_t NOALLOC_MAX_N = 32768;                                  // particles
constexpr size_t IMAGE_BYTES = (size_t)NOALLOC_MAX_N * sizeof(JMixed);    // 2.5 MiB
constexpr size_t PARTIAL_DOUBLES = (size_t)1 << 19;                       // 4 MiB of split partials
constexpr size_t SCRATCH_BYTES = IMAGE_BYTES + PARTIAL_DOUBLES * sizeof(double) + 256;
static_assert(NOALLOC_MAX_N % TILE_J == 0, "the image holds whole tiles");

// The scratch itself: [j image | split partials | error word].  In host code
// this symbol is only a host-side stand-in; its device address comes from
// cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;

struct DeviceSetup {
    std::mutex mu;
    bool done = false;  // set only once the set-up has succeeded
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int nsm = 0;
    int occ[4] = {0, 0, 0, 0};  // CTAs per SM for 1, 2, 4, 8 j-groups (no guard)
    int occ_guard[4] = {0, 0, 0, 0};
};
DeviceSetup g_setup[MAX_DEVICES];

// Once per device, with that device current: the scratch address and the
// numbers the launch shape depends on.  A set-up that fails (for example one
// attempted while the stream is being captured) is not remembered: the next
// call on that device tries again.
cudaError_t setup_device(DeviceSetup &s, int dev)
{
    std::lock_guard<std::mutex> lock(s.mu);
    if (s.done)
        return cudaSuccess;
    void *p = nullptr;
    cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (rc == cudaSuccess)
        rc = cudaDeviceGetAttribute(&s.nsm, cudaDevAttrMultiProcessorCount, dev);
    if (rc != cudaSuccess) {
        cudaGetLastError();  // clear the error the failed attempt left behind
        return rc;
    }
    for (int k = 0; k < 4; ++k) {
        s.occ[k] = std::max(1, force_mixed_ctas_per_sm(1 << k, false, MODE_ACC_JERK_POT));
        s.occ_guard[k] = std::max(1, force_mixed_ctas_per_sm(1 << k, true, MODE_ACC_JERK_POT));
    }
    s.scratch = static_cast<unsigned char *>(p);
    s.done = true;
    return cudaSuccess;
}

// Same trade-off as the context path (waves of CTAs against per-CTA work and
// split overhead), restricted to what the static partial buffer holds.
Shape pick_shape(const DeviceSetup &s, int64_t n_i, int ntiles, bool guard)
{
    Shape best{1, 1};
    double best_cost = 1e300;
    for (int k = 0; k < 4; ++k) {
        const int groups = 1 << k;
        const int i_cta = MIX_I_PER_THREAD * FORCE_THREADS / groups;
        const int64_t iblocks = (n_i + i_cta - 1) / i_cta;
        const double slots = (double)s.nsm * (guard ? s.occ_guard[k] : s.occ[k]);
        for (int ns = 1; ns <= std::min(ntiles, MAX_SPLIT); ++ns) {
            if (ns > 1 && (size_t)ns * 7 * (size_t)(iblocks * i_cta) > PARTIAL_DOUBLES)
                break;
            const double waves = ceil((double)iblocks * ns / slots);
            double cost = waves * (ceil((double)ntiles / ns) + 2.0) * TILE_J * (double)i_cta;
            if (ns > 1)
                cost += (double)ns * 7 * iblocks * i_cta * 4.0 / slots + 5.0e3 * TILE_J;
            if (cost < best_cost * 0.999) {
                best_cost = cost;
                best = Shape{groups, ns};
            }
        }
    }
    return best;
}

}  // namespace

extern "C" int kirin_forces_noalloc(int64_t n, const double *m, const double *x, const double *v, int64_t n_i,
                                    const int32_t *i_list, double eps, double G, double r_min, double *acc,
                                    double *jerk, double *pot, unsigned *status, void *stream)
{
    if (n < 1 || n > NOALLOC_MAX_N || !m || !x || !v)
        return KIRIN_EINVAL;
    if (!i_list)
        n_i = n;
    if (n_i < 0 || n_i > NOALLOC_MAX_N)
        return KIRIN_EINVAL;
    if (!(eps >= 0.0) || !isfinite(eps) || !isfinite(G) || !(r_min >= 0.0) || !isfinite(r_min))
        return KIRIN_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return KIRIN_ECUDA;
    }
    DeviceSetup &s = g_setup[dev];
    if (setup_device(s, dev) != cudaSuccess)
        return KIRIN_ECUDA;

    cudaStream_t st = (cudaStream_t)stream;
    JMixed *image = reinterpret_cast<JMixed *>(s.scratch);
    double *partial = reinterpret_cast<double *>(s.scratch + IMAGE_BYTES);
    unsigned *err = status ? status : reinterpret_cast<unsigned *>(s.scratch + IMAGE_BYTES +
                                                                   PARTIAL_DOUBLES * sizeof(double));
    // error bits accumulate with atomicOr: start from zero on every call
    if (cudaMemsetAsync(err, 0, sizeof(unsigned), st) != cudaSuccess)
        return KIRIN_ECUDA;
    if (n_i == 0)
        return KIRIN_OK;
    const int ntiles = (int)((n + TILE_J - 1) / TILE_J);
    // the pack writes every record of the tiles used, padding included, so
    // nothing left by an earlier call is read
    if (launch_predict_pack((int)n, ntiles * TILE_J, 0.0, 0, m, x, v, nullptr, nullptr, nullptr, nullptr, nullptr,
                            image, nullptr, err, st) != cudaSuccess)
        return KIRIN_ECUDA;
    const bool guard = eps == 0.0 || r_min > 0.0;
    const Shape sh = pick_shape(s, n_i, ntiles, guard);
    ForceArgs a{};
    a.jimg = image;
    a.ilist = i_list;
    a.n_i = (int)n_i;
    a.n_j = (int)n;
    a.ntiles = ntiles;
    a.n_split = sh.n_split;
    a.eps2 = eps * eps;
    a.rmin2 = r_min * r_min;
    a.G = G;
    a.acc = acc;
    a.jerk = jerk;
    a.pot = pot;
    a.partial = sh.n_split > 1 ? partial : nullptr;
    const int i_cta = MIX_I_PER_THREAD * FORCE_THREADS / sh.groups;
    a.n_i_pad = (int)((n_i + i_cta - 1) / i_cta * i_cta);
    a.accumulate = 0;
    a.err = err;
    a.nq = 7;
    if (launch_force_mixed(a, sh, guard, MODE_ACC_JERK_POT, st) != cudaSuccess)
        return KIRIN_ECUDA;
    if (sh.n_split > 1 && launch_reduce_splits(a, st) != cudaSuccess)
        return KIRIN_ECUDA;
    return KIRIN_OK;
}
