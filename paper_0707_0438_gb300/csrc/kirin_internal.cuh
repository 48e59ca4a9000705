// Internal declarations shared by the libkirin translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kirin.h"

namespace kirin {

// ---- j-particle images in HBM ---------------------------------------------
//
// Mixed precision: one 80-byte record per j, every scalar stored twice so
// that a broadcast LDS.128 yields ready-made {v, v} operands for the packed
// FP32x2 instructions (the two lanes hold two different i-particles).
//   q[0] = {xh, xh, yh, yh}   q[1] = {zh, zh, m, m}    q[2] = {xl, xl, yl, yl}
//   q[3] = {zl, zl, vx, vx}   q[4] = {vy, vy, vz, vz}
// with x = xh + xl (double-single: xh = fl32(x), xl = fl32(x - xh)).
struct __align__(16) JMixed {
    float4 q[5];
};
// FP64: {x, y}, {z, m}, {vx, vy}, {vz, 0} as double2 (64 bytes).
struct __align__(16) JF64 {
    double2 q[4];
};

// j tile (shared-memory burst) and pipeline depth of the force kernels
// (overridable at build time for tuning sweeps).
#ifndef KIRIN_TILE_J
#define KIRIN_TILE_J 128
#endif
#ifndef KIRIN_STAGES
#define KIRIN_STAGES 4
#endif
#ifndef KIRIN_MIX_IPAIRS
#define KIRIN_MIX_IPAIRS 1
#endif
constexpr int TILE_J = KIRIN_TILE_J;
constexpr int STAGES = KIRIN_STAGES;
// Mixed kernel: packed FP32x2 i-pairs per thread, hence i-particles per thread.
constexpr int MIX_IPAIRS = KIRIN_MIX_IPAIRS;
constexpr int MIX_I_PER_THREAD = 2 * MIX_IPAIRS;
constexpr int FORCE_THREADS = 256;
constexpr int MAX_SPLIT = 1024;

// Padding particle: zero mass, far away (all its contributions are exact zeros).
constexpr double PAD_POS = 1.0e4;

// Device error bits (ctx->d_err).
enum : unsigned {
    ERR_INDEX = 1u,      // i index outside [0, n_j)
    ERR_TIMEOUT = 2u,    // bounded mbarrier wait gave up
    ERR_DRAIN = 4u,      // in-flight copies did not land after a timeout
    ERR_NONFINITE = 8u,  // NaN / Inf in device-uploaded particle data
    ERR_STALL = 16u,     // block time stopped advancing (t + dt == t in FP64)
};

// Bounded waits: wall-clock limit of one wait, in nanoseconds.
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;

// Launch shape of one force evaluation.
struct Shape {
    int groups;   // j-groups per CTA (1, 2, 4, 8); i per CTA = 2*256/groups (mixed) or 256/groups (fp64);
                  // 0: the tiny-block kernel (mixed, acc+jerk+pot, n_i <= TINY_MAX)
    int n_split;  // CTAs splitting the j range (grid.y; the grid of the tiny-block kernel)
};

// Blocks of at most this many i-particles go to the tiny-block kernel: each
// CTA stages a range of at most TINY_JCHUNK j in shared memory, each warp
// takes one i-particle and its lanes the j.  (At N = 65536 on GB300 it takes
// 7.2 us for one i and 8.5 us for four, against 11.4 us for the best regular
// shape, but loses beyond about 12 i: every further group of 8 i re-stages the
// j range.)
constexpr int TINY_MAX = 8;
constexpr int TINY_JCHUNK = 256;

// i-slots per CTA of a launch shape (the padding unit of the split partials).
inline int shape_i_cta(Shape s, bool mixed)
{
    if (s.groups == 0)
        return TINY_MAX;
    return (mixed ? MIX_I_PER_THREAD : 1) * FORCE_THREADS / s.groups;
}

struct ForceArgs {
    const void *jimg;       // JMixed* or JF64*, padded to a multiple of TILE_J
    const int32_t *ilist;   // device, n_i entries; nullptr = identity
    int n_i;
    int n_j;
    int ntiles;             // j tiles summed: [tile0, tile0 + ntiles) of the padded image
    int tile0;              // first j tile (0 unless the context sums one part of a j partition)
    int n_split;
    double eps2;
    double rmin2;
    double G;
    double *acc;            // final outputs (n_i x 3, n_i x 3, n_i); any may be null
    double *jerk;
    double *pot;
    double *partial;        // [n_split][nq][n_i_pad] when n_split > 1
    int n_i_pad;
    int accumulate;         // 1: add the results to the outputs instead of overwriting them
    unsigned *err;
    int32_t *nn;            // nearest-neighbour mode: index of the nearest j != i (n_i)
    double *nn_r2;          // and its squared distance |d|^2 (n_i); either may be null
    int nq;                 // quantities per i in the partials: 7, or 9 with the neighbour
    const int32_t *n_i_dev; // if set, n_i is read from here at launch (device-driven loops);
                            // the grid then covers an upper bound and the CTAs beyond n_i exit
};

// Final scaling of one of the seven per-i sums and its store (acc and jerk:
// G * sum; pot: -G * sum); shared by the force kernels and the split reduction.
__device__ __forceinline__ void store_final(const ForceArgs &A, int q, int k, double sum)
{
    double *dst;
    double val;
    if (q < 3) {
        dst = A.acc ? A.acc + 3 * (size_t)k + q : nullptr;
        val = A.G * sum;
    } else if (q < 6) {
        dst = A.jerk ? A.jerk + 3 * (size_t)k + (q - 3) : nullptr;
        val = A.G * sum;
    } else {
        dst = A.pot ? A.pot + k : nullptr;
        val = -A.G * sum;
    }
    if (dst)
        *dst = A.accumulate ? *dst + val : val;
}

// Store the nearest neighbour found for output slot k: d2 = |d|^2, j its
// index (-1: none).
__device__ __forceinline__ void store_nn(const ForceArgs &A, int k, double d2, double j)
{
    if (A.nn)
        A.nn[k] = j < 0 ? -1 : (int32_t)j;
    if (A.nn_r2)
        A.nn_r2[k] = j < 0 ? INFINITY : fmax(d2, 0.0);
}

// Lexicographic (r2, j) minimum: the nearer neighbour, the smaller index on ties.
__device__ __forceinline__ void nn_min(double &r2, double &j, double r2b, double jb)
{
    if (jb >= 0 && (j < 0 || r2b < r2 || (r2b == r2 && jb < j))) {
        r2 = r2b;
        j = jb;
    }
}

// What a force launch sums (the seven per-i quantities of ForceArgs):
//  MODE_ACC_JERK_POT: acc, jerk, pot;  MODE_ACC_POT: acc, pot (jerk outputs 0);
//  MODE_ADJOINT: the velocity slots of the j image hold g = dL/da; the jerk
//  outputs receive dL/dx and the pot output dL/dm (acc outputs 0).
//  MODE_NN: as MODE_ACC_JERK_POT, plus the nearest j != i of every i (the
//  neighbour search of Sect. 3.3.1): quantities 7 and 8 of the partials hold
//  its |d|^2 and index, reduced by the lexicographic minimum.
enum { MODE_ACC_JERK_POT = 0, MODE_ACC_POT = 1, MODE_ADJOINT = 2, MODE_NN = 3 };
constexpr int N_MODES = 4;

// Launchers (force_mixed.cu / force_fp64.cu).
cudaError_t launch_force_mixed(const ForceArgs &a, Shape s, bool guard, int mode, cudaStream_t st);
cudaError_t launch_force_fp64(const ForceArgs &a, Shape s, int mode, cudaStream_t st);
int force_mixed_ctas_per_sm(int groups, bool guard, int mode);
int force_fp64_ctas_per_sm(int groups, int mode);

// aux_kernels.cu
cudaError_t launch_reduce_splits(const ForceArgs &a, cudaStream_t st);
cudaError_t launch_predict_pack(int n, int n_pad, double t, int predict, const double *m,
                                const double *x, const double *v, const double *a,
                                const double *jk, const double *t0, double *xp, double *vp,
                                JMixed *jm, JF64 *jd, unsigned *err, cudaStream_t st);
cudaError_t launch_pack_xm(int n, int n_pad, const double *m, const double *x, JMixed *jm,
                           JF64 *jd, unsigned *err, cudaStream_t st);
cudaError_t launch_scatter_state(int first, int n, const double *m, const double *x,
                                 const double *v, const double *a, const double *jk,
                                 const double *t0, double *bm, double *bx, double *bv,
                                 double *ba, double *bj, double *bt0, unsigned *err,
                                 cudaStream_t st);
cudaError_t launch_energy(int n, const double *m, const double *v, const double *pot,
                          double *out2, cudaStream_t st);
cudaError_t launch_hermite_init(int n, double t, const double *acc, const double *jerk,
                                double dt_min, double dt_max, double *ba, double *bj,
                                double *bt, double *bdt, cudaStream_t st);
// counts: ceil(n / 1024) int32 of scratch; minw: one 64-bit word of scratch.
// (t_next_host, count_host: optional mapped host copies of the block's time and size)
cudaError_t launch_block_select(int n, const double *bt, const double *bdt, double t_end, int32_t *ilist,
                                double *t_next_out, int32_t *count_out, unsigned long long *minw,
                                int32_t *counts, cudaStream_t st, double *t_next_host = nullptr,
                                int32_t *count_host = nullptr);
cudaError_t launch_hermite_correct(int n_act, const int32_t *ilist, double t_next, double eta,
                                   double dt_min, double dt_max, int update_dt,
                                   const double *xp, const double *vp, const double *acc,
                                   const double *jerk, double *bx, double *bv, double *ba,
                                   double *bj, double *bt, double *bdt, cudaStream_t st);
cudaError_t launch_lf_kick_drift(int n, double h, double dt, const double *a, double *v, double *x,
                                 double *hist, cudaStream_t st);
cudaError_t launch_axpy(int n, double alpha, const double *x, double *y, cudaStream_t st);
cudaError_t launch_wait_selftest(unsigned long long limit_ns, unsigned *err, cudaStream_t st);
cudaError_t launch_copy(int n, const double *src, double *dst, cudaStream_t st);
cudaError_t launch_pack_adjoint(int n, int n_pad, const double *m, const double *x, const double *lv, double c,
                                JMixed *jm, JF64 *jd, unsigned *err, cudaStream_t st);
// Sum of n_parts consecutive blocks of `count` doubles, part 0 first (the same
// order on every rank), split into acc (3 n_i), jerk (3 n_i) and pot (n_i);
// count = 7 n_i; any output may be null.
cudaError_t launch_sum_parts(int n_parts, int64_t n_i, const double *parts, double *acc, double *jerk,
                             double *pot, cudaStream_t st);

}  // namespace kirin
