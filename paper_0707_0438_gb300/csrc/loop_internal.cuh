// Device-driven block-step loop: the run state shared by the host runtime
// and the two step kernels (Sect. 3.1 block time-steps, with the predictor,
// corrector and scheduler on the device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kirin_internal.cuh"

namespace kirin {

// Parameters and counters of a device-driven block-step run; the host
// writes a fresh copy before every run.
struct RunState {
    double t_end;                   // end time of the run
    long long max_steps;            // step limit, 0 = unbounded
    long long steps;                // blocks selected so far
    double pairs;                   // sum over those blocks of n_active * n_j
    double t_last;                  // time of the last block selected
    long long pending;              // size of the block forced but not yet corrected
    unsigned long long minw[2];     // atomic minimum of the keys of t_i + dt_i, alternating by step parity
    unsigned long long list_done;   // select kernel: (CTAs done) << 32 | members listed so far
};

constexpr int MAX_SEL_CLASSES = 16;

// Everything the two kernels of a device-driven block step touch.  Both run
// the same grid; CTA b owns the particles [b * chunk, (b + 1) * chunk).
struct StepArgs {
    int n, n_pad;
    const double *bm;
    double *bx, *bv, *ba, *bj, *bt, *bdt;
    double *xp, *vp;
    JMixed *jm;
    JF64 *jd;
    const double *acc, *jerk;  // forces of the pending block, in list order
    int32_t *ilist;            // the pending block in, the next block out
    int32_t *chunk_off;        // per CTA: where its members start in ilist
    double eta, dt_min, dt_max;
    RunState *run;
    int32_t *count_out;        // size of the next block (read by the force launches)
    double *t_next_out;        // its time
    unsigned *err;
    cudaGraphConditionalHandle loop, branch;
    int n_classes;
    int32_t class_max[MAX_SEL_CLASSES];
    int n_j;
};

// One block step of a device-driven run in two kernels over `ctas` CTAs.
// The first corrects the pending block (Hermite corrector and new steps),
// each CTA the members among its own particles, and takes the minimum of
// t_i + dt_i over them.  The second, if t_next <= t_end and fewer than
// max_steps blocks were taken, predicts every j to t_next and lists the
// block: each CTA its own members in index order, at a range reserved with
// one atomic add (so the order of the CTAs' ranges varies; each particle's
// force and correction do not depend on its place in the list).  The CTA
// that reserves last publishes the block and sets the graph's WHILE
// condition (a block was selected) and SWITCH value (the first c with
// class_max[c] >= block size; n_classes when there is none).  A block time
// that does not advance stops the loop with ERR_STALL.
cudaError_t launch_block_step(const StepArgs &a, int ctas, cudaStream_t st);
constexpr int STEP_CTAS_PER_SM = 2;

// ---- small active blocks ----------------------------------------------------
//
// A block of at most SMALL_MAX i-particles against N j is a few hundred
// thousand pair interactions: launch and latency, not arithmetic, set its
// time.  The small-block force spreads the j tiles over G CTAs (one chunk
// each; a lane per member, the warps over the chunk's j) and leaves each
// chunk's double-single sums in a scratch; then one CTA per member adds its
// sums over the chunks in one round of loads and a fixed tree.  The
// small-step kernel runs whole block steps of small blocks in one cooperative
// launch: chunk sums, a grid barrier, the member CTAs' sums and correctors, a
// barrier, the selection and prediction of the next block, a barrier, until a
// larger block or the end of the run comes up.
constexpr int SMALL_MAX = 32;

// Scratch of the small-block force for a grid of `chunks` CTAs.
struct SmallScratch {
    float2 *part;  // [chunks][7][SMALL_MAX] (hi, lo) sums of each chunk
    int chunks;
};

struct SmallForceArgs {
    const JMixed *jimg;
    const int32_t *ilist;    // n_i entries (device); nullptr = identity
    int n_i;
    const int32_t *n_i_dev;  // if set, the block size is read here at launch
    int n_j;
    int tile0, ntiles;       // j tiles summed: [tile0, tile0 + ntiles)
    float eps2, rmin2;
    double G;
    double *acc, *jerk, *pot;  // outputs in i-list order; any may be null
    unsigned *err;
    SmallScratch scr;
};
// One small-block force (n_i <= SMALL_MAX): the chunk kernel over scr.chunks CTAs, then the member kernel.
cudaError_t launch_force_small(const SmallForceArgs &a, bool guard, cudaStream_t st);

// The small-step kernel: as long as the selected block has at most SMALL_MAX
// members, force, correct and select in one cooperative launch over `ctas`
// CTAs (the step kernels' grid, so the list layout is theirs).
struct SmallStepArgs {
    StepArgs st;
    SmallScratch scr;
    unsigned *bar;  // grid barrier: [0] arrivals, [1] generation
    int tile0, ntiles;
    float eps2, rmin2;
    double G;
};
cudaError_t launch_small_steps(const SmallStepArgs &a, bool guard, int ctas, cudaStream_t st);
int small_steps_ctas_per_sm(bool guard);

}  // namespace kirin
