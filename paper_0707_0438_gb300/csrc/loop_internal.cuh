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

}  // namespace kirin
