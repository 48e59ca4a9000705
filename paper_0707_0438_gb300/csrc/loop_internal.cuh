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

// Shared-step Hermite runs of at most SH_MAX_N particles in one cooperative
// launch (shared_steps.cu): one CTA per SM owns a slice of the particles and
// predicts and corrects it; the predicted j image goes through two global
// buffers (even and odd steps), and each CTA counts its arrival on a counter
// that only grows; each CTA waits for all arrivals of the step, copies the
// whole image into its shared memory and sums its own particles against it
// (mixed precision).
constexpr int SH_MAX_N = 8192;
struct SharedStepArgs {
    int n, n_pad;             // particles; image records (a multiple of TILE_J)
    const double *m;
    double *x, *v, *a, *jerk_b, *t_b, *dt_b;  // FP64 base state, corrected in place
    double *xp, *vp;          // predicted positions and velocities (the corrector's input)
    double *f_acc, *f_jerk, *f_pot;  // force rows of the last evaluation (pot may be null)
    JMixed *img;              // [2][n_pad] predicted j images of even and odd steps
    unsigned *arrivals;       // the arrival counter: each CTA adds n_steps per launch (mod 2^32)
    unsigned arrivals0;       // its value before this launch
    double eps2, rmin2, G;
    double eta, dt_min, dt_max;
    double t0, dt;            // the run starts at t0 and takes n_steps steps of dt
    int n_steps;
    int init;                 // 1: instead, evaluate at t0 and initialise (a, jerk, t, first step);
                              // the CTAs arrive once
    int ctas;                 // CTAs of the launch (all resident: a cooperative launch)
    unsigned *err;
};
// CTAs of a shared-step launch for n particles on the current device (one per SM, at most n), or 0
// when the kernel does not fit.
int shared_steps_grid(int n, bool guard);
cudaError_t launch_shared_steps(const SharedStepArgs &a, bool guard, cudaStream_t st);
// One CTA waits for an arrival that never comes, giving up after limit_ns (sets ERR_TIMEOUT).
cudaError_t launch_arrival_selftest(unsigned long long limit_ns, unsigned *err, cudaStream_t st);

}  // namespace kirin
