/*
 * kirin.h -- C ABI of libkirin: direct O(N^2) softened gravitational
 * acceleration, jerk and potential on one GB300 (sm_103a) GPU.
 *
 * The call sequence mirrors the GRAPE-6 style library of Appendix A
 * (GPU_open / GPU_set_j_particle / GPU_set_ti / GPUcalc_firsthalf /
 * GPUcalc_lasthalf / GPU_close), with the host-side predictor of Sect. 3.1 moved
 * onto the device and j-particles kept resident in HBM between calls.
 *
 * Conventions for every entry point:
 *  - Return 0 (KIRIN_OK) on success, a negative KIRIN_E* code otherwise.
 *    Nothing aborts or exits; kirin_strerror() names a code and
 *    kirin_last_error() gives the context's last detailed message.
 *  - Host arrays are owned by the caller and only read/written during the call
 *    (kirin_get_* calls synchronise first).  Device memory is owned by the
 *    library and released by kirin_finalize / kirin_batch_destroy.
 *  - Vectors are row-major: x[3*k + c] is component c of particle k.
 *  - *_dev entry points take CUDA device pointers, enqueue work on the
 *    context's stream and return without synchronising; errors detected on
 *    the device (bad index, timed-out wait) are reported by the next
 *    kirin_sync / kirin_get_* call on that context.
 *  - Units: any consistent set; G is a parameter (1 in the Henon units of
 *    Sect. 4).
 *  - A context (or a batch) is used by one host thread at a time: calls on
 *    the same context from several threads must be serialised by the caller.
 *    Different contexts share nothing and may be driven concurrently.
 */
#ifndef KIRIN_H
#define KIRIN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KIRIN_OK 0
#define KIRIN_EINVAL (-1)     /* bad argument: NULL, size, index, eps < 0, ... */
#define KIRIN_ENOMEM (-2)     /* device or pinned host allocation failed */
#define KIRIN_ECUDA (-3)      /* a CUDA runtime call failed (see kirin_last_error) */
#define KIRIN_ENONFINITE (-4) /* NaN or Inf in uploaded particle data */
#define KIRIN_ETIMEOUT (-5)   /* a bounded wait inside a kernel gave up */
#define KIRIN_ESTATE (-6)     /* call out of order (e.g. forces before particles) */
#define KIRIN_EEXCHANGE (-7)  /* the j-partition all-gather callback reported a failure */

typedef struct kirin_ctx kirin_ctx;

/* Arithmetic of the pair interaction.
 * KIRIN_MIXED: positions held as double-single (hi + lo float pairs), the
 *   separation formed in that precision and cast to FP32, FP32 pair arithmetic
 *   with the hardware reciprocal square root, per-tile FP32 partial sums
 *   folded into compensated (double-single) accumulators; results in FP64.
 * KIRIN_FP64: every operation in FP64. */
typedef enum { KIRIN_FP64 = 0, KIRIN_MIXED = 1 } kirin_precision;

typedef struct {
    double eps;      /* Plummer softening length, >= 0 (Sect. 3.3.1); s^2 = r^2 + eps^2 */
    double G;        /* gravitational constant */
    double r_min;    /* separation floor: s^2 = max(s^2, r_min^2), 0 = off; with eps = 0
                        a pair at exactly zero separation contributes nothing (Sect. 3.3.1) */
    int32_t prec;    /* kirin_precision */
    int32_t device;  /* CUDA device ordinal */
    void *stream;    /* cudaStream_t to enqueue on; NULL: the context creates its own
                        non-blocking stream; cudaStreamLegacy for the legacy default stream */
} kirin_config;

/* GPU_open (Appendix A).  Creates a context for up to n_max particles on
 * cfg->device and allocates its device buffers (about 160 bytes per particle
 * plus result and split-partial buffers).  *out receives the context.
 * Errors: EINVAL (NULL out/cfg, n_max < 1 or > 2^31 - 256, eps < 0, r_min < 0,
 * unknown precision), ECUDA (no such device), ENOMEM. */
int kirin_init(kirin_ctx **out, int64_t n_max, const kirin_config *cfg);

/* GPU_close (Appendix A).  Synchronises, frees all device and host buffers
 * and the stream the context created.  NULL is accepted. */
int kirin_finalize(kirin_ctx *ctx);

/* GPU_npipes (Appendix A): the capacity and the current launch shape.
 * tile_i = i-particles per CTA, tile_j = j-particles per shared-memory tile
 * for the context's precision.  Any output pointer may be NULL. */
int kirin_query(const kirin_ctx *ctx, int64_t *n_max, int32_t *tile_i, int32_t *tile_j);

/* Change the softening, G, separation floor or precision of an open context. */
int kirin_set_params(kirin_ctx *ctx, double eps, double G, double r_min, int32_t prec);

/* Make the context enqueue on `stream` (a cudaStream_t; NULL = a stream of its own;
 * cudaStreamLegacy = the legacy default stream). */
int kirin_set_stream(kirin_ctx *ctx, void *stream);

/* Launch shape of the force kernel (the configurable "npipes" of GPU_npipes,
 * Appendix A, and the j-split of Sect. 3.2): `groups` j-groups per CTA
 * (1, 2, 4 or 8; a CTA holds 512 / groups i-particles in mixed precision,
 * 256 / groups in FP64) and `n_split` CTAs sharing the j range (1..1024,
 * reduced on the device).  groups = n_split = 0 restores the automatic choice
 * (a cost model over waves of CTAs).  Errors: EINVAL. */
int kirin_set_launch(kirin_ctx *ctx, int32_t groups, int32_t n_split);

/* A tuned shape table (the paper wishes CUDA picked threads and bundles by
 * itself, Sect. 5): entry k gives the (groups, n_split) of full force calls
 * (acc, jerk, pot) with n_i <= n_i_max[k], for the context's current
 * precision; n_i_max ascending, at most 64 entries; calls beyond the last
 * entry use the cost model.  n_entries = 0 clears the table.  A fixed shape
 * (kirin_set_launch) takes precedence.  Errors: EINVAL. */
int kirin_set_launch_table(kirin_ctx *ctx, int32_t n_entries, const int64_t *n_i_max,
                           const int32_t *groups, const int32_t *n_split);

/* The kinds of force call that each have their own launch table: the full
 * evaluation (acc, jerk, pot), acceleration and potential only (the leapfrog
 * and kirin_accel_dev), and the adjoint (kirin_accel_adjoint_dev and the
 * reverse leapfrog).  Their pair costs differ (about 33, 19 and 40 FP32
 * operations), so do their best shapes. */
typedef enum { KIRIN_CALL_FORCES = 0, KIRIN_CALL_ACC_POT = 1, KIRIN_CALL_ADJOINT = 2 } kirin_call_kind;

/* kirin_set_launch_table / kirin_get_launch for one kind of call.
 * Errors: EINVAL (unknown kind, bad entries). */
int kirin_set_launch_table_for(kirin_ctx *ctx, int32_t kind, int32_t n_entries, const int64_t *n_i_max,
                               const int32_t *groups, const int32_t *n_split);
int kirin_get_launch_for(kirin_ctx *ctx, int32_t kind, int64_t n_i, int32_t *groups, int32_t *n_split);

/* The shape that a force call for n_i i-particles would use now.  groups = 0
 * names the tiny-block kernel, which serves automatic mixed-precision calls
 * with n_i <= 8 (and n_j <= 512 x the SM count): n_split CTAs each stage a
 * range of j in shared memory and give every i a warp. */
int kirin_get_launch(kirin_ctx *ctx, int64_t n_i, int32_t *groups, int32_t *n_split);

/* GPU_set_j_particle (Appendix A), in bulk: particles [first, first + n) get
 * mass m[k], position x[3k..3k+2], velocity v[3k..], and for the predictor
 * acceleration a, jerk and their time t0 (each of a, jerk, t0 may be NULL:
 * zeros).  The number of j-particles becomes max(previous, first + n).
 * The positions used by the force are the given ones until kirin_predict.
 * Host arrays, copied before return.
 * Errors: EINVAL (range outside [0, n_max), NULL m/x/v), ENONFINITE. */
int kirin_set_j_particles(kirin_ctx *ctx, int64_t first, int64_t n, const double *m,
                          const double *x, const double *v, const double *a,
                          const double *jerk, const double *t0);

/* Same as kirin_set_j_particles with device arrays (FP64, same layouts);
 * enqueued on the context's stream.  Non-finite values are reported as
 * ENONFINITE by the next kirin_sync / kirin_get_*. */
int kirin_set_j_particles_dev(kirin_ctx *ctx, int64_t first, int64_t n, const double *m,
                              const double *x, const double *v, const double *a,
                              const double *jerk, const double *t0);

/* Shrink or grow the number of j-particles (<= the highest index ever set + 1). */
int kirin_set_nj(kirin_ctx *ctx, int64_t n_j);

/* GPU_set_ti (Appendix A; Sect. 3.1 does it on the host, here it runs on the
 * device in FP64): predict every j-particle to time t,
 *   x_p = x + v dt + a dt^2/2 + jerk dt^3/6,  v_p = v + a dt + jerk dt^2/2,
 * dt = t - t0_j, and use (x_p, v_p) for subsequent force calls.
 * Errors: ESTATE (no particles). */
int kirin_predict(kirin_ctx *ctx, double t);

/* GPUcalc_firsthalf (Appendix A): start the evaluation, for the n_i
 * i-particles listed in i_list (indices into the j set; NULL = all j in
 * order, n_i ignored), of
 *   a_i    =  G sum_{j != i} m_j d_ij / s^3
 *   jerk_i =  G sum_{j != i} m_j [ w_ij / s^3 - 3 (d_ij . w_ij) d_ij / s^5 ]
 *   phi_i  = -G sum_{j != i} m_j / s
 * with d_ij = x_j - x_i, w_ij = v_j - v_i, s^2 = |d_ij|^2 + eps^2 (Sect. 2
 * Eq. 1 with the attractive sign, Sect. 3 and Sect. 3.1).  Asynchronous;
 * the host i_list is copied before return.  Small active blocks are split
 * over j across thread groups and CTAs and reduced on the device (Sect. 3.2).
 * Errors: EINVAL (n_i < 0 or > n_max, index outside [0, n_j)), ESTATE. */
int kirin_compute_forces(kirin_ctx *ctx, int64_t n_i, const int32_t *i_list);

/* GPUcalc_lasthalf (Appendix A): wait for the last kirin_compute_forces and
 * copy its results, in i_list order, to host arrays acc (n_i x 3),
 * jerk (n_i x 3), pot (n_i).  Any of them may be NULL.
 * Errors: ESTATE (no pending results), ETIMEOUT, ENONFINITE, ECUDA. */
int kirin_get_acc_jerk_pot(kirin_ctx *ctx, double *acc, double *jerk, double *pot);

/* Device twin of compute + get: i_list, acc, jerk, pot are device arrays
 * (int32 n_i; FP64 n_i x 3, n_i x 3, n_i; any output may be NULL).  i_list
 * NULL = all j.  Enqueued on the context's stream, no synchronisation. */
int kirin_compute_forces_dev(kirin_ctx *ctx, int64_t n_i, const int32_t *i_list,
                             double *acc, double *jerk, double *pot);

/* Nearest neighbours (Sect. 3.3.1: the GRAPE hardware returns the nearest
 * neighbour of every i-particle and kira needs it; the search runs inside the
 * force loop).  Device twin of compute + get with, in addition, the index of
 * the nearest j != i (nn, int32, n_i; -1 if there is no other particle) and
 * its squared distance |x_j - x_i|^2 (nn_r2, FP64, n_i), either may be NULL.
 * "Nearest" compares the squared separation |x_j - x_i|^2 itself (softening
 * plays no part) in the precision of the pair arithmetic (FP32 from the
 * double-single separation for KIRIN_MIXED, FP64 for KIRIN_FP64); ties go to
 * the smallest j. */
int kirin_compute_forces_nn_dev(kirin_ctx *ctx, int64_t n_i, const int32_t *i_list, double *acc,
                                double *jerk, double *pot, int32_t *nn, double *nn_r2);

/* Host-pointer path: with enable != 0, every kirin_compute_forces also
 * searches neighbours, and kirin_get_nn copies the last call's results (in
 * i_list order; host arrays of n_i, either may be NULL).  kirin_get_nn
 * synchronises.  Errors: ESTATE (the last compute did not search). */
int kirin_set_nn(kirin_ctx *ctx, int32_t enable);
int kirin_get_nn(kirin_ctx *ctx, int32_t *nn, double *nn_r2);

/* Wait for all work of the context and report device-side errors. */
int kirin_sync(kirin_ctx *ctx);

/* Energies of Eq. 2: kin = sum 1/2 m |v|^2 (v: host n_j x 3, or NULL for the
 * current, possibly predicted, velocities) and pot = 1/2 sum_i m_i phi_i with
 * phi from a full evaluation at the current positions.  Synchronous. */
int kirin_energy(kirin_ctx *ctx, const double *v, double *kin, double *pot);

/* ---- 4th-order Hermite integration on the device (Sect. 3, Sect. 3.1) ----
 * The predictor-corrector scheme the paper runs on the host, executed by
 * device kernels on the context's particles:
 *   corrector  a2 = [-6 (a0 - a1) - dt (4 j0 + 2 j1)] / dt^2,
 *              a3 = [12 (a0 - a1) + 6 dt (j0 + j1)] / dt^3,
 *              x1 = x_p + a2 dt^4/24 + a3 dt^5/120, v1 = v_p + a2 dt^3/6 + a3 dt^4/24
 *   block steps: power-of-two dt in [dt_min, dt_max] from Aarseth's criterion
 *   with accuracy eta; a step shrinks freely and doubles only when the new
 *   time is a multiple of the doubled step. */

/* Evaluate a, jerk for all particles at their current state, set t_i = t and
 * dt_i = 0.01 |a| / |jerk| quantised down to a power of two in [dt_min, dt_max].
 * Where kirin_hermite_shared_run would take its single-launch kernel (see
 * there), the evaluation and the initialisation are one launch of that kernel;
 * otherwise the force kernels and an initialisation kernel.  Errors: EINVAL
 * (eta <= 0, dt_min <= 0, dt_max < dt_min, t not finite), ESTATE (no
 * particles), ETIMEOUT, ENONFINITE. */
int kirin_hermite_init(kirin_ctx *ctx, double t, double eta, double dt_min, double dt_max);

/* One block step: t_next = min_i (t_i + dt_i); if t_next > t_end nothing is
 * done and *n_active = 0.  Otherwise predict all j to t_next, evaluate the
 * block {i : t_i + dt_i = t_next}, correct it and choose its new steps.
 * *t_now receives t_next; *n_active the block size.  Either may be NULL. */
int kirin_hermite_block_step(kirin_ctx *ctx, double t_end, double *t_now, int64_t *n_active);

/* Block steps until no block is due by t_end (then every particle has
 * t_i <= t_end < t_i + dt_i, and all sit at t_end when it is a multiple of
 * dt_max) or max_steps steps were taken (max_steps <= 0: no limit); *n_steps
 * and *n_pairs receive the number of block steps and the sum of
 * n_active * n_j over them (either may be NULL).
 *
 * With the device loop on (the default, see kirin_set_device_loop) the whole
 * run is one CUDA graph launch: a conditional WHILE node repeats two step
 * kernels (correction of the previous block and the minimum of t_i + dt_i;
 * selection of the next block and prediction of all j) and the force
 * evaluation (a SWITCH node picks one of a ladder of launches by block
 * size); the step kernels decide on the device whether another step
 * follows.  The host then waits once per call instead of once per block
 * step.  The graph is built on the first call and rebuilt only when n_j, the
 * parameters or the launch shapes change.  Results are those of the same
 * steps taken one kirin_hermite_block_step at a time, bit for bit when both
 * use the same launch shape (kirin_set_launch); the automatic shapes of the
 * two paths can differ, and so can the summation order.  Errors:
 * KIRIN_ESTATE before kirin_hermite_init, or when a block time does not
 * advance (t + dt rounds to t in FP64; the run stops there); KIRIN_ECUDA if
 * the graph cannot be built or launched. */
int kirin_hermite_run(kirin_ctx *ctx, double t_end, int64_t max_steps, int64_t *n_steps,
                      double *n_pairs);

/* Choose how kirin_hermite_run drives its block steps: enable != 0, one
 * device-driven graph per call (default); 0, one host round trip per step. */
int kirin_set_device_loop(kirin_ctx *ctx, int32_t enable);

/* One shared step of size dt for all particles (no step-size update). */
int kirin_hermite_shared_step(kirin_ctx *ctx, double dt);

/* n_steps shared steps of size dt, with a single synchronisation (and error
 * check) at the end.  A mixed-precision system of at most 8192 particles
 * (no fixed launch shape, no j partition) runs the whole call in one
 * cooperative launch, one CTA per SM: each CTA owns a slice of the particles,
 * corrects it with the step kernels' corrector and predicts it with their
 * FP64 predictor into a global j image (two images, for even and odd steps)
 * and counts its arrival on a counter that only grows; once every CTA has
 * arrived for the step (a bounded wait) each copies the image into its shared
 * memory (above 2048 particles through a ring of tiles) and sums its slice's
 * acc, jerk and pot against all j with the force kernels' pair arithmetic.  Otherwise the steps are the predictor,
 * force and corrector kernels enqueued back to back, the same kernels and
 * results as n_steps calls of kirin_hermite_shared_step.  The two paths sum
 * the j in different orders, so they agree to rounding; each gives the same
 * bits on every call.  kirin_hermite_shared_step is this call with one step.
 * Errors: EINVAL (dt <= 0, n_steps < 0), ESTATE before kirin_hermite_init,
 * ENOMEM (the two images), ETIMEOUT (an arrival or copy wait gave up). */
int kirin_hermite_shared_run(kirin_ctx *ctx, double dt, int64_t n_steps);

/* Tracing (no counterpart in the paper, which times its kernels with host
 * timers and leaves transfers out, Sect. 4.1).  With tracing on, each of these
 * calls, once past its argument checks, opens an NVTX range named after it (seen
 * by an attached profiler; free otherwise) and brackets the stream work it
 * enqueues with two CUDA events: kirin_compute_forces (its i_list copy
 * included), kirin_compute_forces_dev, kirin_compute_forces_nn_dev,
 * kirin_energy, kirin_hermite_init, kirin_hermite_block_step,
 * kirin_hermite_run, kirin_hermite_shared_run, kirin_accel_dev,
 * kirin_accel_adjoint_dev, kirin_leapfrog_dev and kirin_leapfrog_adjoint_dev.
 * A call made inside another (kirin_hermite_run's host-driven steps) is timed
 * as part of the outer one; nothing is timed while the context's stream is
 * being captured into a graph.  Tracing is off by default.
 *
 * kirin_set_tracing: enable != 0 turns it on, 0 off; either way the totals
 * start again from zero (event pairs still pending are waited for and dropped).
 * kirin_get_trace: synchronises on the pending pairs and returns the number of
 * timed calls and their summed device time in milliseconds since the last
 * kirin_set_tracing.  Every 1024 timed calls the pending pairs are folded in
 * the same way, which waits for the stream once.
 * Errors: EINVAL (NULL context or output); ECUDA when an event could not be
 * read (that call is not counted). */
int kirin_set_tracing(kirin_ctx *ctx, int32_t enable);
int kirin_get_trace(kirin_ctx *ctx, int64_t *n_calls, double *device_ms);

/* kirin_set_shared_persistent: enable != 0 (default) lets
 * kirin_hermite_shared_run use the single-launch kernel where it can; 0 keeps
 * the per-kernel steps.  kirin_get_shared_persistent: *active = 1 if the next
 * shared run would use it.  Errors: EINVAL (NULL). */
int kirin_set_shared_persistent(kirin_ctx *ctx, int32_t enable);
int kirin_get_shared_persistent(kirin_ctx *ctx, int32_t *active);

/* Copy the integrator state (host arrays, each may be NULL): x, v, a, jerk
 * (n_j x 3), t and dt (n_j). */
int kirin_get_state(kirin_ctx *ctx, double *x, double *v, double *a, double *jerk, double *t,
                    double *dt);

/* Restore an integrator state saved with kirin_get_state (resume after a
 * checkpoint; no counterpart in the paper): particles 0..n-1 get m, x, v, a,
 * jerk, their times t and steps dt (host arrays, layouts as in
 * kirin_get_state), and the block-step parameters eta, dt_min, dt_max.  The
 * next kirin_hermite_block_step continues exactly where the saved run was.
 * Errors: EINVAL, ENONFINITE. */
int kirin_set_state(kirin_ctx *ctx, int64_t n, const double *m, const double *x, const double *v,
                    const double *a, const double *jerk, const double *t, const double *dt, double eta,
                    double dt_min, double dt_max);

/* Failure-path self-test: one device thread waits on a barrier phase that never
 * completes, with a wait limit of limit_ns, exactly as the force kernels wait on
 * their tile copies; it returns KIRIN_ETIMEOUT (the context stays usable).
 * No counterpart in the paper. */
int kirin_selftest_wait_timeout(kirin_ctx *ctx, int64_t limit_ns);

/* Failure-path self-test of the waits between CTAs of the single-launch shared
 * steps: one CTA waits for an arrival on a counter that nothing increments,
 * with a wait limit of limit_ns, exactly as a CTA waits for the others' step;
 * it returns KIRIN_ETIMEOUT (the context stays usable).  Errors: EINVAL
 * (NULL, limit_ns < 0).  No counterpart in the paper. */
int kirin_selftest_arrival_timeout(kirin_ctx *ctx, int64_t limit_ns);

/* ---- accelerations of device particle sets (leapfrog clients, Sect. 4.3) ----
 * Acceleration (and optionally potential) of all n particles of (m, x), every
 * particle against every other, without jerk: the force-only evaluation the
 * paper's treecode client needs.  m: n, x: n x 3, acc: n x 3, pot: n or NULL,
 * all FP64 device arrays.  Uses the context's eps, G and precision and its
 * j buffers (n <= n_max). */
int kirin_accel_dev(kirin_ctx *ctx, int64_t n, const double *m, const double *x, double *acc,
                    double *pot);

/* Reverse-mode derivative of kirin_accel_dev (no counterpart in the paper):
 * given g = dL/da (n x 3), write dL/dx (n x 3) and dL/dm (n), where
 *   dL/dx_k = G sum_{j != k} K(d_kj) (m_k g_j - m_j g_k),
 *   K(d) = I / s^3 - 3 d d^T / s^5,  d_kj = x_j - x_k,
 *   dL/dm_k = G sum_{i != k} g_i . (x_k - x_i) / s_ik^3.
 * gx or gm may be NULL.  FP64 device arrays; context precision. */
int kirin_accel_adjoint_dev(kirin_ctx *ctx, int64_t n, const double *m, const double *x,
                            const double *g, double *gx, double *gm);

/* Kick-drift-kick leapfrog (Sect. 4.3) on device arrays, in place:
 *   v_h = v + (dt/2) a(x),  x' = x + dt v_h,  v' = v_h + (dt/2) a(x')
 * for n_steps steps; a is the force-only acceleration of kirin_accel_dev.
 * acc (n x 3) holds a(x) on entry when acc_valid != 0 (else it is computed)
 * and a(x) of the final positions on return.  x_hist, if not NULL, receives
 * the n_steps + 1 positions x_0 ... x_{n_steps} ((n_steps + 1) x n x 3).
 * FP64 device arrays; asynchronous. */
int kirin_leapfrog_dev(kirin_ctx *ctx, int64_t n, const double *m, double *x, double *v, double *acc,
                       double dt, int32_t n_steps, int32_t acc_valid, double *x_hist);

/* Reverse sweep of kirin_leapfrog_dev over one segment of n_steps steps whose
 * positions are x_hist ((n_steps + 1) x n x 3): on entry lx, lv hold dL/dx and
 * dL/dv at the segment's last point, on return at its first point; lm (n)
 * accumulates dL/dm.  The two half-kicks that meet at an interior point are
 * applied as one adjoint force call of weight dt.  flags bit 0: the segment
 * ends at the end of the trajectory (its last point gets weight dt/2);
 * bit 1: it starts at the trajectory's start (the first point gets dt/2).
 * A trajectory cut into segments is swept from its last segment to its first.
 * No counterpart in the paper (it is the chain rule of the leapfrog). */
int kirin_leapfrog_adjoint_dev(kirin_ctx *ctx, int64_t n, const double *m, const double *x_hist,
                               int32_t n_steps, double dt, double *lx, double *lv, double *lm,
                               int32_t flags);

/* ---- batched ensembles: many independent clusters in one launch ----
 * Cluster c owns particles [offsets[c], offsets[c+1]) with softening eps[c];
 * clusters do not interact.  State is FP64 on the device; the pair arithmetic
 * is the mixed one. */
typedef struct kirin_batch kirin_batch;

/* offsets: host, n_clusters + 1 entries, offsets[0] = 0, non-decreasing;
 * eps: host, n_clusters entries, >= 0.  Errors: EINVAL, ECUDA, ENOMEM. */
int kirin_batch_create(kirin_batch **out, int32_t n_clusters, const int64_t *offsets,
                       const double *eps, double G, int32_t device, void *stream);
int kirin_batch_destroy(kirin_batch *b);

/* Host FP64 state: m (n_total), x, v (n_total x 3). */
int kirin_batch_set_state(kirin_batch *b, const double *m, const double *x, const double *v);
int kirin_batch_get_state(kirin_batch *b, double *x, double *v);

/* n_steps kick-drift-kick leapfrog steps of size dt for every cluster
 * (Sect. 4.3 integrator); use_graph != 0 captures the steps in a CUDA graph
 * (built on first use for a given (dt, n_steps), then replayed).
 * Asynchronous; kirin_batch_sync waits and reports device errors. */
int kirin_batch_leapfrog(kirin_batch *b, double dt, int32_t n_steps, int32_t use_graph);
int kirin_batch_sync(kirin_batch *b);

/* Accelerations of every particle of every cluster into a host array (n_total x 3). */
int kirin_batch_accel(kirin_batch *b, double *acc);

/* Device-pointer twins of kirin_batch_set_state / _get_state / _accel: the
 * same layouts as CUDA device arrays (FP64), enqueued on the batch's stream
 * without synchronising.  Non-finite uploaded values and device errors are
 * reported by the next kirin_batch_sync (ENONFINITE, ETIMEOUT).
 * Errors here: EINVAL (NULL batch or array), ESTATE (accel before any
 * state), ECUDA (a launch or copy failed to enqueue). */
int kirin_batch_set_state_dev(kirin_batch *b, const double *m, const double *x, const double *v);
int kirin_batch_get_state_dev(kirin_batch *b, double *x, double *v);
int kirin_batch_accel_dev(kirin_batch *b, double *acc);

/* Work decomposition of the batched force launch (the batching is this
 * library's; the paper evaluates one system at a time).  A work item is one
 * cluster's block of 2 * 256 / groups i-particles (groups = 1, 2 or 4 j-groups
 * per CTA: 512, 256 or 128 i) against a range of at most j_tiles tiles of 128
 * j-particles of the same cluster (j_tiles = 0: the whole cluster).  A
 * cluster whose j range is split gets its sums added in split order by the
 * item that finishes last, so results are deterministic for a given
 * decomposition; different decompositions differ by rounding only.  Default:
 * groups 1, j_tiles 0.  Waits for the context's stream, rebuilds the work
 * list and drops the captured leapfrog graph.  Errors: EINVAL (groups not 1,
 * 2 or 4, j_tiles < 0, or the partial sums of the split clusters would exceed
 * 1 GiB), ENOMEM, ECUDA; on error the previous decomposition stays. */
int kirin_batch_set_launch(kirin_batch *b, int32_t groups, int32_t j_tiles);
/* The current decomposition and its number of work items; any pointer may be NULL. */
int kirin_batch_get_launch(const kirin_batch *b, int32_t *groups, int32_t *j_tiles, int32_t *n_items);

/* ---- j partition over several GPUs ----
 * The j-split of Sect. 3.2 (several thread blocks each sum a range of j for
 * the same i, and the host adds their partial sums) lifted across GPUs: each
 * rank keeps the whole particle set (every particle is an i-particle
 * somewhere, and the predictor of every step runs on each rank's own copy),
 * but its force calls sum only its part of the j tiles.  The seven partial
 * sums per i of every part are then gathered and added in part order, so
 * every rank holds the same bits.
 *
 * kirin_j_partition_range: the j-particles [*j_begin, *j_end) that part
 *   `part` of `n_parts` sums for a set of n_j: whole tiles of 128, the
 *   tiles shared out as evenly as they go (a part may be empty when there
 *   are more parts than tiles).  Host-only arithmetic.  Errors: EINVAL.
 *
 * kirin_set_j_partition: from now on the context's force calls sum only
 *   that part's j (n_parts = 1 restores the whole sum).
 *   With allgather == NULL every result is this part's partial sum, for the
 *   caller to add up.  Otherwise the library calls, once per force call,
 *     allgather(user, send, recv, count, stream)
 *   with count = 7 n_i: `send` holds this part's partial sums (device
 *   memory, [acc 3 n_i | jerk 3 n_i | pot n_i], G applied) and the callback
 *   must leave part r's send buffer in recv[r * count ...] for every r
 *   (device memory of n_parts * count doubles), ordered on `stream` (the
 *   context's cudaStream_t): the send buffer is complete once work enqueued
 *   on `stream` before the call has run, and the library's next work on
 *   `stream` may read recv.  It returns 0 on success; anything else makes
 *   the force call return KIRIN_EEXCHANGE.  The callback runs on the calling
 *   host thread, inside the force call.  With a callback every entry point
 *   that evaluates acc + jerk + pot or acc + pot returns whole sums:
 *   compute_forces(_dev), energy, the Hermite and leapfrog integrators (the
 *   block steps of kirin_hermite_run are then driven from the host, one
 *   exchange per step).  The adjoint calls and the neighbour search return
 *   ESTATE on a partitioned context.
 *   The context allocates 7 n_max (send) and 7 n_max n_parts (recv) doubles
 *   here.  Errors: EINVAL (part outside [0, n_parts), n_parts outside
 *   [1, KIRIN_MAX_PARTS]), ENOMEM, ECUDA; on error the context is left
 *   unpartitioned. */
#define KIRIN_MAX_PARTS 4096
typedef int (*kirin_allgather_fn)(void *user, const double *send, double *recv, int64_t count, void *stream);
int kirin_j_partition_range(int64_t n_j, int32_t part, int32_t n_parts, int64_t *j_begin, int64_t *j_end);
int kirin_set_j_partition(kirin_ctx *ctx, int32_t part, int32_t n_parts, kirin_allgather_fn allgather, void *user);

/* ---- allocation-free evaluation ----
 * No counterpart in the paper.  For callers that cannot allocate device
 * memory when they need forces (inside another framework's memory pool that
 * holds the whole device, in callbacks where cudaMalloc/cudaFree would
 * synchronise the device, or in hosts that forbid allocation after start-up):
 * the same mixed-precision evaluation as kirin_compute_forces_dev (acc, jerk
 * and pot of the n_i listed i against all n j, i_list NULL = all), with no
 * context and no allocation.  Its scratch (the j image and the j-split
 * partial sums) is one fixed device array of about 6.6 MB inside the library,
 * which every GPU that loads the library holds until the process exits.
 *   n, n_i <= KIRIN_NOALLOC_MAX_N; larger sizes return EINVAL.
 *   m (n), x, v (n x 3), i_list (n_i, int32), acc, jerk (n_i x 3), pot (n_i):
 *   FP64 device arrays on the current device; any output may be NULL.
 *   status: device word set to 0 and then to the OR of KIRIN_STATUS_* bits
 *   found while the work runs (NULL: not reported).
 *   stream: cudaStream_t (NULL or cudaStreamLegacy: the legacy default stream).
 * Asynchronous.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and must come before any stream capture on
 * that device; if that set-up fails the call returns ECUDA, nothing of it is
 * kept, and the next call on the device tries again.  Every call on a device shares the one array, which keeps the
 * last call's contents: calls whose work overlaps on the GPU (other streams,
 * other host threads) race and must be ordered by the caller. */
#define KIRIN_NOALLOC_MAX_N 32768
#define KIRIN_STATUS_BAD_INDEX 1u  /* an i_list entry outside [0, n) */
#define KIRIN_STATUS_TIMEOUT 2u    /* a bounded device wait gave up */
#define KIRIN_STATUS_NONFINITE 8u  /* NaN or Inf in m, x or v */
int kirin_forces_noalloc(int64_t n, const double *m, const double *x, const double *v, int64_t n_i,
                         const int32_t *i_list, double eps, double G, double r_min, double *acc,
                         double *jerk, double *pot, unsigned *status, void *stream);

/* ---- roofline denominators ----
 * Sustained fused multiply-add rate of the GPU `device` (2 flops per lane):
 * kind 0 = FP32 FFMA, 1 = packed FP32x2 FFMA2, 2 = FP64 DFMA, measured with
 * independent FMA chains on every SM (no counterpart in the paper, whose
 * Sect. 4.1 derives the 8800GTX peak from its unit count and clock).
 * Synchronous.  Errors: EINVAL, ECUDA. */
int kirin_measure_fma_rate(int32_t device, int32_t kind, double *flops_per_s);

/* Human-readable name of a return code (static string). */
const char *kirin_strerror(int code);

/* The context's last detailed error message (static storage owned by ctx). */
const char *kirin_last_error(const kirin_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* KIRIN_H */
