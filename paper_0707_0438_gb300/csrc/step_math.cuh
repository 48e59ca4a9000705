// The FP64 step arithmetic of the Hermite integrator (Sect. 3: predictor,
// Hermite interpolation, corrector and Aarseth's block step; Sect. 3.1: the
// j images the force kernels read), shared by the step kernels and the
// single-launch shared-step kernel so that both compute the same bits.
#pragma once

#include <cuda_runtime.h>

#include "f32_pack.cuh"
#include "kirin_internal.cuh"

namespace kirin {
namespace {

// hi = RN32(v), lo = RN32(v - hi), built on the integer pipes (f32_pack.cuh).
__device__ __forceinline__ void split_ds(double v, float &hi, float &lo) { f32pack::split(v, hi, lo); }

__device__ __forceinline__ void write_images(int k, double X, double Y, double Z, double M, double VX,
                                             double VY, double VZ, JMixed *jm, JF64 *jd)
{
    if (jm) {
        float xh, xl, yh, yl, zh, zl;
        split_ds(X, xh, xl);
        split_ds(Y, yh, yl);
        split_ds(Z, zh, zl);
        const float m = f32pack::to_f32(M);
        const float vx = f32pack::to_f32(VX), vy = f32pack::to_f32(VY), vz = f32pack::to_f32(VZ);
        JMixed r;
        r.q[0] = make_float4(xh, xh, yh, yh);
        r.q[1] = make_float4(zh, zh, m, m);
        r.q[2] = make_float4(xl, xl, yl, yl);
        r.q[3] = make_float4(zl, zl, vx, vx);
        r.q[4] = make_float4(vy, vy, vz, vz);
        jm[k] = r;
    }
    if (jd) {
        JF64 r;
        r.q[0] = make_double2(X, Y);
        r.q[1] = make_double2(Z, M);
        r.q[2] = make_double2(VX, VY);
        r.q[3] = make_double2(VZ, 0.0);
        jd[k] = r;
    }
}

// Powers of the prediction interval dt and one component of the predictor
// x_p = x + v dt + a dt^2/2 + jerk dt^3/6, v_p = v + a dt + jerk dt^2/2.
struct PredictDt {
    double dt, dt2, dt3;  // dt, dt^2 / 2, dt^3 / 6
};

__device__ __forceinline__ PredictDt predict_dt(double dt)
{
    PredictDt P;
    P.dt = dt;
    P.dt2 = dt * dt * 0.5;
    P.dt3 = P.dt2 * dt * (1.0 / 3.0);
    return P;
}

__device__ __forceinline__ void predict_xv(const PredictDt &P, double x, double v, double a, double j, double &X,
                                           double &V)
{
    X = x + v * P.dt + a * P.dt2 + j * P.dt3;
    V = v + a * P.dt + j * P.dt2;
}

// Predictor x_p = x + v dt + a dt^2/2 + jerk dt^3/6, v_p = v + a dt + jerk dt^2/2
// (dt = t - t0) of record k, then its j images; records [n, n_pad) are
// zero-mass padding.  Loads bypass L1: inside the fused step kernel other
// CTAs have just corrected some of these particles.
__device__ __forceinline__ void predict_one(int k, int n, double t, int predict, const double *m, const double *x,
                                            const double *v, const double *a, const double *jk, const double *t0,
                                            double *xp, double *vp, JMixed *jm, JF64 *jd, unsigned *err)
{
    if (k >= n) {
        write_images(k, PAD_POS, PAD_POS, PAD_POS, 0.0, 0.0, 0.0, 0.0, jm, jd);
        return;
    }
    double X[3], V[3];
    if (predict) {
        const PredictDt P = predict_dt(t - __ldcg(t0 + k));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t o = 3 * (size_t)k + c;
            predict_xv(P, __ldcg(x + o), __ldcg(v + o), __ldcg(a + o), __ldcg(jk + o), X[c], V[c]);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            X[c] = __ldcg(x + 3 * (size_t)k + c);
            V[c] = __ldcg(v + 3 * (size_t)k + c);
        }
    }
    if (xp) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xp[3 * (size_t)k + c] = X[c];
            vp[3 * (size_t)k + c] = V[c];
        }
    }
    const double M = m[k];
    using f32pack::finite;
    if (!(finite(X[0]) && finite(X[1]) && finite(X[2]) && finite(V[0]) && finite(V[1]) && finite(V[2]) &&
          finite(M)))
        atomicOr(err, ERR_NONFINITE);
    write_images(k, X[0], X[1], X[2], M, V[0], V[1], V[2], jm, jd);
}

__device__ __forceinline__ double norm3(const double *p)
{
    return sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
}

// Largest power of two <= d within [dt_min, dt_max].
__device__ __forceinline__ double quantise_down(double d, double dt_min, double dt_max)
{
    double q = dt_max;
    while (q > d && q > dt_min)
        q *= 0.5;
    return q;
}

// Initial block step of a particle from its first a and jerk: 0.01 |a| / |j|
// on the power-of-two ladder.
__device__ __forceinline__ double initial_step(const double *a, const double *j, double dt_min, double dt_max)
{
    return quantise_down(0.01 * norm3(a) / norm3(j), dt_min, dt_max);
}

// Hermite corrector for the block (Sect. 3): a2, a3 from the two (a, jerk)
// pairs, corrected x and v, and (update_dt) Aarseth's step on the
// power-of-two ladder.
__device__ __forceinline__ bool is_pow2(double d)
{
    return (__double_as_longlong(d) & 0x000fffffffffffffll) == 0 && d > 0.0 && isfinite(d);
}

// The step's interval dt and the powers the corrector needs: 1/dt of a
// power-of-two step from its exponent (exact), else a divide; the powers of
// dt shared by the three components.
struct CorrectDt {
    double dt, idt, idt2, idt3, dt2, c3, c4, c5, dt6;
    bool p2;
};

__device__ __forceinline__ CorrectDt correct_dt(double dt)
{
    CorrectDt S;
    S.dt = dt;
    S.p2 = is_pow2(dt);
    S.idt = S.p2 ? __longlong_as_double((2046ll << 52) - (__double_as_longlong(dt) & 0x7ff0000000000000ll))
                 : 1.0 / dt;
    S.idt2 = S.idt * S.idt;
    S.idt3 = S.idt2 * S.idt;
    S.dt2 = dt * dt;
    const double dt4 = S.dt2 * S.dt2;
    S.c3 = S.dt2 * dt * (1.0 / 6.0);
    S.c4 = dt4 * (1.0 / 24.0);
    S.c5 = dt4 * dt * (1.0 / 120.0);
    S.dt6 = 6.0 * dt;
    return S;
}

// One component of the Hermite corrector: a2 and a3 (Hermite interpolation
// of the old a0, j0 and the new a1, j1 over the step), corrected x and v.
__device__ __forceinline__ void correct_xv(const CorrectDt &S, double a0, double j0, double a1, double j1,
                                           double xp, double vp, double &x1, double &v1, double &a2, double &a3)
{
    const double da = a0 - a1;
    a2 = fma(-S.dt, fma(4.0, j0, 2.0 * j1), -6.0 * da) * S.idt2;
    a3 = fma(S.dt6, j0 + j1, 12.0 * da) * S.idt3;
    x1 = fma(a3, S.c5, fma(a2, S.c4, xp));
    v1 = fma(a3, S.c4, fma(a2, S.c3, vp));
}

// Component c of the Hermite corrector of block member k (particle i): the
// new a and jerk (acc/jerk row k) are stored, x and v corrected; a1, j1, the
// a2 at the end of the step (a2e) and a3 go to Aarseth's criterion.
__device__ __forceinline__ void correct_component(const CorrectDt &S, int c, size_t i, int k, const double *xp,
                                                  const double *vp, const double *acc, const double *jerk,
                                                  double *bx, double *bv, double *ba, double *bj, double &a1,
                                                  double &j1, double &a2e, double &a3)
{
    a1 = acc[3 * (size_t)k + c];
    j1 = jerk[3 * (size_t)k + c];
    double a2;
    correct_xv(S, ba[3 * i + c], bj[3 * i + c], a1, j1, xp[3 * i + c], vp[3 * i + c], bx[3 * i + c], bv[3 * i + c],
               a2, a3);
    ba[3 * i + c] = a1;
    bj[3 * i + c] = j1;
    a2e = fma(S.dt, a3, a2);
}

// Aarseth's block step after a step of dt ending at t_next, from the squared
// norms A = |a|^2, J = |jerk|^2, N2 = |a2e|^2, N3 = |a3|^2 (each summed over
// the components in order x, y, z): the criterion quantised to a power of two
// that may shrink freely and double only where t_next is a multiple of the
// doubled step.  FP64 is the scarce pipe on this part, so this spends it
// sparingly:
//  - dt_A = sqrt(X / Y), X = eta (|a||a2| + |j|^2), Y = |j||a3| + |a2|^2, is
//    compared in squared form (q < dt_A <=> q^2 Y < X), with
//    |a||a2| = sqrt(|a|^2 |a2|^2): two square roots, no divide;
//  - "t_next is a multiple of 2 dt" is tested exactly by scaling when 2 dt is
//    a power of two (idt = 1/dt from the exponent), by fmod otherwise.
__device__ __forceinline__ double aarseth_step(double A, double J, double N2, double N3, double dt, double dt2,
                                               bool p2, double idt, double t_next, double eta, double dt_min,
                                               double dt_max)
{
    const double X = eta * (sqrt(A * N2) + J), Y = sqrt(J * N3) + N2;
    double q = dt;
    if (X == 0.0 && Y == 0.0) {
        // no criterion (0 / 0): keep the step
    } else if (X < dt2 * Y) {
        while (q > dt_min && X < q * q * Y)
            q *= 0.5;
    } else if (X >= 4.0 * dt2 * Y && 2.0 * dt <= dt_max) {
        bool multiple;
        if (p2) {
            const double r = t_next * (0.5 * idt);  // exact: a power-of-two scaling
            multiple = r == trunc(r);
        } else {
            multiple = fmod(t_next, 2.0 * dt) == 0.0;
        }
        if (multiple)
            q = 2.0 * dt;
    }
    return fmin(fmax(q, dt_min), dt_max);
}

// Hermite corrector of block member k (particle ilist[k], or k) at t_next
// from its new a, jerk (acc/jerk row k), and with update_dt its new block
// step (aarseth_step).  The powers of dt are shared by the three components
// (correct_dt).  Member k of the block is particle i; returns its new
// t_i + dt_i.
__device__ __forceinline__ double correct_at(size_t i, int k, double t_next, double eta, double dt_min,
                                             double dt_max, int update_dt, const double *xp, const double *vp,
                                             const double *acc, const double *jerk, double *bx, double *bv,
                                             double *ba, double *bj, double *bt, double *bdt)
{
    const CorrectDt S = correct_dt(t_next - bt[i]);
    double A = 0.0, J = 0.0, N2 = 0.0, N3 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double a1, j1, a2e, a3;
        correct_component(S, c, i, k, xp, vp, acc, jerk, bx, bv, ba, bj, a1, j1, a2e, a3);
        A = fma(a1, a1, A);
        J = fma(j1, j1, J);
        N2 = fma(a2e, a2e, N2);
        N3 = fma(a3, a3, N3);
    }
    bt[i] = t_next;
    if (update_dt) {
        const double q = aarseth_step(A, J, N2, N3, S.dt, S.dt2, S.p2, S.idt, t_next, eta, dt_min, dt_max);
        bdt[i] = q;
        return t_next + q;
    }
    return t_next + bdt[i];
}

}  // namespace
}  // namespace kirin
