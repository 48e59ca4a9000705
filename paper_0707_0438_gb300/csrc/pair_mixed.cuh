// The mixed-precision pair interaction, shared by the single-system and the
// batched kernels.  Two i-particles ride in the two lanes of packed FP32x2
// registers; one call accumulates one j record into the tile sums of both.
//
// Per pair (Sect. 3: acceleration, jerk and potential by direct summation):
//   d = (x_j,hi - x_i,hi) + (x_j,lo - x_i,lo)  (double-single, rounded once)
//   s^2 = |d|^2 + eps^2,  r = rsqrt(s^2) (MUFU),  mr = m_j r,  mr3 = mr r^2
//   pot += mr;  acc += mr3 d;  jerk1 += mr3 w;  jerk2 += mr3 (d.w) r^2 d
// with w = v_j - v_i; the jerk is jerk1 - 3 jerk2, formed when tile sums are
// folded.  In adjoint mode the velocity slots carry g and the jerk1 registers
// collect K(d) w = w/s^3 - 3 (d.w) d/s^5 with w = m_k g_j - m_j g_k, combined
// per pair (the two parts cancel to the tidal term across j, so summing them
// separately in FP32 would lose digits), and the pot registers g_j.d / s^3.
//
// MASK: the pair whose j index equals a lane's i index contributes nothing
// (used only on the tile holding a thread's own i-particles).
//
// In adjoint mode the MUFU estimate of 1/s is refined by one Newton-Raphson
// step, y' = y (3 - s^2 y^2) / 2: the hardware estimate's small systematic
// error enters w/s^3 and d(d.w)/s^5 with different weights (3 and 5), and the
// two halves cancel across j, which would amplify it.
#pragma once

#include <cuda_runtime.h>

#include "kirin_internal.cuh"

namespace kirin {

__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Error-free transformation hi + t = s + e (Knuth two-sum); lo collects e.
__device__ __forceinline__ void two_sum(float &hi, float &lo, float t)
{
    const float s = __fadd_rn(hi, t);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(t, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// Negated i-particle data of the two lanes, and the softening.
struct IPair {
    float2 nxh, nyh, nzh, nxl, nyl, nzl, nvx, nvy, nvz;
    float2 mk;
    float2 eps2v;
    float rmin2;
};

// Load the i data of two records (pass the same record twice for a lone i).
__device__ __forceinline__ IPair load_ipair(const JMixed *r0, const JMixed *r1, float eps2, float rmin2)
{
    IPair p;
    const float4 a0 = r0->q[0], a1 = r0->q[1], a2 = r0->q[2], a3 = r0->q[3], a4 = r0->q[4];
    const float4 b0 = r1->q[0], b1 = r1->q[1], b2 = r1->q[2], b3 = r1->q[3], b4 = r1->q[4];
    p.nxh = f2(-a0.x, -b0.x);
    p.nyh = f2(-a0.z, -b0.z);
    p.nzh = f2(-a1.x, -b1.x);
    p.mk = f2(a1.z, b1.z);
    p.nxl = f2(-a2.x, -b2.x);
    p.nyl = f2(-a2.z, -b2.z);
    p.nzl = f2(-a3.x, -b3.x);
    p.nvx = f2(-a3.z, -b3.z);
    p.nvy = f2(-a4.x, -b4.x);
    p.nvz = f2(-a4.z, -b4.z);
    p.eps2v = f2(eps2, eps2);
    p.rmin2 = rmin2;
    return p;
}

// FP32x2 partial sums over the current block of j.
struct Tile7 {
    float2 ax, ay, az, pt, j1x, j1y, j1z, j2x, j2y, j2z;
    __device__ __forceinline__ void zero()
    {
        ax = ay = az = pt = f2(0.f, 0.f);
        j1x = j1y = j1z = j2x = j2y = j2z = f2(0.f, 0.f);
    }
};

// Compensated per-lane accumulators of the seven outputs (acc 3, jerk 3, pot).
struct Lane7 {
    float h[7];
    float l[7];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int q = 0; q < 7; ++q)
            h[q] = l[q] = 0.f;
    }
};

// Nearest j of the two lanes so far: |d|^2 as computed in FP32 (the kernel's
// own precision decides), and its index.
struct NNPair {
    float r0, r1;
    int j0, j1;
    __device__ __forceinline__ void reset()
    {
        r0 = r1 = INFINITY;
        j0 = j1 = -1;
    }
};

template <int MODE>
__device__ __forceinline__ void fold(Tile7 &t, Lane7 &L0, Lane7 &L1)
{
    constexpr bool JERK = MODE != MODE_ACC_POT;
    if (MODE != MODE_ADJOINT) {
        two_sum(L0.h[0], L0.l[0], t.ax.x);
        two_sum(L1.h[0], L1.l[0], t.ax.y);
        two_sum(L0.h[1], L0.l[1], t.ay.x);
        two_sum(L1.h[1], L1.l[1], t.ay.y);
        two_sum(L0.h[2], L0.l[2], t.az.x);
        two_sum(L1.h[2], L1.l[2], t.az.y);
    }
    if (MODE == MODE_ADJOINT) {
        two_sum(L0.h[3], L0.l[3], t.j1x.x);
        two_sum(L1.h[3], L1.l[3], t.j1x.y);
        two_sum(L0.h[4], L0.l[4], t.j1y.x);
        two_sum(L1.h[4], L1.l[4], t.j1y.y);
        two_sum(L0.h[5], L0.l[5], t.j1z.x);
        two_sum(L1.h[5], L1.l[5], t.j1z.y);
    } else if (JERK) {
        two_sum(L0.h[3], L0.l[3], __fmaf_rn(-3.f, t.j2x.x, t.j1x.x));
        two_sum(L1.h[3], L1.l[3], __fmaf_rn(-3.f, t.j2x.y, t.j1x.y));
        two_sum(L0.h[4], L0.l[4], __fmaf_rn(-3.f, t.j2y.x, t.j1y.x));
        two_sum(L1.h[4], L1.l[4], __fmaf_rn(-3.f, t.j2y.y, t.j1y.y));
        two_sum(L0.h[5], L0.l[5], __fmaf_rn(-3.f, t.j2z.x, t.j1z.x));
        two_sum(L1.h[5], L1.l[5], __fmaf_rn(-3.f, t.j2z.y, t.j1z.y));
    }
    two_sum(L0.h[6], L0.l[6], t.pt.x);
    two_sum(L1.h[6], L1.l[6], t.pt.y);
    t.zero();
}

template <bool GUARD, int MODE, bool MASK = false>
__device__ __forceinline__ void pair(const JMixed &J, const IPair &I, Tile7 &t, int j = 0, int i0 = -1,
                                     int i1 = -1, NNPair *nn = nullptr, int jlim = 0)
{
    constexpr bool JERK = MODE != MODE_ACC_POT;
    constexpr bool ADJ = MODE == MODE_ADJOINT;
    constexpr bool NN = MODE == MODE_NN;
    const float4 q0 = J.q[0];
    const float4 q1 = J.q[1];
    const float4 q2 = J.q[2];
    const float4 q3 = J.q[3];
    const float2 dx = __fadd2_rn(__fadd2_rn(f2(q0.x, q0.y), I.nxh), __fadd2_rn(f2(q2.x, q2.y), I.nxl));
    const float2 dy = __fadd2_rn(__fadd2_rn(f2(q0.z, q0.w), I.nyh), __fadd2_rn(f2(q2.z, q2.w), I.nyl));
    const float2 dz = __fadd2_rn(__fadd2_rn(f2(q1.x, q1.y), I.nzh), __fadd2_rn(f2(q3.x, q3.y), I.nzl));
    float2 r2;
    if (NN) {
        // the search compares |d|^2 itself (one more add than the fused chain);
        // padding records (j >= jlim) and the self pair are skipped, and strict <
        // in increasing j keeps the smallest index on ties
        float2 d2 = __fmul2_rn(dx, dx);
        d2 = __ffma2_rn(dy, dy, d2);
        d2 = __ffma2_rn(dz, dz, d2);
        r2 = __fadd2_rn(d2, I.eps2v);
        const float ra = (MASK && j == i0) ? INFINITY : d2.x;
        const float rb = (MASK && j == i1) ? INFINITY : d2.y;
        if (j < jlim) {
            if (ra < nn->r0) {
                nn->r0 = ra;
                nn->j0 = j;
            }
            if (rb < nn->r1) {
                nn->r1 = rb;
                nn->j1 = j;
            }
        }
    } else {
        r2 = __ffma2_rn(dx, dx, I.eps2v);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
    }
    float2 ri;
    if (GUARD) {
        ri.x = rsqrt_mufu(fmaxf(r2.x, I.rmin2));
        ri.y = rsqrt_mufu(fmaxf(r2.y, I.rmin2));
        ri.x = (r2.x == 0.f) ? 0.f : ri.x;
        ri.y = (r2.y == 0.f) ? 0.f : ri.y;
    } else {
        ri.x = rsqrt_mufu(r2.x);
        ri.y = rsqrt_mufu(r2.y);
    }
    if (MASK) {
        ri.x = (j == i0) ? 0.f : ri.x;
        ri.y = (j == i1) ? 0.f : ri.y;
    }
    float2 ri2 = __fmul2_rn(ri, ri);
    if (ADJ) {
        const float2 e = __ffma2_rn(__fmul2_rn(r2, ri2), f2(-0.5f, -0.5f), f2(1.5f, 1.5f));
        ri = __fmul2_rn(ri, e);
        ri2 = __fmul2_rn(ri, ri);
        const float4 q4 = J.q[4];
        const float2 mj = f2(q1.z, q1.w);
        const float2 gjx = f2(q3.z, q3.w), gjy = f2(q4.x, q4.y), gjz = f2(q4.z, q4.w);
        const float2 ri3 = __fmul2_rn(ri, ri2);
        // w = m_k g_j - m_j g_k, one rounding fewer with the multiply-add (the self pair, where the
        // two products are equal, is masked by the caller or has r = 0 under the eps = 0 guard)
        const float2 wx = __ffma2_rn(I.mk, gjx, __fmul2_rn(mj, I.nvx));
        const float2 wy = __ffma2_rn(I.mk, gjy, __fmul2_rn(mj, I.nvy));
        const float2 wz = __ffma2_rn(I.mk, gjz, __fmul2_rn(mj, I.nvz));
        float2 dw = __fmul2_rn(dx, wx);
        dw = __ffma2_rn(dy, wy, dw);
        dw = __ffma2_rn(dz, wz, dw);
        const float2 nb3 = __fmul2_rn(__fmul2_rn(dw, __fmul2_rn(ri2, f2(-3.f, -3.f))), ri3);  // -3 (d.w) / s^5
        t.j1x = __ffma2_rn(nb3, dx, __ffma2_rn(ri3, wx, t.j1x));
        t.j1y = __ffma2_rn(nb3, dy, __ffma2_rn(ri3, wy, t.j1y));
        t.j1z = __ffma2_rn(nb3, dz, __ffma2_rn(ri3, wz, t.j1z));
        float2 gd = __fmul2_rn(gjx, dx);
        gd = __ffma2_rn(gjy, dy, gd);
        gd = __ffma2_rn(gjz, dz, gd);
        t.pt = __ffma2_rn(gd, ri3, t.pt);
        return;
    }
    const float2 mr = __fmul2_rn(f2(q1.z, q1.w), ri);  // m_j / s
    const float2 mr3 = __fmul2_rn(mr, ri2);             // m_j / s^3
    t.pt = __fadd2_rn(t.pt, mr);
    t.ax = __ffma2_rn(mr3, dx, t.ax);
    t.ay = __ffma2_rn(mr3, dy, t.ay);
    t.az = __ffma2_rn(mr3, dz, t.az);
    if (JERK) {
        const float4 q4 = J.q[4];
        const float2 dvx = __fadd2_rn(f2(q3.z, q3.w), I.nvx);
        const float2 dvy = __fadd2_rn(f2(q4.x, q4.y), I.nvy);
        const float2 dvz = __fadd2_rn(f2(q4.z, q4.w), I.nvz);
        float2 rv = __fmul2_rn(dx, dvx);
        rv = __ffma2_rn(dy, dvy, rv);
        rv = __ffma2_rn(dz, dvz, rv);
        const float2 b = __fmul2_rn(__fmul2_rn(rv, ri2), mr3);  // m (d.w) / s^5
        t.j1x = __ffma2_rn(mr3, dvx, t.j1x);
        t.j1y = __ffma2_rn(mr3, dvy, t.j1y);
        t.j1z = __ffma2_rn(mr3, dvz, t.j1z);
        t.j2x = __ffma2_rn(b, dx, t.j2x);
        t.j2y = __ffma2_rn(b, dy, t.j2y);
        t.j2z = __ffma2_rn(b, dz, t.j2z);
    }
}

}  // namespace kirin
