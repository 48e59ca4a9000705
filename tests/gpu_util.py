"""Shared helpers of the GPU parity tests: error metrics and tolerances.

Tolerances (per particle, against the FP64 oracle on the same inputs):
* mixed path, acceleration: median relative error <= 1e-6 and max <= 1e-5
  (the stated target of the mixed-precision path);
* mixed path, potential: same bounds (all terms have one sign, no cancellation);
* mixed path, jerk: median <= 1e-6, max <= 1e-4.  The jerk sums terms of both
  signs built from FP32 velocity differences, so a particle whose jerk nearly
  cancels carries a larger relative error than its acceleration does; measured
  at N = 2^20 the median is ~3e-7 and the worst of ~17000 sampled i ~1e-5;
* FP64 path: median <= 1e-12 and max <= 1e-10 for every quantity (the order
  of summation differs from the oracle's, so results agree to the rounding of
  a sum of N terms, amplified where the sum cancels).
"""
import numpy as np

from paper_0707_0438_gb300 import metrics

TOL = {
    "mixed": {"acc": (1e-6, 1e-5), "pot": (1e-6, 1e-5), "jerk": (1e-6, 1e-4)},
    "fp64": {"acc": (1e-12, 1e-10), "pot": (1e-12, 1e-10), "jerk": (1e-12, 1e-10)},
}


def errors(got, ref):
    acc, jerk, pot = got
    racc, rjerk, rpot = ref
    return {
        "acc": metrics.summary(metrics.rel_err_vec(acc, racc)),
        "jerk": metrics.summary(metrics.rel_err_vec(jerk, rjerk)),
        "pot": metrics.summary(metrics.rel_err_scalar(pot, rpot)),
    }


def assert_parity(got, ref, precision, what=""):
    errs = errors(got, ref)
    for q, (med, mx) in TOL[precision].items():
        e = errs[q]
        assert e["median"] <= med and e["max"] <= mx, f"{what} {precision} {q}: {e} (tolerance {med}, {mx})"
    return errs
