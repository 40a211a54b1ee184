"""Fit of the polynomial Q(s) = acos(1 - s) / sqrt(s) on s in [0, s_max] used
by the sweeps (theta = sqrt(s) Q(s)): on [0, 1] (theta <= pi/2) degree 6 in
the far-field sweep's general form (sweep.cu), degree 7 in cc_math.cuh
(near-field sweep, refinement, ring build); on [0, 0.8] (theta <= 78.46 deg)
degree 5 in the far-field sweep's one-sided forms, as accurate as degree 6
on [0, 1] (9.3e-8 rad with exact coefficients, 2.6e-7 evaluated in FP32).

Criterion: minimise the maximum absolute error of theta = sqrt(s) Q(s), i.e.
max |sqrt(s) (P(s) - Q(s))|, by weighted least squares on Chebyshev nodes with
Lawson-style reweighting toward the equioscillating minimax solution.  The
printed coefficients (increasing powers, rounded to binary32) are the ones in
the kernels; the report gives the error of the rounded coefficients evaluated
with FP32 fused multiply-adds (degree 6: 2.7e-7 rad, degree 7: 2.3e-7 rad -
the FP32 evaluation dominates both).

Run: python paper_2411_04785_gb300/csrc/fit_acos.py [degree] [s_max]
"""
import sys

import numpy as np


def target(s):
    return np.arccos(1.0 - s) / np.sqrt(s)


def fit(deg, smax=1.0, n=4000, iters=60):
    s = smax * (0.5 - 0.5 * np.cos(np.pi * (np.arange(n) + 0.5) / n))
    w = np.sqrt(s)
    lam = np.ones(n)
    for _ in range(iters):
        A = np.vander(s, deg + 1, increasing=True) * (w * lam)[:, None]
        c, *_ = np.linalg.lstsq(A, target(s) * w * lam, rcond=None)
        err = np.abs(w * (np.polynomial.polynomial.polyval(s, c) - target(s)))
        lam = lam * (err / err.max()) ** 0.3 + 1e-12
        lam /= lam.max()
    return c


def report(c, smax=1.0):
    s = np.linspace(1e-9, smax, 2_000_001)
    exact = np.arccos(1.0 - s)
    e64 = np.abs(np.sqrt(s) * np.polynomial.polynomial.polyval(s, c) - exact).max()
    c32 = c.astype(np.float32)
    s32 = s.astype(np.float32)
    acc = np.full_like(s32, c32[-1])
    for k in range(len(c32) - 2, -1, -1):   # FMA: one rounding per step
        acc = (acc.astype(np.float64) * s32 + c32[k]).astype(np.float32)
    th = (np.sqrt(s32.astype(np.float64)).astype(np.float32).astype(np.float64) * acc)
    e32 = np.abs(th.astype(np.float32).astype(np.float64) - np.arccos(1.0 - s32.astype(np.float64)))
    return e64, e32.max(), e32.mean(), c32


if __name__ == "__main__":
    deg = int(sys.argv[1]) if len(sys.argv) > 1 else 7
    smax = float(sys.argv[2]) if len(sys.argv) > 2 else 1.0
    e64, e32max, e32mean, c32 = report(fit(deg, smax), smax)
    print(f"degree {deg} on [0, {smax}]: max |error| {e64:.3e} rad (exact coefficients), "
          f"FP32 evaluation max {e32max:.3e} mean {e32mean:.3e}")
    print("coefficients (increasing powers):")
    for v in c32:
        print(f"  {float(v):.8e}f")
