"""Fit of the polynomial used by the sweeps' equatorial form: angles within
asin(0.55) = 33.4 degrees of pi/2 from the ring axis, theta = pi/2 + asin(x)
with x = -cos(theta) = sigma s.  Far field (sweep.cu): s = a'.(-c') with both vectors
scaled by 1/sqrt(2), sigma = 2.  Near field (voxel.cu): s = (-a/sqrt(2)).d
/ |d|, sigma = sqrt(2).

asin(x) = x R(x^2) with R(z) = sum_n c_n z^n; the kernel evaluates it on s
directly as asin(sigma s) = s P(s^2), P(w) = sum_n sigma^(2n+1) c_n w^n.  For
sigma = 2 the scaling is a power of two and commutes with FP32 rounding (the
same arithmetic as evaluating R at x = 2 s, without the doubling); for
sigma = sqrt(2) the scaled coefficients are rounded once more.

Criterion: minimise max |x (R(x^2) - asin(x)/x)| on |x| <= X (the absolute
error of the angle) by weighted least squares on Chebyshev nodes with
Lawson-style reweighting toward the minimax solution.  The printed
coefficients (P's, increasing powers, binary32) are the ones in the kernel;
the report evaluates them as the kernel does (w = s*s rounded, Horner with
fused multiply-adds, v = s P(w) rounded) against FP64 asin.  Degree 4 in w on
X = 0.55: 7.3e-8 rad with exact coefficients, 1.4e-7 rad (sigma = 2) and
1.3e-7 rad (sigma = sqrt(2)) evaluated in FP32.

Run: python paper_2411_04785_gb300/csrc/fit_asin.py [degree] [X] [sigma]
(the kernels: 4 0.55 2 and 4 0.55 1.41421356)
(sigma: 2 for the far field, the default, or 1.41421356 for the near field)
"""
import sys

import numpy as np


def fit(deg, X, n=4000, iters=80):
    x = np.maximum(X * (0.5 - 0.5 * np.cos(np.pi * (np.arange(n) + 0.5) / n)), 1e-6)
    t = np.arcsin(x) / x
    lam = np.ones(n)
    for _ in range(iters):
        A = np.vander(x * x, deg + 1, increasing=True) * (x * lam)[:, None]
        c, *_ = np.linalg.lstsq(A, t * x * lam, rcond=None)
        err = np.abs(x * (np.polynomial.polynomial.polyval(x * x, c) - t))
        lam = lam * (err / err.max()) ** 0.3 + 1e-12
        lam /= lam.max()
    return c


def report(c, X, sigma=2.0):
    x = np.linspace(0.0, X, 2_000_001)
    e64 = np.abs(x * np.polynomial.polynomial.polyval(x * x, c) - np.arcsin(x)).max()
    p32 = (c * sigma ** (2 * np.arange(len(c)) + 1)).astype(np.float32)
    s = np.linspace(0.0, X / sigma, 2_000_001).astype(np.float32)
    w = (s.astype(np.float64) ** 2).astype(np.float32)
    acc = np.full_like(s, p32[-1])
    for k in range(len(p32) - 2, -1, -1):   # FMA: one rounding per step
        acc = (acc.astype(np.float64) * w + p32[k]).astype(np.float32)
    v = (s.astype(np.float64) * acc).astype(np.float32)
    e32 = np.abs(v.astype(np.float64) - np.arcsin(sigma * s.astype(np.float64)))
    return e64, e32.max(), e32.mean(), p32


if __name__ == "__main__":
    deg = int(sys.argv[1]) if len(sys.argv) > 1 else 4
    X = float(sys.argv[2]) if len(sys.argv) > 2 else 0.55
    sigma = float(sys.argv[3]) if len(sys.argv) > 3 else 2.0
    e64, e32max, e32mean, p32 = report(fit(deg, X), X, sigma)
    print(f"degree {deg} on |x| <= {X}: max |error| {e64:.3e} rad (exact coefficients), "
          f"FP32 evaluation max {e32max:.3e} mean {e32mean:.3e}")
    print("coefficients of P (increasing powers of w = s^2):")
    for v in p32:
        print(f"  {float(v):.8e}f")
