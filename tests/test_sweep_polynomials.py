"""The sweeps' angle polynomials and class limits, read from the CUDA sources
and checked on the CPU against the error bounds the sources state: every
coefficient list evaluated as the kernels do (FP32, one rounding per fused
multiply-add) against FP64 acos / asin over its stated range, and every
angle constant against its definition.  A mistyped coefficient or limit
fails here before any GPU run.  CPU only."""
import math
import re
from pathlib import Path

import numpy as np
import pytest

CSRC = Path(__file__).resolve().parent.parent / "paper_2411_04785_gb300" / "csrc"
F32 = np.float32


def block_coeffs(src, marker, count):
    """The first `count` float literals inside pair(...) from the line of
    `marker` on, in the order written (highest power first: Horner)."""
    i = src.rindex("\n", 0, src.index(marker)) + 1
    vals = re.findall(r"pair\(([-+0-9.eE]+)f\)", src[i:i + 2000])
    assert len(vals) >= count, marker
    return [float(v) for v in vals[:count]]


def fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def horner32(coef_high_first, x):
    acc = np.full_like(x, F32(coef_high_first[0]))
    for c in coef_high_first[1:]:
        acc = fma32(acc, x, np.full_like(x, F32(c)))
    return acc


def acos_error(coef_high_first, smax):
    """max |sqrt(s) Q(s) - acos(1 - s)| on [0, smax], Q evaluated in FP32."""
    s = np.linspace(0.0, smax, 400_001).astype(F32)
    q = horner32(coef_high_first, s)
    rt = np.sqrt(s.astype(np.float64)).astype(F32)
    th = (rt.astype(np.float64) * q.astype(np.float64)).astype(F32)
    return np.abs(th.astype(np.float64) - np.arccos(1.0 - s.astype(np.float64))).max()


def asin_error(coef_high_first, xmax, sigma):
    """max |s P(s^2) - asin(sigma s)| for |sigma s| <= xmax, in FP32."""
    s = np.linspace(0.0, xmax / sigma, 400_001).astype(F32)
    w = (s.astype(np.float64) ** 2).astype(F32)
    p = horner32(coef_high_first, w)
    v = (s.astype(np.float64) * p.astype(np.float64)).astype(F32)
    return np.abs(v.astype(np.float64) - np.arcsin(sigma * s.astype(np.float64))).max()


@pytest.fixture(scope="module")
def sweep_src():
    return (CSRC / "sweep.cu").read_text()


@pytest.fixture(scope="module")
def voxel_src():
    return (CSRC / "voxel.cu").read_text()


@pytest.mark.parametrize("marker,deg,smax,bound", [
    ("// Q(s) on [0, 1], degree 6", 6, 1.0, 2.7e-7),
    ("// Q(s) on [0, 0.8], degree 5", 5, 0.8, 2.6e-7),
    ("// Q(s) on [0, 0.55], degree 4", 4, 0.55, 2.4e-7),
])
def test_far_field_acos_polynomials(sweep_src, marker, deg, smax, bound):
    coef = block_coeffs(sweep_src, marker, deg + 1)
    assert acos_error(coef, smax) <= bound


def test_far_field_asin_polynomial(sweep_src):
    coef = block_coeffs(sweep_src, "// P(w), degree 4, FP32x2", 5)
    assert asin_error(coef, 0.55, 2.0) <= 1.45e-7


@pytest.mark.parametrize("marker,deg,smax,bound", [
    ("// acos_q on [0, 1], degree 7", 7, 1.0, 2.4e-7),
    ("// on [0, 0.8], degree 5", 5, 0.8, 2.6e-7),
    ("// on [0, 0.55], degree 4", 4, 0.55, 2.4e-7),
])
def test_near_field_acos_polynomials(voxel_src, marker, deg, smax, bound):
    coef = block_coeffs(voxel_src, marker, deg + 1)
    assert acos_error(coef, smax) <= bound


def test_near_field_asin_polynomial(voxel_src):
    i = voxel_src.index("if constexpr (SIDE == 5)")
    coef = block_coeffs(voxel_src[i:], "float2 p = pair(", 5)
    assert asin_error(coef, 0.55, math.sqrt(2.0)) <= 1.3e-7


def const(src, name):
    m = re.search(r"constexpr float %s = ([-+0-9.eE]+)f;" % name, src)
    assert m, name
    return float(m.group(1))


def test_class_limits(sweep_src, voxel_src):
    """The bands and side limits are the angles their comments define, to
    FP32 rounding: the equatorial band asin(0.55) in both sweeps, the
    one-sided limits acos(0.2) and acos(0.45), the dot form's pi/6."""
    eps = 2e-7
    assert abs(const(sweep_src, "kEquAngle") - math.asin(0.55)) < eps
    assert abs(const(sweep_src, "kSideAngle") - math.acos(0.2)) < eps
    assert abs(const(sweep_src, "kSide2Angle") - math.acos(0.45)) < eps
    assert abs(const(sweep_src, "kDotAngle") - math.pi / 6) < eps
    a = math.asin(0.55) - 1e-3
    assert abs(const(voxel_src, "kEquSin") - math.sin(a)) < eps
    assert abs(const(voxel_src, "kEquCos") - math.cos(a)) < eps
    t = math.acos(0.2) - 1e-3
    assert abs(const(voxel_src, "kSideCos") - math.cos(t)) < eps
    assert abs(const(voxel_src, "kSideSin") - math.sin(t)) < eps
    t2 = math.acos(0.45) - 1e-3
    assert abs(const(voxel_src, "kSide2Cos") - math.cos(t2)) < eps
    assert abs(const(voxel_src, "kSide2Sin") - math.sin(t2)) < eps


def test_short_polynomial_ranges_cover_the_one_sided_pairs():
    """With the equatorial band |cos theta| <= 0.55, a one-sided ring that is
    not equatorial has every pair within (pi/2 - asin 0.55) + 2 rho + 2e-3 of
    its axis; the per-launch levels admit caps that keep this inside the
    polynomials' ranges (s = 1 - cos theta <= 0.8 and <= 0.55)."""
    band = math.pi / 2 - math.asin(0.55)
    for limit, smax in ((math.acos(0.2), 0.8), (math.acos(0.45), 0.55)):
        rho = 0.5 * (limit - band) - 1e-3            # the largest admitted cap
        assert 1.0 - math.cos(band + 2 * rho + 2e-3) <= smax + 1e-12
