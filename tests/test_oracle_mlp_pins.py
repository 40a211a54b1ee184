"""Pins of the learned-ring-filter oracle (oracle/mlp.py): BF16 rounding,
analytic gradients against finite differences, a closed-form loss, and the
features of a constructed event.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp


def test_bf16_rounding_matches_an_independent_implementation():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 65504.0, 1e-38]])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), want)
    assert mlp.bf16(np.float32(1.0 + 2 ** -8))[()] == 1.0          # tie to even
    assert mlp.bf16(np.float32(1.0 + 3 * 2 ** -8))[()] == 1.0 + 2 ** -6


def _batch(seed, B=64):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, 16))
    y = (rng.uniform(size=B) < 0.4).astype(float)
    res = rng.standard_normal(B) * 0.3
    w = (rng.uniform(size=B) < 0.9).astype(float)
    return X, y, res, w


def test_gradient_matches_finite_differences():
    p = mlp.init_params(3).astype(np.float64)
    p[-2:] = [0.3, -1.2]
    X, y, res, w = _batch(1)
    f0, g = mlp.loss_and_grad(p, X, y, res, w, round_points=False)
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.integers(0, 2048, 6), [2048, 2049], rng.integers(2176, 18560, 6),
                          rng.integers(18688, 35072, 6), np.arange(35200, 35458, 40)])
    for i in idx:
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, y, res, w, False)[0] -
              mlp.loss_and_grad(pm, X, y, res, w, False)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_zero_network_loss_closed_form():
    p = np.zeros(mlp.N_PARAMS)
    c = 0.7
    p[-1] = c                                     # b4 = (0, c): out = (0, c)
    X, y, res, w = _batch(4)
    f, g = mlp.loss_and_grad(p, X, y, res, w, round_points=False)
    want = np.sum(w * (math.log(2.0) + y * (c + 0.5 * res ** 2 * math.exp(-2 * c)))) / len(y)
    assert f == pytest.approx(want, rel=1e-12)
    # with zero weights only the output biases have a gradient
    assert np.all(g[:-2] == 0.0)
    assert g[-2] == pytest.approx(np.sum(w * (0.5 - y)) / len(y), rel=1e-12)


def test_features_of_a_constructed_event():
    # two sites: slot 0 at the origin with 200 keV, slot 1 at (3, 4, 0) cm with
    # 300 keV; a ring built from order (0, 1)
    ev = {"n": np.array([2], np.uint8)}
    for k in "xyze":
        ev[k] = np.zeros((4, 1))
    ev["x"][1, 0], ev["y"][1, 0] = 3.0, 4.0
    ev["e"][0, 0], ev["e"][1, 0] = 200.0, 300.0
    rings = {"valid": np.array([1], np.uint8), "perm": np.array([0], np.uint8),
             "eta": np.array([1.0]), "deta": np.array([0.2]), "az": np.array([0.0])}
    F = mlp.features(ev, rings)[0]
    want = [1.0 / math.pi, math.cos(1.0), math.sin(1.0), math.log(0.2) / 4, 1, 0, 0,
            math.log(500 / 500), 200 / 500, 300 / 500, 300 / 500, math.log(5.0 / 5.0), 0.0,
            0.0, 0.0, math.sqrt(2) / 5.0 / 0.2]
    np.testing.assert_allclose(F, want, rtol=1e-14, atol=1e-15)


def test_filter_rule():
    out = np.array([[2.0, math.log(0.05)], [-2.0, 0.0], [0.0, math.log(10.0)]])
    keep, deta = mlp.apply_filter(out, np.array([1, 1, 1], np.uint8), None, 0.5, 0.01, 1.0)
    assert list(keep) == [1, 0, 1]
    np.testing.assert_allclose(deta, [0.05, 1.0, 1.0])
