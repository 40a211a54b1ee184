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


# --------------------------------------------------------------------------
# The element-wise bounds the GPU parity tests apply (tests/mlp_bounds.py),
# checked here against an emulation of the GPU's arithmetic in FP32
# (numpy float32: other summation orders, fused multiply-adds, the same BF16
# rounding points), including the rare one-ulp BF16 flips.
# --------------------------------------------------------------------------
def _emulate_fp32(p, X, y, res, w, order_seed):
    """The GPU network's arithmetic in float32 with the products summed in a
    shuffled order (any order the bounds must cover)."""
    rng = np.random.default_rng(order_seed)
    f32 = np.float32
    layers = mlp.unpack(np.asarray(p, np.float32))
    B = X.shape[0]

    def matmul(a, b):                    # a [m,k] @ b [k,n], shuffled k order
        perm = rng.permutation(a.shape[1])
        acc = np.zeros((a.shape[0], b.shape[1]), f32)
        for k in perm:
            acc = (acc + np.outer(a[:, k], b[k, :]).astype(f32)).astype(f32)
        return acc

    A = [mlp.bf16(X).astype(f32)]
    for li, (W, b) in enumerate(layers):
        z = (matmul(A[-1], mlp.bf16(W).astype(f32).T) + b.astype(f32)).astype(f32)
        if li < 3:
            A.append(mlp.bf16(np.maximum(z, 0)).astype(f32))
        else:
            out = z
    zz, v = out[:, 0], out[:, 1]
    inv = f32(1.0) / f32(B)
    sg = f32(1.0) / (f32(1.0) + np.exp(-zz).astype(f32))
    e2v = np.exp(f32(-2.0) * v).astype(f32)
    d0 = (w.astype(f32) * (sg - y.astype(f32)) * inv).astype(f32)
    d1 = (w.astype(f32) * y.astype(f32) * (f32(1.0) - res.astype(f32) ** 2 * e2v) * inv)
    dP = mlp.bf16(np.stack([d0, d1.astype(f32)], 1)).astype(f32)
    trace = {"hidden": [a.astype(np.float64) for a in A[1:]], "out": out.astype(np.float64),
             "dout": dP.astype(np.float64), "signals": [None] * 3}
    grads = [None] * 4
    for li in range(3, -1, -1):
        W, _ = layers[li]
        grads[li] = (matmul(dP.T, A[li]), dP.sum(0, dtype=f32))
        if li > 0:
            dA = matmul(dP, mlp.bf16(W).astype(f32))
            dP = mlp.bf16(np.where(A[li] > 0, dA, f32(0))).astype(f32)
            trace["signals"][li - 1] = dP.astype(np.float64)
    return out.astype(np.float64), mlp.pack([(g.astype(np.float64), b.astype(np.float64))
                                             for g, b in grads]), trace


@pytest.mark.parametrize("seed", [0, 1])
def test_elementwise_bounds_contain_fp32_arithmetic(seed):
    from tests.mlp_bounds import forward_bounds, grad_bounds
    rng = np.random.default_rng(seed)
    B = 300
    p = mlp.init_params(seed)
    p[-2:] = [0.2, -1.0]
    X = mlp.bf16(rng.standard_normal((B, 16)))
    y = (rng.uniform(size=B) < 0.3).astype(float)
    res = rng.standard_normal(B) * 0.4
    w = (rng.uniform(size=B) < 0.95).astype(float)
    want, bound, _, dA = forward_bounds(p, X)
    g_want, g_bound = grad_bounds(p, X, y, res, w)
    flips = sum(int((d > 0).sum()) for d in dA[1:])
    from tests import mlp_bounds as mb
    layers = mlp.unpack(p.astype(np.float64))
    n_amb = 0
    for order_seed in range(3):
        out, g, t = _emulate_fp32(p, X, y, res, w, order_seed)
        assert (np.abs(out - want) <= bound).all()
        assert (np.abs(g - g_want) <= g_bound).all()
        # the stage-by-stage intervals of the GPU tests, on the emulation's
        # own inputs to each stage
        H = [X] + t["hidden"]
        for li, (W, b) in enumerate(layers):
            ok, amb = mb.check_layer(H[li], W, b, out if li == 3 else H[li + 1], relu=li < 3)
            assert ok.all()
            n_amb += int(amb.sum())
        assert mb.check_dout(out, y, res, w, t["dout"])[0].all()
        S = [None] + t["signals"]
        above = t["dout"]
        for li in (3, 2, 1):
            assert mb.check_signal(above, layers[li][0], H[li], S[li])[0].all()
            above = S[li]
        gl = mlp.unpack(g)
        for li, sg in enumerate([S[1], S[2], S[3], t["dout"]]):
            okW, okb = mb.check_weight_grad(sg, H[li], gl[li][0], gl[li][1])
            assert okW.all() and okb.all()
    # a stage's interval admits two BF16 values only near a rounding boundary
    assert 0 < n_amb < 0.05 * 3 * X.shape[0] * 128 * 3
    # BF16 flips are possible on this batch, so the carried bounds are used
    assert flips > 0


def test_stage_checks_catch_a_wrong_column():
    """The stage intervals are tight enough to catch what a norm-wise check
    would pass: one hidden unit's column off by 1 %, one output column off by
    1e-4 relative, one weight-gradient column off by 1e-3."""
    from tests import mlp_bounds as mb
    rng = np.random.default_rng(4)
    B = 300
    p = mlp.init_params(4)
    X = mlp.bf16(rng.standard_normal((B, 16)))
    y = (rng.uniform(size=B) < 0.3).astype(float)
    res = rng.standard_normal(B) * 0.4
    w = np.ones(B)
    out, g, t = _emulate_fp32(p, X, y, res, w, 0)
    layers = mlp.unpack(p.astype(np.float64))
    H = [X] + t["hidden"]
    bad_h = H[2].copy()
    bad_h[:, 5] = mlp.bf16(bad_h[:, 5] * 1.01)
    assert not mb.check_layer(H[1], *layers[1], bad_h, relu=True)[0].all()
    bad_out = out.copy()
    bad_out[:, 1] *= 1 + 1e-4
    assert not mb.check_layer(H[3], *layers[3], bad_out, relu=False)[0].all()
    gl = mlp.unpack(g)
    gW = gl[2][0].copy()
    gW[:, 7] *= 1 + 1e-3
    assert not mb.check_weight_grad(t["signals"][2], H[2], gW, gl[2][1])[0].all()
