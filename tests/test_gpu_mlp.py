"""GPU parity of the learned ring filter (tensor-core MLP) against its oracle
(oracle/mlp.py, FP64 with BF16 rounding at the GPU's rounding points), and
what the trained filter gains over the plain method."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2411_04785_gb300 import synth
from tests.helpers import grid32, grid_to_dev, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
D2R = math.pi / 180


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_04785_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def dev(cc):
    return torch.device("cuda:0")


def random_case(seed, B):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    p[-2:] = [0.2, -1.0]
    X = mlp.bf16(rng.standard_normal((B, 16)))
    y = (rng.uniform(size=B) < 0.3).astype(np.uint8)
    res = (rng.standard_normal(B) * 0.4).astype(np.float32)
    w = (rng.uniform(size=B) < 0.95).astype(np.uint8)
    return p, X, y, res, w


def SMS():
    return torch.cuda.get_device_properties(0).multi_processor_count


def f64(t):
    return t.float().cpu().numpy().astype(np.float64)


# 128-row tiles on at most one CTA per SM: one partial tile, exact tiles, a
# ragged tail, one tile per CTA (3000), several tile pairs per CTA plus an odd
# tile (70,001 and 500,000 rows)
@pytest.mark.parametrize("R", [1, 127, 128, 129, 3000, 70_001, 500_000])
def test_forward_matches_oracle(cc, dev, R):
    """Inference outputs element by element: each within the bound the
    network's arithmetic allows against the oracle's FP64 network with the
    same BF16 rounding points (FP32 accumulation of every product, and a
    hidden activation rounded one BF16 ulp apart wherever its value lies
    within its bound of a rounding boundary, carried through the later
    layers; tests/mlp_bounds.py)."""
    from tests.mlp_bounds import forward_bounds
    p, X, _, _, _ = random_case(1, R)
    f = cc.RingFilter(dev, params=p)
    out = f.forward(to_dev(X.astype(np.float32), dev).to(torch.bfloat16).contiguous())
    torch.cuda.synchronize()
    want, bound, _, _ = forward_bounds(p, X)
    got = out.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all()
    bad = np.argwhere(np.abs(got - want) > bound)
    assert bad.size == 0, (bad[:5], got[tuple(bad[0])], want[tuple(bad[0])])


def test_forward_rejects_misaligned_features(cc, dev):
    p, X, _, _, _ = random_case(1, 64)
    f = cc.RingFilter(dev, params=p)
    flat = torch.zeros(64 * 16 + 8, dtype=torch.bfloat16, device=dev)
    feats = flat[1:1 + 64 * 16].view(64, 16)       # contiguous, 2 bytes off 16
    with pytest.raises(cc.CCError):
        f.forward(feats)


@pytest.mark.parametrize("B", [1, 777, 65536])
def test_training_step_stage_by_stage(cc, dev, B):
    """Every stage of a training step, element by element, on the GPU's own
    inputs to that stage (kept by cc_mlp_grad_trace): the three hidden
    layers and the outputs, the output gradient, the three backward signals
    and every weight and bias gradient, each within the interval its own
    FP32 accumulation and BF16 rounding allow (tests/mlp_bounds.py); the
    traced step equals the plain one bit for bit, and the inference kernel's
    outputs equal the training forward's."""
    from tests import mlp_bounds as mb
    p, X, y, res, w = random_case(2, B)
    f = cc.RingFilter(dev, params=p)
    Xd = to_dev(X.astype(np.float32), dev).to(torch.bfloat16).contiguous()
    yd, rd, wd = to_dev(y, dev), to_dev(res, dev), to_dev(w, dev)
    loss, g, t = f.grad_trace(Xd, yd, rd, wd)
    torch.cuda.synchronize()
    g_tr, l_tr = g.clone(), float(loss.item())
    loss2, g2 = f.grad(Xd, yd, rd, wd)
    inf = f.forward(Xd)
    torch.cuda.synchronize()
    assert torch.equal(g2, g_tr) and float(loss2.item()) == l_tr
    assert torch.equal(inf, t["out"])

    layers = mlp.unpack(p.astype(np.float64))
    H = [X] + [f64(t["hidden"][l]) for l in range(3)]
    out = t["out"].cpu().numpy().astype(np.float64)
    for li, (W, b) in enumerate(layers):
        got = out if li == 3 else H[li + 1]
        ok, amb = mb.check_layer(H[li], W, b, got, relu=li < 3)
        assert ok.all(), ("layer", li + 1, np.argwhere(~ok)[:3])
    yf, rf, wf = y.astype(float), res.astype(np.float64), w.astype(float)
    dout = f64(t["dout"])
    ok, _ = mb.check_dout(out, yf, rf, wf, dout)
    assert ok.all(), np.argwhere(~ok)[:3]
    S = [None] + [f64(t["signals"][l]) for l in range(3)]   # S[l]: signal of layer l
    sig_above = dout
    for li in (3, 2, 1):
        ok, _ = mb.check_signal(sig_above, layers[li][0], H[li], S[li])
        assert ok.all(), ("signal", li, np.argwhere(~ok)[:3])
        sig_above = S[li]
    grad = g_tr.cpu().numpy().astype(np.float64)
    gl = mlp.unpack(grad)
    sigs = [S[1], S[2], S[3], dout]
    for li in range(4):
        okW, okb = mb.check_weight_grad(sigs[li], H[li], gl[li][0], gl[li][1], sms=SMS())
        assert okW.all() and okb.all(), ("grad", li + 1, np.argwhere(~okW)[:3])
    want_loss, _ = mlp.loss_and_grad(p, X, yf, rf, wf, round_points=True)
    assert l_tr == pytest.approx(want_loss, rel=1e-4, abs=1e-7)


@pytest.mark.parametrize("B", [777, 65536])
def test_gradient_matches_oracle(cc, dev, B):
    """The whole gradient against the oracle's, element by element, within
    the bound carried through the step from the forward pass's own (the
    stage-by-stage test holds each stage to its own tight interval)."""
    from tests.mlp_bounds import grad_bounds
    p, X, y, res, w = random_case(2, B)
    f = cc.RingFilter(dev, params=p)
    Xd = to_dev(X.astype(np.float32), dev).to(torch.bfloat16).contiguous()
    _, g = f.grad(Xd, to_dev(y, dev), to_dev(res, dev), to_dev(w, dev))
    torch.cuda.synchronize()
    want, bound = grad_bounds(p, X, y.astype(float), res.astype(np.float64), w.astype(float),
                              sms=SMS())
    got = g.cpu().numpy().astype(np.float64)
    bad = np.nonzero(np.abs(got - want) > bound)[0]
    assert bad.size == 0, (bad[:5], got[bad[:5]], want[bad[:5]], bound[bad[:5]])


def test_features_match_oracle(cc, dev):
    ev = synth.simulate_events(n_src=3000, n_bkg=7000, seed=17)
    p = cc.Params()
    n = to_dev(ev["n"], dev)
    x, y, z, e = (to_dev(np.asarray(ev[k], np.float32), dev) for k in "xyze")
    rings = cc.rings_from_events(n, x, y, z, e, p)
    F = cc.ring_features(n, x, y, z, e, rings, p)
    torch.cuda.synchronize()
    r = oracle.rings_from_events(ev, p.sigma_e_frac, p.sigma_pos_cm, p.deta_min, p.deta_max)
    want = mlp.features(ev, r, p.sigma_pos_cm)
    got = F.float().cpu().numpy().astype(np.float64)
    # GPU features are FP32 values rounded to BF16 (relative 2^-9) from FP32
    # rings; the oracle's are FP64 from FP64 rings
    tol = 2.0 ** -7 * np.abs(want) + 1e-5        # one BF16 ulp
    bad = np.abs(got - want) > tol
    assert bad.mean() < 1e-4, np.argwhere(bad)[:5]


def test_adam_step(cc, dev):
    p, X, y, res, w = random_case(5, 512)
    f = cc.RingFilter(dev, params=p)
    Xd = to_dev(X.astype(np.float32), dev).to(torch.bfloat16).contiguous()
    f.grad(Xd, to_dev(y, dev), to_dev(res, dev), to_dev(w, dev))
    g = f.grad_buf.cpu().numpy().astype(np.float64)
    f.adam(lr=1e-2)
    torch.cuda.synchronize()
    # first Adam step: m_hat = g, v_hat = g^2 -> p - lr g / (|g| + eps)
    want = p.astype(np.float64) - 1e-2 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(f.p.cpu().numpy(), want, rtol=1e-5, atol=1e-6)
    np.testing.assert_array_equal(f.wb.float().cpu().numpy(), mlp.bf16(f.p.cpu().numpy()))


def localize_error(cc, rings, grid, source, params):
    loc = cc.Localizer(grid, params)
    loc.from_rings(rings)
    torch.cuda.synchronize()
    d = loc.dir.cpu().numpy()
    return math.degrees(math.atan2(np.linalg.norm(np.cross(d, source)), float(d @ source)))


def test_trained_filter_gains_over_the_plain_method(cc, dev):
    """Train on 400k simulated events (random source per 20k-event chunk,
    background 3:1) on the GPU; apply the filter to the 200k-event burst (its
    own seed) before the sweep; the refined direction must come closer to the
    true source than the plain method's.  The plain rings are also the
    fallback: with the filter removed the result is the plain one."""
    p = cc.Params()
    tr = synth.training_events(400_000, seed=11)
    n = to_dev(tr["n"], dev)
    x, y, z, e = (to_dev(np.asarray(tr[k], np.float32), dev) for k in "xyze")
    rings = cc.rings_from_events(n, x, y, z, e, p)
    F = cc.ring_features(n, x, y, z, e, rings, p)
    res = cc.ring_residuals(rings, to_dev(tr["sources"], dev))
    ys = to_dev(tr["is_source"].astype(np.uint8), dev)
    f = cc.RingFilter(dev, seed=0)
    losses = f.train(F, ys, res, rings["valid"], epochs=8, batch=8192, lr=2e-3)
    assert losses[-1] < losses[0]

    ev = synth.simulate_events(seed=2)
    n = to_dev(ev["n"], dev)
    x, y, z, e = (to_dev(np.asarray(ev[k], np.float32), dev) for k in "xyze")
    grid = grid_to_dev(oracle.grid_healpix_ring(64), dev)
    plain = cc.rings_from_events(n, x, y, z, e, p)
    err_plain = localize_error(cc, plain, grid, ev["source"], p)
    learned = {k: v.clone() for k, v in plain.items()}
    out = f.forward(cc.ring_features(n, x, y, z, e, plain, p))
    f.apply(learned, out, tau=0.0, deta_min=p.deta_min, deta_max=p.deta_max)
    err_learned = localize_error(cc, learned, grid, ev["source"], p)
    print(f"plain {err_plain:.3f} deg, learned {err_learned:.3f} deg, losses {losses}")
    assert err_learned < err_plain
    # the width head learned something per ring: on these held-out events its
    # width (before the clamp) ranks the source rings' actual residuals
    src = torch.from_numpy(ev["is_source"]).to(dev) & plain["valid"].bool()
    res = cc.ring_residuals(plain, to_dev(np.repeat(ev["source"][None, :], ev["n"].size, 0), dev))
    w = torch.exp(out[:, 1].float())[src].cpu().numpy()
    r = res.abs()[src].cpu().numpy()
    rank = lambda a: np.argsort(np.argsort(a)).astype(np.float64)
    rho = float(np.corrcoef(rank(w), rank(r))[0, 1])
    print(f"rank correlation of learned width and |residual| on {w.size} source rings: {rho:.3f}")
    assert rho > 0.3


def test_checkpoint_resumes_training(cc, dev, tmp_path):
    p, X, y, res, w = random_case(7, 4096)
    Xd = to_dev(X.astype(np.float32), dev).to(torch.bfloat16).contiguous()
    yd, rd, wd = to_dev(y, dev), to_dev(res, dev), to_dev(w, dev)
    f = cc.RingFilter(dev, params=p)
    for _ in range(3):
        f.grad(Xd, yd, rd, wd)
        f.adam(lr=1e-3)
    f.save(tmp_path / "filter.bin")
    g = cc.RingFilter.load(tmp_path / "filter.bin", dev)
    assert g.step == f.step
    torch.testing.assert_close(g.forward(Xd), f.forward(Xd), rtol=0, atol=0)
    for h in (f, g):                     # one more step from each: bit-identical
        h.grad(Xd, yd, rd, wd)
        h.adam(lr=1e-3)
    torch.cuda.synchronize()
    assert torch.equal(f.p, g.p) and torch.equal(f.m, g.m) and torch.equal(f.v, g.v)
