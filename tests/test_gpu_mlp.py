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


# 128-row tiles on at most one CTA per SM: one partial tile, exact tiles, a
# ragged tail, one tile per CTA (3000), several tile pairs per CTA plus an odd
# tile (70,001 and 500,000 rows)
@pytest.mark.parametrize("R", [1, 127, 128, 129, 3000, 70_001, 500_000])
def test_forward_matches_oracle(cc, dev, R):
    p, X, _, _, _ = random_case(1, R)
    f = cc.RingFilter(dev, params=p)
    out = f.forward(to_dev(X.astype(np.float32), dev).to(torch.bfloat16).contiguous())
    torch.cuda.synchronize()
    want, _, _ = mlp.forward(p, X, round_points=True)
    got = out.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all()
    # FP32 accumulation vs FP64 over K <= 128 BF16 products, plus rare
    # one-ulp BF16 flips of a hidden activation: norm-wise half a BF16 ulp
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 2.0 ** -9, err
    # row by row: a row read from or written to the wrong place would be off
    # by the outputs' own scale
    dev_ = np.abs(got - want).max(1)
    assert dev_.max() < 0.05 * np.abs(want).mean(), (dev_.argmax(), dev_.max())


def test_forward_rejects_misaligned_features(cc, dev):
    p, X, _, _, _ = random_case(1, 64)
    f = cc.RingFilter(dev, params=p)
    flat = torch.zeros(64 * 16 + 8, dtype=torch.bfloat16, device=dev)
    feats = flat[1:1 + 64 * 16].view(64, 16)       # contiguous, 2 bytes off 16
    with pytest.raises(cc.CCError):
        f.forward(feats)


@pytest.mark.parametrize("B", [1, 777, 65536])
def test_gradient_matches_oracle(cc, dev, B):
    p, X, y, res, w = random_case(2, B)
    f = cc.RingFilter(dev, params=p)
    Xd = to_dev(X.astype(np.float32), dev).to(torch.bfloat16).contiguous()
    loss, g = f.grad(Xd, to_dev(y, dev), to_dev(res, dev), to_dev(w, dev))
    torch.cuda.synchronize()
    want_loss, want_g = mlp.loss_and_grad(p, X, y.astype(float), res.astype(float),
                                          w.astype(float), round_points=True)
    assert float(loss.item()) == pytest.approx(want_loss, rel=1e-4, abs=1e-7)
    got = g.cpu().numpy().astype(np.float64)
    off = 0
    for o, i in mlp.SIZES:
        for n in (o * i, o):
            a, b = got[off:off + n], want_g[off:off + n]
            off += n
            scale = np.linalg.norm(b)
            if scale == 0:
                assert np.linalg.norm(a) < 1e-7
                continue
            assert np.linalg.norm(a - b) / scale < 2.0 ** -9, (o, i, n)


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
