"""The sweep's direction order and the angular selection with block
skipping.  The sweep takes any grid's directions in their NESTED HEALPix
order (cc_grid_order), so each warp owns a compact patch: per warp and tile
it skips the rings that cannot reach the patch.  A skipped ring's terms are
all cut to 0 anyway, so the map must be within the oracle's k_cut bracket,
and a NESTED grid's map bit for bit the map of the same pixels in RING order
(swept in the same order)."""
import math

import numpy as np
import pytest

import oracle
from paper_2411_04785_gb300 import synth
from tests.helpers import rings_to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_04785_gb300 as m
    m.lib()
    return m


def nest_to_ring_perm(nside):
    """RING index of every NESTED pixel, from the two oracle grids (the
    nearest RING centre; pixel centres are at least ~0.1 / nside rad apart)."""
    from scipy.spatial import cKDTree
    nv = np.stack(oracle.grid_healpix_nest(nside), 1)
    rv = np.stack(oracle.grid_healpix_ring(nside), 1)
    dist, out = cKDTree(rv).query(nv)
    assert dist.max() < 1e-9
    return out.astype(np.int64)


@pytest.mark.parametrize("nside", [1, 2, 16, 64])
def test_nest_grid_is_the_ring_grid_permuted(cc, nside):
    perm = nest_to_ring_perm(nside)
    gn = [t.cpu().numpy() for t in cc.grid_healpix_nest(nside, "cuda:0")]
    gr = [t.cpu().numpy() for t in cc.grid_healpix_ring(nside, "cuda:0")]
    for a, b in zip(gn, gr):
        np.testing.assert_array_equal(a, b[perm])
    on = oracle.grid_healpix_nest(nside)
    for a, b in zip(gn, on):
        assert np.abs(a - b).max() < 3e-7


@pytest.mark.parametrize("nside", [1, 4, 16, 64])
def test_ring_grid_is_swept_in_nested_order(cc, nside):
    perm = nest_to_ring_perm(nside)
    order = cc.grid_order(cc.grid_healpix_ring(nside, "cuda:0")).cpu().numpy()
    np.testing.assert_array_equal(order, perm)
    order = cc.grid_order(cc.grid_healpix_nest(nside, "cuda:0")).cpu().numpy()
    np.testing.assert_array_equal(order, np.arange(12 * nside * nside))


@pytest.mark.parametrize("M", [1, 2, 257, 5003, 100003])
def test_grid_order_is_a_compact_permutation(cc, M):
    g = cc.grid_fibonacci(M, "cuda:0")
    o = cc.grid_order(g).cpu().numpy()
    np.testing.assert_array_equal(np.sort(o), np.arange(M))
    if M >= 5003:      # runs of 256 in the order span small patches
        v = np.stack([t.cpu().numpy() for t in g], 1).astype(np.float64)[o]
        n = M // 256 * 256
        c = v[:n].reshape(-1, 256, 3).sum(1)
        c /= np.linalg.norm(c, axis=1, keepdims=True)
        spread = np.degrees(np.arccos(np.clip(np.einsum("wkd,wd->wk", v[:n].reshape(-1, 256, 3), c), -1, 1)).max(1))
        assert np.median(spread) < 2.5 * math.degrees(math.sqrt(4 * math.pi * 256 / M))


def test_grid_order_ties_and_bad_directions(cc):
    """Equal directions keep their index order; zero and NaN directions go last."""
    dev = "cuda:0"
    M = 3000
    x = torch.zeros(M, device=dev)
    y = torch.zeros(M, device=dev)
    z = torch.ones(M, device=dev)
    x[::7] = 1.0
    z[::7] = 0.0
    z[5] = 0.0
    x[11] = float("nan")
    o = cc.grid_order((x, y, z)).cpu().numpy()
    np.testing.assert_array_equal(np.sort(o), np.arange(M))
    assert set(o[-2:].tolist()) == {5, 11}
    for grp in (np.arange(M)[::7], np.setdiff1d(np.arange(M), np.r_[np.arange(M)[::7], 5, 11])):
        pos = np.argsort(o)[grp]             # where each index landed
        assert (np.diff(pos) > 0).all()       # in index order among equals


def test_kept_order_equals_computed_order(cc):
    """A grid's order kept with it (cc_grid.order) gives the map computed with
    the order the call finds itself, bit for bit; any other permutation is a
    valid traversal too (a different FP32 summation), within the map rule."""
    r, _, _ = synth.rings_burst(n=20000, seed=5)
    rd = rings_to_dev(r, "cuda:0")
    g = cc.grid_healpix_ring(32, "cuda:0")
    m1, a1, _, st1 = cc.localize(rd, g)
    m2, a2, _, st2 = cc.localize(rd, tuple(g) + (cc.grid_order(g),))
    assert int(st1.item()) == 0 and int(st2.item()) == 0
    assert torch.equal(m1, m2) and torch.equal(a1, a2)
    ident = torch.arange(g[0].numel(), dtype=torch.int32, device="cuda:0")
    m3 = cc.localize(rd, tuple(g) + (ident,))[0]
    want = oracle.likelihood_map({k: np.asarray(r[k], np.float32) for k in ("ax", "ay", "az", "eta", "deta")},
                                 oracle.grid_healpix_ring(32))
    for m in (m1, m3):
        got = m.cpu().numpy()
        assert (np.abs(got - want) <= 1e-5 * np.maximum(want, 1e-3 * want.max())).all()
    with pytest.raises(ValueError):
        cc.localize(rd, tuple(g) + (ident[:-1],))


@pytest.mark.parametrize("dmax_deg,kcut,nside", [(2.0, 5.0, 64), (10.0, 3.0, 64), (0.6, 8.0, 64),
                                                 (2.0, 5.0, 256)])
def test_skipping_is_exact(cc, dmax_deg, kcut, nside):
    perm = nest_to_ring_perm(nside)
    rng = np.random.default_rng(int(dmax_deg * 10))
    r, s, _ = synth.rings_burst(n=30000, seed=int(kcut))
    r = dict(r)
    lo, hi = math.log(math.radians(0.5)), math.log(math.radians(dmax_deg))
    r["deta"] = np.exp(rng.uniform(lo, hi, 30000)).astype(np.float32)
    rd = rings_to_dev(r, "cuda:0")
    p = cc.Params(k_cut=kcut)
    m_nest = cc.localize(rd, cc.grid_healpix_nest(nside, "cuda:0"), p)[0].cpu().numpy()
    m_ring = cc.localize(rd, cc.grid_healpix_ring(nside, "cuda:0"), p)[0].cpu().numpy()
    np.testing.assert_array_equal(m_nest, m_ring[perm])
    # and within the oracle's bracket of the cut
    g = oracle.grid_healpix_nest(nside)
    idx = np.arange(0, g[0].size, 97)
    r32 = {k: np.asarray(r[k], np.float32) for k in ("ax", "ay", "az", "eta", "deta")}
    lo_m = oracle.likelihood_map(r32, g, idx=idx, k_cut=kcut * (1 - 1e-4))
    hi_m = oracle.likelihood_map(r32, g, idx=idx, k_cut=kcut * (1 + 1e-4))
    b = 1e-5 * np.maximum(hi_m, 1e-3 * hi_m.max()) + 1e-6
    assert ((m_nest[idx] >= lo_m - b) & (m_nest[idx] <= hi_m + b)).all()


@pytest.mark.parametrize("nside,kept_order", [(32, False), (128, True), (256, True)])
def test_batched_sweep_with_skipping_equals_alone(cc, nside, kept_order):
    """With the angular selection, each burst of a batched sweep alone and in
    the batch bit for bit, and close to the single-burst sweep (a different
    ring split, so a different FP32 summation).  A NESTED grid as given, and
    RING grids kept with their order at nside 128 and 256, where the sweeps
    take the short polynomials."""
    from tests.test_gpu_serve import batch_localize
    if kept_order:
        g = cc.grid_healpix_ring(nside, "cuda:0")
        g = tuple(g) + (cc.grid_order(g),)
    else:
        g = cc.grid_healpix_nest(nside, "cuda:0")
    p = cc.Params(k_cut=5.0, topk=2, nms_rad=math.radians(5))
    sets = []
    for n, seed in ((3000, 1), (20000, 2), (700, 3)):
        r = dict(synth.rings_burst(n=n, seed=seed)[0])
        r["deta"] = np.full(n, math.radians(1.5), np.float32)
        sets.append(rings_to_dev(r, "cuda:0"))
    mixed = batch_localize(cc, sets, g, p)
    for rs, m in zip(sets, mixed):
        alone = batch_localize(cc, [rs], g, p)[0]
        np.testing.assert_array_equal(m["map"], alone["map"])
        single = cc.localize(rs, g, p)[0].cpu().numpy()
        np.testing.assert_allclose(m["map"], single, rtol=2e-6, atol=1e-6 * single.max())
