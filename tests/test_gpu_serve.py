"""The serving path: batched sweeps give each burst the same result as when
it is swept alone, and the continuous-batching server returns, for every
burst of a mixed stream, the same map and direction as serving it alone."""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
from paper_2411_04785_gb300 import synth
from tests.helpers import grid_to_dev, rings_to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_04785_gb300 as m
    m.lib()
    return m


def batch_localize(cc, ring_sets, grid, params):
    from paper_2411_04785_gb300 import api
    dev = grid[0].device
    n = len(ring_sets)
    M = grid[0].numel()
    outs = []
    for r in ring_sets:
        nb = api.lib().cc_localize_batch_workspace_bytes(r["ax"].numel(), M, C.byref(params.c()))
        outs.append({"map": torch.empty(M, device=dev), "am": torch.empty(1, dtype=torch.int32, device=dev),
                     "sd": torch.empty(params.topk, dtype=torch.int32, device=dev),
                     "st": torch.empty(1, dtype=torch.int32, device=dev),
                     "ws": torch.empty(nb, dtype=torch.uint8, device=dev)})
    P = C.c_void_p
    rings = (api.cc_rings * n)(*[api._rings_struct(r) for r in ring_sets])
    arr = lambda k: (P * n)(*[o[k].data_ptr() for o in outs])
    wsb = (C.c_size_t * n)(*[o["ws"].numel() for o in outs])
    st = api.lib().cc_localize_batch(n, rings, C.byref(api._grid_struct(grid)), C.byref(params.c()),
                                     arr("map"), arr("am"), arr("sd"), arr("st"), arr("ws"), wsb,
                                     None)
    assert st == 0, api.lib().cc_last_error()
    torch.cuda.synchronize()
    return [{k: o[k].cpu().numpy() for k in ("map", "am", "sd", "st")} for o in outs]


def test_batched_sweep_equals_alone_and_matches_oracle(cc):
    dev = torch.device("cuda:0")
    grid_np = oracle.grid_healpix_ring(32)
    grid = grid_to_dev(grid_np, dev)
    p = cc.Params(topk=3, nms_rad=math.radians(5))
    sets_np = [synth.rings_burst(n=n, seed=s)[0] for n, s in ((500, 1), (3000, 2), (20000, 3),
                                                             (129, 4), (150000, 5))]
    sets = [rings_to_dev(r, dev) for r in sets_np]
    mixed = batch_localize(cc, sets, grid, p)
    for r, r_np, m in zip(sets, sets_np, mixed):
        alone = batch_localize(cc, [r], grid, p)[0]
        np.testing.assert_array_equal(m["map"], alone["map"])      # bit for bit
        assert m["am"][0] == alone["am"][0] and (m["sd"] == alone["sd"]).all()
        assert m["st"][0] == 0
        # and the batched map satisfies the parity rule against the oracle
        idx = np.arange(0, grid_np[0].size, 7)
        want = oracle.likelihood_map({k: np.asarray(r_np[k], np.float32) for k in
                                      ("ax", "ay", "az", "eta", "deta")}, grid_np, idx=idx)
        bound = 1e-5 * np.maximum(want, 1e-3 * want.max())
        assert (np.abs(m["map"][idx] - want) <= bound).all()


def test_batched_sweep_on_a_fine_ordered_grid(cc):
    """A HEALPix nside 128 grid kept with its order: the batched sweep takes
    the short polynomial of the one-sided forms there; each burst alone and
    in the batch bit for bit, and within the map rule of the oracle."""
    dev = torch.device("cuda:0")
    grid_np = oracle.grid_healpix_ring(128)
    g = cc.grid_healpix_ring(128, dev)
    grid = tuple(g) + (cc.grid_order(g),)
    p = cc.Params(topk=2, nms_rad=math.radians(5))
    sets_np = [synth.rings_burst(n=n, deta_deg=(0.5, 20.0), seed=s)[0]
               for n, s in ((2000, 21), (700, 22))]
    sets = [rings_to_dev(r, dev) for r in sets_np]
    mixed = batch_localize(cc, sets, grid, p)
    idx = np.arange(0, grid_np[0].size, 13)
    for r, r_np, m in zip(sets, sets_np, mixed):
        alone = batch_localize(cc, [r], grid, p)[0]
        np.testing.assert_array_equal(m["map"], alone["map"])
        assert m["st"][0] == 0
        want = oracle.likelihood_map({k: np.asarray(r_np[k], np.float32) for k in
                                      ("ax", "ay", "az", "eta", "deta")}, grid_np, idx=idx)
        bound = 1e-5 * np.maximum(want, 1e-3 * want.max())
        assert (np.abs(m["map"][idx] - want) <= bound).all()


def test_server_mixed_stream_equals_alone(cc):
    from paper_2411_04785_gb300 import serve
    dev = torch.device("cuda:0")
    grid = cc.grid_healpix_ring(32, dev)
    p = cc.Params()
    bursts = serve.make_bursts(16, rate_hz=4000.0, seed=7, median=4000, hi=60000, n_dirs=3,
                               pool_src=30000, pool_bkg=60000)
    srv = serve.Server(grid, p, hbm_budget=256 << 20, max_active=8)
    mixed, stats = srv.run(bursts, realtime=True, keep_maps=True)
    assert len(mixed) == 16 and max(stats["batches"]) > 1        # bursts were batched
    for b in bursts:
        alone, _ = serve.Server(grid, p).run([b], realtime=False, keep_maps=True)
        a, m = alone[b.bid], mixed[b.bid]
        np.testing.assert_array_equal(m["map"], a["map"])
        assert m["argmax"] == a["argmax"]
        np.testing.assert_array_equal(m["dir"], a["dir"])
        assert (m["status"] == 0).all() or m["status"][1] == -5
    lat = np.array([r["latency"] for r in mixed.values()])
    assert (lat > 0).all()


def test_sweep_compacts_to_the_kept_rings(cc):
    """Rings that are invalid, non-finite or of zero width are left out of
    the sweep (compacted away before it): the map equals the oracle's over
    the kept rings, and the localisation of the kept subset alone."""
    dev = torch.device("cuda:0")
    grid_np = oracle.grid_healpix_ring(32)
    grid = grid_to_dev(grid_np, dev)
    p = cc.Params()
    r_np = synth.rings_burst(n=40000, seed=9)[0]
    rng = np.random.default_rng(9)
    valid = (rng.uniform(size=40000) < 0.6).astype(np.uint8)
    deta = np.asarray(r_np["deta"], np.float32).copy()
    bad = rng.choice(40000, 300, replace=False)
    deta[bad[:100]] = np.nan
    deta[bad[100:200]] = 0.0
    deta[bad[200:]] = -1.0
    r_np = dict(r_np, deta=deta, valid=valid)
    keep = (valid == 1) & np.isfinite(deta) & (deta > 0)
    full = cc.localize(rings_to_dev(r_np, dev), grid, p)
    sub = cc.localize(rings_to_dev({k: np.asarray(v)[keep] for k, v in r_np.items()}, dev), grid, p)
    torch.cuda.synchronize()
    got, want_sub = full[0].cpu().numpy(), sub[0].cpu().numpy()
    np.testing.assert_allclose(got, want_sub, rtol=2e-6, atol=1e-6 * want_sub.max())
    idx = np.arange(0, grid_np[0].size, 5)
    want = oracle.likelihood_map({k: np.asarray(r_np[k], np.float32)[keep] for k in
                                  ("ax", "ay", "az", "eta", "deta")}, grid_np, idx=idx)
    bound = 1e-5 * np.maximum(want, 1e-3 * want.max())
    assert (np.abs(got[idx] - want) <= bound).all()


def test_server_learned_path_mixed_equals_alone(cc):
    """The learned path (features, MLP, filter with tau > 0, then the sweep)
    served in a mixed stream gives every burst its alone result."""
    from paper_2411_04785_gb300 import serve
    dev = torch.device("cuda:0")
    grid = cc.grid_healpix_ring(32, dev)
    p = cc.Params()
    f = cc.RingFilter(dev, seed=3)
    bursts = serve.make_bursts(12, rate_hz=4000.0, seed=8, median=4000, hi=60000, n_dirs=2,
                               pool_src=30000, pool_bkg=60000)
    kw = dict(ring_filter=f, tau=0.3)
    mixed, stats = serve.Server(grid, p, hbm_budget=256 << 20, max_active=8, **kw).run(
        bursts, realtime=True, keep_maps=True)
    assert len(mixed) == 12 and max(stats["batches"]) > 1
    for b in bursts:
        alone, _ = serve.Server(grid, p, **kw).run([b], realtime=False, keep_maps=True)
        a, m = alone[b.bid], mixed[b.bid]
        np.testing.assert_array_equal(m["map"], a["map"])
        assert m["argmax"] == a["argmax"]
        np.testing.assert_array_equal(m["dir"], a["dir"])


@pytest.mark.parametrize("learned", [False, True])
def test_graph_front_ends_equal_the_launched_path(cc, learned):
    """The per-size-bucket CUDA graphs of the front end give every burst the
    same map, argmax and direction as launching the kernels one by one."""
    from paper_2411_04785_gb300 import serve
    dev = torch.device("cuda:0")
    grid = cc.grid_healpix_ring(32, dev)
    p = cc.Params()
    kw = dict(ring_filter=cc.RingFilter(dev, seed=5), tau=0.2) if learned else {}
    bursts = serve.make_bursts(10, rate_hz=4000.0, seed=9, median=3000, hi=40000, n_dirs=2,
                               pool_src=20000, pool_bkg=40000)
    plain, _ = serve.Server(grid, p, max_active=8, **kw).run(bursts, realtime=False,
                                                             keep_maps=True)
    srv = serve.Server(grid, p, max_active=8, graphs=True, **kw)
    srv.prepare([b.count for b in bursts])
    graphed, stats = srv.run(bursts, realtime=True, keep_maps=True)
    for b in bursts:
        a, g = plain[b.bid], graphed[b.bid]
        np.testing.assert_array_equal(g["map"], a["map"])
        assert g["argmax"] == a["argmax"]
        np.testing.assert_array_equal(g["dir"], a["dir"])


def test_events_copy_of_pool_slices(cc):
    """cc_events_copy: slices of a wider host pool land at an offset of a
    device event set, slot rows and counts intact."""
    from paper_2411_04785_gb300 import api
    rng = np.random.default_rng(2)
    P, cap = 5000, 3000
    pool = {"n": rng.integers(0, 5, P).astype(np.uint8)}
    for k in "xyze":
        pool[k] = rng.standard_normal((4, P)).astype(np.float32)
    host = {k: torch.from_numpy(v).pin_memory() for k, v in pool.items()}
    dev = {"n": torch.zeros(cap, dtype=torch.uint8, device="cuda:0")}
    for k in "xyze":
        dev[k] = torch.zeros((4, cap), dtype=torch.float32, device="cuda:0")
    dst = tuple(dev[k] for k in ("n", "x", "y", "z", "e"))
    a, n1, b, n2 = 1234, 700, 4000, 900
    part1 = (host["n"][a:a + n1],) + tuple(host[k][:, a:a + n1] for k in "xyze")
    part2 = (host["n"][b:b + n2],) + tuple(host[k][:, b:b + n2] for k in "xyze")
    api.events_copy(dst, 10, part1)
    api.events_copy(dst, 10 + n1, part2)
    torch.cuda.synchronize()
    got_n = dev["n"].cpu().numpy()
    np.testing.assert_array_equal(got_n[10:10 + n1], pool["n"][a:a + n1])
    np.testing.assert_array_equal(got_n[10 + n1:10 + n1 + n2], pool["n"][b:b + n2])
    assert (got_n[:10] == 0).all() and (got_n[10 + n1 + n2:] == 0).all()
    for k in "xyze":
        g = dev[k].cpu().numpy()
        np.testing.assert_array_equal(g[:, 10:10 + n1], pool[k][:, a:a + n1])
        np.testing.assert_array_equal(g[:, 10 + n1:10 + n1 + n2], pool[k][:, b:b + n2])
