"""GPU parity: the CUDA path, called through the C ABI (ctypes binding),
against the CPU oracle on the same seeded inputs.  The oracle never consumes a
value the GPU produced: shared inputs come from the generators or from the
oracle itself (its grids, its rings rounded to FP32)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2411_04785_gb300 import synth
from tests.helpers import (EPS32, REFINE_TOL_DEG, ang_deg, eta_tol, grid32, grid_to_dev,
                           extreme_events, map_violations, rings_to_dev, to_dev)

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


def run_localize(cc, rings_np, grid_np, dev, **pk):
    p = cc.Params(**pk)
    m, am, sd, st = cc.localize(rings_to_dev(rings_np, dev), grid_to_dev(grid_np, dev), p)
    torch.cuda.synchronize()
    return m.cpu().numpy(), int(am.item()), sd.cpu().numpy(), int(st.item())


def fp32_term_bound(r32, grid):
    """sum_i |dterm/dr| * dr_i with dr_i = 3 eps (theta + pi) / deta_i: the
    first-order effect on each term of rounding theta (and eta or pi - eta)
    to binary32, from the arithmetic of the FP32 evaluation."""
    a = np.stack([r32["ax"], r32["ay"], r32["az"]], 1).astype(np.float64)
    c = np.stack(grid, 1).astype(np.float64)
    a /= np.linalg.norm(a, axis=1)[:, None]
    c /= np.linalg.norm(c, axis=1)[:, None]
    th = np.arccos(np.clip(c @ a.T, -1, 1))
    r = (th - r32["eta"].astype(np.float64)) / r32["deta"].astype(np.float64)
    dr = 3 * EPS32 * (th + math.pi) / r32["deta"].astype(np.float64)
    return (np.abs(r) * np.exp(-0.5 * r * r) * dr * r32["valid"]).sum(1)


def oracle_rings32(r):
    out = {k: np.asarray(r[k], np.float32) for k in ("ax", "ay", "az", "eta", "deta")}
    out["valid"] = np.asarray(r.get("valid", np.ones(len(r["ax"]))), np.uint8)
    return out


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nside", [1, 2, 3, 64, 256])
def test_healpix_grid_matches_oracle(cc, dev, nside):
    g = cc.grid_healpix_ring(nside, dev)
    torch.cuda.synchronize()
    want = oracle.grid_healpix_ring(nside)
    for a, b in zip(g, want):
        np.testing.assert_allclose(a.cpu().numpy(), b, rtol=0, atol=4e-7)


@pytest.mark.parametrize("n", [1, 7, 3072, 49152, 1000003])
def test_fibonacci_grid_matches_oracle(cc, dev, n):
    g = cc.grid_fibonacci(n, dev)
    torch.cuda.synchronize()
    want = oracle.grid_fibonacci(n)
    for a, b in zip(g, want):
        np.testing.assert_allclose(a.cpu().numpy(), b, rtol=0, atol=1e-6)


# --------------------------------------------------------------------------
# reconstruction
# --------------------------------------------------------------------------
def check_rings(got, want, ev):
    valid = want["valid"] == 1
    np.testing.assert_array_equal(got["valid"], want["valid"])
    np.testing.assert_array_equal(got["perm"][valid], want["perm"][valid])
    assert (got["perm"][~valid] == 255).all()
    for k in ("ax", "ay", "az"):
        np.testing.assert_allclose(got[k][valid], want[k][valid], rtol=0, atol=8 * EPS32)
    # eta: bound from the FP32 arithmetic of cos eta = 1 - u
    u = 1.0 - np.cos(want["eta"][valid])
    err = np.abs(got["eta"][valid] - want["eta"][valid])
    tol = eta_tol(u, want["eta"][valid])
    assert (err <= tol).all(), f"eta: worst {np.max(err / tol):.2f} x tol"
    np.testing.assert_allclose(got["deta"][valid], want["deta"][valid], rtol=2e-5)


def gpu_rings(cc, ev, dev, p):
    n = to_dev(ev["n"], dev)
    x, y, z, e = (to_dev(np.asarray(ev[k], np.float32), dev) for k in "xyze")
    r = cc.rings_from_events(n, x, y, z, e, p)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


@pytest.mark.parametrize("n_src,n_bkg,seed", [(18182, 181818, 2), (333, 1000, 5)])
def test_rings_match_oracle(cc, dev, n_src, n_bkg, seed):
    ev = synth.simulate_events(n_src=n_src, n_bkg=n_bkg, seed=seed)
    p = cc.Params()
    want = oracle.rings_from_events(ev, p.sigma_e_frac, p.sigma_pos_cm, p.deta_min, p.deta_max)
    got = gpu_rings(cc, ev, dev, p)
    check_rings(got, want, ev)
    assert want["valid"].mean() > 0.5


def test_rings_edge_cases(cc, dev):
    """Invalid site counts, coincident sites, impossible energies, a padded
    stride and noise-free tracks, all decided exactly as the oracle does."""
    ev = synth.simulate_events(n_src=200, n_bkg=300, seed=31, sigma_e_frac=0.0,
                               sigma_pos_cm=0.0)
    N = ev["n"].size
    ev["n"][:5] = [0, 1, 5, 255, 4]
    ev["x"][:, 10] = ev["x"][0, 10]       # all sites at one point
    ev["y"][:, 10] = ev["y"][0, 10]
    ev["z"][:, 10] = ev["z"][0, 10]
    ev["e"][:3, 11] = [33.0, 33.0, 34.0]   # no kinematic solution
    ev["n"][11] = 3
    ev["e"][1, 12] = -5.0                  # negative deposit
    pad = {k: np.zeros((4, N + 37), np.float32) for k in "xyze"}
    for k in "xyze":
        pad[k][:, :N] = ev[k]
    ev2 = dict(ev, **pad)
    p = cc.Params()
    want = oracle.rings_from_events(
        {"n": ev["n"], **{k: pad[k] for k in "xyze"}}, p.sigma_e_frac, p.sigma_pos_cm,
        p.deta_min, p.deta_max)
    got = gpu_rings(cc, ev2, dev, p)
    check_rings(got, want, ev2)
    assert not want["valid"][[0, 1, 2, 3, 10, 11]].any()


def test_rings_many_windows_and_misaligned(cc, dev):
    """1.26M events (more 768-event windows than resident CTAs, so every CTA
    runs several windows through its double buffer, and a ragged last
    window), then the same events through arrays that start 4 bytes off a
    16-byte boundary (plain loads) into ring arrays that start 4 or 1 bytes
    off (scalar stores): all equal to the oracle's rings."""
    ev = synth.tile_events(synth.simulate_events(n_src=6000, n_bkg=54000, seed=12), 21)
    N = ev["n"].size
    p = cc.Params()
    want = oracle.rings_from_events(ev, p.sigma_e_frac, p.sigma_pos_cm, p.deta_min, p.deta_max)
    got = gpu_rings(cc, ev, dev, p)
    check_rings(got, want, ev)

    def off(arr, dtype, o):
        flat = torch.zeros(arr.size + o, dtype=dtype, device=dev)
        v = flat[o:].view(arr.shape)
        v.copy_(torch.from_numpy(np.ascontiguousarray(arr)).to(dev))
        return v

    n = off(ev["n"], torch.uint8, 1)
    x, y, z, e = (off(np.asarray(ev[k], np.float32), torch.float32, 1) for k in "xyze")
    out = {k: torch.zeros(N + 1, dtype=torch.float32, device=dev)[1:] for k in
           ("ax", "ay", "az", "eta", "deta")}
    out["valid"] = torch.zeros(N + 1, dtype=torch.uint8, device=dev)[1:]
    out["perm"] = torch.zeros(N + 1, dtype=torch.uint8, device=dev)[1:]
    cc.rings_from_events(n, x, y, z, e, p, out)
    torch.cuda.synchronize()
    check_rings({k: v.cpu().numpy() for k, v in out.items()}, want, ev)


def test_rings_order_extremes(cc, dev):
    """The ordering decision on extreme and degenerate events (see
    extreme_events): validity and the chosen order equal the oracle's bit for
    bit."""
    ev = extreme_events(60000, 91)
    p = cc.Params()
    want = oracle.rings_from_events(ev, p.sigma_e_frac, p.sigma_pos_cm, p.deta_min, p.deta_max)
    with np.errstate(all="ignore"):
        got = gpu_rings(cc, ev, dev, p)
    v = want["valid"] == 1
    np.testing.assert_array_equal(got["valid"], want["valid"])
    np.testing.assert_array_equal(got["perm"][v], want["perm"][v])
    assert (got["perm"][~v] == 255).all()
    assert 0.05 < v.mean() < 0.95
    # the symmetric tracks produce exact chi2 ties between an order and its reverse
    ties = 0
    for i in ev["sym"][:300]:
        x, y, z, e = (ev[k][:3, i] for k in "xyze")
        c = [oracle.order_chi2(x, y, z, e, list(o)) for o in itertools.permutations(range(3))]
        ties += v[i] and sum(1 for t in c if t == min(c)) > 1
    assert ties > 50


def test_rings_empty(cc, dev):
    z = torch.zeros((4, 0), dtype=torch.float32, device=dev)
    r = cc.rings_from_events(torch.zeros(0, dtype=torch.uint8, device=dev), z, z, z, z)
    torch.cuda.synchronize()
    assert r["ax"].numel() == 0


# --------------------------------------------------------------------------
# likelihood map, argmax, seeds
# --------------------------------------------------------------------------
def check_argmax(got_map, am, want_map):
    # exact on the GPU's own map (ties to the lowest index) ...
    assert am == int(np.argmax(got_map))
    # ... and a maximum of the oracle map up to the map tolerance (ties)
    js = int(np.argmax(want_map))
    tol = 1e-5 * max(want_map[js], 1e-3 * want_map[js])
    assert want_map[am] >= want_map[js] - 2 * tol


def test_map_noise_free_burst_full(cc, dev):
    """2,000 noise-free rings x 3,072 Fibonacci directions: every direction."""
    rings, s = synth.rings_noise_free(n=2000, seed=1)
    grid = grid32(oracle.grid_fibonacci(3072))
    got, am, _, st = run_localize(cc, rings, grid, dev)
    want = oracle.likelihood_map(oracle_rings32(rings), grid)
    assert st == 0
    bad = map_violations(got, want, want.max())
    assert bad.size == 0, f"{bad.size} directions off, worst rel " \
        f"{np.max(np.abs(got - want)[bad] / want[bad]):.2e}"
    check_argmax(got, am, want)
    assert ang_deg([grid[0][am], grid[1][am], grid[2][am]], s) < 3.0


@pytest.mark.parametrize("R,M,seed", [(1, 1, 1), (127, 300, 2), (129, 4097, 3),
                                      (1000, 5003, 4), (4096, 257, 5), (20000, 3000, 6)])
def test_map_ragged_sizes(cc, dev, R, M, seed):
    """Sizes that leave ragged ring tiles, ragged direction blocks, one
    direction, and several ring splits."""
    rings, _, _ = synth.rings_burst(n=R, seed=seed)
    grid = grid32(oracle.grid_fibonacci(M))
    got, am, _, st = run_localize(cc, rings, grid, dev)
    want = oracle.likelihood_map(oracle_rings32(rings), grid)
    assert st == 0
    assert map_violations(got, want, want.max()).size == 0
    check_argmax(got, am, want)


def test_map_no_rings_and_invalid_rings(cc, dev):
    grid = grid32(oracle.grid_fibonacci(1000))
    empty = {k: np.zeros(0, np.float32) for k in ("ax", "ay", "az", "eta", "deta")}
    got, am, _, st = run_localize(cc, empty, grid, dev)
    assert st == 0 and (got == 0).all() and am == 0
    rings, _, _ = synth.rings_burst(n=3000, seed=9)
    rings["valid"][::2] = 0
    rings["eta"][1::4] = np.nan                   # garbage in invalid... and valid rings
    rings["valid"][1::4] = 0
    got, am, _, st = run_localize(cc, rings, grid, dev)
    want = oracle.likelihood_map(oracle_rings32(rings), grid)
    assert map_violations(got, want, want.max()).size == 0


def test_map_angular_cut(cc, dev):
    """The cut is a decision taken in floating point: a pair within 1e-5
    (relative) of |r| = k_cut may fall on either side, so the GPU map must lie
    between the oracle maps cut at k_cut (1 -+ 1e-5), up to the map rule."""
    rings, _, _ = synth.rings_burst(n=5000, seed=10)
    grid = grid32(oracle.grid_healpix_ring(16))
    got, am, _, _ = run_localize(cc, rings, grid, dev, k_cut=3.0)
    r32 = oracle_rings32(rings)
    want = oracle.likelihood_map(r32, grid, k_cut=3.0)
    lo = oracle.likelihood_map(r32, grid, k_cut=3.0 * (1 - 1e-5))
    hi = oracle.likelihood_map(r32, grid, k_cut=3.0 * (1 + 1e-5))
    tol = 1e-5 * np.maximum(want, 1e-3 * want.max())
    assert ((got >= lo - tol) & (got <= hi + tol)).all()
    assert am == int(np.argmax(got))
    assert hi[am] + tol[am] >= lo.max() - tol.max()


def test_map_rings_near_poles_and_backscatter(cc, dev):
    """Rings with eta near 0 and pi (mirrored on the GPU) and directions at
    tiny and near-pi angles from ring axes."""
    rng = np.random.default_rng(3)
    a = synth.random_units(rng, 400)
    eta = np.concatenate([rng.uniform(0, 0.02, 100), rng.uniform(math.pi - 0.02, math.pi, 100),
                          rng.uniform(0, math.pi, 200)])
    deta = np.full(400, 0.5 * D2R)
    rings = {"ax": a[:, 0], "ay": a[:, 1], "az": a[:, 2], "eta": eta, "deta": deta}
    # probes: the axes themselves, their antipodes, and random directions
    c = np.concatenate([a[:50], -a[50:100], synth.random_units(rng, 2000)])
    grid = grid32((c[:, 0], c[:, 1], c[:, 2]))
    got, am, _, _ = run_localize(cc, rings, grid, dev)
    r32 = oracle_rings32(rings)
    want = oracle.likelihood_map(r32, grid)
    # directions carried by a few rings of the narrowest width: add the FP32
    # conditioning bound of each term (theta and eta rounded at ~3 eps)
    bound = 1e-5 * np.maximum(want, 1e-3 * want.max()) + fp32_term_bound(r32, grid)
    assert (np.abs(got - want) <= bound).all(), np.max(np.abs(got - want) / bound)


def test_seeds_greedy_suppression_on_gpu_map(cc, dev):
    """Seeds follow the greedy rule on the GPU's own map exactly (borderline
    suppression within 1e-6 of the cosine either way), and agree with the
    oracle's seeds up to ties."""
    rings, s, _ = synth.rings_burst(n=20000, seed=11)
    gnp = grid32(oracle.grid_healpix_ring(32))
    nms = 5 * D2R
    got, am, seeds, st = run_localize(cc, rings, gnp, dev, topk=8, nms_rad=nms)
    c = np.stack(gnp, 1).astype(np.float64)
    cos_nms = math.cos(nms)
    acc = []
    for t in range(8):
        dots = c @ c[acc].T if acc else np.zeros((c.shape[0], 0))
        ambiguous = np.abs(dots - cos_nms) < 1e-6
        sup = (dots > cos_nms).any(1)
        sup[acc] = True
        cand = np.nonzero(~sup)[0]
        best = cand[np.lexsort((cand, -got[cand]))[0]]
        if seeds[t] != best:
            assert ambiguous.any(1)[best] or ambiguous.any(1)[seeds[t]]
        acc.append(int(seeds[t]))
    assert seeds[0] == am
    want = oracle.likelihood_map(oracle_rings32(rings), gnp)
    osd = oracle.seeds(want, gnp, 8, nms)
    tolv = 2e-5 * want.max()
    for a, b in zip(seeds, osd):
        assert abs(want[a] - want[b]) <= tolv


# --------------------------------------------------------------------------
# workload-size parity (sampled)
# --------------------------------------------------------------------------
def sample_dirs(M, am, grid, extra=(), n=256, radius_deg=2.0, seed=0):
    rng = np.random.default_rng(seed)
    c = np.stack(grid, 1).astype(np.float64)
    near = np.nonzero(c @ c[am] > math.cos(radius_deg * D2R))[0]
    idx = np.unique(np.concatenate([rng.choice(M, n, replace=False), near, [am], list(extra)]))
    return idx.astype(np.int64), near


def test_map_event_workload_full(cc, dev):
    """200k simulated events -> oracle rings (FP32) x HEALPix nside 64: every
    one of the 49,152 directions under the map rule against the oracle's full
    FP64 map, and the GPU's argmax the oracle's global maximum up to ties
    (its oracle value within twice the map tolerance of the maximum)."""
    ev = synth.simulate_events(seed=2)
    p = cc.Params()
    r = oracle.rings_from_events(ev, p.sigma_e_frac, p.sigma_pos_cm, p.deta_min, p.deta_max)
    rings = oracle_rings32(r)
    grid = grid32(oracle.grid_healpix_ring(64))
    got, am, _, st = run_localize(cc, rings, grid, dev)
    assert st == 0
    want = oracle.likelihood_map(rings, grid)
    ref_max = want.max()
    bad = map_violations(got, want, ref_max)
    assert bad.size == 0, f"{bad.size} of {want.size} off"
    assert want[am] >= ref_max - 2 * 1e-5 * ref_max
    assert am == int(np.argmax(got))
    assert ang_deg([grid[0][am], grid[1][am], grid[2][am]], ev["source"]) < 3.0


def test_map_large_burst_sampled(cc, dev):
    """1M rings (70 % background, deta 0.5-10 deg) x HEALPix nside 256
    (786,432 directions), top-8 seeds: the full-size workload, checked on
    sampled directions, the argmax neighbourhood and the seeds."""
    rings, s, _ = synth.rings_burst(n=1_000_000, seed=3)
    grid = grid32(oracle.grid_healpix_ring(256))
    got, am, seeds, st = run_localize(cc, rings, grid, dev, topk=8, nms_rad=1 * D2R)
    assert st == 0
    idx, near = sample_dirs(grid[0].size, am, grid, extra=seeds, n=128, radius_deg=0.6)
    want = oracle.likelihood_map(rings, grid, idx=idx)
    ref_max = want.max()
    bad = map_violations(got[idx], want, ref_max)
    assert bad.size == 0, f"{bad.size} of {idx.size} off"
    wn = dict(zip(idx.tolist(), want))
    assert wn[am] >= max(wn[j] for j in near) - 2e-5 * ref_max
    assert ang_deg([grid[0][am], grid[1][am], grid[2][am]], s) < 1.0
    assert (seeds >= 0).all() and len(set(seeds.tolist())) == 8


@pytest.mark.parametrize("nside,R", [(128, 10000), (256, 2000)])
def test_map_fine_grid_full(cc, dev, nside, R):
    """Rings of widths 0.5-20 deg x HEALPix nside 128 (196,608 directions) and
    256 (786,432): every direction under the map rule.  At these nsides the
    warps' patches are narrow enough for the short polynomials of the
    one-sided forms (degree 5 on s <= 0.8 at nside 128, degree 4 on s <= 0.55
    at nside 256), and the widths put rings in every form (equatorial, chord,
    dot)."""
    rings, s, _ = synth.rings_burst(n=R, deta_deg=(0.5, 20.0), seed=13)
    grid = grid32(oracle.grid_healpix_ring(nside))
    got, am, _, st = run_localize(cc, rings, grid, dev)
    assert st == 0
    want = oracle.likelihood_map(oracle_rings32(rings), grid)
    bad = map_violations(got, want, want.max())
    assert bad.size == 0, f"{bad.size} of {want.size} off"
    check_argmax(got, am, want)


# --------------------------------------------------------------------------
# refinement
# --------------------------------------------------------------------------
def run_refine(cc, rings_np, seed_dirs, dev, **pk):
    p = cc.Params(**pk)
    d, obj, it, st = cc.refine(rings_to_dev(rings_np, dev),
                               to_dev(np.asarray(seed_dirs, np.float64).reshape(-1, 3), dev), p)
    torch.cuda.synchronize()
    return d.cpu().numpy(), float(obj.item()), int(it.item()), int(st.item())


def test_refine_noise_free_burst(cc, dev):
    rings, s = synth.rings_noise_free(n=2000, seed=1)
    r32 = oracle_rings32(rings)
    grid = grid32(oracle.grid_fibonacci(3072))
    want_map = oracle.likelihood_map(r32, grid)
    j = oracle.argmax(want_map)
    seed = np.array([grid[0][j], grid[1][j], grid[2][j]], np.float64)
    od, oobj, _, ost = oracle.refine(r32, seed, tol_rad=1e-10)
    gd, gobj, git, gst = run_refine(cc, rings, seed, dev)
    assert ost == 0 and gst == 0
    assert ang_deg(gd, od) < REFINE_TOL_DEG
    assert ang_deg(gd, s) < 0.001
    assert gobj == pytest.approx(oobj, rel=1e-4)


def test_refine_several_seeds_and_status(cc, dev):
    rings, s, _ = synth.rings_burst(n=50000, seed=13)
    rng = np.random.default_rng(1)
    seeds = [s + 0.02 * rng.standard_normal(3) for _ in range(3)] + [-s]
    seeds = np.array([v / np.linalg.norm(v) for v in seeds])
    od, oobj, oit, ost = oracle.refine(oracle_rings32(rings), seeds, tol_rad=1e-10)
    gd, gobj, git, gst = run_refine(cc, rings, seeds, dev)
    assert gst == 0
    assert ang_deg(gd, od) < REFINE_TOL_DEG
    assert gobj == pytest.approx(oobj, rel=1e-4)
    # one iteration allowed: not converged, reported as such
    _, _, it1, st1 = run_refine(cc, rings, seeds, dev, max_iter=1)
    assert st1 == -5 and it1 == 1


def test_refine_from_gpu_seeds_large_burst(cc, dev):
    """The whole plain path at full size on the GPU (sweep -> top-8 -> refine)
    against the oracle refined from its own seeds (the GPU's seed indices are
    never given to the oracle: it seeds from a coarse grid of its own)."""
    rings, s, _ = synth.rings_burst(n=1_000_000, seed=3)
    gnp = grid32(oracle.grid_healpix_ring(256))
    p = cc.Params(topk=8, nms_rad=1 * D2R)
    loc = cc.Localizer(grid_to_dev(gnp, dev), p)
    loc.from_rings(rings_to_dev(rings, dev))
    torch.cuda.synchronize()
    assert int(loc.ref_status.item()) == 0
    gd = loc.dir.cpu().numpy()
    coarse = grid32(oracle.grid_healpix_ring(16))
    cm = oracle.likelihood_map(oracle_rings32(rings), coarse)
    osd = oracle.seeds(cm, coarse, 3, 10 * D2R)
    seeds = np.stack([[coarse[0][j], coarse[1][j], coarse[2][j]] for j in osd]).astype(float)
    od, _, _, ost = oracle.refine(oracle_rings32(rings), seeds, tol_rad=1e-10)
    assert ang_deg(gd, od) < REFINE_TOL_DEG
    assert ang_deg(gd, s) < 0.2


# --------------------------------------------------------------------------
# end to end: events -> rings -> map -> argmax -> refined direction
# --------------------------------------------------------------------------
def test_end_to_end_event_workload(cc, dev):
    ev = synth.simulate_events(seed=2)
    p = cc.Params()
    gnp = grid32(oracle.grid_healpix_ring(64))
    loc = cc.Localizer(grid_to_dev(gnp, dev), p)
    x, y, z, e = (to_dev(np.asarray(ev[k], np.float32), dev) for k in "xyze")
    loc.from_events(to_dev(ev["n"], dev), x, y, z, e)
    torch.cuda.synchronize()
    assert int(loc.loc_status.item()) == 0 and int(loc.ref_status.item()) == 0
    r = oracle.rings_from_events(ev, p.sigma_e_frac, p.sigma_pos_cm, p.deta_min, p.deta_max)
    np.testing.assert_array_equal(loc._rings["perm"].cpu().numpy(), r["perm"])
    coarse = grid32(oracle.grid_healpix_ring(16))
    cm = oracle.likelihood_map(r, coarse)
    j = oracle.argmax(cm)
    od, _, _, ost = oracle.refine(r, [coarse[0][j], coarse[1][j], coarse[2][j]],
                                  tol_rad=1e-10)
    gd = loc.dir.cpu().numpy()
    assert ang_deg(gd, od) < REFINE_TOL_DEG
    # where the likelihood peaks is the method's, not the GPU's: the GPU's
    # distance to the true source is the oracle's own, to the parity bound
    err_gpu, err_or = ang_deg(gd, ev["source"]), ang_deg(od, ev["source"])
    print(f"\nplain method, event workload: {err_gpu:.3f} deg from the source "
          f"(oracle {err_or:.3f} deg; target 0.5 deg)")
    assert abs(err_gpu - err_or) < REFINE_TOL_DEG


@pytest.mark.xfail(strict=True, reason="the plain method's likelihood peaks ~1.46 deg from "
                   "the source on the event workload (background 10:1); the 0.5 deg target "
                   "is not reached by it")
def test_plain_method_reaches_half_a_degree_on_event_workload(cc, dev):
    """The accuracy target on the event workload, for the plain method: an
    explicit, visible gap (strict: it fails loudly once it passes)."""
    ev = synth.simulate_events(seed=2)
    gnp = grid32(oracle.grid_healpix_ring(64))
    loc = cc.Localizer(grid_to_dev(gnp, dev), cc.Params())
    x, y, z, e = (to_dev(np.asarray(ev[k], np.float32), dev) for k in "xyze")
    loc.from_events(to_dev(ev["n"], dev), x, y, z, e)
    torch.cuda.synchronize()
    assert ang_deg(loc.dir.cpu().numpy(), ev["source"]) <= 0.5


# --------------------------------------------------------------------------
# C ABI error behaviour (host-side checks: nothing is launched)
# --------------------------------------------------------------------------
def test_abi_rejects_bad_arguments(cc, dev):
    import ctypes as C
    from paper_2411_04785_gb300 import api
    rings, _, _ = synth.rings_burst(n=100, seed=1)
    rd = rings_to_dev(rings, dev)
    grid = grid_to_dev(oracle.grid_fibonacci(64), dev)
    with pytest.raises(cc.CCError) as ei:
        cc.localize(rd, grid, cc.Params(topk=0))
    assert ei.value.status == -1
    with pytest.raises(cc.CCError) as ei:
        cc.localize(rd, grid, cc.Params(max_iter=0))
    assert ei.value.status == -1
    # a workspace smaller than the query: CC_ENOMEM, nothing launched
    rs, gs, pc = api._rings_struct(rd), api._grid_struct(grid), cc.Params().c()
    m = torch.zeros(64, device=dev)
    am = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(256, dtype=torch.uint8, device=dev)
    st = cc.lib().cc_localize(C.byref(rs), C.byref(gs), C.byref(pc), api._ptr(m),
                              api._ptr(am), None, None, api._ptr(ws), 16, None)
    assert st == -3 and b"workspace" in cc.lib().cc_last_error()
    # misaligned workspace
    st = cc.lib().cc_localize(C.byref(rs), C.byref(gs), C.byref(pc), api._ptr(m),
                              api._ptr(am), None, None, C.c_void_p(ws.data_ptr() + 4),
                              1 << 30, None)
    assert st == -1
    with pytest.raises(cc.CCError) as ei:
        cc.grid_healpix_ring(0, dev)
    assert ei.value.status == -1
    with pytest.raises(cc.CCError):
        cc.refine(rd, torch.zeros((65, 3), dtype=torch.float64, device=dev))
    torch.cuda.synchronize()


def test_exact_reciprocal_and_root_match_the_intrinsics(cc):
    """The ordering decision's correctly rounded reciprocal and square root
    equal __frcp_rn / __fsqrt_rn on every float of [1, 4), hence (the result
    depending only on mantissa and exponent parity there) on [2^-100, 2^100];
    its two-correction quotient equals __fdiv_rn on every float of [1, 2)
    against 64 divisor mantissas, both ways."""
    from paper_2411_04785_gb300 import api
    out = api.selftest_exact_ops("cuda:0")
    torch.cuda.synchronize()
    assert out.view(torch.int64).cpu().tolist() == [0, 0, 0]
