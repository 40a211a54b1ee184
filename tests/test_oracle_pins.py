"""Pins of the CPU oracle against facts fixed outside the oracle itself:
the paper's Compton formula run forward, closed forms, textbook limits,
invariants of noise-free data, brute force on tiny inputs and high-precision
re-evaluation.  CPU only."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2411_04785_gb300 import synth

ME = 510.99895
D2R = math.pi / 180.0


def unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v)


def perp_basis(u):
    ref = np.array([0.0, 0.0, 1.0]) if abs(u[2]) < 0.9 else np.array([1.0, 0, 0])
    p1 = unit(np.cross(u, ref))
    return p1, np.cross(u, p1)


def rotate_from(u, theta, phi):
    """Unit vector at angle theta from u, azimuth phi around it."""
    p1, p2 = perp_basis(u)
    return (math.cos(theta) * u + math.sin(theta) *
            (math.cos(phi) * p1 + math.sin(phi) * p2))


def scattered_energy(e, theta):
    """Sec. 1.1: E' = E / (1 + (E / m_e c^2)(1 - cos theta)), as printed."""
    return e / (1.0 + (e / ME) * (1.0 - math.cos(theta)))


def forward_event(s, e0, thetas, lengths, x1, phis):
    """A noise-free track: photon from direction s (travelling along -s)
    scatters at each of len(thetas) sites, then is absorbed.  Returns site
    positions (true order), deposits and the first scatter angle."""
    u = -unit(s)
    x = np.asarray(x1, float)
    pos, dep = [x.copy()], []
    e = e0
    for th, L, ph in zip(thetas, lengths, phis):
        e_after = scattered_energy(e, th)
        dep.append(e - e_after)
        e = e_after
        u = rotate_from(u, th, ph)
        x = x + L * u
        pos.append(x.copy())
    dep.append(e)
    return np.array(pos), np.array(dep)


def as_events(tracks, slot_orders=None, dtype=np.float64):
    N = len(tracks)
    ev = {"n": np.zeros(N, np.uint8)}
    for k in "xyze":
        ev[k] = np.zeros((4, N), dtype)
    for i, (pos, dep) in enumerate(tracks):
        k = len(dep)
        ev["n"][i] = k
        order = slot_orders[i] if slot_orders is not None else list(range(k))
        for j in range(k):          # true site j goes to slot order[j]
            sl = order[j]
            ev["x"][sl, i], ev["y"][sl, i], ev["z"][sl, i] = pos[j]
            ev["e"][sl, i] = dep[j]
    return ev


PERMS = {k: list(itertools.permutations(range(k))) for k in (2, 3, 4)}


# --------------------------------------------------------------------------
# Compton formula and the noise-free invariant
# --------------------------------------------------------------------------
@pytest.mark.parametrize("e0", [60.0, 200.0, 662.0, 1500.0, 2000.0])
def test_cone_angle_round_trips_the_compton_formula(e0):
    """eta recovered from the deposits equals the forward scatter angle to
    1e-12 (Sec. 1.1 formula inverted), and the axis points at the source."""
    rng = np.random.default_rng(11)
    s = unit([0.3, -0.2, 0.93])
    tracks, first = [], []
    for th in np.linspace(0.15, 2.9, 12):
        th2 = rng.uniform(0.4, 2.6)
        if scattered_energy(scattered_energy(e0, th), th2) <= 0:
            continue
        pos, dep = forward_event(s, e0, [th, th2], [7.0, 9.0], [1.0, 2.0, 0.0],
                                 [rng.uniform(0, 6.28), rng.uniform(0, 6.28)])
        tracks.append((pos, dep))
        first.append(th)
    ev = as_events(tracks)
    r = oracle.rings_from_events(ev, 0.05, 1.0, 0.0, 10.0)
    assert r["valid"].all()
    assert (r["perm"] == 0).all()            # true order is slot order 0,1,2
    np.testing.assert_allclose(r["eta"], first, rtol=0, atol=1e-12)
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    np.testing.assert_allclose(a @ s, np.cos(first), rtol=0, atol=1e-12)


def test_noise_free_rings_pass_through_source():
    """Noise-free simulated events (FP64): every event of 3-4 sites is ordered
    as simulated, and every correctly ordered ring passes through the true
    source: |angle(a, s) - eta| < 1e-11."""
    ev = synth.simulate_events(n_src=3000, n_bkg=0, seed=21, sigma_e_frac=0.0,
                               sigma_pos_cm=0.0, dtype=np.float64)
    r = oracle.rings_from_events(ev, 0.05, 1.0, 0.0, 10.0)
    s = ev["source"]
    good = np.zeros(len(ev["n"]), bool)
    for i, k in enumerate(ev["n"]):
        if r["valid"][i]:
            chosen = PERMS[k][r["perm"][i]]
            good[i] = chosen == tuple(int(v) for v in ev["order"][i][:k])
    k34 = ev["n"] >= 3
    assert good[k34].mean() > 0.995
    assert good[~k34].mean() > 0.8          # 2-site rule: physics only
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)[good]
    th = np.array([oracle.angle(v, s) for v in a])
    assert np.abs(th - r["eta"][good]).max() < 1e-11


# --------------------------------------------------------------------------
# Ordering
# --------------------------------------------------------------------------
def test_true_order_has_zero_chi2_and_wins():
    """For noise-free 3- and 4-site tracks, the true order's Compton chi2 is
    zero to binary32 rounding, and the oracle returns it whatever slot order
    the sites are stored in (rank changes, physical sequence does not)."""
    rng = np.random.default_rng(5)
    s = unit([0.1, 0.4, 0.9])
    for trial in range(60):
        k = 3 + trial % 2
        e0 = rng.uniform(300, 2000)
        ths = rng.uniform(0.3, 2.0, k - 1)
        pos, dep = forward_event(s, e0, ths, rng.uniform(4, 12, k - 1),
                                 rng.uniform(-10, 10, 3),
                                 rng.uniform(0, 6.28, k - 1))
        if dep.min() < 5.0:
            continue
        for order in PERMS[k][:: max(1, len(PERMS[k]) // 5)]:
            ev = as_events([(pos, dep)], [order], np.float32)
            x, y, z, e = (ev[c][:k, 0] for c in "xyze")
            truth = tuple(order)
            chi_true = oracle.order_chi2(x, y, z, e, list(truth))
            assert chi_true < 1e-9
            got = oracle.order_event(x, y, z, e)
            assert got is not None
            assert got[0] == truth
            assert PERMS[k][got[1]] == truth


def test_ordering_is_exhaustive_argmin_lowest_rank():
    """Brute force on tiny events: the chosen rank is the lowest rank among the
    orders of minimal chi2 (ties included: two sites with equal deposits and
    mirror geometry)."""
    rng = np.random.default_rng(7)
    for trial in range(200):
        k = 3 + trial % 2
        x, y, z = (rng.normal(0, 5, k).astype(np.float32) for _ in range(3))
        e = rng.uniform(20, 600, k).astype(np.float32)
        if trial % 10 == 0:           # plant an exact tie
            e[1] = e[0]
        chis = [oracle.order_chi2(x, y, z, e, list(p)) for p in PERMS[k]]
        got = oracle.order_event(x, y, z, e)
        finite = [c for c in chis if np.isfinite(c)]
        if not finite:
            assert got is None
            continue
        best = min(finite)
        want = chis.index(best)
        assert got[1] == want and got[2] == best


def test_order_invalid_when_no_kinematic_solution():
    # a 100 keV photon cannot leave less than 100/(1 + 2*100/511) = 71.9 keV
    # after its first scatter; with three ~33 keV deposits every first site
    # leaves ~67 keV, so cos eta < -1 for every order
    x = np.array([0, 5, 10], np.float32)
    y = np.zeros(3, np.float32)
    z = np.zeros(3, np.float32)
    e = np.array([33.0, 33.0, 34.0], np.float32)
    assert oracle.order_event(x, y, z, e) is None
    # coincident first two sites of every order (all three sites equal)
    assert oracle.order_event(np.zeros(2, np.float32), np.zeros(2, np.float32),
                              np.zeros(2, np.float32),
                              np.array([100, 200], np.float32)) is None


@pytest.mark.parametrize("kappa", [1e-3, 0.2, 1.0, 3.0])
def test_klein_nishina_weight_integrates_to_total_cross_section(kappa):
    """The 2-site rule's weight P^2 (P + 1/P - sin^2) integrated over the
    sphere equals the Klein-Nishina total cross section (in units of
    r_e^2 / 2); its kappa -> 0 limit is the Thomson value 16 pi / 3."""
    c = np.linspace(-1, 1, 200001)
    P = 1.0 / (1.0 + kappa * (1.0 - c))
    w = np.array([oracle.kn_weight_f32(p, cc) for p, cc in
                  zip(P[::50], c[::50])])
    integral = 2 * math.pi * np.trapezoid(w, c[::50])
    k = kappa
    L = math.log(1 + 2 * k)
    sigma = 2 * math.pi * ((1 + k) / k ** 2 * (2 * (1 + k) / (1 + 2 * k) - L / k)
                           + L / (2 * k) - (1 + 3 * k) / (1 + 2 * k) ** 2)
    if kappa < 0.01:
        sigma = 8 * math.pi / 3 * (1 - 2 * k)     # series, avoids cancellation
    assert integral == pytest.approx(2 * sigma, rel=2e-4)


# --------------------------------------------------------------------------
# Ordering: the binary32 decision against the FP64 definition
# --------------------------------------------------------------------------
def _exact_chi2(pos, dep, order):
    """chi2 of one order from the FP32 inputs in 50-digit arithmetic: sums,
    differences and products of the inputs are exact rationals, and only the
    segment lengths are square roots (exact integers on the tracks below,
    wherever the order follows the track)."""
    import mpmath as mp
    from fractions import Fraction as F
    mp.mp.dps = 50
    me = F("510.99895")
    E = [F(float(v)) for v in dep]
    P = [[F(float(c)) for c in p] for p in pos]
    chi2 = mp.mpf(0)
    for j in range(1, len(order) - 1):
        eb = sum(E[order[m]] for m in range(j, len(order)))
        ea = eb - E[order[j]]
        ce = 1 - me * (1 / ea - 1 / eb)
        p, q, r = (P[order[i]] for i in (j - 1, j, j + 1))
        d1 = [b - a for a, b in zip(p, q)]
        d2 = [b - a for a, b in zip(q, r)]
        dot = sum(a * b for a, b in zip(d1, d2))
        nn = sum(v * v for v in d1) * sum(v * v for v in d2)
        n1n2 = mp.sqrt(mp.mpf(nn.numerator) / nn.denominator)
        cg = mp.mpf(dot.numerator) / dot.denominator / n1n2
        chi2 += (mp.mpf(ce.numerator) / ce.denominator - cg) ** 2
    return chi2


def test_order_chi2_f64_closed_forms():
    """The FP64 definition on tracks with integer segment lengths: a right
    angle whose chi2 is (1 - 510.99895/511)^2 in closed form, a 3-4-5 turn
    (cos_G = 3/5) and a 4-site track of two Pythagorean turns; every order
    of each against a 50-digit evaluation, to 1e-14 in sqrt(chi2) (FP64
    rounding of each residual)."""
    cases = [
        ([(0, 0, 0), (3, 0, 0), (3, 4, 0)], [255.5, 255.5, 255.5]),
        ([(0, 0, 0), (5, 0, 0), (8, 4, 0)], [300.0, 420.0, 180.0]),
        ([(1, 2, 3), (1, 2, 15), (4, 6, 15), (4, 6, 27)], [100.0, 250.0, 75.0, 320.0]),
    ]
    # the right angle along the track: cos_G = 0 exactly, cos_E = 1 - m/511
    x, y, z = (np.array([p[c] for p in cases[0][0]], np.float32) for c in range(3))
    got = oracle.order_chi2_f64(x, y, z, np.array(cases[0][1], np.float32), [0, 1, 2])
    assert math.sqrt(got) == pytest.approx(1.0 - ME / 511.0, abs=1e-15)
    for pos, dep in cases:
        k = len(dep)
        x, y, z = (np.array([p[c] for p in pos], np.float32) for c in range(3))
        e = np.array(dep, np.float32)
        for order in PERMS[k]:
            got = oracle.order_chi2_f64(x, y, z, e, list(order))
            try:
                want = float(_exact_chi2(pos, dep, order))
            except ZeroDivisionError:
                want = math.inf
            # the definition's invalid orders (no energy after a site,
            # |cos_E| > 1) are +inf; the exact value is then irrelevant
            if not math.isfinite(got):
                continue
            # each residual cos_E - cos_G carries FP64 rounding of ~1e-16
            # absolute; compare the root of the sum of their squares
            assert abs(math.sqrt(got) - math.sqrt(want)) < 1e-14


def test_order_f64_picks_the_simulated_order_on_noise_free_tracks():
    """On noise-free simulated 3- and 4-site tracks (FP32 inputs) the FP64
    definition's choice is the simulated order, all but a few degenerate
    events; the binary32 decision agrees wherever the bound decides."""
    ev = synth.simulate_events(n_src=3000, n_bkg=0, seed=23, sigma_e_frac=0.0,
                               sigma_pos_cm=0.0)
    chk = oracle.order_check(ev)
    k34 = ev["n"] >= 3
    truth = np.array([PERMS[k].index(tuple(int(v) for v in ev["order"][i][:k]))
                      for i, k in enumerate(ev["n"])])
    assert (chk["rank64"][k34] == truth[k34]).mean() > 0.995
    dec = chk["status"] == oracle.ORDER_DECIDED
    np.testing.assert_array_equal(chk["rank32"][dec], chk["rank64"][dec])


def test_kn_weight_f64_integrates_to_total_cross_section():
    c = np.linspace(-1, 1, 200001)
    for kappa in (0.2, 1.0, 3.0):
        P = 1.0 / (1.0 + kappa * (1.0 - c))
        w = np.array([oracle.kn_weight_f64(p, cc) for p, cc in zip(P[::50], c[::50])])
        integral = 2 * math.pi * np.trapezoid(w, c[::50])
        k = kappa
        L = math.log(1 + 2 * k)
        sigma = 2 * math.pi * ((1 + k) / k ** 2 * (2 * (1 + k) / (1 + 2 * k) - L / k)
                               + L / (2 * k) - (1 + 3 * k) / (1 + 2 * k) ** 2)
        assert integral == pytest.approx(2 * sigma, rel=2e-4)


def test_binary32_bound_holds_for_every_order():
    """The bound the oracle derives on binary32's rounding of each order's
    chi2 (the Klein-Nishina weight for 2 sites) contains the binary32
    sequence's actual value for every valid order of 6,000 simulated
    events, and it is tight enough to decide: its median is below 1e-5 of
    the value wherever the value exceeds 1e-3."""
    ev = synth.simulate_events(n_src=1000, n_bkg=5000, seed=41)
    rel = []
    checked = 0
    for i in range(ev["n"].size):
        k = int(ev["n"][i])
        x, y, z, e = (np.asarray(ev[c][:k, i], np.float32) for c in "xyze")
        e0 = np.float32(e.sum(dtype=np.float32))
        for order in PERMS[k]:
            st, val, bnd = oracle.order_bound(x, y, z, e, list(order))
            c32 = oracle.order_chi2(x, y, z, e, list(order))
            assert (st == 1) == np.isfinite(c32) or st < 0
            if st != 1:
                continue
            if k == 2:
                e2 = np.float32(0.0) + e[order[1]]
                e0 = (np.float32(0.0) + e[0]) + e[1]
                ce = np.float32(1.0) - np.float32(oracle.ME_KEV) * (
                    np.float32(1.0) / e2 - np.float32(1.0) / e0)
                got = oracle.kn_weight_f32(np.float32(e2 / e0), ce)
            else:
                got = c32
            assert abs(float(got) - val) <= bnd, (i, order, got, val, bnd)
            checked += 1
            if abs(val) > 1e-3:
                rel.append(bnd / abs(val))
    assert checked > 10000
    assert np.median(rel) < 1e-5


def _order_report(name, chk):
    st = np.bincount(chk["status"], minlength=4)
    print(f"\n{name}: {st[0]} decided, {st[1]} near ties, {st[2]} near a validity "
          f"threshold, {st[3]} outside the model; ranks differ on "
          f"{int((chk['rank32'] != chk['rank64']).sum())} events in all")
    return st


def test_binary32_decision_is_the_fp64_argmin_event_workload():
    """The 200,000 events of the event workload: on every event the bound
    decides (the FP64 winner's chi2 margin over every other valid order
    exceeds both orders' binary32 bounds, every validity threshold is
    cleared by more than its bound), the binary32 decision is the FP64
    definition's argmin; fewer than 0.1 % of the events are left undecided."""
    ev = synth.simulate_events(n_src=18182, n_bkg=181818, seed=2)
    chk = oracle.order_check(ev)
    st = _order_report("event workload", chk)
    dec = chk["status"] == oracle.ORDER_DECIDED
    np.testing.assert_array_equal(chk["rank32"][dec], chk["rank64"][dec])
    assert st[3] == 0
    assert (~dec).mean() < 1e-3


def test_binary32_decision_is_the_fp64_argmin_extremes():
    """The 60,000 extreme and degenerate events of the GPU ordering test
    (magnitudes from 1e-40 to 1e38, zeros, negative deposits, infinities,
    NaNs, coincident pairs, mirror-symmetric tracks): on every event the
    bound decides, the binary32 decision is the FP64 argmin.  Most of the
    rest lies outside the binary32 range or on an exact tie, which the
    lowest-rank rule settles in both precisions alike."""
    from tests.helpers import extreme_events
    ev = extreme_events(60000, 91)
    with np.errstate(all="ignore"):
        chk = oracle.order_check(ev)
    st = _order_report("extreme events", chk)
    dec = chk["status"] == oracle.ORDER_DECIDED
    np.testing.assert_array_equal(chk["rank32"][dec], chk["rank64"][dec])
    assert dec.sum() > 15000 and (chk["rank64"][dec] >= 0).sum() > 8000


# --------------------------------------------------------------------------
# Ring width
# --------------------------------------------------------------------------
def _ring_stats(sig_e, sig_pos, n_draw=6000, seed=3):
    rng = np.random.default_rng(seed)
    s = unit([0.2, 0.1, 0.97])
    pos, dep = forward_event(s, 800.0, [1.1, 1.3], [20.0, 15.0],
                             [0.0, 0.0, 0.0], [0.7, 2.0])
    tracks = []
    for _ in range(n_draw):
        p = pos + sig_pos * rng.standard_normal(pos.shape)
        d = dep * (1 + sig_e * rng.standard_normal(dep.shape))
        tracks.append((p, d))
    ev = as_events(tracks)
    r = oracle.rings_from_events(ev, sig_e, sig_pos, 0.0, 10.0)
    ok = (r["valid"] == 1) & (r["perm"] == 0)
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)[ok]
    resid = np.arccos(np.clip(a @ s, -1, 1)) - r["eta"][ok]
    return resid, r["deta"][ok], ok.mean()


def test_deta_energy_term_matches_scatter_of_eta():
    resid, deta, frac = _ring_stats(0.02, 0.0)
    assert frac > 0.95
    assert np.std(resid) / np.mean(deta) == pytest.approx(1.0, abs=0.1)


def test_deta_position_term_matches_scatter_of_axis():
    resid, deta, frac = _ring_stats(0.0, 0.3)
    assert frac > 0.95
    assert np.std(resid) / np.mean(deta) == pytest.approx(1.0, abs=0.1)


def test_deta_combined_and_clamped():
    resid, deta, _ = _ring_stats(0.02, 0.3)
    assert np.std(resid) / np.mean(deta) == pytest.approx(1.0, abs=0.1)
    ev = synth.simulate_events(n_src=500, n_bkg=500, seed=9)
    lo, hi = 0.5 * D2R, 20 * D2R
    r = oracle.rings_from_events(ev, 0.05, 1.0, lo, hi)
    d = r["deta"][r["valid"] == 1]
    assert d.min() >= lo and d.max() <= hi
    assert (d == lo).any() or (d == hi).any()


# --------------------------------------------------------------------------
# Likelihood map
# --------------------------------------------------------------------------
def test_noise_free_source_probe_sums_to_ring_count():
    rings, s = synth.rings_noise_free(n=2000, dtype=np.float64)
    assert oracle.likelihood(rings, s) == pytest.approx(2000.0, abs=1e-9)


def test_single_ring_closed_form_including_poles():
    a = unit([0.3, 0.5, -0.4])
    eta, deta = 0.9, 0.02
    ring = {"ax": [a[0]], "ay": [a[1]], "az": [a[2]], "eta": [eta],
            "deta": [deta]}
    thetas = np.array([1e-7, 1e-4, 0.3, 0.88, 0.9, 0.93, 1.5, 2.5,
                       math.pi - 1e-4, math.pi - 1e-7])
    dirs = np.array([rotate_from(a, t, 0.37 * i) for i, t in enumerate(thetas)])
    L = oracle.likelihood_map(ring, (dirs[:, 0], dirs[:, 1], dirs[:, 2]))
    want = np.exp(-0.5 * ((thetas - eta) / deta) ** 2)
    np.testing.assert_allclose(L, want, rtol=1e-12, atol=1e-300)
    # a ring through the pole direction
    ring2 = dict(ring, eta=[1e-5], deta=[1e-5])
    L2 = oracle.likelihood_map(ring2, (dirs[:2, 0], dirs[:2, 1], dirs[:2, 2]))
    np.testing.assert_allclose(L2, np.exp(-0.5 * ((thetas[:2] - 1e-5) / 1e-5) ** 2),
                               rtol=1e-9)


def test_map_matches_high_precision_evaluation():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rings, _, _ = synth.rings_burst(n=40, seed=4)
    gx, gy, gz = oracle.grid_fibonacci(64)
    L = oracle.likelihood_map(rings, (gx, gy, gz))
    for j in range(0, 64, 7):
        tot = mpmath.mpf(0)
        c = [mpmath.mpf(float(v)) for v in (gx[j], gy[j], gz[j])]
        for i in range(40):
            a = [mpmath.mpf(float(rings[k][i])) for k in ("ax", "ay", "az")]
            na = mpmath.sqrt(sum(v * v for v in a))
            nc = mpmath.sqrt(sum(v * v for v in c))
            cosang = sum(p * q for p, q in zip(a, c)) / (na * nc)
            th = mpmath.acos(max(min(cosang, 1), -1))
            r = (th - mpmath.mpf(float(rings["eta"][i]))) / mpmath.mpf(float(rings["deta"][i]))
            tot += mpmath.exp(-r * r / 2)
        assert float(tot) == pytest.approx(L[j], rel=1e-12, abs=1e-300)


def test_map_is_linear_and_order_free():
    rings, _, _ = synth.rings_burst(n=3000, seed=8)
    grid = oracle.grid_healpix_ring(4)
    full = oracle.likelihood_map(rings, grid)
    A = {k: v[:1200] for k, v in rings.items()}
    B = {k: v[1200:] for k, v in rings.items()}
    np.testing.assert_allclose(full, oracle.likelihood_map(A, grid) +
                               oracle.likelihood_map(B, grid), rtol=1e-12)
    p = np.random.default_rng(1).permutation(3000)
    np.testing.assert_allclose(full, oracle.likelihood_map(
        {k: v[p] for k, v in rings.items()}, grid), rtol=1e-12)
    # an invalid ring contributes nothing
    inv = {k: v.copy() for k, v in rings.items()}
    inv["valid"][::3] = 0
    keep = {k: v[inv["valid"] == 1] for k, v in rings.items()}
    np.testing.assert_allclose(oracle.likelihood_map(inv, grid),
                               oracle.likelihood_map(keep, grid), rtol=1e-12)


def test_angular_cut_drops_only_far_terms():
    a = unit([0.0, 0.6, 0.8])
    ring = {"ax": [a[0]], "ay": [a[1]], "az": [a[2]], "eta": [0.5],
            "deta": [0.1]}
    thetas = np.array([0.5, 0.7, 0.99, 1.01, 1.2])   # r = 0, 2, 4.9, 5.1, 7
    d = np.array([rotate_from(a, t, 1.0) for t in thetas])
    L = oracle.likelihood_map(ring, (d[:, 0], d[:, 1], d[:, 2]), k_cut=5.0)
    r = (thetas - 0.5) / 0.1
    want = np.where(np.abs(r) > 5.0, 0.0, np.exp(-0.5 * r * r))
    np.testing.assert_allclose(L, want, rtol=1e-12, atol=0)


# --------------------------------------------------------------------------
# Argmax and seeds
# --------------------------------------------------------------------------
def test_argmax_ties_go_to_lowest_index():
    assert oracle.argmax(np.array([0.0, 2.0, 5.0, 5.0, 1.0])) == 2
    assert oracle.argmax(np.array([7.0])) == 0


def test_seeds_greedy_suppression():
    grid = oracle.grid_healpix_ring(16)
    c = np.stack(grid, 1)
    peaks = [unit([0, 0, 1]), unit([1, 0, 0.2]), unit([-0.3, -1, -0.5])]
    heights = [10.0, 8.0, 6.0]
    m = np.zeros(c.shape[0])
    for p, h in zip(peaks, heights):   # smooth bumps: shoulders are near-max
        m += h * np.exp(-0.5 * (np.arccos(np.clip(c @ p, -1, 1)) / 0.1) ** 2)
    nms = 20 * D2R
    got = oracle.seeds(m, grid, 3, nms)
    for g, p in zip(got, peaks):
        assert np.arccos(np.clip(c[g] @ p, -1, 1)) < 5 * D2R
    # without suppression the top 3 are all on the first bump
    got0 = oracle.seeds(m, grid, 3, 0.0)
    assert all(np.arccos(np.clip(c[g] @ peaks[0], -1, 1)) < 10 * D2R for g in got0)
    assert list(got0) == list(np.lexsort((np.arange(m.size), -m))[:3])


# --------------------------------------------------------------------------
# Refinement
# --------------------------------------------------------------------------
def test_refine_recovers_planted_source_exactly():
    rings, s = synth.rings_noise_free(n=2000, dtype=np.float64)
    rng = np.random.default_rng(2)
    for _ in range(4):
        seed = rotate_from(s, rng.uniform(0.5, 3.0) * D2R, rng.uniform(0, 6.28))
        d, obj, iters, st = oracle.refine(rings, seed, tol_rad=1e-12)
        assert st == 0
        assert oracle.angle(d, s) < 1e-9
        assert obj == pytest.approx(2000.0, abs=1e-6)


def test_refine_finds_local_maximum_of_noisy_burst():
    rings, s, _ = synth.rings_burst(n=600, bkg_frac=0.5, seed=12,
                                    source=unit([0.5, 0.5, 0.7]))
    d, obj, iters, st = oracle.refine(rings, s, tol_rad=1e-12)
    assert st == 0
    # dense FP64 search on a local tangent grid around the result: no
    # direction within 0.5 deg beats it, coarse-to-fine down to 0.0005 deg
    p1, p2 = perp_basis(d)
    best, best_L = d, oracle.likelihood(rings, d)
    centre = d
    for step_deg, half in ((0.05, 10), (0.005, 10), (0.0005, 10)):
        u = np.arange(-half, half + 1) * step_deg * D2R
        pts = [unit(centre + a * p1 + b * p2) for a in u for b in u]
        Ls = oracle.likelihood_map(rings, tuple(np.array(pts).T))
        k = int(np.argmax(Ls))
        if Ls[k] > best_L:
            best, best_L = pts[k], Ls[k]
        centre = pts[k]
    assert oracle.angle(best, d) < 0.002 * D2R
    assert obj == pytest.approx(oracle.likelihood(rings, d), rel=1e-12)


def test_refine_picks_best_of_several_seeds():
    rings, s = synth.rings_noise_free(n=500, dtype=np.float64)
    far = unit(-s + np.array([0.1, 0.0, 0.0]))
    near = rotate_from(s, 1.0 * D2R, 0.3)
    d, obj, _, st = oracle.refine(rings, np.stack([far, near]))
    assert oracle.angle(d, s) < 1e-8 and st == 0


# --------------------------------------------------------------------------
# Grids
# --------------------------------------------------------------------------
def test_healpix_base_pixels():
    """nside 1: the 12 base pixels sit at z = 2/3, 0, -2/3 with azimuths
    pi/4 + k pi/2 (polar rows) and k pi/2 (equatorial row)."""
    x, y, z = oracle.grid_healpix_ring(1)
    phi = np.mod(np.arctan2(y, x), 2 * math.pi)
    np.testing.assert_allclose(z, [2 / 3] * 4 + [0] * 4 + [-2 / 3] * 4, atol=1e-15)
    want = np.array([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7]) * math.pi / 4
    np.testing.assert_allclose(phi, want, atol=1e-12)


@pytest.mark.parametrize("nside", [2, 4, 16, 64])
def test_healpix_ring_structure_and_equal_area(nside):
    x, y, z = oracle.grid_healpix_ring(nside)
    npix = 12 * nside * nside
    assert x.size == npix
    np.testing.assert_allclose(x * x + y * y + z * z, 1.0, atol=1e-14)
    # rings: z non-increasing with index, 4 nside - 1 rings
    assert np.all(np.diff(z) <= 1e-15)
    zr, start, counts = np.unique(-z, return_index=True, return_counts=True)
    zr = -zr
    assert zr.size == 4 * nside - 1
    want_counts = [min(4 * i, 4 * nside, 4 * (4 * nside - i))
                   for i in range(1, 4 * nside)]
    assert list(counts) == want_counts
    # equal area: the solid angle above a ring's centre line holds the
    # pixels of earlier rings plus half of this ring's pixels
    above = np.concatenate([[0], np.cumsum(counts)[:-1]]) + counts / 2
    np.testing.assert_allclose(2 * math.pi * (1 - zr), above * 4 * math.pi / npix,
                               atol=1e-12)
    # azimuths: equally spaced within a ring, increasing, first one at half a
    # step (shifted rings) or at 0
    for r0, cnt in zip(start, counts):
        ph = np.mod(np.arctan2(y[r0:r0 + cnt], x[r0:r0 + cnt]), 2 * math.pi)
        step = 2 * math.pi / cnt
        off = ph[0] / step
        assert min(abs(off - 0.5), abs(off)) < 1e-9
        np.testing.assert_allclose(np.diff(ph), step, atol=1e-9)
    assert np.linalg.norm([x.sum(), y.sum(), z.sum()]) < 1e-9 * npix


def test_healpix_neighbour_spacing():
    nside = 32
    c = np.stack(oracle.grid_healpix_ring(nside), 1)
    spacing = math.sqrt(4 * math.pi / c.shape[0])
    sub = c[::97]
    d = np.arccos(np.clip(sub @ c.T, -1, 1))
    d[d < 1e-6] = 9
    nn = d.min(1)
    assert nn.min() > 0.6 * spacing and nn.max() < 1.3 * spacing


def test_fibonacci_grid_properties():
    n = 3072
    x, y, z = oracle.grid_fibonacci(n)
    np.testing.assert_allclose(x * x + y * y + z * z, 1.0, atol=1e-14)
    np.testing.assert_allclose(np.diff(z), -2.0 / n, atol=1e-14)
    assert z[0] == pytest.approx(1 - 1.0 / n) and z[-1] == pytest.approx(-1 + 1.0 / n)
    phi = np.arctan2(y, x)
    dphi = np.mod(np.diff(phi), 2 * math.pi)
    golden = math.pi * (3 - math.sqrt(5))
    np.testing.assert_allclose(dphi, golden, atol=1e-12)
    c = np.stack([x, y, z], 1)
    d = np.arccos(np.clip(c[::50] @ c.T, -1, 1))
    d[d < 1e-6] = 9
    spacing = math.sqrt(4 * math.pi / n)
    assert d.min(1).min() > 0.5 * spacing
    assert np.linalg.norm(c.sum(0)) < 1e-4 * n


# --------------------------------------------------------------------------
# HEALPix NESTED: the same pixels as RING, ordered hierarchically
# --------------------------------------------------------------------------
def test_healpix_nest_is_a_permutation_of_ring():
    assert np.array_equal(np.stack(oracle.grid_healpix_nest(1)), np.stack(oracle.grid_healpix_ring(1)))
    for nside in (2, 4, 8, 16):
        nv = np.stack(oracle.grid_healpix_nest(nside), 1)
        rv = np.stack(oracle.grid_healpix_ring(nside), 1)
        d = nv @ rv.T                                     # cosines, nest x ring
        best = d.argmax(1)
        assert np.unique(best).size == nv.shape[0]        # a bijection
        assert (1.0 - d[np.arange(nv.shape[0]), best]).max() < 1e-12


def test_healpix_nest_hierarchy():
    """NESTED index p at nside n has children 4p .. 4p+3 at nside 2n: each
    child's nearest pixel centre at nside n is its parent's."""
    for n in (1, 2, 4, 8):
        par = np.stack(oracle.grid_healpix_nest(n), 1)
        kid = np.stack(oracle.grid_healpix_nest(2 * n), 1)
        nearest = (kid @ par.T).argmax(1)
        np.testing.assert_array_equal(nearest, np.arange(kid.shape[0]) // 4)


def test_healpix_nest_patches_are_compact():
    # 1024 consecutive NESTED pixels at nside 64 form a 32 x 32 block of one
    # base face (radius <= 26 deg); 1024 consecutive RING pixels are
    # latitude strips around the sphere (wide except near the poles)
    def radius(blk):
        c = blk.sum(0)
        c /= np.linalg.norm(c)
        return np.degrees(np.arccos(np.clip(blk @ c, -1, 1)).max())
    v = np.stack(oracle.grid_healpix_nest(64), 1)
    r = np.stack(oracle.grid_healpix_ring(64), 1)
    rn = [radius(v[b * 1024:(b + 1) * 1024]) for b in range(48)]
    rr = [radius(r[b * 1024:(b + 1) * 1024]) for b in range(48)]
    assert max(rn) < 26.0 and np.mean(rr) > 2.0 * np.mean(rn)
