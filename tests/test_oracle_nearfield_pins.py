"""Pins of the near-field back-projection oracle (Sec. 3) against facts
independent of its code: a planted point source, the closed form of one
cone, the far-field limit, linearity, the angular cut, the volume fractions
the paper states for the cylinder and sphere universes, and the apex of a
hand-ordered event."""
import math

import numpy as np
import pytest

import oracle


def random_units(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def cones_through(rng, S, R, deta_deg=1.0):
    """R cones with random apexes in a detector slab, random axes, and eta
    the exact angle at which each passes through the point S (FP64 via the
    normalised dot product)."""
    p = np.column_stack([rng.uniform(-25, 25, R), rng.uniform(-25, 25, R),
                         rng.uniform(-31, 1, R)])
    a = random_units(rng, R)
    d = S[None, :] - p
    cosang = np.sum(d * a, 1) / np.linalg.norm(d, axis=1)
    eta = np.arccos(np.clip(cosang, -1, 1))
    rings = {"ax": a[:, 0], "ay": a[:, 1], "az": a[:, 2], "eta": eta,
             "deta": np.full(R, math.radians(deta_deg)), "valid": np.ones(R, np.uint8)}
    return rings, p


def test_planted_point_source_gets_every_ring():
    rng = np.random.default_rng(1)
    S = np.array([2.0, -3.0, 20.0])
    rings, p = cones_through(rng, S, 3000)
    vox = tuple(np.array([S[c], S[c] + 1.0, S[c]]) for c in range(3))
    L = oracle.backproject(rings, p, vox)
    assert abs(L[0] - 3000) < 3000 * 1e-9          # every term exp(0) = 1
    assert L[1] < 0.9 * 3000                        # off-source voxels lose terms


def test_single_cone_closed_form_at_any_distance():
    eta, deta = math.radians(40.0), math.radians(2.0)
    rings = {"ax": [0.0], "ay": [0.0], "az": [1.0], "eta": [eta], "deta": [deta]}
    p = np.array([[1.0, 2.0, -5.0]])
    th = np.radians([0.0, 10.0, 38.0, 40.0, 43.0, 90.0, 170.0, 180.0])
    for rho in (0.5, 7.0, 300.0):
        for phi in (0.0, 2.1):
            v = p[0][:, None] + rho * np.array([np.sin(th) * np.cos(phi),
                                                np.sin(th) * np.sin(phi), np.cos(th)])
            L = oracle.backproject(rings, p, (v[0], v[1], v[2]))
            want = np.exp(-0.5 * ((th - eta) / deta) ** 2)
            np.testing.assert_allclose(L, want, rtol=1e-12, atol=1e-300)
    # angular selection: |r| > k_cut contributes nothing
    v = p[0][:, None] + 5.0 * np.array([np.sin(th), 0 * th, np.cos(th)])
    L = oracle.backproject(rings, p, (v[0], v[1], v[2]), k_cut=1.6)
    r = np.abs((th - eta) / deta)
    np.testing.assert_allclose(L, np.where(r > 1.6, 0.0, np.exp(-0.5 * r * r)), rtol=1e-12)


def test_far_field_limit_and_linearity():
    rng = np.random.default_rng(3)
    R = 500
    a = random_units(rng, R)
    rings = {"ax": a[:, 0], "ay": a[:, 1], "az": a[:, 2], "eta": rng.uniform(0.1, 3.0, R),
             "deta": rng.uniform(0.01, 0.2, R), "valid": (rng.uniform(size=R) < 0.9).astype(np.uint8)}
    P = np.array([0.5, -1.0, 2.0])
    apex = np.tile(P, (R, 1))
    c = random_units(rng, 40)
    for lam in (0.3, 1.0, 250.0):          # every apex equal: the image along a ray is the sky map
        v = P[None, :] + lam * c
        L = oracle.backproject(rings, apex, (v[:, 0], v[:, 1], v[:, 2]))
        want = [oracle.likelihood(rings, ci) for ci in c]
        np.testing.assert_allclose(L, want, rtol=1e-10, atol=1e-12)
    apex = rng.uniform(-20, 20, (R, 3))
    v = tuple(rng.uniform(-10, 10, 60) for _ in range(3))
    half = {k: np.asarray(x)[:250] for k, x in rings.items()}
    rest = {k: np.asarray(x)[250:] for k, x in rings.items()}
    np.testing.assert_allclose(oracle.backproject(rings, apex, v),
                               oracle.backproject(half, apex[:250], v) +
                               oracle.backproject(rest, apex[250:], v), rtol=1e-12)
    perm = rng.permutation(R)
    shuf = {k: np.asarray(x)[perm] for k, x in rings.items()}
    np.testing.assert_allclose(oracle.backproject(shuf, apex[perm], v),
                               oracle.backproject(rings, apex, v), rtol=1e-12)


def brute_universe(shape, n):
    off = 2 * np.arange(n) + 1 - n
    k, j, i = np.meshgrid(off, off, off, indexing="ij")
    keep = np.ones_like(i, bool)
    if shape == "cylinder":
        keep = i * i + j * j <= n * n
    if shape == "sphere":
        keep = i * i + j * j + k * k <= n * n
    return i[keep], j[keep], k[keep]


@pytest.mark.parametrize("shape", ["cube", "cylinder", "sphere"])
def test_universe_voxels(shape):
    for n in (1, 2, 3, 4, 7, 16):
        i, j, k = brute_universe(shape, n)
        x, y, z = oracle.universe(shape, n, 0.5, center=(1.0, -2.0, 3.0))
        np.testing.assert_array_equal(x, 1.0 + 0.25 * i)          # z-major, then y, x
        np.testing.assert_array_equal(y, -2.0 + 0.25 * j)
        np.testing.assert_array_equal(z, 3.0 + 0.25 * k)


def test_universe_volumes_match_the_paper():
    # Sec. 3: the cylinder has about 21.5 % less volume than its cube, the
    # sphere 47.6 % less, i.e. 1 - pi/4 and 1 - pi/6
    assert abs((1 - math.pi / 4) - 0.215) < 5e-4 and abs((1 - math.pi / 6) - 0.476) < 5e-4
    for n in (64, 128, 256):
        cube = oracle.universe("cube", n, 1.0, count_only=True)
        cyl = oracle.universe("cylinder", n, 1.0, count_only=True)
        sph = oracle.universe("sphere", n, 1.0, count_only=True)
        assert cube == n ** 3
        assert abs(cyl / cube - math.pi / 4) < 4.0 / n      # lattice-point error O(1/n)
        assert abs(sph / cube - math.pi / 6) < 4.0 / n
    assert abs(1 - cyl / cube - 0.215) < 2e-3 and abs(1 - sph / cube - 0.476) < 2e-3


def test_apex_is_the_first_site_of_the_chosen_order():
    # one 3-site event and one 2-site event with known slot orders
    rng = np.random.default_rng(5)
    from paper_2411_04785_gb300 import synth
    ev = synth.simulate_events(n_src=300, n_bkg=0, seed=5, sigma_e_frac=0.0, sigma_pos_cm=0.0,
                               dtype=np.float64)
    r = oracle.rings_from_events(ev, 0.05, 1.0, math.radians(0.5), math.radians(20))
    apex = oracle.ring_apex(ev, r)
    for i in np.flatnonzero(r["valid"])[:100]:
        k = int(ev["n"][i])
        order, rank, _ = oracle.order_event(ev["x"][:k, i], ev["y"][:k, i], ev["z"][:k, i],
                                            ev["e"][:k, i])
        assert rank == r["perm"][i]
        np.testing.assert_array_equal(apex[i], [ev["x"][order[0], i], ev["y"][order[0], i],
                                                ev["z"][order[0], i]])
        # the first rank-th permutation's first slot is rank // (k-1)!
        assert order[0] == rank // math.factorial(k - 1)
    del rng


def test_noise_free_near_field_cones_pass_through_the_point_source():
    """Sec. 1.1 in the near field: noise-free events from a point source give
    cones (oracle rings and apexes) through the source point, except where
    the chosen order is not the true one."""
    from paper_2411_04785_gb300 import synth
    S = np.array([1.0, -2.0, 20.0])
    ev = synth.simulate_events(n_src=2000, n_bkg=0, seed=3, sigma_e_frac=0.0, sigma_pos_cm=0.0,
                               dtype=np.float64, source_point=tuple(S))
    r = oracle.rings_from_events(ev, 0.05, 1.0, math.radians(0.5), math.radians(20))
    v = r["valid"] == 1
    ap = oracle.ring_apex(ev, r)[v]
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)[v]
    d = S[None, :] - ap
    th = np.arctan2(np.linalg.norm(np.cross(d, a), axis=1), np.sum(d * a, 1))
    hit = np.abs(th - r["eta"][v]) < 1e-9
    assert v.mean() > 0.99 and hit.mean() > 0.95
    img = oracle.backproject({k: np.asarray(r[k])[v] for k in ("ax", "ay", "az", "eta", "deta")},
                             ap, tuple(np.array([S[c], S[c] + 2.0]) for c in range(3)))
    assert img[0] >= hit.sum() - 1e-6 and img[0] > img[1]
