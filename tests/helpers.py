"""Shared test helpers: tensors on the device, oracle grids rounded to FP32,
and the tolerance rules the parity tests apply."""
import math

import numpy as np

EPS32 = 2.0 ** -24
MAP_RTOL = 1e-5          # map: |L_gpu - L_or| <= 1e-5 max(L_or, 1e-3 max L_or)
MAP_FLOOR = 1e-3
REFINE_TOL_DEG = 0.01    # refined direction within 0.01 deg of the oracle


def to_dev(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def rings_to_dev(r, dev):
    out = {k: to_dev(np.asarray(r[k], np.float32), dev) for k in ("ax", "ay", "az", "eta", "deta")}
    out["valid"] = to_dev(np.asarray(r.get("valid", np.ones(len(r["ax"]))), np.uint8), dev)
    return out


def grid32(g):
    return tuple(np.asarray(v, np.float32) for v in g)


def grid_to_dev(g, dev):
    return tuple(to_dev(v, dev) for v in grid32(g))


def map_violations(got, want, ref_max):
    """Indices where the map rule fails."""
    bound = MAP_RTOL * np.maximum(want, MAP_FLOOR * ref_max)
    return np.nonzero(np.abs(got - want) > bound)[0]


def ang_deg(a, b):
    a = np.asarray(a, float) / np.linalg.norm(a)
    b = np.asarray(b, float) / np.linalg.norm(b)
    return math.degrees(math.atan2(np.linalg.norm(np.cross(a, b)), float(a @ b)))


def eta_tol(u, eta):
    """Bound on |eta_fp32 - eta_fp64| from the FP32 arithmetic of the ring:
    cos eta = 1 - u with u = m E1 / (E2 E0) rounded ~4 times (relative
    4 eps), then 1 - u (half an ulp of 1) and acosf (2 ulp)."""
    dc = 6.0 * EPS32 * (1.0 + np.abs(u))
    s = np.sin(eta)
    return dc / np.maximum(s, np.sqrt(dc)) * 2.0 + 4.0 * EPS32 * np.maximum(eta, 1e-30)


def extreme_events(N, seed):
    """Events built to reach every branch of the binary32 ordering rule:
    log-uniform magnitudes from 1e-40 to 1e38 with random signs (subnormal,
    overflowing and negative deposits and distances), zeros, infinities and
    NaNs, nearly coincident and coincident pairs, and mirror-symmetric 3-site
    tracks with equal end deposits, whose two directions have bitwise equal
    chi2 (the lower rank must win)."""
    rng = np.random.default_rng(seed)
    n = rng.integers(2, 5, N).astype(np.uint8)
    kind = rng.integers(0, 6, N)
    ev = {k: rng.normal(0.0, 10.0, (4, N)).astype(np.float32) for k in "xyz"}
    ev["e"] = rng.uniform(20.0, 800.0, (4, N)).astype(np.float32)
    ev["n"] = n

    def logu(lo, hi, shape):
        return (10.0 ** rng.uniform(lo, hi, shape)) * rng.choice([-1.0, 1.0], shape)

    m = kind == 0                          # wild magnitudes everywhere
    for k in "xyz":
        ev[k][:, m] = logu(-40, 38, (4, m.sum())).astype(np.float32)
    ev["e"][:, m] = np.abs(logu(-40, 38, (4, m.sum()))).astype(np.float32)
    m = kind == 1                          # wild deposits, some negative or zero
    ev["e"][:, m] = logu(-42, 38, (4, m.sum())).astype(np.float32)
    ev["e"][:, m & (rng.random(N) < 0.2)] = 0.0
    m = np.flatnonzero(kind == 2)          # one pair nearly or exactly coincident
    d = (10.0 ** rng.uniform(-45, -3, m.size)) * rng.choice([0.0, 1.0, 1.0, 1.0], m.size)
    for k in "xyz":
        ev[k][1, m] = (ev[k][0, m] + d).astype(np.float32)
    m = np.flatnonzero(kind == 3)          # mirror-symmetric 3-site tracks
    ev["n"][m] = 3
    c = rng.normal(0.0, 10.0, (3, m.size))
    u = rng.normal(0.0, 2.0, (3, m.size))
    pts = np.stack([c - u, c, c + u])      # [site, coord, event], exact in FP32 below
    pts = np.round(pts * 64.0) / 64.0
    ends = rng.uniform(50.0, 400.0, m.size).astype(np.float32)
    mid = rng.uniform(50.0, 400.0, m.size).astype(np.float32)
    for j, ev_i in enumerate(m):
        slots = rng.permutation(3)        # which slot holds which site
        for s_i, site in enumerate(slots):
            for a, k in enumerate("xyz"):
                ev[k][s_i, ev_i] = pts[site, a, j]
            ev["e"][s_i, ev_i] = mid[j] if site == 1 else ends[j]
    m = kind == 4                          # infinities and NaNs
    bad = rng.choice(np.array([np.inf, -np.inf, np.nan], np.float32), (4, m.sum()))
    which = rng.integers(0, 4, m.sum())
    arr = ev[("x", "y", "z", "e")[int(rng.integers(0, 4))]]
    arr[which, np.flatnonzero(m)] = bad[which, np.arange(m.sum())]
    ev["sym"] = np.setdiff1d(np.flatnonzero(kind == 3), np.flatnonzero(m))
    return ev
