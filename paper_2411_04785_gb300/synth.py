"""Seeded synthetic inputs for the Compton ring-localisation path.

This module only generates inputs: rings and detector events with the shapes
and distributions of the three plain-method workloads (2,000 noise-free rings
on a 3,072-direction Fibonacci grid; 200k simulated 2-4-site events in a
4-layer 50 x 50 cm detector on a HEALPix nside-64 grid; 1M rings with 70 %
background on a HEALPix nside-256 grid).  It holds none of the localisation
arithmetic (no ordering, no cone reconstruction, no likelihood): the event
simulator runs the physics forward (Compton scattering with Klein-Nishina
angles, full absorption at the last site) and the ring generators place rings
around a chosen source.  Both the CUDA path and the CPU oracle consume what it
returns.

Everything is numpy with an explicit ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math

import numpy as np

ME_KEV = 510.99895  # electron rest energy, keV (CODATA)

# Detector of the event workload: 4 square layers, 50 x 50 cm, 1.5 cm thick,
# centred at z = 0, -10, -20, -30 cm.
LAYER_HALF_XY = 25.0
LAYER_HALF_T = 0.75
LAYER_Z = np.array([0.0, -10.0, -20.0, -30.0])
MEAN_PATH_CM = 5.0
SITE_PROBS = (0.5, 0.3, 0.2)  # k = 2, 3, 4
E_MIN, E_MAX = 50.0, 2000.0


def unit_from_angles(theta_deg: float, phi_deg: float) -> np.ndarray:
    """Unit vector at colatitude theta (from +z) and azimuth phi (from +x)."""
    t, p = math.radians(theta_deg), math.radians(phi_deg)
    return np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p),
                     math.cos(t)])


def random_units(rng: np.random.Generator, n: int) -> np.ndarray:
    """n directions uniform on the sphere (z ~ U[-1,1], phi ~ U[0, 2 pi))."""
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def _rings_dict(a, eta, deta):
    a32 = a.astype(np.float32)
    return {"ax": np.ascontiguousarray(a32[:, 0]),
            "ay": np.ascontiguousarray(a32[:, 1]),
            "az": np.ascontiguousarray(a32[:, 2]),
            "eta": eta.astype(np.float32),
            "deta": deta.astype(np.float32),
            "valid": np.ones(a.shape[0], dtype=np.uint8)}


# --------------------------------------------------------------------------
# Ring workloads
# --------------------------------------------------------------------------
def rings_noise_free(n: int = 2000, theta_deg: float = 30.0,
                     phi_deg: float = 45.0, deta_deg: float = 1.0,
                     seed: int = 1, dtype=np.float32):
    """Noise-free rings through one source: axes uniform on the sphere, eta
    the exact angle between axis and source (FP64), then rounded to ``dtype``.
    Returns (rings dict, source unit vector)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = unit_from_angles(theta_deg, phi_deg)
    a = random_units(rng, n)
    eta = np.arccos(np.clip(a @ s, -1.0, 1.0))
    deta = np.full(n, math.radians(deta_deg))
    if dtype == np.float64:
        r = {"ax": a[:, 0].copy(), "ay": a[:, 1].copy(), "az": a[:, 2].copy(),
             "eta": eta, "deta": deta, "valid": np.ones(n, np.uint8)}
        return r, s
    return _rings_dict(a, eta, deta), s


def rings_burst(n: int = 1_000_000, bkg_frac: float = 0.7,
                deta_deg=(0.5, 10.0), seed: int = 3, source=None):
    """Large burst: source rings with axes uniform and eta = angle(axis, s) +
    deta * N(0,1); background rings with axes uniform and cos eta ~ U[-1,1];
    deta log-uniform over ``deta_deg``.  The source direction is a seeded
    random direction unless given.  Returns (rings dict, source, is_source)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = random_units(rng, 1)[0] if source is None else np.asarray(source, float)
    n_bkg = int(round(n * bkg_frac))
    n_src = n - n_bkg
    a = random_units(rng, n)
    lo, hi = (math.radians(v) for v in deta_deg)
    deta = np.exp(rng.uniform(math.log(lo), math.log(hi), n))
    eta = np.empty(n)
    eta[:n_src] = np.arccos(np.clip(a[:n_src] @ s, -1.0, 1.0)) + \
        deta[:n_src] * rng.standard_normal(n_src)
    eta[n_src:] = np.arccos(rng.uniform(-1.0, 1.0, n_bkg))
    is_src = np.zeros(n, bool)
    is_src[:n_src] = True
    perm = rng.permutation(n)
    return _rings_dict(a[perm], eta[perm], deta[perm]), s, is_src[perm]


# --------------------------------------------------------------------------
# Event simulator
# --------------------------------------------------------------------------
def _band_table(alpha=-1.0, beta=-2.3, e_peak=300.0, n=20000):
    """Inverse-CDF table of the Band photon spectrum on [E_MIN, E_MAX]."""
    e = np.geomspace(E_MIN, E_MAX, n)
    e0 = e_peak / (2.0 + alpha)
    eb = (alpha - beta) * e0
    low = e ** alpha * np.exp(-e / e0)
    high = eb ** (alpha - beta) * math.exp(beta - alpha) * e ** beta
    f = np.where(e < eb, low, high)
    # trapezoid CDF on the log grid
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(e))])
    return e, cdf / cdf[-1]


def _sample_band(rng, n):
    e, cdf = _band_table()
    return np.interp(rng.uniform(0.0, 1.0, n), cdf, e)


def _sample_power_m2(rng, n):
    """E^-2 over [E_MIN, E_MAX] by its closed-form inverse CDF."""
    u = rng.uniform(0.0, 1.0, n)
    return 1.0 / (1.0 / E_MIN - u * (1.0 / E_MIN - 1.0 / E_MAX))


def _sample_kn_cos(rng, energy):
    """Scatter cosines from the Klein-Nishina distribution by rejection
    against its maximum (2, at cos = 1)."""
    out = np.empty(energy.shape[0])
    todo = np.arange(energy.shape[0])
    while todo.size:
        c = rng.uniform(-1.0, 1.0, todo.size)
        p = 1.0 / (1.0 + energy[todo] / ME_KEV * (1.0 - c))
        f = p * p * (p + 1.0 / p - (1.0 - c * c))
        acc = rng.uniform(0.0, 2.0, todo.size) < f
        out[todo[acc]] = c[acc]
        todo = todo[~acc]
    return out


def _rotate(u, cos_t, phi):
    """Directions at angle acos(cos_t) from u, azimuth phi around u."""
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    ref = np.where(np.abs(u[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]),
                   np.array([[1.0, 0.0, 0.0]]))
    p1 = np.cross(u, ref)
    p1 /= np.linalg.norm(p1, axis=1, keepdims=True)
    p2 = np.cross(u, p1)
    return (cos_t[:, None] * u + (sin_t * np.cos(phi))[:, None] * p1 +
            (sin_t * np.sin(phi))[:, None] * p2)


def _inside(p):
    inxy = (np.abs(p[:, 0]) <= LAYER_HALF_XY) & (np.abs(p[:, 1]) <= LAYER_HALF_XY)
    inz = np.any(np.abs(p[:, 2:3] - LAYER_Z[None, :]) <= LAYER_HALF_T, axis=1)
    return inxy & inz


def _first_points(rng, n):
    layer = rng.integers(0, LAYER_Z.size, n)
    return np.stack([rng.uniform(-LAYER_HALF_XY, LAYER_HALF_XY, n),
                     rng.uniform(-LAYER_HALF_XY, LAYER_HALF_XY, n),
                     LAYER_Z[layer] + rng.uniform(-LAYER_HALF_T, LAYER_HALF_T, n)],
                    axis=1)


def _simulate_tracks(rng, e0, u0, k, max_tries=64, point=None, from_point=None):
    """Forward Compton tracks: k-1 Klein-Nishina scatters then full
    absorption.  Rows in ``from_point`` come from the point ``point`` (their
    direction is the one from it to their first site) instead of u0.
    Returns positions [n,4,3], deposits [n,4] and a mask of the tracks whose
    every site fell inside a layer."""
    n = e0.shape[0]
    pos = np.zeros((n, 4, 3))
    dep = np.zeros((n, 4))
    ok = np.ones(n, bool)
    p = _first_points(rng, n)
    u = u0.copy()
    if point is not None and from_point is not None and from_point.any():
        d = p[from_point] - np.asarray(point, float)[None, :]
        u[from_point] = d / np.linalg.norm(d, axis=1, keepdims=True)
    e = e0.copy()
    pos[:, 0] = p
    for j in range(3):
        scat = k > j + 1          # site j scatters, a later site exists
        if not scat.any():
            break
        idx = np.nonzero(scat)[0]
        c = _sample_kn_cos(rng, e[idx])
        e_after = e[idx] / (1.0 + e[idx] / ME_KEV * (1.0 - c))
        dep[idx, j] = e[idx] - e_after
        e[idx] = e_after
        u[idx] = _rotate(u[idx], c, rng.uniform(0.0, 2.0 * math.pi, idx.size))
        nxt = np.zeros((idx.size, 3))
        pending = np.arange(idx.size)
        for _ in range(max_tries):
            if not pending.size:
                break
            d = rng.exponential(MEAN_PATH_CM, pending.size)
            cand = p[idx[pending]] + d[:, None] * u[idx[pending]]
            good = _inside(cand)
            nxt[pending[good]] = cand[good]
            pending = pending[~good]
        ok[idx[pending]] = False
        p[idx] = nxt
        pos[idx, j + 1] = nxt
    last = k - 1
    dep[np.arange(n), last] = e
    return pos, dep, ok


def simulate_events(n_src: int = 18182, n_bkg: int = 181818, seed: int = 2,
                    theta_deg: float = 30.0, phi_deg: float = 45.0,
                    sigma_e_frac: float = 0.05, sigma_pos_cm: float = 1.0,
                    source=None, dtype=np.float32, source_point=None):
    """Detector events: source photons (Band spectrum, alpha -1, beta -2.3,
    E_peak 300 keV, 50 keV - 2 MeV) from one direction and isotropic
    background photons (E^-2, 50 keV - 2 MeV); k = 2/3/4 sites with
    probabilities 0.5/0.3/0.2; Gaussian noise sigma_e_frac of each deposit and
    sigma_pos_cm per axis.  Sites are stored in a random slot order.  With
    ``source_point`` (cm) the source is a point at that position instead of a
    direction at infinity (near field): each source photon travels from it to
    its first site.

    Returns a dict: n [N] u8; x, y, z, e [4, N] ``dtype`` (slot-major, unused
    slots 0); truth: order [N, 4] (slot of the j-th true site), is_source [N],
    energy [N] (keV), source (unit vector)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = unit_from_angles(theta_deg, phi_deg) if source is None else \
        np.asarray(source, float)
    n = n_src + n_bkg
    is_src = np.zeros(n, bool)
    is_src[:n_src] = True
    pos = np.zeros((n, 4, 3))
    dep = np.zeros((n, 4))
    kk = np.zeros(n, np.int64)
    energy = np.zeros(n)
    todo = np.arange(n)
    while todo.size:
        m = todo.size
        src = is_src[todo]
        e0 = np.where(src, _sample_band(rng, m), _sample_power_m2(rng, m))
        u0 = np.where(src[:, None], -s[None, :], -random_units(rng, m))
        k = rng.choice(np.array([2, 3, 4]), size=m, p=SITE_PROBS)
        p_, d_, ok = _simulate_tracks(rng, e0, u0, k, point=source_point,
                                      from_point=src if source_point is not None else None)
        done = todo[ok]
        pos[done], dep[done], kk[done], energy[done] = p_[ok], d_[ok], k[ok], e0[ok]
        todo = todo[~ok]

    # noise
    if sigma_e_frac > 0:
        dep = dep * (1.0 + sigma_e_frac * rng.standard_normal(dep.shape))
    if sigma_pos_cm > 0:
        pos = pos + sigma_pos_cm * rng.standard_normal(pos.shape)
    slot_mask = np.arange(4)[None, :] < kk[:, None]
    dep = np.where(slot_mask, dep, 0.0)
    pos = np.where(slot_mask[:, :, None], pos, 0.0)

    # random slot order per event: slot[i, j] = slot holding true site j
    keys = rng.uniform(size=(n, 4)) + np.where(slot_mask, 0.0, 2.0)
    slot_of_site = np.argsort(np.argsort(keys, axis=1), axis=1)
    x = np.zeros((4, n))
    y = np.zeros((4, n))
    z = np.zeros((4, n))
    e = np.zeros((4, n))
    rows = np.arange(n)
    for j in range(4):
        sl = slot_of_site[:, j]
        x[sl, rows] = pos[:, j, 0]
        y[sl, rows] = pos[:, j, 1]
        z[sl, rows] = pos[:, j, 2]
        e[sl, rows] = dep[:, j]
    order = np.where(slot_mask, slot_of_site, -1).astype(np.int8)

    perm = rng.permutation(n)
    cast = lambda a: np.ascontiguousarray(a[:, perm], dtype=dtype)
    return {"n": kk[perm].astype(np.uint8), "x": cast(x), "y": cast(y),
            "z": cast(z), "e": cast(e), "order": order[perm],
            "is_source": is_src[perm], "energy": energy[perm], "source": s}


def tile_events(ev: dict, copies: int) -> dict:
    """A larger pile made of ``copies`` copies of an event set (for bandwidth
    measurements that need more bytes than one workload holds)."""
    out = {"n": np.tile(ev["n"], copies)}
    for k in ("x", "y", "z", "e"):
        out[k] = np.ascontiguousarray(np.tile(ev[k], (1, copies)))
    return out


def training_events(n_events: int, seed: int, bkg_ratio: float = 3.0, chunk: int = 20000):
    """Training data of the learned ring filter: chunks of simulated events,
    each chunk with its own random source direction (so that no direction is
    learned), background bkg_ratio times the source.  Returns the event dict
    of simulate_events over all chunks plus 'sources' [N, 3] (the true source
    of each event's chunk; meaningful for source events)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for c in range((n_events + chunk - 1) // chunk):
        m = min(chunk, n_events - c * chunk)
        s = random_units(rng, 1)[0]
        n_src = int(round(m / (1.0 + bkg_ratio)))
        ev = simulate_events(n_src=n_src, n_bkg=m - n_src, seed=seed * 100003 + c, source=s)
        ev["sources"] = np.repeat(s[None, :], m, axis=0)
        parts.append(ev)
    out = {"n": np.concatenate([p["n"] for p in parts]),
           "is_source": np.concatenate([p["is_source"] for p in parts]),
           "sources": np.concatenate([p["sources"] for p in parts]),
           "order": np.concatenate([p["order"] for p in parts])}
    for k in ("x", "y", "z", "e"):
        out[k] = np.ascontiguousarray(np.concatenate([p[k] for p in parts], axis=1))
    return out



def serving_bursts(n_bursts: int = 2000, rate_hz: float = 50.0, seed: int = 5,
                   median: int = 20000, sigma: float = 1.0, lo: int = 500, hi: int = 300000,
                   bkg_lo: float = 1.0, bkg_hi: float = 50.0, n_dirs: int = 16,
                   pool_src: int = 160000, pool_bkg: int = 320000):
    """The serving workload: Poisson arrivals at rate_hz; event counts
    log-normal (median, sigma) truncated to [lo, hi]; background ratio uniform
    in [bkg_lo, bkg_hi]; the source one of n_dirs random directions.

    Events come from pools simulated once (pool_src source events per
    direction, pool_bkg isotropic background events, each pool in random
    order): a burst is a contiguous slice of its direction's source pool plus
    a contiguous slice of the background pool, at random offsets.  Returns
    (pools, specs): pools = {"src": [event dict per direction], "bkg": event
    dict}; specs = list of {"arrival" (s), "dir", "source", "src": (offset,
    count), "bkg": (offset, count)}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dirs = random_units(rng, n_dirs)
    pools = {"src": [simulate_events(n_src=pool_src, n_bkg=0, seed=seed * 7919 + d,
                                     source=dirs[d]) for d in range(n_dirs)],
             "bkg": simulate_events(n_src=0, n_bkg=pool_bkg, seed=seed * 7919 + n_dirs)}
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_bursts))
    specs = []
    for i in range(n_bursts):
        while True:
            N = int(round(median * math.exp(sigma * rng.standard_normal())))
            if lo <= N <= hi:
                break
        ratio = rng.uniform(bkg_lo, bkg_hi)
        n_src = min(pool_src, max(1, int(round(N / (1.0 + ratio)))))
        n_bkg = min(pool_bkg, N - n_src)
        d = int(rng.integers(n_dirs))
        a = int(rng.integers(pool_src - n_src + 1))
        b = int(rng.integers(pool_bkg - n_bkg + 1))
        specs.append({"arrival": float(t[i]), "dir": d, "source": dirs[d],
                      "src": (a, n_src), "bkg": (b, n_bkg)})
    return pools, specs


def burst_events(pools, spec):
    """The events of one serving burst as one event dict (source slice then
    background slice), with is_source."""
    (a, ns), (b, nb) = spec["src"], spec["bkg"]
    S, B = pools["src"][spec["dir"]], pools["bkg"]
    ev = {"n": np.concatenate([S["n"][a:a + ns], B["n"][b:b + nb]]),
          "is_source": np.concatenate([np.ones(ns, bool), np.zeros(nb, bool)]),
          "source": spec["source"]}
    for k in ("x", "y", "z", "e"):
        ev[k] = np.ascontiguousarray(np.concatenate([S[k][:, a:a + ns], B[k][:, b:b + nb]], 1))
    return ev


def detection_stream(n_events: int = 400_000, seed: int = 21, event_rate_hz: float = 2.0e5,
                     mean_det: float = 12.0, tau_ns: float = 28.0, jitter_ns: float = 0.5,
                     dark_rate_hz: float = 1.0e6, adc_per_kev: float = 10.0,
                     pe_adc: int = 8, photopeak_frac: float = 0.35):
    """Time-sorted detections of a monolithic scintillator read out by a
    pixelated photodetector under a 662 keV (137Cs-like) source.

    Events arrive as a Poisson process at event_rate_hz; each gives
    1 + Poisson(mean_det - 1) detections, delayed from the event time by the
    scintillation decay (exponential, tau_ns) plus Gaussian jitter
    (jitter_ns).  Its energy is the 662 keV photopeak (photopeak_frac of
    events) or the Compton continuum (uniform below the 477 keV edge), split
    among its detections by a flat Dirichlet draw.  Dark counts (single
    detections of 1-3 photoelectrons, pe_adc channels each) arrive as a
    Poisson process at dark_rate_hz.  Times are int64 picoseconds from 0,
    amplitudes uint32 ADC channels.

    Returns (t [N] int64 sorted, adc [N] uint32, truth [N] int64: the
    generating event of each detection, -1 for dark counts)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t_ev = np.cumsum(rng.exponential(1e12 / event_rate_hz, n_events))     # ps
    span = t_ev[-1] + 1e6 if n_events else 0.0
    k = 1 + rng.poisson(mean_det - 1.0, n_events)
    e_kev = np.where(rng.uniform(size=n_events) < photopeak_frac, 662.0,
                     rng.uniform(0.0, 477.0, n_events))
    owner = np.repeat(np.arange(n_events), k)
    delay = rng.exponential(tau_ns * 1e3, owner.size) + rng.normal(0.0, jitter_ns * 1e3, owner.size)
    t_det = t_ev[owner] + np.abs(delay)
    share = rng.exponential(1.0, owner.size)                 # flat Dirichlet per event
    tot = np.bincount(owner, weights=share, minlength=n_events)
    adc_det = np.maximum(1, np.round(share / tot[owner] * e_kev[owner] * adc_per_kev))
    n_dark = rng.poisson(dark_rate_hz * span * 1e-12)
    t_dark = rng.uniform(0.0, span, n_dark)
    adc_dark = pe_adc * rng.integers(1, 4, n_dark)
    t = np.concatenate([t_det, t_dark])
    adc = np.concatenate([adc_det, adc_dark])
    truth = np.concatenate([owner, -np.ones(n_dark, np.int64)])
    order = np.argsort(t, kind="stable")
    return (np.round(t[order]).astype(np.int64), adc[order].astype(np.uint32), truth[order])


def tile_stream(t, adc, copies: int, gap_ps: int = 1_000_000):
    """A longer sorted stream made of `copies` copies of (t, adc), each
    shifted past the end of the previous one by gap_ps."""
    t = np.asarray(t, np.int64)
    span = int(t[-1] - t[0]) + gap_ps if t.size else gap_ps
    off = (np.arange(copies, dtype=np.int64) * span)[:, None]
    return (t[None, :] + off).ravel(), np.tile(np.asarray(adc, np.uint32), copies)
