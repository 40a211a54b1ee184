"""Plain FP64 CPU oracle for the Compton ring-localisation hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path (the CUDA
library and its Python binding) never imports this package, and this package
never imports the product.  It shares no code with the CUDA library.

The arithmetic lives in ``oracle.c`` (plain C, FP64; the site-ordering
decision alone is taken in IEEE binary32, the precision the GPU decides in).
This module compiles it with gcc and wraps each function for numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "cluster.c"), os.path.join(_HERE, "nearfield.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# -ffp-contract=off: every binary32 operation of the ordering decision is
# rounded on its own (no fused multiply-add), as the decision rule defines.
CFLAGS = ["-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
          "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-Wall"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, a few seconds)."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < max([os.path.getmtime(s) for s in _SRCS] +
                                         [os.path.getmtime(os.path.join(_HERE, "oracle.h"))]):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, *_SRCS, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        i64, i32, f64, f32 = C.c_int64, C.c_int, C.c_double, C.c_float
        lib.or_order_event.argtypes = [i32, P, P, P, P, P, P, P]
        lib.or_order_event.restype = i32
        lib.or_order_chi2.argtypes = [i32, P, P, P, P, P]
        lib.or_order_chi2.restype = f32
        lib.or_kn_weight_f32.argtypes = [f32, f32]
        lib.or_kn_weight_f32.restype = f32
        lib.or_order_chi2_f64.argtypes = [i32, P, P, P, P, P]
        lib.or_order_chi2_f64.restype = f64
        lib.or_kn_weight_f64.argtypes = [f64, f64]
        lib.or_kn_weight_f64.restype = f64
        lib.or_order_event_f64.argtypes = [i32, P, P, P, P]
        lib.or_order_event_f64.restype = i32
        lib.or_order_bound.argtypes = [i32, P, P, P, P, P, P, P]
        lib.or_order_bound.restype = i32
        lib.or_order_check.argtypes = [i64, i64, P, P, P, P, P, P, P, P, P]
        lib.or_order_check.restype = None
        lib.or_rings_from_events.argtypes = [i64, i64, P, P, P, P, P, f64, f64,
                                             f64, f64, P, P, P, P, P, P, P]
        lib.or_rings_from_events.restype = None
        lib.or_angle.argtypes = [P, P]
        lib.or_angle.restype = f64
        lib.or_map.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, i64, f64,
                               i32, P]
        lib.or_map.restype = None
        lib.or_likelihood.argtypes = [i64, P, P, P, P, P, P, P, f64]
        lib.or_likelihood.restype = f64
        lib.or_argmax.argtypes = [i64, P]
        lib.or_argmax.restype = i64
        lib.or_seeds.argtypes = [i64, P, P, P, P, i32, f64, P]
        lib.or_seeds.restype = i32
        lib.or_refine.argtypes = [i64, P, P, P, P, P, P, P, i32, f64, i32, f64,
                                  P, P, P]
        lib.or_refine.restype = i32
        lib.or_grid_fibonacci.argtypes = [i64, P, P, P]
        lib.or_grid_fibonacci.restype = None
        lib.or_grid_healpix_ring.argtypes = [i64, P, P, P]
        lib.or_grid_healpix_ring.restype = i32
        lib.or_grid_healpix_nest.argtypes = [i64, P, P, P]
        lib.or_grid_healpix_nest.restype = i32
        lib.or_maxstep_edges.argtypes = [P, i64, i64, P]
        lib.or_maxstep_edges.restype = None
        lib.or_events_from_edges.argtypes = [P, P, i64, P, P, P, P]
        lib.or_events_from_edges.restype = i64
        lib.or_fixed_window.argtypes = [P, P, i64, i64, i64, C.c_uint64, P, P, P, P]
        lib.or_fixed_window.restype = i64
        lib.or_spectrum.argtypes = [P, i64, C.c_uint64, i32, P]
        lib.or_spectrum.restype = None
        lib.or_ring_apex.argtypes = [i64, i64, P, P, P, P, P, P, P, P, P]
        lib.or_ring_apex.restype = None
        lib.or_backproject.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P, P, P, i64, f64,
                                       i32, P]
        lib.or_backproject.restype = None
        lib.or_universe.argtypes = [i32, i64, f64, f64, f64, f64, P, P, P]
        lib.or_universe.restype = i64
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


ME_KEV = 510.99895


# --------------------------------------------------------------------------
# Ordering
# --------------------------------------------------------------------------
def order_event(x, y, z, e):
    """Ordering decision for one event (arrays of its k sites, binary32).

    Returns (order tuple, lexicographic rank, chi2) or None when no order is
    kinematically valid."""
    x, y, z, e = (_f32(v) for v in (x, y, z, e))
    k = len(x)
    order = np.zeros(4, dtype=np.int32)
    rank = C.c_int(0)
    chi2 = C.c_float(0)
    ok = _load().or_order_event(k, _p(x), _p(y), _p(z), _p(e), _p(order),
                                C.addressof(rank), C.addressof(chi2))
    if not ok:
        return None
    return tuple(int(v) for v in order[:k]), rank.value, chi2.value


def order_chi2(x, y, z, e, order):
    """Compton chi-square of one order (binary32); +inf when invalid."""
    x, y, z, e = (_f32(v) for v in (x, y, z, e))
    o = np.ascontiguousarray(order, dtype=np.int32)
    return _load().or_order_chi2(len(x), _p(x), _p(y), _p(z), _p(e), _p(o))


def kn_weight_f32(P, cos_eta):
    return _load().or_kn_weight_f32(float(P), float(cos_eta))


def order_chi2_f64(x, y, z, e, order):
    """The definition's chi2 of one order in FP64 (FP32 inputs); +inf when
    the order is invalid, 0 for a valid 2-site order."""
    x, y, z, e = (_f32(v) for v in (x, y, z, e))
    o = np.ascontiguousarray(order, dtype=np.int32)
    return _load().or_order_chi2_f64(len(x), _p(x), _p(y), _p(z), _p(e), _p(o))


def kn_weight_f64(P, cos_eta):
    return _load().or_kn_weight_f64(float(P), float(cos_eta))


def order_event_f64(x, y, z, e):
    """Rank the ordering rule picks on the FP64 definition (-1: none valid)."""
    x, y, z, e = (_f32(v) for v in (x, y, z, e))
    return _load().or_order_event_f64(len(x), _p(x), _p(y), _p(z), _p(e))


def order_bound(x, y, z, e, order):
    """(validity, value, bound) of one order: validity 1/0 as both precisions
    decide it, -1 within a bound of a threshold, -2 outside the model; value
    the FP64 chi2 (Klein-Nishina weight for 2 sites) and bound the most the
    binary32 sequence can differ from it."""
    x, y, z, e = (_f32(v) for v in (x, y, z, e))
    o = np.ascontiguousarray(order, dtype=np.int32)
    val, bnd = C.c_double(0), C.c_double(0)
    st = _load().or_order_bound(len(x), _p(x), _p(y), _p(z), _p(e), _p(o),
                                C.addressof(val), C.addressof(bnd))
    return st, val.value, bnd.value


ORDER_DECIDED, ORDER_NEAR_TIE, ORDER_NEAR_THRESHOLD, ORDER_OUTSIDE = 0, 1, 2, 3


def order_check(ev):
    """Binary32 decision vs the FP64 definition for an event set (FP32 inputs).

    Returns dict(rank32, rank64, status, margin); see ``or_order_check``:
    status 0 = decided (ranks must agree), 1 = near tie within the binary32
    bound, 2 = a validity threshold within its bound, 3 = outside the model."""
    n = np.ascontiguousarray(ev["n"], dtype=np.uint8)
    N = n.shape[0]
    x, y, z, e = (_f32(ev[k]) for k in ("x", "y", "z", "e"))
    stride = x.shape[1] if x.ndim == 2 else N
    out = {"rank32": np.empty(N, np.int32), "rank64": np.empty(N, np.int32),
           "status": np.empty(N, np.uint8), "margin": np.empty(N)}
    _load().or_order_check(N, stride, _p(n), _p(x), _p(y), _p(z), _p(e),
                           _p(out["rank32"]), _p(out["rank64"]), _p(out["status"]),
                           _p(out["margin"]))
    return out


# --------------------------------------------------------------------------
# Rings
# --------------------------------------------------------------------------
def rings_from_events(ev, sigma_e_frac, sigma_pos_cm, deta_min, deta_max):
    """Rings of an event set ``ev`` (dict with n[N] u8 and x, y, z, e as
    [4, N] arrays).  Returns a dict of FP64 ring arrays + valid + perm."""
    n = np.ascontiguousarray(ev["n"], dtype=np.uint8)
    N = n.shape[0]
    x, y, z, e = (_f64(ev[k]) for k in ("x", "y", "z", "e"))
    stride = x.shape[1] if x.ndim == 2 else N
    out = {k: np.zeros(N) for k in ("ax", "ay", "az", "eta", "deta")}
    out["valid"] = np.zeros(N, dtype=np.uint8)
    out["perm"] = np.zeros(N, dtype=np.uint8)
    _load().or_rings_from_events(
        N, stride, _p(n), _p(x), _p(y), _p(z), _p(e), sigma_e_frac,
        sigma_pos_cm, deta_min, deta_max, _p(out["ax"]), _p(out["ay"]),
        _p(out["az"]), _p(out["eta"]), _p(out["deta"]), _p(out["valid"]),
        _p(out["perm"]))
    return out


# --------------------------------------------------------------------------
# Map, argmax, seeds
# --------------------------------------------------------------------------
def _rings64(r):
    ax, ay, az, eta, deta = (_f64(r[k]) for k in ("ax", "ay", "az", "eta", "deta"))
    v = r.get("valid")
    valid = np.ones(ax.shape[0], np.uint8) if v is None else \
        np.ascontiguousarray(v, dtype=np.uint8)
    return ax, ay, az, eta, deta, valid


def angle(a, c):
    a, c = _f64(a), _f64(c)
    return _load().or_angle(_p(a), _p(c))


def likelihood_map(rings, grid, idx=None, k_cut=0.0, nthreads=None):
    """L_j for the directions ``idx`` (all when None).  ``grid`` = (x, y, z)."""
    ax, ay, az, eta, deta, valid = _rings64(rings)
    cx, cy, cz = (_f64(v) for v in grid)
    if idx is None:
        idx_a, nidx = None, cx.shape[0]
    else:
        idx_a = np.ascontiguousarray(idx, dtype=np.int64)
        nidx = idx_a.shape[0]
    out = np.zeros(nidx)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    _load().or_map(ax.shape[0], _p(ax), _p(ay), _p(az), _p(eta), _p(deta),
                   _p(valid), _p(cx), _p(cy), _p(cz), _p(idx_a), nidx,
                   float(k_cut), int(nthreads), _p(out))
    return out


def likelihood(rings, s, k_cut=0.0):
    ax, ay, az, eta, deta, valid = _rings64(rings)
    s = _f64(s)
    return _load().or_likelihood(ax.shape[0], _p(ax), _p(ay), _p(az), _p(eta),
                                 _p(deta), _p(valid), _p(s), float(k_cut))


def argmax(m):
    m = _f64(m)
    return int(_load().or_argmax(m.shape[0], _p(m)))


def seeds(m, grid, topk, nms_rad):
    m = _f64(m)
    cx, cy, cz = (_f64(v) for v in grid)
    out = np.zeros(topk, dtype=np.int64)
    got = _load().or_seeds(m.shape[0], _p(m), _p(cx), _p(cy), _p(cz), topk,
                           nms_rad, _p(out))
    return out[:got]


# --------------------------------------------------------------------------
# Refinement
# --------------------------------------------------------------------------
def refine(rings, seed_dirs, k_cut=0.0, max_iter=50, tol_rad=1e-10):
    """Returns (dir[3], objective, iterations, status)."""
    ax, ay, az, eta, deta, valid = _rings64(rings)
    sd = _f64(np.atleast_2d(seed_dirs))
    out = np.zeros(3)
    obj = C.c_double(0)
    iters = C.c_int(0)
    st = _load().or_refine(ax.shape[0], _p(ax), _p(ay), _p(az), _p(eta),
                           _p(deta), _p(valid), _p(sd), sd.shape[0],
                           float(k_cut), int(max_iter), float(tol_rad),
                           _p(out), C.addressof(obj), C.addressof(iters))
    return out, obj.value, iters.value, st


# --------------------------------------------------------------------------
# Grids
# --------------------------------------------------------------------------
def grid_fibonacci(n):
    x, y, z = np.zeros(n), np.zeros(n), np.zeros(n)
    _load().or_grid_fibonacci(n, _p(x), _p(y), _p(z))
    return x, y, z


def grid_healpix_ring(nside):
    npix = 12 * nside * nside
    x, y, z = np.zeros(npix), np.zeros(npix), np.zeros(npix)
    if _load().or_grid_healpix_ring(nside, _p(x), _p(y), _p(z)) != 0:
        raise ValueError("nside must be >= 1")
    return x, y, z


def grid_healpix_nest(nside):
    """HEALPix pixel centres in NESTED order (nside a power of two)."""
    npix = 12 * nside * nside
    x, y, z = np.zeros(npix), np.zeros(npix), np.zeros(npix)
    if _load().or_grid_healpix_nest(nside, _p(x), _p(y), _p(z)) != 0:
        raise ValueError("nside must be a power of two")
    return x, y, z


# --------------------------------------------------------------------------
# Event clustering of detections (cluster.c, Sec. 2)
# --------------------------------------------------------------------------
def _events_out(N):
    K = N // 2 + 1
    return (np.empty(N, np.int32), np.empty(K, np.int64), np.empty(K, np.int32),
            np.empty(K, np.uint64))


def maxstep_edges(t, dt_max):
    """The edge array E of the max-step clustering (uint8 [N])."""
    t = np.ascontiguousarray(t, dtype=np.int64)
    edge = np.empty(t.size, np.uint8)
    _load().or_maxstep_edges(_p(t), t.size, int(dt_max), _p(edge))
    return edge


def maxstep_events(t, adc, dt_max):
    """Max-step clustering: dict of edge [N], event_id [N] (-1 isolated),
    first [K], count [K], adc [K] (uint64 sums)."""
    t = np.ascontiguousarray(t, dtype=np.int64)
    adc = np.ascontiguousarray(adc, dtype=np.uint32)
    edge = maxstep_edges(t, dt_max)
    eid, first, count, s = _events_out(t.size)
    K = _load().or_events_from_edges(_p(edge), _p(adc), t.size, _p(eid), _p(first),
                                     _p(count), _p(s))
    return {"edge": edge, "event_id": eid, "first": first[:K], "count": count[:K],
            "adc": s[:K]}


def fixed_window_events(t, adc, window, n_min, adc_min):
    """The prior-art fixed-length non-overlapping window (sequential)."""
    t = np.ascontiguousarray(t, dtype=np.int64)
    adc = np.ascontiguousarray(adc, dtype=np.uint32)
    N = t.size
    eid, first, count, s = (np.empty(N, np.int32), np.empty(N + 1, np.int64),
                            np.empty(N + 1, np.int32), np.empty(N + 1, np.uint64))
    K = _load().or_fixed_window(_p(t), _p(adc), N, int(window), int(n_min), int(adc_min),
                                _p(eid), _p(first), _p(count), _p(s))
    return {"event_id": eid, "first": first[:K], "count": count[:K], "adc": s[:K]}


def spectrum(adc_sum, bin_width, nbins):
    a = np.ascontiguousarray(adc_sum, dtype=np.uint64)
    h = np.empty(nbins, np.uint64)
    _load().or_spectrum(_p(a), a.size, int(bin_width), int(nbins), _p(h))
    return h


# --------------------------------------------------------------------------
# Near-field back projection (nearfield.c, Sec. 3)
# --------------------------------------------------------------------------
UNIVERSES = {"cube": 0, "cylinder": 1, "sphere": 2}


def ring_apex(ev, rings):
    """Apex (first interaction site) of each valid ring: [N, 3] float64."""
    n = np.ascontiguousarray(ev["n"], dtype=np.uint8)
    N = n.size
    x, y, z = (_f64(ev[k]) for k in ("x", "y", "z"))
    stride = x.shape[1] if x.ndim == 2 else N
    out = [np.zeros(N) for _ in range(3)]
    _load().or_ring_apex(N, stride, _p(n), _p(x), _p(y), _p(z),
                         _p(np.ascontiguousarray(rings["perm"], dtype=np.uint8)),
                         _p(np.ascontiguousarray(rings["valid"], dtype=np.uint8)), *map(_p, out))
    return np.stack(out, 1)


def backproject(rings, apex, vox, idx=None, k_cut=0.0, nthreads=None):
    """Image value at voxels vox[idx] (all voxels when idx is None)."""
    ax, ay, az, eta, deta, valid = _rings64(rings)
    p = _f64(apex)
    px, py, pz = (np.ascontiguousarray(p[:, c]) for c in range(3))
    vx, vy, vz = (_f64(v) for v in vox)
    idx = np.arange(vx.size, dtype=np.int64) if idx is None else \
        np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(idx.size)
    _load().or_backproject(ax.size, _p(px), _p(py), _p(pz), _p(ax), _p(ay),
                           _p(az), _p(eta), _p(deta), _p(valid), _p(vx), _p(vy),
                           _p(vz), _p(idx), idx.size, float(k_cut),
                           int(nthreads or os.cpu_count() or 1), _p(out))
    return out


def universe(shape, n, pitch, center=(0.0, 0.0, 0.0), count_only=False):
    """Voxel centres of the image universe ('cube', 'cylinder', 'sphere')."""
    L = _load()
    s = UNIVERSES[shape]
    m = L.or_universe(s, n, pitch, *center, None, None, None)
    if count_only:
        return m
    out = [np.zeros(m) for _ in range(3)]
    L.or_universe(s, n, pitch, *center, *map(_p, out))
    return tuple(out)
