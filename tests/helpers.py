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
