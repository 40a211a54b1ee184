"""Python binding of libcompton.so (the C ABI declared in include/compton.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch provides device memory (tensors, workspaces) and the stream.  There is
no CPU fallback: if the library is missing the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import struct
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# CC_LIBRARY=debug selects the debug build (libcompton_debug.so, index bounds
# checks; see cc_debug_bounds); the default is the optimised build.
LIB_PATH = os.path.join(HERE, "libcompton_debug.so" if os.environ.get("CC_LIBRARY") == "debug"
                        else "libcompton.so")

CC_OK, CC_EINVAL, CC_ECUDA, CC_ENOMEM, CC_ETIMEOUT, CC_ENOCONV = 0, -1, -2, -3, -4, -5
STATUS_NAMES = {0: "CC_OK", -1: "CC_EINVAL", -2: "CC_ECUDA", -3: "CC_ENOMEM",
                -4: "CC_ETIMEOUT", -5: "CC_ENOCONV"}

_P = C.c_void_p


class cc_params(C.Structure):
    _fields_ = [("sigma_e_frac", C.c_float), ("sigma_pos_cm", C.c_float),
                ("deta_min", C.c_float), ("deta_max", C.c_float),
                ("k_cut", C.c_float), ("topk", C.c_int32), ("nms_rad", C.c_float),
                ("max_iter", C.c_int32), ("tol_rad", C.c_double)]


class cc_events(C.Structure):
    _fields_ = [("n", _P), ("x", _P), ("y", _P), ("z", _P), ("e", _P),
                ("count", C.c_int64), ("stride", C.c_int64)]


class cc_rings(C.Structure):
    _fields_ = [("ax", _P), ("ay", _P), ("az", _P), ("eta", _P), ("deta", _P),
                ("valid", _P), ("perm", _P), ("count", C.c_int64)]


class cc_grid(C.Structure):
    _fields_ = [("x", _P), ("y", _P), ("z", _P), ("count", C.c_int64), ("order", _P)]


class cc_detections(C.Structure):
    _fields_ = [("t", _P), ("adc", _P), ("count", C.c_int64)]


class cc_stage_time(C.Structure):
    _fields_ = [("launches", C.c_int64), ("ms", C.c_double)]


STAGES = ("recon", "pack", "sweep", "reduce", "select", "gather", "refine", "grid", "mlp",
          "cluster", "voxel")


class CCError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """The loaded libcompton.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -m paper_2411_04785_gb300.build` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        S = C.c_int
        L.cc_abi_version.restype = C.c_int32
        L.cc_last_error.restype = C.c_char_p
        L.cc_params_default.argtypes = [C.POINTER(cc_params)]
        L.cc_params_default.restype = None
        L.cc_rings_from_events.argtypes = [C.POINTER(cc_events), C.POINTER(cc_rings),
                                           C.POINTER(cc_params), _P]
        L.cc_rings_from_events.restype = S
        L.cc_localize_workspace_bytes.argtypes = [C.c_int64, C.c_int64, C.POINTER(cc_params)]
        L.cc_localize_workspace_bytes.restype = C.c_size_t
        L.cc_localize.argtypes = [C.POINTER(cc_rings), C.POINTER(cc_grid), C.POINTER(cc_params),
                                  _P, _P, _P, _P, _P, C.c_size_t, _P]
        L.cc_localize.restype = S
        L.cc_refine_workspace_bytes.argtypes = [C.c_int64, C.c_int32]
        L.cc_refine_workspace_bytes.restype = C.c_size_t
        L.cc_refine.argtypes = [C.POINTER(cc_rings), _P, C.c_int32, C.POINTER(cc_params),
                                _P, _P, _P, _P, _P, C.c_size_t, _P]
        L.cc_refine.restype = S
        L.cc_grid_fibonacci.argtypes = [C.c_int64, _P, _P, _P, _P]
        L.cc_grid_fibonacci.restype = S
        L.cc_grid_healpix_ring.argtypes = [C.c_int32, _P, _P, _P, _P]
        L.cc_grid_healpix_ring.restype = S
        L.cc_grid_healpix_nest.argtypes = [C.c_int32, _P, _P, _P, _P]
        L.cc_grid_healpix_nest.restype = S
        L.cc_grid_gather.argtypes = [C.POINTER(cc_grid), _P, C.c_int32, _P, _P]
        L.cc_grid_gather.restype = S
        L.cc_grid_order_workspace_bytes.argtypes = [C.c_int64]
        L.cc_grid_order_workspace_bytes.restype = C.c_size_t
        L.cc_grid_order.argtypes = [C.POINTER(cc_grid), _P, _P, C.c_size_t, _P]
        L.cc_grid_order.restype = S
        L.cc_localize_static.argtypes = [C.POINTER(cc_rings), C.POINTER(cc_grid),
                                         C.POINTER(cc_params), _P, _P, _P, _P, _P]
        L.cc_localize_static.restype = S
        L.cc_ring_features.argtypes = [C.POINTER(cc_events), C.POINTER(cc_rings),
                                       C.POINTER(cc_params), _P, _P]
        L.cc_ring_features.restype = S
        L.cc_mlp_workspace_bytes.argtypes = [C.c_int64]
        L.cc_mlp_workspace_bytes.restype = C.c_size_t
        L.cc_mlp_forward.argtypes = [_P, _P, _P, C.c_int64, _P, _P, C.c_size_t, _P]
        L.cc_mlp_forward.restype = S
        L.cc_mlp_grad.argtypes = [_P, _P, _P, _P, _P, _P, C.c_int64, _P, _P, _P, C.c_size_t, _P]
        L.cc_mlp_grad.restype = S
        L.cc_mlp_grad_trace.argtypes = [_P, _P, _P, _P, _P, _P, C.c_int64, _P, _P, _P,
                                        C.c_size_t, _P, _P, _P, _P, _P]
        L.cc_mlp_grad_trace.restype = S
        L.cc_mlp_adam.argtypes = [_P, _P, _P, _P, _P, C.c_int32, C.c_float, C.c_float,
                                  C.c_float, C.c_float, _P]
        L.cc_mlp_adam.restype = S
        L.cc_mlp_params_to_bf16.argtypes = [_P, _P, _P]
        L.cc_mlp_params_to_bf16.restype = S
        L.cc_mlp_apply_filter.argtypes = [_P, C.POINTER(cc_rings), C.c_float, C.c_float,
                                          C.c_float, _P]
        L.cc_mlp_apply_filter.restype = S
        L.cc_localize_batch_workspace_bytes.argtypes = [C.c_int64, C.c_int64, C.POINTER(cc_params)]
        L.cc_localize_batch_workspace_bytes.restype = C.c_size_t
        L.cc_localize_batch.argtypes = [C.c_int32, C.POINTER(cc_rings), C.POINTER(cc_grid),
                                        C.POINTER(cc_params), _P, _P, _P, _P, _P, _P, _P]
        L.cc_localize_batch.restype = S
        L.cc_cluster_workspace_bytes.argtypes = [C.c_int64]
        L.cc_cluster_workspace_bytes.restype = C.c_size_t
        L.cc_cluster_maxstep.argtypes = [C.POINTER(cc_detections), C.c_int64, _P, _P, _P, _P, _P,
                                         C.c_int64, _P, _P, _P, C.c_size_t, _P]
        L.cc_cluster_maxstep.restype = S
        L.cc_cluster_spectrum.argtypes = [_P, _P, C.c_uint64, C.c_int32, _P, _P]
        L.cc_cluster_spectrum.restype = S
        L.cc_ring_apex.argtypes = [C.POINTER(cc_events), C.POINTER(cc_rings), _P, _P, _P, _P]
        L.cc_ring_apex.restype = S
        L.cc_voxel_count.argtypes = [C.c_int32, C.c_int32]
        L.cc_voxel_count.restype = C.c_int64
        L.cc_voxel_universe.argtypes = [C.c_int32, C.c_int32, C.c_float, C.c_float, C.c_float,
                                        C.c_float, _P, _P, _P, _P]
        L.cc_voxel_universe.restype = S
        L.cc_backproject_workspace_bytes.argtypes = [C.c_int64, C.c_int64, C.POINTER(cc_params)]
        L.cc_backproject_workspace_bytes.restype = C.c_size_t
        L.cc_backproject.argtypes = [C.POINTER(cc_rings), _P, _P, _P, C.POINTER(cc_grid),
                                     C.POINTER(cc_params), _P, _P, _P, _P, C.c_size_t, _P]
        L.cc_backproject.restype = S
        L.cc_events_copy.argtypes = [C.POINTER(cc_events), C.c_int64, C.POINTER(cc_events),
                                     C.c_int64, C.c_int64, _P]
        L.cc_events_copy.restype = S
        L.cc_selftest_exact_ops.argtypes = [_P, _P]
        L.cc_selftest_exact_ops.restype = S
        L.cc_selftest_wait_timeout.argtypes = [C.c_int32, C.c_int64, _P, _P, _P]
        L.cc_selftest_wait_timeout.restype = S
        L.cc_debug_bounds.argtypes = [C.POINTER(C.c_uint64), C.c_int32]
        L.cc_debug_bounds.restype = S
        L.cc_debug_selftest_bounds.argtypes = [_P, C.c_int64, _P]
        L.cc_debug_selftest_bounds.restype = S
        L.cc_trace_enable.argtypes = [C.c_int32]
        L.cc_trace_enable.restype = S
        L.cc_trace_read.argtypes = [C.POINTER(cc_stage_time), C.c_int32, C.c_int32]
        L.cc_trace_read.restype = S
        if L.cc_abi_version() != 2:
            raise RuntimeError("libcompton.so ABI version mismatch")
        _lib = L
    return _lib


def debug_bounds(reset: bool = False) -> int:
    """The debug build's bounds word: 0 when no checked index was out of
    bounds, else site << 48 | index (raises CCError in the normal build)."""
    w = C.c_uint64(0)
    _check("cc_debug_bounds", lib().cc_debug_bounds(C.byref(w), 1 if reset else 0))
    return int(w.value)


def _check(fn, st):
    if st != CC_OK:
        raise CCError(fn, st, lib().cc_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _need(t, dtype, name):
    if t is None:
        return
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
@dataclass
class Params:
    sigma_e_frac: float = 0.05
    sigma_pos_cm: float = 1.0
    deta_min: float = math.radians(0.5)
    deta_max: float = math.radians(20.0)
    k_cut: float = 0.0
    topk: int = 1
    nms_rad: float = math.radians(1.0)
    max_iter: int = 50
    tol_rad: float = 1e-7

    def c(self) -> cc_params:
        return cc_params(self.sigma_e_frac, self.sigma_pos_cm, self.deta_min,
                         self.deta_max, self.k_cut, self.topk, self.nms_rad,
                         self.max_iter, self.tol_rad)


def default_params() -> Params:
    p = cc_params()
    lib().cc_params_default(C.byref(p))
    return Params(p.sigma_e_frac, p.sigma_pos_cm, p.deta_min, p.deta_max, p.k_cut,
                  p.topk, p.nms_rad, p.max_iter, p.tol_rad)


# --------------------------------------------------------------------------
# rings
# --------------------------------------------------------------------------
RING_KEYS = ("ax", "ay", "az", "eta", "deta")


def empty_rings(n: int, device) -> dict:
    r = {k: torch.empty(n, dtype=torch.float32, device=device) for k in RING_KEYS}
    r["valid"] = torch.empty(n, dtype=torch.uint8, device=device)
    r["perm"] = torch.empty(n, dtype=torch.uint8, device=device)
    return r


def _rings_struct(r: dict) -> cc_rings:
    n = r["ax"].numel()
    for k in RING_KEYS:
        _need(r[k], torch.float32, k)
        if r[k].numel() != n:
            raise ValueError("ring arrays differ in length")
    for k in ("valid", "perm"):
        if r.get(k) is not None:
            _need(r[k], torch.uint8, k)
    return cc_rings(*(_ptr(r[k]) for k in RING_KEYS), _ptr(r.get("valid")),
                    _ptr(r.get("perm")), n)


def rings_from_events(n, x, y, z, e, params: Params | None = None, out: dict | None = None,
                      stream=None) -> dict:
    """Rings from events.  ``n`` [N] uint8; x, y, z, e [4, S] float32 with
    S >= N (slot s of event i at [s, i]).  Returns the ring dict."""
    params = params or Params()
    N = n.numel()
    _need(n, torch.uint8, "n")
    for t, nm in ((x, "x"), (y, "y"), (z, "z"), (e, "e")):
        _need(t, torch.float32, nm)
        if t.dim() != 2 or t.shape[0] != 4 or t.shape[1] < N:
            raise ValueError(f"{nm} must be [4, S] with S >= N")
    stride = x.shape[1]
    if any(t.shape[1] != stride for t in (y, z, e)):
        raise ValueError("x, y, z, e must share one stride")
    out = out if out is not None else empty_rings(N, n.device)
    ev = cc_events(_ptr(n), _ptr(x), _ptr(y), _ptr(z), _ptr(e), N, stride)
    rs = _rings_struct(out)
    if rs.count != N:
        raise ValueError("out rings have the wrong length")
    pc = params.c()
    _check("cc_rings_from_events", lib().cc_rings_from_events(
        C.byref(ev), C.byref(rs), C.byref(pc), _stream(stream)))
    return out


# --------------------------------------------------------------------------
# localisation
# --------------------------------------------------------------------------
def localize_workspace_bytes(R: int, M: int, params: Params | None = None) -> int:
    pc = (params or Params()).c()
    return int(lib().cc_localize_workspace_bytes(R, M, C.byref(pc)))


def _grid_struct(grid) -> cc_grid:
    """(x, y, z) or (x, y, z, order): order from grid_order, reused by the sweep."""
    gx, gy, gz = grid[:3]
    for t, nm in ((gx, "grid x"), (gy, "grid y"), (gz, "grid z")):
        _need(t, torch.float32, nm)
    order = None
    if len(grid) > 3 and grid[3] is not None:
        _need(grid[3], torch.int32, "grid order")
        if grid[3].numel() != gx.numel():
            raise ValueError("grid order has the wrong length")
        order = _ptr(grid[3])
    return cc_grid(_ptr(gx), _ptr(gy), _ptr(gz), gx.numel(), order)


def localize(rings: dict, grid, params: Params | None = None, workspace=None, out=None,
             stream=None):
    """Likelihood map, argmax and seeds.  Returns (map [M] f32, argmax [1]
    i32, seeds [topk] i32, status [1] i32) as device tensors (asynchronous)."""
    params = params or Params()
    rs = _rings_struct(rings)
    gs = _grid_struct(grid)
    dev = grid[0].device
    M = gs.count
    need = localize_workspace_bytes(rs.count, M, params)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    if out is None:
        out = (torch.empty(M, dtype=torch.float32, device=dev),
               torch.empty(1, dtype=torch.int32, device=dev),
               torch.empty(params.topk, dtype=torch.int32, device=dev),
               torch.empty(1, dtype=torch.int32, device=dev))
    m, am, sd, st = out
    pc = params.c()
    _check("cc_localize", lib().cc_localize(
        C.byref(rs), C.byref(gs), C.byref(pc), _ptr(m), _ptr(am), _ptr(sd), _ptr(st),
        _ptr(workspace), workspace.numel(), _stream(stream)))
    return m, am, sd, st


STATIC_SCRATCH_BYTES = 32 << 20


def localize_static(rings: dict, grid, params: Params | None = None, out=None, stream=None):
    """cc_localize_static: localize without a workspace (the library's static
    device scratch, STATIC_SCRATCH_BYTES; calls that overlap on the GPU race).
    Returns (map, argmax, seeds, status) like localize()."""
    params = params or Params()
    rs = _rings_struct(rings)
    gs = _grid_struct(grid)
    dev = grid[0].device
    M = gs.count
    if out is None:
        out = (torch.empty(M, dtype=torch.float32, device=dev),
               torch.empty(1, dtype=torch.int32, device=dev),
               torch.empty(params.topk, dtype=torch.int32, device=dev),
               torch.empty(1, dtype=torch.int32, device=dev))
    m, am, sd, st = out
    pc = params.c()
    _check("cc_localize_static", lib().cc_localize_static(
        C.byref(rs), C.byref(gs), C.byref(pc), _ptr(m), _ptr(am), _ptr(sd), _ptr(st),
        _stream(stream)))
    return m, am, sd, st


def refine_workspace_bytes(R: int, k: int) -> int:
    return int(lib().cc_refine_workspace_bytes(R, k))


def refine(rings: dict, seed_dirs, params: Params | None = None, workspace=None, out=None,
           stream=None):
    """Gauss-Newton refinement from seed_dirs [k, 3] float64 (device).
    Returns (dir [3] f64, obj [1] f64, iters [1] i32, status [1] i32)."""
    params = params or Params()
    rs = _rings_struct(rings)
    _need(seed_dirs, torch.float64, "seed_dirs")
    k = seed_dirs.numel() // 3
    dev = seed_dirs.device
    need = max(refine_workspace_bytes(rs.count, k), 256)   # 0: bad sizes, the call says why
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    if out is None:
        out = (torch.empty(3, dtype=torch.float64, device=dev),
               torch.empty(1, dtype=torch.float64, device=dev),
               torch.empty(1, dtype=torch.int32, device=dev),
               torch.empty(1, dtype=torch.int32, device=dev))
    d, obj, it, st = out
    pc = params.c()
    _check("cc_refine", lib().cc_refine(
        C.byref(rs), _ptr(seed_dirs), k, C.byref(pc), _ptr(d), _ptr(obj), _ptr(it),
        _ptr(st), _ptr(workspace), workspace.numel(), _stream(stream)))
    return d, obj, it, st


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------
def grid_fibonacci(n: int, device="cuda", stream=None):
    g = [torch.empty(n, dtype=torch.float32, device=device) for _ in range(3)]
    _check("cc_grid_fibonacci", lib().cc_grid_fibonacci(n, *(_ptr(t) for t in g),
                                                        _stream(stream)))
    return tuple(g)


def grid_healpix_ring(nside: int, device="cuda", stream=None):
    npix = 12 * nside * nside
    g = [torch.empty(npix, dtype=torch.float32, device=device) for _ in range(3)]
    _check("cc_grid_healpix_ring", lib().cc_grid_healpix_ring(nside, *(_ptr(t) for t in g),
                                                              _stream(stream)))
    return tuple(g)


def grid_healpix_nest(nside: int, device="cuda", stream=None):
    """HEALPix pixel centres in NESTED order (compact blocks for the angular
    selection's block skipping)."""
    npix = 12 * nside * nside
    g = [torch.empty(npix, dtype=torch.float32, device=device) for _ in range(3)]
    _check("cc_grid_healpix_nest", lib().cc_grid_healpix_nest(nside, *(_ptr(t) for t in g),
                                                              _stream(stream)))
    return tuple(g)


def grid_gather(grid, idx, out=None, stream=None):
    """FP64 unit vectors of grid directions idx [k] int32 -> [k, 3]."""
    gs = _grid_struct(grid)
    _need(idx, torch.int32, "idx")
    k = idx.numel()
    out = out if out is not None else torch.empty((k, 3), dtype=torch.float64,
                                                  device=idx.device)
    _check("cc_grid_gather", lib().cc_grid_gather(C.byref(gs), _ptr(idx), k, _ptr(out),
                                                  _stream(stream)))
    return out


def grid_order(grid, stream=None):
    """The order in which localize sweeps the grid's directions (int32 [M])."""
    gs = _grid_struct(grid)
    dev = grid[0].device
    M = grid[0].numel()
    out = torch.empty(M, dtype=torch.int32, device=dev)
    nb = lib().cc_grid_order_workspace_bytes(M)
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
    _check("cc_grid_order", lib().cc_grid_order(C.byref(gs), _ptr(out), _ptr(ws), nb,
                                                _stream(stream)))
    return out


# --------------------------------------------------------------------------
# the whole path
# --------------------------------------------------------------------------
class Localizer:
    """Events (or rings) -> map, argmax, seeds, refined direction, with
    workspaces and outputs allocated once and reused across calls."""

    def __init__(self, grid, params: Params | None = None, max_rings: int = 0):
        # the grid's direction order, computed once and reused by every sweep
        self.grid = tuple(grid[:3]) + (grid[3] if len(grid) > 3 else grid_order(grid),)
        self.params = params or Params()
        self.M = grid[0].numel()
        self.dev = grid[0].device
        self._ws_loc = None
        self._ws_ref = None
        self._rings = None
        self.map = torch.empty(self.M, dtype=torch.float32, device=self.dev)
        self.argmax = torch.empty(1, dtype=torch.int32, device=self.dev)
        self.seeds = torch.empty(self.params.topk, dtype=torch.int32, device=self.dev)
        self.loc_status = torch.empty(1, dtype=torch.int32, device=self.dev)
        self.seed_dirs = torch.empty((self.params.topk, 3), dtype=torch.float64,
                                     device=self.dev)
        self.dir = torch.empty(3, dtype=torch.float64, device=self.dev)
        self.obj = torch.empty(1, dtype=torch.float64, device=self.dev)
        self.iters = torch.empty(1, dtype=torch.int32, device=self.dev)
        self.ref_status = torch.empty(1, dtype=torch.int32, device=self.dev)
        if max_rings:
            self._reserve(max_rings)

    def _reserve(self, R):
        nl = localize_workspace_bytes(R, self.M, self.params)
        if self._ws_loc is None or self._ws_loc.numel() < nl:
            self._ws_loc = torch.empty(nl, dtype=torch.uint8, device=self.dev)
        nr = refine_workspace_bytes(R, self.params.topk)
        if self._ws_ref is None or self._ws_ref.numel() < nr:
            self._ws_ref = torch.empty(nr, dtype=torch.uint8, device=self.dev)
        if self._rings is None or self._rings["ax"].numel() != R:
            self._rings = empty_rings(R, self.dev)

    def from_rings(self, rings, stream=None):
        R = rings["ax"].numel()
        self._reserve(R)
        localize(rings, self.grid, self.params, self._ws_loc,
                 (self.map, self.argmax, self.seeds, self.loc_status), stream)
        grid_gather(self.grid, self.seeds, self.seed_dirs, stream)
        refine(rings, self.seed_dirs, self.params, self._ws_ref,
               (self.dir, self.obj, self.iters, self.ref_status), stream)
        return self

    def from_events(self, n, x, y, z, e, stream=None):
        self._reserve(n.numel())
        rings_from_events(n, x, y, z, e, self.params, self._rings, stream)
        return self.from_rings(self._rings, stream)


# --------------------------------------------------------------------------
# tracing
# --------------------------------------------------------------------------
def trace_enable(on: bool = True):
    _check("cc_trace_enable", lib().cc_trace_enable(1 if on else 0))


def trace_read(reset: bool = False) -> dict:
    """Per-stage {launches, ms} since the last reset (waits for events)."""
    arr = (cc_stage_time * len(STAGES))()
    _check("cc_trace_read", lib().cc_trace_read(arr, len(STAGES), 1 if reset else 0))
    return {n: {"launches": int(a.launches), "ms": float(a.ms)} for n, a in zip(STAGES, arr)}


# --------------------------------------------------------------------------
# learned ring filter
# --------------------------------------------------------------------------
MLP_FEATURES = 16
MLP_PARAMS = 35458
MLP_HIDDEN = 128
MLP_MAX_BATCH = 65536
MLP_SIZES = ((128, 16), (128, 128), (128, 128), (2, 128))


def ring_features(n, x, y, z, e, rings: dict, params: Params | None = None, out=None,
                  stream=None):
    """[N, 16] BF16 features of the rings of an event set (cc_ring_features)."""
    params = params or Params()
    N = n.numel()
    stride = x.shape[1]
    ev = cc_events(_ptr(n), _ptr(x), _ptr(y), _ptr(z), _ptr(e), N, stride)
    rs = _rings_struct(rings)
    out = out if out is not None else torch.empty((N, MLP_FEATURES), dtype=torch.bfloat16,
                                                  device=n.device)
    pc = params.c()
    _check("cc_ring_features", lib().cc_ring_features(C.byref(ev), C.byref(rs), C.byref(pc),
                                                      _ptr(out), _stream(stream)))
    return out


# Checkpoint of the ring filter: a flat little-endian file, a 32-byte header
# (magic, format version, parameter count, Adam step) followed by the FP32
# parameters and the two FP32 Adam moments.
_CKPT_MAGIC = b"CCFILTR\0"
_CKPT_VERSION = 1


def pack_filter_state(params, m, v, step: int) -> bytes:
    """Bytes of a ring-filter checkpoint (host numpy float32 arrays)."""
    import numpy as np
    arrs = [np.ascontiguousarray(a, dtype="<f4") for a in (params, m, v)]
    n = arrs[0].size
    if any(a.size != n for a in arrs):
        raise ValueError("params and moments differ in length")
    head = _CKPT_MAGIC + struct.pack("<IIq", _CKPT_VERSION, n, int(step)) + bytes(8)
    return head + b"".join(a.tobytes() for a in arrs)


def unpack_filter_state(buf: bytes):
    """(params, m, v, step) from checkpoint bytes; ValueError on a bad file."""
    import numpy as np
    if len(buf) < 32 or buf[:8] != _CKPT_MAGIC:
        raise ValueError("not a ring-filter checkpoint")
    version, n, step = struct.unpack("<IIq", buf[8:24])
    if version != _CKPT_VERSION:
        raise ValueError(f"checkpoint format version {version}, expected {_CKPT_VERSION}")
    if len(buf) != 32 + 12 * n:
        raise ValueError(f"checkpoint of {len(buf)} bytes, expected {32 + 12 * n}")
    body = np.frombuffer(buf, dtype="<f4", offset=32)
    return body[:n].copy(), body[n:2 * n].copy(), body[2 * n:].copy(), int(step)


class RingFilter:
    """The MLP of the learned ring filter with its FP32 parameters, BF16 copy
    and Adam state on the device; every product runs in libcompton.so."""

    def __init__(self, device, seed: int = 0, params=None):
        import numpy as np
        self.dev = torch.device(device)
        if params is None:
            rng = np.random.default_rng(seed)
            parts = []
            for o, i in MLP_SIZES:        # He-uniform weights, zero biases
                lim = math.sqrt(6.0 / i)
                parts += [rng.uniform(-lim, lim, o * i), np.zeros(o)]
            params = np.concatenate(parts).astype(np.float32)
            params[-1] = math.log(0.3)    # initial predicted width ~17 deg
        self.p = torch.as_tensor(params, dtype=torch.float32).to(self.dev).contiguous()
        assert self.p.numel() == MLP_PARAMS
        self.wb = torch.empty(MLP_PARAMS, dtype=torch.bfloat16, device=self.dev)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.grad_buf = torch.zeros_like(self.p)
        self.loss_buf = torch.zeros(1, dtype=torch.float32, device=self.dev)
        self.step = 0
        self._ws = None
        _check("cc_mlp_params_to_bf16", lib().cc_mlp_params_to_bf16(
            _ptr(self.p), _ptr(self.wb), _stream(None)))

    def save(self, path) -> None:
        """Write parameters and Adam state (see pack_filter_state)."""
        buf = pack_filter_state(self.p.cpu().numpy(), self.m.cpu().numpy(),
                                self.v.cpu().numpy(), self.step)
        with open(path, "wb") as fh:
            fh.write(buf)

    @classmethod
    def load(cls, path, device):
        """A filter restored from save(): same outputs, training resumes."""
        with open(path, "rb") as fh:
            p, m, v, step = unpack_filter_state(fh.read())
        if p.size != MLP_PARAMS:
            raise ValueError(f"checkpoint has {p.size} parameters, the network {MLP_PARAMS}")
        f = cls(device, params=p)
        f.m.copy_(torch.from_numpy(m))
        f.v.copy_(torch.from_numpy(v))
        f.step = step
        return f

    def _workspace(self, rows):
        need = max(int(lib().cc_mlp_workspace_bytes(rows)), 256)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.dev)
        return self._ws

    def forward(self, feats, out=None, stream=None, workspace=None):
        """MLP outputs [R, 2] (the forward needs no workspace; the argument is
        accepted and ignored)."""
        _need(feats, torch.bfloat16, "feats")
        if feats.dim() != 2 or feats.shape[1] != MLP_FEATURES:
            raise ValueError(f"feats must be [R, {MLP_FEATURES}]")
        R = feats.shape[0]
        out = out if out is not None else torch.empty((R, 2), dtype=torch.float32,
                                                      device=self.dev)
        _check("cc_mlp_forward", lib().cc_mlp_forward(
            _ptr(self.p), _ptr(self.wb), _ptr(feats), R, _ptr(out), None, 0, _stream(stream)))
        return out

    def grad(self, feats, is_source, residual, weight, stream=None):
        """Loss and gradient of one batch (<= MLP_MAX_BATCH rows)."""
        B = feats.shape[0]
        ws = self._workspace(B)
        _check("cc_mlp_grad", lib().cc_mlp_grad(
            _ptr(self.p), _ptr(self.wb), _ptr(feats), _ptr(is_source), _ptr(residual),
            _ptr(weight), B, _ptr(self.grad_buf), _ptr(self.loss_buf), _ptr(ws), ws.numel(),
            _stream(stream)))
        return self.loss_buf, self.grad_buf

    def grad_trace(self, feats, is_source, residual, weight, stream=None):
        """grad() keeping the step's intermediate values: returns (loss, grad,
        trace) with trace = dict(hidden [3, B, 128] bf16, out [B, 2] f32,
        dout [B, 2] bf16, signals [3, B, 128] bf16)."""
        B = feats.shape[0]
        ws = self._workspace(B)
        t = {"hidden": torch.empty((3, B, MLP_HIDDEN), dtype=torch.bfloat16, device=self.dev),
             "out": torch.empty((B, 2), dtype=torch.float32, device=self.dev),
             "dout": torch.empty((B, 2), dtype=torch.bfloat16, device=self.dev),
             "signals": torch.empty((3, B, MLP_HIDDEN), dtype=torch.bfloat16, device=self.dev)}
        _check("cc_mlp_grad_trace", lib().cc_mlp_grad_trace(
            _ptr(self.p), _ptr(self.wb), _ptr(feats), _ptr(is_source), _ptr(residual),
            _ptr(weight), B, _ptr(self.grad_buf), _ptr(self.loss_buf), _ptr(ws), ws.numel(),
            _ptr(t["hidden"]), _ptr(t["out"]), _ptr(t["dout"]), _ptr(t["signals"]),
            _stream(stream)))
        return self.loss_buf, self.grad_buf, t

    def adam(self, lr=2e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self.step += 1
        _check("cc_mlp_adam", lib().cc_mlp_adam(
            _ptr(self.p), _ptr(self.m), _ptr(self.v), _ptr(self.grad_buf), _ptr(self.wb),
            self.step, lr, beta1, beta2, eps, _stream(stream)))

    def train(self, feats, is_source, residual, weight, epochs=4, batch=MLP_MAX_BATCH,
              lr=2e-3, seed=0):
        """Adam over shuffled batches; returns the mean loss of each epoch."""
        R = feats.shape[0]
        g = torch.Generator(device="cpu").manual_seed(seed)
        losses = []
        for _ in range(epochs):
            order = torch.randperm(R, generator=g).to(self.dev)
            tot = torch.zeros(1, device=self.dev)
            nb = 0
            for b0 in range(0, R, batch):
                ix = order[b0:b0 + batch]
                loss, _ = self.grad(feats[ix].contiguous(), is_source[ix].contiguous(),
                                    residual[ix].contiguous(), weight[ix].contiguous())
                tot += loss
                self.adam(lr)
                nb += 1
            losses.append(float(tot.item()) / nb)
        return losses

    def apply(self, rings: dict, out, tau: float, deta_min: float, deta_max: float,
              stream=None):
        """Filter rings in place: keep sigmoid(z) >= tau, width exp(v)."""
        rs = _rings_struct(rings)
        _check("cc_mlp_apply_filter", lib().cc_mlp_apply_filter(
            _ptr(out), C.byref(rs), tau, deta_min, deta_max, _stream(stream)))


def mlp_workspace_bytes(rows: int) -> int:
    return max(int(lib().cc_mlp_workspace_bytes(rows)), 256)


def ring_residuals(rings: dict, sources):
    """Angle between each ring's axis and its true source minus eta (training
    labels; sources [N, 3] device float)."""
    a = torch.stack([rings["ax"], rings["ay"], rings["az"]], 1).double()
    s = sources.double()
    cr = torch.linalg.cross(a, s, dim=1).norm(dim=1)
    th = torch.atan2(cr, (a * s).sum(1))
    return (th - rings["eta"].double()).float().contiguous()


# --------------------------------------------------------------------------
# event clustering of detections (Sec. 2)
# --------------------------------------------------------------------------
CLUSTER_OUTPUTS = ("edge", "event_id", "first", "count", "adc")


def cluster_workspace_bytes(n: int) -> int:
    return int(lib().cc_cluster_workspace_bytes(n))


def cluster_maxstep(t, adc, dt_max: int, outputs=CLUSTER_OUTPUTS, out: dict | None = None,
                    workspace=None, stream=None) -> dict:
    """Max-step clustering of time-sorted detections: t [N] int64, adc [N]
    uint32 (or None) device tensors.  Returns device tensors: the requested
    outputs among edge [N] u8, event_id [N] i32, first / count / adc
    [N // 2 + 1] (i64 / i32 / u64; the first n_events entries are events), and
    n_events [1] i64, status [1] i32 (asynchronous)."""
    _need(t, torch.int64, "t")
    _need(adc, torch.uint32, "adc")
    N = t.numel()
    dev = t.device
    K = N // 2 + 1
    shapes = {"edge": (N, torch.uint8), "event_id": (N, torch.int32), "first": (K, torch.int64),
              "count": (K, torch.int32), "adc": (K, torch.uint64)}
    o = dict(out or {})
    for k in outputs:
        if k not in o:
            n, dt = shapes[k]
            o[k] = torch.empty(n, dtype=dt, device=dev)
    o.setdefault("n_events", torch.empty(1, dtype=torch.int64, device=dev))
    o.setdefault("status", torch.empty(1, dtype=torch.int32, device=dev))
    need = cluster_workspace_bytes(N)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    d = cc_detections(t.data_ptr() if N else None, adc.data_ptr() if adc is not None and N else None, N)
    g = lambda k: _ptr(o.get(k)) if k in outputs else None
    _check("cc_cluster_maxstep", lib().cc_cluster_maxstep(
        C.byref(d), int(dt_max), g("edge"), g("event_id"), g("first"), g("count"), g("adc"), K,
        _ptr(o["n_events"]), _ptr(o["status"]), _ptr(workspace), workspace.numel(),
        _stream(stream)))
    return o


def cluster_spectrum(ev_adc, n_events, bin_width: int, nbins: int, out=None, stream=None):
    """Histogram (uint64 [nbins], device) of event amplitude sums."""
    h = out if out is not None else torch.empty(nbins, dtype=torch.uint64, device=ev_adc.device)
    _check("cc_cluster_spectrum", lib().cc_cluster_spectrum(
        _ptr(ev_adc), _ptr(n_events), int(bin_width), int(nbins), _ptr(h), _stream(stream)))
    return h


# --------------------------------------------------------------------------
# near-field back projection (Sec. 3)
# --------------------------------------------------------------------------
UNIVERSES = {"cube": 0, "cylinder": 1, "sphere": 2}


def ring_apex(n, x, y, z, rings: dict, out=None, stream=None):
    """Apex (first site of the chosen order) of every ring: (px, py, pz)."""
    N = n.numel()
    dev = n.device
    o = out if out is not None else tuple(torch.empty(N, dtype=torch.float32, device=dev)
                                          for _ in range(3))
    _need(n, torch.uint8, "n")
    for t, nm in ((x, "x"), (y, "y"), (z, "z")):
        _need(t, torch.float32, nm)
        if t.dim() != 2 or t.shape[0] != 4 or t.shape[1] < N or t.shape[1] != x.shape[1]:
            raise ValueError(f"{nm} must be [4, S] with S >= N, one stride for x, y, z")
    ev = cc_events(_ptr(n), _ptr(x), _ptr(y), _ptr(z), None, N, x.shape[1])
    _check("cc_ring_apex", lib().cc_ring_apex(C.byref(ev), C.byref(_rings_struct(rings)),
                                               *(_ptr(t) for t in o), _stream(stream)))
    return o


def voxel_count(shape: str, n: int) -> int:
    c = int(lib().cc_voxel_count(UNIVERSES[shape], n))
    if c < 0:
        raise ValueError(f"bad universe ({shape}, {n})")
    return c


def voxel_universe(shape: str, n: int, pitch: float, center=(0.0, 0.0, 0.0), device="cuda",
                   stream=None):
    """Voxel centres of the image universe as (x, y, z) device tensors."""
    m = voxel_count(shape, n)
    out = tuple(torch.empty(m, dtype=torch.float32, device=device) for _ in range(3))
    _check("cc_voxel_universe", lib().cc_voxel_universe(
        UNIVERSES[shape], n, float(pitch), *(float(c) for c in center), *(_ptr(t) for t in out),
        _stream(stream)))
    return out


def backproject_workspace_bytes(R: int, V: int, params: Params | None = None) -> int:
    params = params or Params()
    return int(lib().cc_backproject_workspace_bytes(R, V, C.byref(params.c())))


def backproject(rings: dict, apex, voxels, params: Params | None = None, workspace=None,
                out=None, stream=None):
    """Near-field image over the voxels.  Returns (image [V] f32, argmax [1]
    i32, status [1] i32) device tensors (asynchronous)."""
    params = params or Params()
    rs = _rings_struct(rings)
    vs = _grid_struct(voxels)
    dev = voxels[0].device
    V = vs.count
    need = backproject_workspace_bytes(rs.count, V, params)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    if out is None:
        out = (torch.empty(V, dtype=torch.float32, device=dev),
               torch.empty(1, dtype=torch.int32, device=dev),
               torch.empty(1, dtype=torch.int32, device=dev))
    _check("cc_backproject", lib().cc_backproject(
        C.byref(rs), *(_ptr(t) for t in apex), C.byref(vs), C.byref(params.c()),
        _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _ptr(workspace), workspace.numel(),
        _stream(stream)))
    return out


def selftest_wait_timeout(which: int, limit_ns: int, device="cuda", stream=None):
    """Run a bounded device wait against a signal that never comes; returns
    the device status tensor [1] (CC_ETIMEOUT once limit_ns has passed)."""
    counter = torch.empty(1, dtype=torch.int32, device=device)
    status = torch.full((1,), 99, dtype=torch.int32, device=device)
    _check("cc_selftest_wait_timeout", lib().cc_selftest_wait_timeout(
        int(which), int(limit_ns), _ptr(counter), _ptr(status), _stream(stream)))
    return status


def selftest_exact_ops(device="cuda", stream=None):
    """Mismatches of the decision's correctly rounded reciprocal, square root
    and quotient against the CUDA intrinsics: (rcp, sqrt, div)."""
    out = torch.empty(3, dtype=torch.uint64, device=device)
    _check("cc_selftest_exact_ops", lib().cc_selftest_exact_ops(_ptr(out), _stream(stream)))
    return out


def events_copy(dst: tuple, dst_offset: int, src: tuple, src_offset: int = 0, count=None,
                stream=None):
    """Copy events between event sets given as (n, x, y, z, e) tensors with
    x, y, z, e of shape [4, S] (views of a wider buffer allowed: each row's
    stride is its own).  One library call: n plus one 2D copy per array."""
    def struct(ev):
        n, x, y, z, e = ev
        stride = x.stride(0)
        if any(t.stride(0) != stride or t.stride(1) != 1 for t in (y, z, e)) or x.stride(1) != 1:
            raise ValueError("x, y, z, e must share one row stride and have unit column stride")
        return cc_events(_ptr(n), _ptr(x), _ptr(y), _ptr(z), _ptr(e), n.numel(), stride)
    count = src[0].numel() - src_offset if count is None else count
    d, s = struct(dst), struct(src)
    _check("cc_events_copy", lib().cc_events_copy(C.byref(d), dst_offset, C.byref(s), src_offset,
                                                   count, _stream(stream)))
