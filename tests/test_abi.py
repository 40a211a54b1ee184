"""The C-ABI library builds, loads and exports every entry point that
include/compton.h declares; host-side argument checks need no GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "compton.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2411_04785_gb300 import build
    return build.build()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("cc_rings_from_events", "cc_localize", "cc_refine",
                 "cc_localize_workspace_bytes", "cc_refine_workspace_bytes",
                 "cc_grid_fibonacci", "cc_grid_healpix_ring", "cc_grid_gather",
                 "cc_last_error", "cc_params_default", "cc_abi_version"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = C.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_host_side_calls_without_gpu(libpath):
    import paper_2411_04785_gb300 as cc
    L = cc.lib()
    assert L.cc_abi_version() == 2
    p = cc.default_params()
    assert p.topk == 1 and p.max_iter == 50 and abs(p.tol_rad - 1e-7) < 1e-20
    # argument errors are caught before any CUDA call
    from paper_2411_04785_gb300 import api
    assert L.cc_grid_healpix_ring(0, None, None, None, None) == -1
    assert b"nside" in L.cc_last_error()
    assert L.cc_grid_fibonacci(0, None, None, None, None) == -1
    bad = api.cc_params(0.05, 1.0, 0.01, 0.3, 0.0, 0, 0.01, 50, 1e-7)   # topk 0
    rs = api.cc_rings(None, None, None, None, None, None, None, 0)
    gs = api.cc_grid(None, None, None, 10)
    assert L.cc_localize(C.byref(rs), C.byref(gs), C.byref(bad), None, None, None, None,
                         None, 0, None) == -1
    assert b"topk" in L.cc_last_error()
    assert L.cc_refine_workspace_bytes(-1, 1) == 0


def test_cluster_argument_checks_without_gpu(libpath):
    import paper_2411_04785_gb300 as cc
    from paper_2411_04785_gb300 import api
    L = cc.lib()
    ws = L.cc_cluster_workspace_bytes(10_000)
    assert ws >= 256 and L.cc_cluster_workspace_bytes(-1) == 0
    fake = C.c_void_p(1 << 20)                     # never dereferenced: checks come first
    call = lambda d, cap=5000, wsb=ws, ev=None: L.cc_cluster_maxstep(
        d, 10, None, None, ev, None, None, cap, None, None, fake, wsb, None)
    assert call(None) == -1 and b"NULL" in L.cc_last_error()
    assert call(C.byref(api.cc_detections(fake, fake, 1 << 31))) == -1
    assert call(C.byref(api.cc_detections(None, None, 10))) == -1            # t NULL
    d = C.byref(api.cc_detections(fake, fake, 10_000))
    assert call(d, cap=4999, ev=fake) == -1 and b"capacity" in L.cc_last_error()
    assert call(d, wsb=ws - 1) == -1 and b"workspace" in L.cc_last_error()
    assert L.cc_cluster_spectrum(fake, fake, 0, 10, fake, None) == -1
    assert L.cc_cluster_spectrum(fake, fake, 4, 0, fake, None) == -1


def test_debug_calls_refused_by_the_normal_build(libpath):
    import paper_2411_04785_gb300 as cc
    L = cc.lib()
    w = C.c_uint64(5)
    assert L.cc_debug_bounds(C.byref(w), 0) == -1 and w.value == 0
    assert b"debug" in L.cc_last_error()
    assert L.cc_debug_selftest_bounds(None, 8, None) == -1


def test_debug_build_links_and_exports_every_declared_symbol():
    from paper_2411_04785_gb300 import build
    path = build.build(debug=True)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert not [n for n in declared_functions() if n not in exported]


def test_voxel_universe_counts_without_gpu(libpath):
    import oracle
    import paper_2411_04785_gb300 as cc
    L = cc.lib()
    for shape, s in (("cube", 0), ("cylinder", 1), ("sphere", 2)):
        for n in (1, 2, 5, 16, 37):
            assert L.cc_voxel_count(s, n) == oracle.universe(shape, n, 1.0, count_only=True)
    assert L.cc_voxel_count(3, 4) == -1 and L.cc_voxel_count(0, 0) == -1
    assert L.cc_voxel_count(0, 1025) == -1
    assert L.cc_voxel_universe(1, 0, 1.0, 0, 0, 0, None, None, None, None) == -1
    assert L.cc_voxel_universe(1, 8, 0.0, 0, 0, 0, None, None, None, None) == -1


def test_events_copy_argument_checks_without_gpu(libpath):
    import paper_2411_04785_gb300 as cc
    from paper_2411_04785_gb300 import api
    L = cc.lib()
    fake = C.c_void_p(1 << 20)
    ev = lambda stride: api.cc_events(fake, fake, fake, fake, fake, stride, stride)
    assert L.cc_events_copy(None, 0, C.byref(ev(10)), 0, 5, None) == -1
    assert L.cc_events_copy(C.byref(ev(10)), 6, C.byref(ev(10)), 0, 5, None) == -1   # past dst
    assert L.cc_events_copy(C.byref(ev(10)), 0, C.byref(ev(4)), 0, 5, None) == -1    # past src
    assert L.cc_events_copy(C.byref(ev(10)), 0, C.byref(ev(10)), 0, -1, None) == -1
    assert L.cc_events_copy(C.byref(ev(10)), 0, C.byref(ev(10)), 0, 0, None) == 0     # nothing


def test_wait_selftest_argument_checks_without_gpu(libpath):
    import paper_2411_04785_gb300 as cc
    L = cc.lib()
    fake = C.c_void_p(1 << 20)                     # never dereferenced: checks come first
    assert L.cc_selftest_wait_timeout(2, 10**6, fake, fake, None) == -1
    assert L.cc_selftest_wait_timeout(0, 999, fake, fake, None) == -1
    assert L.cc_selftest_wait_timeout(1, 10**10 + 1, fake, fake, None) == -1
    assert L.cc_selftest_wait_timeout(0, 10**6, None, fake, None) == -1
    assert b"NULL" in L.cc_last_error()
