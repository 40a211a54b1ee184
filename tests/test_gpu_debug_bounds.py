"""The debug build (build(debug=True), libcompton_debug.so): every checked
index of the hot path's kernels is compared with its buffer's bound, and a
failure is recorded in a device word instead of being accessed - the
stand-in for a memory checker.  The small cases of tests/debug_bounds_cases.py
run once on each build in a child process: the debug build must leave the
word at 0 and give the optimised build's results (integers bit for bit,
floating point within the map rule's relative 1e-5, the rounding of a
differently compiled build), and its self-test, one checked access one past
the end of a buffer, must be recorded as such and skipped."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def runs(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_04785_gb300 import build
    build.build()
    build.build(debug=True)
    out = {}
    for name in ("normal", "debug"):
        path = str(tmp_path_factory.mktemp(name) / "res.npz")
        env = dict(os.environ)
        env.pop("CC_LIBRARY", None)
        if name == "debug":
            env["CC_LIBRARY"] = "debug"
        r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_bounds_cases.py"),
                            path], env=env, capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stderr[-3000:]
        out[name] = dict(np.load(path))
    return out


def test_no_checked_index_out_of_bounds(runs):
    assert int(runs["debug"]["word"][0]) == 0, hex(int(runs["debug"]["word"][0]))


def test_debug_build_gives_the_same_results(runs):
    a, b = runs["normal"], runs["debug"]
    for k, v in a.items():
        w = b[k]
        if v.dtype.kind in "iub":
            np.testing.assert_array_equal(w, v, err_msg=k)
        else:
            scale = np.maximum(np.abs(v), 1e-3 * np.abs(v).max() + 1e-30)
            assert (np.abs(w - v) <= 1e-5 * scale).all(), k


def test_selftest_records_the_index_and_skips_the_access(runs):
    word = int(runs["debug"]["selftest_word"][0])
    assert word >> 48 == 0x7fff and word & ((1 << 48) - 1) == 8
    assert not runs["debug"]["selftest_buf"].any()


def test_normal_build_refuses_the_debug_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_04785_gb300 as cc
    from paper_2411_04785_gb300 import api
    if os.environ.get("CC_LIBRARY") == "debug":
        pytest.skip("this process runs the debug build")
    with pytest.raises(cc.CCError):
        api.debug_bounds()
