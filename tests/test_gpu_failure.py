"""Failure detection on the GPU without a fault: the library's bounded
device waits (the mbarrier wait of the TMA / tensor-core pipelines and the
global-counter spin of the refinement's grid barrier) are made to run out on
a signal that never comes; each reports CC_ETIMEOUT after its limit and the
context stays usable for the next call."""
import time

import numpy as np
import pytest

import oracle
from tests.helpers import grid_to_dev, rings_to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CC_ETIMEOUT = -4


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_04785_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_reports_timeout_and_context_survives(cc, which):
    dev = torch.device("cuda:0")
    limit_ns = 50_000_000                                    # 50 ms
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = cc.api.selftest_wait_timeout(which, limit_ns, device=dev)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(st.item()) == CC_ETIMEOUT
    assert limit_ns * 1e-9 <= dt < 30.0
    # the context is usable: a small localisation still matches the oracle
    rng = np.random.default_rng(which)
    a = rng.standard_normal((500, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    rings = {"ax": a[:, 0], "ay": a[:, 1], "az": a[:, 2],
             "eta": rng.uniform(0.2, 1.2, 500), "deta": np.full(500, 0.1)}
    r32 = {k: np.asarray(v, np.float32) for k, v in rings.items()}
    g = oracle.grid_healpix_ring(8)
    loc = cc.Localizer(grid_to_dev(g, dev), cc.Params())
    loc.from_rings(rings_to_dev(r32, dev))
    torch.cuda.synchronize()
    want = oracle.likelihood_map(r32, tuple(np.asarray(v, np.float32) for v in g))
    got = loc.map.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-5 * want.max()
