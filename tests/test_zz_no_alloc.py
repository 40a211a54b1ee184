"""cc_localize_static, the localisation entry point for callers that cannot
allocate device memory (a real-time acquisition loop that must not allocate
once running, an application whose pool owns all device memory): its scratch
is a static device array inside the library instead of a caller workspace.

It is called here through the C ABI (ctypes) and checked against
cc_localize, the workspace entry point: both run the same plan and the same
kernels, so the map, the argmax and the seeds must be bit-equal, on two calls
in a row (the shared array keeps the previous call's contents, so a stale
value left in it would show as a difference in the last bits).  One burst is
also checked against the oracle's map.  This file is collected last and
passes alone in a fresh process as well as after the other tests."""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
from paper_2411_04785_gb300 import synth
from tests.helpers import grid_to_dev, map_violations, rings_to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_04785_gb300 as m
    m.lib()
    return m


def call_static(cc, rd, gd, params, dev):
    from paper_2411_04785_gb300 import api
    M = gd[0].numel()
    m = torch.full((M,), -1.0, dtype=torch.float32, device=dev)
    am = torch.full((1,), -7, dtype=torch.int32, device=dev)
    sd = torch.full((params.topk,), -7, dtype=torch.int32, device=dev)
    st = torch.full((1,), 99, dtype=torch.int32, device=dev)
    rs, gs, pc = api._rings_struct(rd), api._grid_struct(gd), params.c()
    rc = cc.lib().cc_localize_static(C.byref(rs), C.byref(gs), C.byref(pc), api._ptr(m),
                                     api._ptr(am), api._ptr(sd), api._ptr(st),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, cc.lib().cc_last_error()
    torch.cuda.synchronize()
    return m.cpu().numpy(), am.cpu().numpy(), sd.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("R,M,seed,topk", [(2000, 3072, 1, 1), (50000, 3000, 2, 8),
                                           (7777, 49152, 3, 4)])
def test_static_scratch_matches_workspace_entry_point(cc, R, M, seed, topk):
    dev = torch.device("cuda:0")
    rings, _, _ = synth.rings_burst(n=R, seed=seed)
    rd = rings_to_dev(rings, dev)
    gd = grid_to_dev(oracle.grid_fibonacci(M), dev)
    p = cc.Params(topk=topk, nms_rad=math.radians(2.0))
    ref = cc.localize(rd, gd, p)
    torch.cuda.synchronize()
    ref_map = ref[0].cpu().numpy()
    for _ in range(2):                   # two calls in a row share the array
        m, am, sd, st = call_static(cc, rd, gd, p, dev)
        assert st == 0
        np.testing.assert_array_equal(m, ref_map)
        assert int(am[0]) == int(ref[1].item())
        np.testing.assert_array_equal(sd, ref[2].cpu().numpy())


def test_static_scratch_matches_oracle(cc):
    """The noise-free 2,000-ring burst over the 3,072-direction Fibonacci
    grid, after a larger call has filled the shared array: every direction
    within the map rule of the oracle's FP64 map, and the argmax the oracle's
    (the true source's neighbourhood)."""
    dev = torch.device("cuda:0")
    big, _, _ = synth.rings_burst(n=60000, seed=9)
    gbig = grid_to_dev(oracle.grid_fibonacci(20000), dev)
    call_static(cc, rings_to_dev(big, dev), gbig, cc.Params(), dev)
    rings, source = synth.rings_noise_free()
    g = oracle.grid_fibonacci(3072)
    want = oracle.likelihood_map(rings, tuple(np.asarray(v, np.float32) for v in g))
    for _ in range(2):
        m, am, _, st = call_static(cc, rings_to_dev(rings, dev), grid_to_dev(g, dev),
                                   cc.Params(), dev)
        assert st == 0
        assert map_violations(m.astype(np.float64), want, want.max()).size == 0
        assert want[int(am[0])] >= want.max() * (1 - 2e-5)


def test_static_scratch_rejects_sizes_beyond_its_maximum(cc):
    from paper_2411_04785_gb300 import api
    dev = torch.device("cuda:0")
    R, M = 2_000_000, 3072               # 2M packed rings alone need 64 MB
    rd = {k: torch.zeros(R, dtype=torch.float32, device=dev)
          for k in ("ax", "ay", "az", "eta", "deta")}
    gd = grid_to_dev(oracle.grid_fibonacci(M), dev)
    assert cc.localize_workspace_bytes(R, M) > api.STATIC_SCRATCH_BYTES
    with pytest.raises(cc.CCError) as ei:
        cc.localize_static(rd, gd)
    assert ei.value.status == -1 and "static scratch" in str(ei.value)
