"""GPU max-step clustering (Sec. 2) against the oracle: every output is
integer, so every output must be equal bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2411_04785_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FULL_COPIES = 12          # the benchmark's stream: 12 copies of the 400k-event segment


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_04785_gb300 as m
    m.lib()
    return m


def run(cc, t, adc, dt_max):
    dev = torch.device("cuda:0")
    td = torch.from_numpy(np.ascontiguousarray(t, np.int64)).to(dev)
    ad = torch.from_numpy(np.ascontiguousarray(adc, np.uint32)).to(dev)
    o = cc.cluster_maxstep(td, ad, dt_max)
    torch.cuda.synchronize()
    K = int(o["n_events"].item())
    assert int(o["status"].item()) == 0
    return {"edge": o["edge"].cpu().numpy(), "event_id": o["event_id"].cpu().numpy(),
            "first": o["first"][:K].cpu().numpy(), "count": o["count"][:K].cpu().numpy(),
            "adc": o["adc"][:K].cpu().numpy()}, o


def assert_same(got, want):
    for k in ("edge", "event_id", "first", "count", "adc"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)


@pytest.mark.parametrize("dt_max", [10_000, 15_000, 25_000])
def test_stream_matches_oracle(cc, dt_max):
    t, adc, _ = synth.detection_stream(n_events=3000, seed=4)
    t, adc = t[:4096 * 9 + 123], adc[:4096 * 9 + 123]           # 10 tiles, ragged tail
    got, _ = run(cc, t, adc, dt_max)
    assert_same(got, oracle.maxstep_events(t, adc, dt_max))


@pytest.mark.parametrize("N", [1, 2, 31, 32, 33, 511, 512, 513, 2047, 2048, 2049, 4095, 4096, 4097, 12289])
def test_sizes_and_tile_boundaries(cc, N):
    rng = np.random.default_rng(N)
    t = np.cumsum(rng.integers(0, 20, N))
    adc = rng.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
    for dt_max in (1, 8, 15):
        got, _ = run(cc, t, adc, dt_max)
        assert_same(got, oracle.maxstep_events(t, adc, dt_max))


def test_one_event_across_every_tile_and_none(cc):
    N = 4096 * 5 + 77
    t = np.arange(N, dtype=np.int64) * 3
    adc = np.full(N, 0xFFFFFFFF, np.uint32)                   # sums beyond 32 bits
    got, _ = run(cc, t, adc, 4)
    want = oracle.maxstep_events(t, adc, 4)
    assert_same(got, want)
    assert got["count"].tolist() == [N] and int(got["adc"][0]) == N * 0xFFFFFFFF
    got, _ = run(cc, t, adc, 3)                                # step == dt_max: no event
    assert got["count"].size == 0 and not got["edge"].any() and (got["event_id"] == -1).all()


def test_long_events_that_cross_tiles(cc):
    """Events of 1 to 9,000 detections (lengths around 256, the tail a tile
    reads ahead, and longer than a tile) in random order: a tile's last event
    starts anywhere in it and runs on into later tiles."""
    rng = np.random.default_rng(21)
    lens = rng.choice(np.array([1, 2, 3, 17, 200, 255, 256, 257, 300, 1000, 4095, 4097, 9000]),
                      size=80)
    steps = []
    for L in lens:
        steps += [1] * (int(L) - 1) + [50]          # joined inside an event, a gap after it
    t = np.concatenate([[0], np.cumsum(steps[:-1])]).astype(np.int64)
    adc = rng.integers(0, 1 << 32, t.size, dtype=np.uint64).astype(np.uint32)
    got, _ = run(cc, t, adc, 2)
    want = oracle.maxstep_events(t, adc, 2)
    assert_same(got, want)
    assert got["count"].size == int((lens > 1).sum())


def test_pairs_steps_at_the_limit_and_large_times(cc):
    # alternating pair / gap pattern puts starts and ends on every lane and
    # row boundary; times near 2^62 exercise the 64-bit steps
    N = 4096 * 3 + 5
    steps = np.where(np.arange(N) % 2 == 0, 7, 8)
    t = (1 << 62) + np.concatenate([[0], np.cumsum(steps[:-1])])
    adc = np.arange(N, dtype=np.uint32)
    for dt_max in (7, 8, 9):
        got, _ = run(cc, t, adc, dt_max)
        assert_same(got, oracle.maxstep_events(t, adc, dt_max))


def test_empty_stream(cc):
    dev = torch.device("cuda:0")
    o = cc.cluster_maxstep(torch.empty(0, dtype=torch.int64, device=dev),
                           torch.empty(0, dtype=torch.uint32, device=dev), 10)
    torch.cuda.synchronize()
    assert int(o["n_events"].item()) == 0 and int(o["status"].item()) == 0


def test_full_size_stream_and_spectrum(cc):
    """The benchmark's stream (12 tiled copies of the 400k-event 137Cs-like
    segment, ~75M detections, 15 ns step), every output against the oracle;
    then the amplitude spectrum of its events."""
    t0, a0, _ = synth.detection_stream()
    t, adc = synth.tile_stream(t0, a0, FULL_COPIES)
    got, o = run(cc, t, adc, 15_000)
    want = oracle.maxstep_events(t, adc, 15_000)
    assert_same(got, want)
    h = cc.cluster_spectrum(o["adc"], o["n_events"], 64, 160)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(h.cpu().numpy(), oracle.spectrum(want["adc"], 64, 160))
    h = cc.cluster_spectrum(o["adc"], o["n_events"], 3, 20000)   # global-atomic path
    torch.cuda.synchronize()
    np.testing.assert_array_equal(h.cpu().numpy(), oracle.spectrum(want["adc"], 3, 20000))


def test_output_subsets_and_no_amplitudes(cc):
    """Outputs may be asked for one by one, and amplitudes left out."""
    t, adc, _ = synth.detection_stream(n_events=1500, seed=6)
    want = oracle.maxstep_events(t, adc, 15_000)
    td = torch.from_numpy(t).to("cuda:0")
    o = cc.cluster_maxstep(td, None, 15_000, outputs=("edge", "event_id", "first", "count"))
    torch.cuda.synchronize()
    K = int(o["n_events"].item())
    np.testing.assert_array_equal(o["edge"].cpu().numpy(), want["edge"])
    np.testing.assert_array_equal(o["event_id"].cpu().numpy(), want["event_id"])
    np.testing.assert_array_equal(o["first"][:K].cpu().numpy(), want["first"])
    np.testing.assert_array_equal(o["count"][:K].cpu().numpy(), want["count"])
    o = cc.cluster_maxstep(td, torch.from_numpy(adc).to("cuda:0"), 15_000, outputs=("adc",))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(o["adc"][:K].cpu().numpy(), want["adc"])
