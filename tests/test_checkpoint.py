"""The ring filter's checkpoint format (host side, no GPU): a round trip
keeps every bit, and a damaged or foreign file is refused."""
import numpy as np
import pytest

from paper_2411_04785_gb300 import api


def state(seed, n=api.MLP_PARAMS):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(n).astype(np.float32) for _ in range(3)]


def test_round_trip_keeps_every_bit():
    p, m, v = state(1)
    p[0], m[1], v[2] = np.float32(-0.0), np.float32(np.inf), np.float32(1e-45)
    buf = api.pack_filter_state(p, m, v, 1234)
    assert len(buf) == 32 + 12 * p.size
    q, mq, vq, step = api.unpack_filter_state(buf)
    assert step == 1234
    for a, b in ((p, q), (m, mq), (v, vq)):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_damaged_or_foreign_files_are_refused():
    p, m, v = state(2, 10)
    buf = api.pack_filter_state(p, m, v, 7)
    with pytest.raises(ValueError):
        api.unpack_filter_state(b"NOTAFILE" + buf[8:])
    with pytest.raises(ValueError):
        api.unpack_filter_state(buf[:-4])
    with pytest.raises(ValueError):
        api.unpack_filter_state(buf[:8] + (2).to_bytes(4, "little") + buf[12:])
    with pytest.raises(ValueError):
        api.pack_filter_state(p, m[:5], v, 0)
