"""Pins of the event-clustering oracle (Sec. 2) against facts independent of
its code: hand-worked streams, a union-find over the masked steps, the
invariants of the edge array, limits of dt_max, and the behaviour the paper
states for the fixed window it replaces."""
import numpy as np
import pytest

import oracle


def union_find_events(t, adc, dt_max):
    """Brute force: join i and i+1 when their step is below dt_max (union-
    find), events = components of two or more detections, numbered by their
    first detection."""
    N = len(t)
    parent = list(range(N))

    def root(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    for i in range(N - 1):
        if int(t[i + 1]) - int(t[i]) < dt_max:
            parent[root(i + 1)] = root(i)
    comps = {}
    for i in range(N):
        comps.setdefault(root(i), []).append(i)
    events = sorted((m for m in comps.values() if len(m) > 1), key=lambda m: m[0])
    eid = -np.ones(N, np.int32)
    for k, m in enumerate(events):
        eid[m] = k
    return eid, [m[0] for m in events], [len(m) for m in events], \
        [int(sum(int(adc[i]) for i in m)) for m in events]


def test_hand_worked_stream():
    # steps: 5 3 22 70 4 96 1 1 198 ; dt_max = 10
    t = np.array([0, 5, 8, 30, 100, 104, 200, 201, 202, 400])
    adc = np.arange(1, 11)
    r = oracle.maxstep_events(t, adc, 10)
    #        M_i (step after i): T T F F T F T T F (F beyond the end)
    #        E_i = M_{i-1} ^ M_i: 1 0 1 0 1 1 1 0 1 0
    assert r["edge"].tolist() == [1, 0, 1, 0, 1, 1, 1, 0, 1, 0]
    assert r["event_id"].tolist() == [0, 0, 0, -1, 1, 1, 2, 2, 2, -1]
    assert r["first"].tolist() == [0, 4, 6]
    assert r["count"].tolist() == [3, 2, 3]
    assert r["adc"].tolist() == [1 + 2 + 3, 5 + 6, 7 + 8 + 9]


def test_strict_inequality_and_single_detections():
    # a step equal to dt_max does not join (M uses "<")
    r = oracle.maxstep_events(np.array([0, 10, 20]), np.ones(3), 10)
    assert r["edge"].tolist() == [0, 0, 0] and len(r["count"]) == 0
    r = oracle.maxstep_events(np.array([0, 9, 19]), np.ones(3), 10)
    assert r["edge"].tolist() == [1, 1, 0] and r["count"].tolist() == [2]
    assert oracle.maxstep_edges(np.array([7]), 10).tolist() == [0]
    assert oracle.maxstep_edges(np.array([], np.int64), 10).size == 0


@pytest.mark.parametrize("seed", range(6))
def test_matches_union_find(seed):
    rng = np.random.default_rng(seed)
    N = 400
    t = np.sort(rng.integers(0, 4000, N))             # ties (step 0) included
    adc = rng.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
    for dt_max in (1, 5, 12, 40):
        r = oracle.maxstep_events(t, adc, dt_max)
        eid, first, count, s = union_find_events(t, adc, dt_max)
        np.testing.assert_array_equal(r["event_id"], eid)
        assert r["first"].tolist() == first and r["count"].tolist() == count
        assert [int(v) for v in r["adc"]] == s        # exact 64-bit sums


def test_edge_invariants_and_limits():
    rng = np.random.default_rng(7)
    t = np.sort(rng.integers(0, 10**6, 5000))
    adc = rng.integers(1, 100, 5000)
    r = oracle.maxstep_events(t, adc, 300)
    K = len(r["count"])
    e = np.flatnonzero(r["edge"])
    assert e.size == 2 * K                                   # a begin and an end per event
    np.testing.assert_array_equal(e[0::2], r["first"])
    np.testing.assert_array_equal(e[1::2], r["first"] + r["count"] - 1)
    assert r["count"].min() >= 2
    assert (r["event_id"] >= 0).sum() == r["count"].sum()
    # dt_max above every step: one event of everything; dt_max <= 0: none
    big = oracle.maxstep_events(t, adc, 10**7)
    assert big["count"].tolist() == [5000] and int(big["adc"][0]) == int(adc.sum())
    none = oracle.maxstep_events(t, adc, 0)
    assert len(none["count"]) == 0 and not none["edge"].any()


def test_fixed_window_hand_worked_and_paper_claims():
    # prior art: window 10, at least 2 detections.  [0, 10) holds 0 4 9: an
    # event; [12, 22) holds 12 alone and [30, 40) holds 30 alone: the window
    # moves on; [50, 60) holds 50 55: an event
    t = np.array([0, 4, 9, 12, 30, 50, 55])
    r = oracle.fixed_window_events(t, np.ones(7), 10, 2, 0)
    assert r["event_id"].tolist() == [0, 0, 0, -1, -1, 1, 1]
    # Sec. 2: simultaneous (pile-up) events are grouped by the max step,
    # where a fixed window cuts them
    t = np.array([0, 3, 6, 9, 12, 15, 18, 21])             # two overlapping bursts
    assert oracle.maxstep_events(t, np.ones(8), 5)["count"].tolist() == [8]
    assert oracle.fixed_window_events(t, np.ones(8), 12, 2, 0)["count"].tolist() == [4, 4]
    # Sec. 2: a noise detection does not break an event: a dark count ahead
    # of the event opens the fixed window early and the event's tail falls
    # out of it; the max step keeps the event in one piece
    t = np.array([0, 7, 9, 11, 13, 15, 17, 19])             # dark count at 0
    fw = oracle.fixed_window_events(t, np.ones(8), 12, 2, 0)  # [0, 12) and [13, 25)
    assert fw["count"].tolist() == [4, 4] and fw["event_id"][0] == 0
    r = oracle.maxstep_events(t, np.ones(8), 3)
    assert r["count"].tolist() == [7] and r["event_id"][0] == -1


def test_spectrum():
    rng = np.random.default_rng(3)
    s = rng.integers(0, 1000, 3000).astype(np.uint64)
    h = oracle.spectrum(s, 16, 50)
    want = np.bincount(np.minimum(s // 16, 49).astype(np.int64), minlength=50)
    np.testing.assert_array_equal(h, want)
    assert h.sum() == 3000
