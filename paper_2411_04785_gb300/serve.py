"""Serving loop for burst localisation with continuous batching.

Bursts (event sets of uneven size) arrive over time.  A burst is admitted as
soon as a slot and its device-memory budget are free; its events are copied
to the device and reconstructed into rings (and, on the learned path, scored
and re-widthed by the ring filter) on a stream of its own.  Every pass of the
loop sweeps ALL bursts admitted since the last sweep in one batched launch
(cc_localize_batch: one persistent kernel over the work units of every
burst), on one of two sweep streams that wait for the bursts' front ends on
the device, so a new batch overlaps a running one on the GPU; each burst's
refinement and result read-back then run on its own stream again.  The host
only polls for completed results; it never waits for the GPU while bursts
remain.

A burst's results do not depend on the batch it was swept in (the batched
sweep keeps each burst's own plan), which the tests check against the same
burst served alone.  Host code here only schedules and moves buffers: every
step of the localisation runs in libcompton.so.

With graphs=True the per-burst front end (reconstruction and, on the learned
path, features, MLP and filter) is a CUDA graph captured once per size bucket
(powers of two) with static buffers: a burst copies its events in, marks the
padding events empty (n = 0, so their rings are invalid and compacted away
before the sweep) and replays one graph instead of launching a dozen kernels
from the host.  Every event and every MLP row is computed independently, so
the results equal the graph-less path's bit for bit.
"""
from __future__ import annotations

import ctypes as C
import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api

BATCH_MAX = 64


@dataclass
class Burst:
    """One request: its events on the host as one or more parts, each
    (n [k] uint8, x, y, z, e [4, k] float32) pinned tensors or views of
    pinned tensors whose rows are contiguous; arrival time in seconds."""
    bid: int
    arrival: float
    parts: list
    source: np.ndarray | None = None

    @property
    def count(self):
        return sum(p[0].numel() for p in self.parts)


@dataclass
class _Active:
    burst: Burst
    stream: torch.cuda.Stream
    bytes: int
    t_admit: float
    dev: dict = field(default_factory=dict)
    ready: torch.cuda.Event | None = None
    swept: bool = False
    done: torch.cuda.Event | None = None
    out_host: dict = field(default_factory=dict)
    front: "_Front | None" = None
    ev0: torch.cuda.Event | None = None       # breakdown: front end starts
    swept_ev: torch.cuda.Event | None = None  # breakdown: its batch's sweep ended
    t_sweep: float = 0.0                      # breakdown: host time the sweep was issued


class _Front:
    """A captured front end for bursts of up to `cap` events."""

    def __init__(self, srv: "Server", cap: int):
        dev = srv.dev
        self.cap = cap
        self.n = torch.zeros(cap, dtype=torch.uint8, device=dev)
        self.xyze = {k: torch.zeros((4, cap), dtype=torch.float32, device=dev) for k in "xyze"}
        self.rings = api.empty_rings(cap, dev)
        learned = srv.filter is not None
        # the burst's outputs and scratch, sized for the bucket
        pc = srv.params.c()
        tk = srv.params.topk
        self.out = {
            "ws": torch.empty(max(api.lib().cc_localize_batch_workspace_bytes(cap, srv.M, C.byref(pc)),
                                  256), dtype=torch.uint8, device=dev),
            "map": torch.empty(srv.M, dtype=torch.float32, device=dev),
            "argmax": torch.empty(1, dtype=torch.int32, device=dev),
            "seeds": torch.empty(tk, dtype=torch.int32, device=dev),
            "status": torch.empty(1, dtype=torch.int32, device=dev),
            "seed_dirs": torch.empty((tk, 3), dtype=torch.float64, device=dev),
            "ref_ws": torch.empty(max(api.refine_workspace_bytes(cap, tk), 256), dtype=torch.uint8,
                                  device=dev),
            "ref": (torch.empty(3, dtype=torch.float64, device=dev),
                    torch.empty(1, dtype=torch.float64, device=dev),
                    torch.empty(1, dtype=torch.int32, device=dev),
                    torch.empty(1, dtype=torch.int32, device=dev))}
        if learned:
            self.feats = torch.empty((cap, api.MLP_FEATURES), dtype=torch.bfloat16, device=dev)
            self.mlp_out = torch.empty((cap, 2), dtype=torch.float32, device=dev)
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        x, y, z, e = (self.xyze[k] for k in "xyze")

        def body():
            api.rings_from_events(self.n, x, y, z, e, srv.params, out=self.rings, stream=s)
            if learned:
                api.ring_features(self.n, x, y, z, e, self.rings, srv.params, out=self.feats,
                                  stream=s)
                srv.filter.forward(self.feats, out=self.mlp_out, stream=s)
                srv.filter.apply(self.rings, self.mlp_out, srv.tau, srv.params.deta_min,
                                 srv.filter_deta_max, stream=s)

        with torch.cuda.stream(s):
            body()                                   # once outside capture (lazy setup)
        s.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=s, capture_error_mode="relaxed"):
            body()
        torch.cuda.synchronize(dev)

    def ring_views(self, N: int) -> dict:
        return {k: v[:N] for k, v in self.rings.items()}


def burst_bytes(N: int, M: int, params: api.Params, learned: bool) -> int:
    """Device bytes one burst holds while in flight."""
    b = N * (1 + 4 * 4 * 4) + N * (5 * 4 + 2)                 # events + rings
    b += api.lib().cc_localize_batch_workspace_bytes(N, M, C.byref(params.c()))
    b += api.refine_workspace_bytes(N, params.topk) + M * 4 + 1024
    if learned:
        b += N * (api.MLP_FEATURES * 2 + 8)                      # features + outputs
    return int(b)


class Server:
    """Continuous-batching server over one GPU."""

    def __init__(self, grid, params: api.Params | None = None, hbm_budget: int = 2 << 30,
                 max_active: int = 48, ring_filter: api.RingFilter | None = None,
                 tau: float = 0.0, filter_deta_max: float | None = None, graphs: bool = False):
        # the grid's direction order, computed once for every batched sweep
        grid = tuple(grid[:3]) + (grid[3] if len(grid) > 3 else api.grid_order(grid),)
        self.grid = grid
        self.M = grid[0].numel()
        self.dev = grid[0].device
        self.params = params or api.Params()
        self.budget = hbm_budget
        self.max_active = max_active
        self.filter = ring_filter
        self.tau = tau
        self.filter_deta_max = filter_deta_max or self.params.deta_max
        # bursts' own streams (front end, refinement, read-back) outrank the
        # sweep streams, so a burst's short kernels take SMs as soon as sweep
        # CTAs retire instead of queueing behind a whole batch
        self.sweep_streams = [torch.cuda.Stream(self.dev, priority=0) for _ in range(2)]
        self._ss = 0
        self._gs = api._grid_struct(grid)
        self.graphs = graphs
        self.breakdown = False
        self.keep_maps = False
        self._fronts: dict[int, list[_Front]] = {}     # free captured front ends per bucket

    @staticmethod
    def bucket(N: int) -> int:
        return max(512, 1 << max(0, (N - 1).bit_length()))

    def _front(self, N: int) -> _Front:
        cap = self.bucket(N)
        free = self._fronts.setdefault(cap, [])
        return free.pop() if free else _Front(self, cap)

    def prepare(self, counts):
        """Capture front ends ahead of time, one per distinct bucket of `counts`."""
        if self.graphs:
            for cap in sorted({self.bucket(c) for c in counts}):
                if not self._fronts.get(cap):
                    self._fronts.setdefault(cap, []).append(_Front(self, cap))

    # -- per-burst front end ------------------------------------------------
    def _event(self):
        return torch.cuda.Event(enable_timing=self.breakdown)

    def _admit(self, b: Burst, now: float) -> _Active:
        s = torch.cuda.Stream(self.dev, priority=-1)
        a = _Active(b, s, burst_bytes(b.count, self.M, self.params, self.filter is not None), now)
        if self.breakdown:
            a.ev0 = self._event()
            a.ev0.record(s)
        if self.graphs:
            return self._admit_graph(a)
        d = a.dev
        N = b.count
        with torch.cuda.stream(s):
            d["n"] = torch.empty(N, dtype=torch.uint8, device=self.dev)
            for k in "xyze":
                d[k] = torch.empty((4, N), dtype=torch.float32, device=self.dev)
            dst = (d["n"], d["x"], d["y"], d["z"], d["e"])
            off = 0
            for part in b.parts:                 # n + one 2D copy per array
                api.events_copy(dst, off, part, stream=s)
                off += part[0].numel()
            d["rings"] = api.rings_from_events(d["n"], d["x"], d["y"], d["z"], d["e"],
                                               self.params, stream=s)
            if self.filter is not None:
                F = api.ring_features(d["n"], d["x"], d["y"], d["z"], d["e"], d["rings"],
                                      self.params, stream=s)
                out = self.filter.forward(F, stream=s)
                self.filter.apply(d["rings"], out, self.tau, self.params.deta_min,
                                  self.filter_deta_max, stream=s)
            ws_b = api.lib().cc_localize_batch_workspace_bytes(b.count, self.M,
                                                               C.byref(self.params.c()))
            d["ws"] = torch.empty(max(ws_b, 256), dtype=torch.uint8, device=self.dev)
            d["map"] = torch.empty(self.M, dtype=torch.float32, device=self.dev)
            d["argmax"] = torch.empty(1, dtype=torch.int32, device=self.dev)
            d["seeds"] = torch.empty(self.params.topk, dtype=torch.int32, device=self.dev)
            d["status"] = torch.empty(1, dtype=torch.int32, device=self.dev)
            a.ready = self._event()
            a.ready.record(s)
        return a

    def _admit_graph(self, a: _Active) -> _Active:
        b, s, d = a.burst, a.stream, a.dev
        N = b.count
        f = a.front = self._front(N)
        s.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(s):
            dst = (f.n, f.xyze["x"], f.xyze["y"], f.xyze["z"], f.xyze["e"])
            off = 0
            for part in b.parts:                 # n + one 2D copy per array
                api.events_copy(dst, off, part, stream=s)
                off += part[0].numel()
            if N < f.cap:
                f.n[N:].zero_()                  # padding events: no sites, no ring
            f.graph.replay()
            d["rings"] = f.ring_views(N)
            d.update(f.out)                       # outputs and scratch of the bucket
            a.ready = self._event()
            a.ready.record(s)
        return a

    # -- one batched sweep ----------------------------------------------------
    def _sweep(self, batch: list[_Active]):
        n = len(batch)
        stream = self.sweep_streams[self._ss]
        self._ss = (self._ss + 1) % len(self.sweep_streams)
        rings = (api.cc_rings * n)(*[api._rings_struct(a.dev["rings"]) for a in batch])
        P = C.c_void_p
        maps = (P * n)(*[a.dev["map"].data_ptr() for a in batch])
        am = (P * n)(*[a.dev["argmax"].data_ptr() for a in batch])
        sd = (P * n)(*[a.dev["seeds"].data_ptr() for a in batch])
        st = (P * n)(*[a.dev["status"].data_ptr() for a in batch])
        ws = (P * n)(*[a.dev["ws"].data_ptr() for a in batch])
        wsb = (C.c_size_t * n)(*[a.dev["ws"].numel() for a in batch])
        for a in batch:
            stream.wait_event(a.ready)
        pc = self.params.c()
        api._check("cc_localize_batch", api.lib().cc_localize_batch(
            n, rings, C.byref(self._gs), C.byref(pc), maps, am, sd, st, ws, wsb,
            C.c_void_p(stream.cuda_stream)))
        swept = self._event()
        swept.record(stream)
        t_issue = time.perf_counter()
        for a in batch:                       # refine + read-back on the burst's stream
            s = a.stream
            s.wait_event(swept)
            d = a.dev
            with torch.cuda.stream(s):
                seeds_dir = api.grid_gather(self.grid, d["seeds"], out=d.get("seed_dirs"), stream=s)
                res = api.refine(d["rings"], seeds_dir, self.params, workspace=d.get("ref_ws"),
                                 out=d.get("ref"), stream=s)
                a.out_host = {"dir": res[0].to("cpu", non_blocking=True),
                              "obj": res[1].to("cpu", non_blocking=True),
                              "status": torch.cat([d["status"], res[3]]).to("cpu", non_blocking=True),
                              "argmax": d["argmax"].to("cpu", non_blocking=True)}
                if self.keep_maps:
                    a.out_host["map"] = d["map"].to("cpu", non_blocking=True)
                a.done = self._event()
                a.done.record(s)
            a.swept = True
            a.swept_ev = swept
            a.t_sweep = t_issue

    # -- the loop -------------------------------------------------------------
    def run(self, bursts: list[Burst], realtime: bool = True, keep_maps: bool = False,
            breakdown: bool = False):
        """Serve the bursts; returns per-burst results and latencies (s).
        With realtime, bursts become available at their arrival times;
        otherwise all are available at once (arrivals then only order them).
        With breakdown, each result also carries where its latency went:
        host admission delay, device front end, wait + batched sweep, refine +
        read-back (CUDA events), and the host's delay in seeing it done."""
        self.keep_maps = keep_maps
        self.breakdown = breakdown
        pending = deque(sorted(bursts, key=lambda b: b.arrival))
        active: list[_Active] = []
        used = 0
        results = {}
        batches = []
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            progressed = False
            # admit
            while pending and (not realtime or pending[0].arrival <= now) and \
                    len(active) < self.max_active:
                need = burst_bytes(pending[0].count, self.M, self.params, self.filter is not None)
                if used + need > self.budget and active:
                    break                                   # wait for memory to free up
                b = pending.popleft()
                active.append(self._admit(b, now))
                used += active[-1].bytes
                progressed = True
            # sweep every admitted burst not yet swept, in one batched launch;
            # the sweep stream waits for their front ends on the device, so
            # the host never waits for a burst's rings
            ready = [a for a in active if not a.swept]
            for i in range(0, len(ready), BATCH_MAX):
                self._sweep(ready[i:i + BATCH_MAX])
                batches.append(len(ready[i:i + BATCH_MAX]))
                progressed = True
            # complete
            still = []
            for a in active:
                if a.swept and a.done.query():
                    t = time.perf_counter() - t0
                    b = a.burst
                    arrival = b.arrival if realtime else 0.0
                    results[b.bid] = {"latency": t - arrival, "t_done": t,
                                      "dir": a.out_host["dir"].numpy(),
                                      "obj": float(a.out_host["obj"][0]),
                                      "status": a.out_host["status"].numpy(),
                                      "argmax": int(a.out_host["argmax"][0]),
                                      "rings": b.count}
                    if keep_maps:
                        results[b.bid]["map"] = a.out_host["map"].numpy()
                    if breakdown:
                        results[b.bid]["breakdown_ms"] = {
                            "admit_delay": 1e3 * (a.t_admit - arrival),
                            "front": a.ev0.elapsed_time(a.ready),
                            "to_swept": a.ready.elapsed_time(a.swept_ev),
                            "back": a.swept_ev.elapsed_time(a.done),
                            "issue_after_admit": 1e3 * (a.t_sweep - t0 - a.t_admit)}
                    if a.front is not None:      # its buffers are free again
                        self._fronts[a.front.cap].append(a.front)
                    used -= a.bytes
                    progressed = True
                else:
                    still.append(a)
            active = still
            if not progressed:
                if realtime and pending and not active:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.002)))
                else:
                    time.sleep(20e-6)
        wall = time.perf_counter() - t0
        return results, {"wall_s": wall, "batches": batches}


def pin_pools(pools):
    """The serving pools as pinned host tensors."""
    conv = lambda ev: {k: torch.from_numpy(np.ascontiguousarray(ev[k])).pin_memory()
                       for k in ("n", "x", "y", "z", "e")}
    return {"src": [conv(p) for p in pools["src"]], "bkg": conv(pools["bkg"])}


def to_bursts(pinned, specs) -> list[Burst]:
    """Bursts from synth.serving_bursts specs over pinned pools: two parts
    each (the source slice and the background slice), no copies on the host."""
    out = []
    for i, sp in enumerate(specs):
        parts = []
        for pool, (a, n) in ((pinned["src"][sp["dir"]], sp["src"]), (pinned["bkg"], sp["bkg"])):
            if n > 0:
                parts.append((pool["n"][a:a + n],) +
                             tuple(pool[k][:, a:a + n] for k in ("x", "y", "z", "e")))
        out.append(Burst(i, sp["arrival"], parts, source=sp["source"]))
    return out


def make_bursts(n_bursts: int, rate_hz: float, seed: int, **kw) -> list[Burst]:
    """Bursts of the serving workload (synth.serving_bursts)."""
    from . import synth
    pools, specs = synth.serving_bursts(n_bursts, rate_hz, seed, **kw)
    return to_bursts(pin_pools(pools), specs)
