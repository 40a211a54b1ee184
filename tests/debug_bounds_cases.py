"""Small cases of every checked kernel, run in a child process by
tests/test_gpu_debug_bounds.py, once on the optimised library and once on the
debug build (CC_LIBRARY=debug): ragged and padded event windows, misaligned
arrays, split sweeps, the angular selection on a NESTED grid, the
refinement, the grids, the clustering, the near-field image and a training
step of the ring filter.  Writes every result to an .npz file and, on the
debug build, the bounds word (0: no checked index was out of bounds) and the
word the bounds self-test leaves.

    python tests/debug_bounds_cases.py OUT.npz
"""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_2411_04785_gb300 as cc  # noqa: E402
from paper_2411_04785_gb300 import api, synth  # noqa: E402


def main(path):
    dev = torch.device("cuda:0")
    res = {}
    debug = os.environ.get("CC_LIBRARY") == "debug"
    if debug:
        api.debug_bounds(reset=True)

    # reconstruction: several windows and a ragged last one, a padded stride,
    # then arrays 4 bytes off a 16-byte boundary (plain loads, scalar stores)
    ev = synth.tile_events(synth.simulate_events(n_src=3000, n_bkg=27000, seed=12), 3)
    N = ev["n"].size
    n = torch.from_numpy(ev["n"]).to(dev)
    xyz = [torch.from_numpy(np.ascontiguousarray(ev[k], np.float32)).to(dev) for k in "xyze"]
    p = cc.Params()
    rings = cc.rings_from_events(n, *xyz, p)
    pad = [torch.zeros((4, N + 37), dtype=torch.float32, device=dev) for _ in range(4)]
    for d, s in zip(pad, xyz):
        d[:, :N] = s
    r_pad = cc.rings_from_events(n, *pad, p)
    off = []
    for s in xyz:
        flat = torch.zeros(s.numel() + 1, dtype=torch.float32, device=dev)
        v = flat[1:].view(s.shape)
        v.copy_(s)
        off.append(v)
    r_off = cc.rings_from_events(n, *off, p)
    for k in ("valid", "perm", "eta", "deta"):
        res[f"rings_{k}"] = rings[k].cpu().numpy()
        res[f"rings_off_{k}"] = r_off[k].cpu().numpy()
        res[f"rings_pad_{k}"] = r_pad[k].cpu().numpy()

    # the sweep: ring splits over a small grid, seeds, the refinement
    grid = cc.grid_healpix_ring(16, dev)
    m, am, sd, st = cc.localize(rings, grid, cc.Params(topk=4, nms_rad=math.radians(5.0)))
    res["map"], res["argmax"], res["seeds"] = m.cpu().numpy(), am.cpu().numpy(), sd.cpu().numpy()
    seeds = cc.grid_gather(grid, sd)
    d, obj, it, rst = cc.refine(rings, seeds, cc.Params(topk=4))
    res["dir"] = d.cpu().numpy()
    # the angular selection on a NESTED grid (warps skip rings)
    burst, _, _ = synth.rings_burst(n=20000, seed=4)
    bd = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in burst.items()}
    nest = cc.grid_healpix_nest(32, dev)
    mk, _, _, _ = cc.localize(bd, nest, cc.Params(k_cut=3.0))
    res["map_kcut"] = mk.cpu().numpy()
    res["grid_fib"] = torch.stack(cc.grid_fibonacci(1001, dev)).cpu().numpy()
    res["grid_nest"] = torch.stack(nest).cpu().numpy()

    # clustering of a detection stream
    t0, a0, _ = synth.detection_stream(n_events=3000, seed=3)
    oc = cc.cluster_maxstep(torch.from_numpy(t0).to(dev), torch.from_numpy(a0).to(dev), 15000)
    res["cluster_id"] = oc["event_id"].cpu().numpy()
    res["cluster_adc"] = oc["adc"][:int(oc["n_events"].item())].cpu().numpy()

    # near-field image over a small sphere
    vox = cc.voxel_universe("sphere", 12, 1.0, (0.0, 0.0, 20.0), device=dev)
    apex = cc.ring_apex(n, *xyz[:3], rings)
    img, _, _ = cc.backproject(rings, apex, vox, p)
    res["image"] = img.cpu().numpy()

    # one training step of the ring filter (forward and backward on the tensor cores)
    from oracle import mlp
    rng = np.random.default_rng(2)
    X = torch.from_numpy(mlp.bf16(rng.standard_normal((777, 16))).astype(np.float32))
    f = cc.RingFilter(dev, params=mlp.init_params(2))
    _, g = f.grad(X.to(dev).to(torch.bfloat16).contiguous(),
                  torch.from_numpy((rng.uniform(size=777) < 0.3).astype(np.uint8)).to(dev),
                  torch.from_numpy(rng.standard_normal(777).astype(np.float32)).to(dev),
                  torch.ones(777, dtype=torch.uint8, device=dev))
    res["grad"] = g.cpu().numpy()
    torch.cuda.synchronize()

    if debug:
        res["word"] = np.array([api.debug_bounds(reset=True)], np.uint64)
        buf = torch.zeros(8, dtype=torch.int32, device=dev)
        api._check("cc_debug_selftest_bounds", api.lib().cc_debug_selftest_bounds(
            api._ptr(buf), 8, api._stream(None)))
        torch.cuda.synchronize()
        res["selftest_word"] = np.array([api.debug_bounds(reset=True)], np.uint64)
        res["selftest_buf"] = buf.cpu().numpy()
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
