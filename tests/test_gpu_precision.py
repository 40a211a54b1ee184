"""The error of every GPU output against the FP64 oracle, measured on one
workload per stage and checked against the stage's parity rule.  With
CC_PRECISION_REPORT=<file> the measured errors are also written there as JSON
(the table of measured errors is made from that file)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2411_04785_gb300 import synth
from tests.helpers import EPS32, MAP_FLOOR, MAP_RTOL, REFINE_TOL_DEG, ang_deg, eta_tol, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_04785_gb300 as m
    m.lib()
    return m


def rel_floor(got, want):
    """max |got - want| / max(want, 1e-3 max want): the map rule's measure."""
    return float((np.abs(got - want) / np.maximum(want, MAP_FLOOR * want.max())).max())


def test_error_of_every_output(cc):
    dev = torch.device("cuda:0")
    out = {}
    p = cc.Params()

    # reconstruction: 60k events (k = 2/3/4), all rings
    ev = synth.simulate_events(n_src=20000, n_bkg=40000, seed=41)
    n = to_dev(ev["n"], dev)
    x, y, z, e = (to_dev(np.asarray(ev[k], np.float32), dev) for k in "xyze")
    r = cc.rings_from_events(n, x, y, z, e, p)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in r.items()}
    w = oracle.rings_from_events(ev, p.sigma_e_frac, p.sigma_pos_cm, p.deta_min, p.deta_max)
    v = w["valid"] == 1
    same = (g["valid"] == w["valid"]) & ((g["perm"] == w["perm"]) | ~v)
    out["site_order_and_validity_identical"] = float(same.mean())
    out["axis_max_abs"] = float(max(np.abs(g[k][v] - w[k][v]).max() for k in ("ax", "ay", "az")))
    eta_err = np.abs(g["eta"][v] - w["eta"][v])
    out["eta_max_abs_rad"] = float(eta_err.max())
    out["eta_max_over_bound"] = float(
        (eta_err / eta_tol(1.0 - np.cos(w["eta"][v]), w["eta"][v])).max())
    out["deta_max_rel"] = float((np.abs(g["deta"][v] - w["deta"][v]) / w["deta"][v]).max())
    assert out["site_order_and_validity_identical"] == 1.0
    assert out["axis_max_abs"] <= 8 * EPS32
    assert out["eta_max_over_bound"] <= 1.0
    assert out["deta_max_rel"] <= 2e-5

    # map, argmax and refinement from the oracle's rings rounded to FP32
    r32 = {k: w[k].astype(np.float32) for k in ("ax", "ay", "az", "eta", "deta")}
    r32["valid"] = w["valid"]
    grid = tuple(a.astype(np.float32) for a in oracle.grid_healpix_ring(32))
    rd = {k: to_dev(r32[k], dev) for k in r32}
    loc = cc.Localizer(tuple(to_dev(a, dev) for a in grid), p)
    loc.from_rings(rd)
    torch.cuda.synchronize()
    want = oracle.likelihood_map(r32, grid)
    out["map_max_rel_floor"] = rel_floor(loc.map.cpu().numpy(), want)
    jo = oracle.argmax(want)
    out["argmax_equal"] = int(loc.argmax.item()) == jo
    od, _, _, _ = oracle.refine(r32, [grid[0][jo], grid[1][jo], grid[2][jo]], tol_rad=1e-10)
    out["refined_direction_deg"] = ang_deg(loc.dir.cpu().numpy(), od)
    assert out["map_max_rel_floor"] <= MAP_RTOL
    assert out["argmax_equal"]
    assert out["refined_direction_deg"] <= REFINE_TOL_DEG

    # learned filter: features and the MLP forward
    F = cc.ring_features(n, x, y, z, e, r, p)
    torch.cuda.synchronize()
    fw = mlp.features(ev, w, p.sigma_pos_cm)
    fg = F.float().cpu().numpy().astype(np.float64)
    ok = np.abs(fg - fw) <= 2.0 ** -7 * np.abs(fw) + 1e-5
    out["features_outside_one_bf16_ulp"] = float(1.0 - ok.mean())
    pm = mlp.init_params(3)
    pm[-2:] = [0.2, -1.0]
    X = mlp.bf16(np.random.default_rng(3).standard_normal((70_001, 16)))
    f = cc.RingFilter(dev, params=pm)
    o = f.forward(to_dev(X.astype(np.float32), dev).to(torch.bfloat16).contiguous())
    torch.cuda.synchronize()
    wo, _, _ = mlp.forward(pm, X, round_points=True)
    out["mlp_forward_rel_norm"] = float(np.linalg.norm(o.cpu().numpy() - wo) / np.linalg.norm(wo))
    assert out["features_outside_one_bf16_ulp"] < 1e-4
    assert out["mlp_forward_rel_norm"] < 2.0 ** -9

    # clustering: integer, bit-exact
    t0, a0, _ = synth.detection_stream(n_events=20000, seed=5)
    oc = cc.cluster_maxstep(to_dev(t0, dev), to_dev(a0, dev), 15000)
    torch.cuda.synchronize()
    wc = oracle.maxstep_events(t0, a0, 15000)
    K = int(oc["n_events"].item())
    out["cluster_bit_exact"] = bool(
        K == wc["count"].size
        and np.array_equal(oc["event_id"].cpu().numpy(), wc["event_id"])
        and np.array_equal(oc["first"][:K].cpu().numpy(), wc["first"])
        and np.array_equal(oc["count"][:K].cpu().numpy(), wc["count"])
        and np.array_equal(oc["adc"][:K].cpu().numpy().astype(np.uint64), wc["adc"]))
    assert out["cluster_bit_exact"]

    # near field: apexes and the image over a 16^3-inscribed sphere
    ap_g = cc.ring_apex(n, x, y, z, r)
    torch.cuda.synchronize()
    ap_w = oracle.ring_apex({k: ev[k] for k in ("n", "x", "y", "z")}, w)
    out["apex_bit_exact"] = bool(all(np.array_equal(ap_g[c].cpu().numpy()[v],
                                                    ap_w[v, c].astype(np.float32))
                                     for c in range(3)))
    vox = tuple(a.astype(np.float32) for a in oracle.universe("sphere", 16, 1.0, (0.0, 0.0, 20.0)))
    ap32 = ap_w.astype(np.float32)
    img, _, _ = cc.backproject(rd, tuple(to_dev(np.ascontiguousarray(ap32[:, c]), dev)
                                         for c in range(3)),
                               tuple(to_dev(a, dev) for a in vox), p)
    torch.cuda.synchronize()
    out["image_max_rel_floor"] = rel_floor(img.cpu().numpy(), oracle.backproject(r32, ap32, vox))
    assert out["apex_bit_exact"]
    assert out["image_max_rel_floor"] <= MAP_RTOL

    path = os.environ.get("CC_PRECISION_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump(out, fh, indent=1)
    print(json.dumps(out))
