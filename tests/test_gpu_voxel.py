"""GPU near-field back projection (Sec. 3) against the oracle: ring apexes
and universes bit for bit, images within the parity rule plus the FP32 bound
of the per-pair apex difference."""
import math

import numpy as np
import pytest

import oracle
from paper_2411_04785_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def cc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_04785_gb300 as m
    m.lib()
    return m


def dev(a, dt=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dt)).to(DEV)


def near_rings(rng, R, S, frac_src=0.3, deta_deg=(0.5, 10.0)):
    """Synthetic near-field cones: apexes in the detector slab, a share of
    them through the point S (eta exact), the rest random; widths
    log-uniform."""
    p = np.column_stack([rng.uniform(-25, 25, R), rng.uniform(-25, 25, R), rng.uniform(-31, 1, R)])
    a = rng.standard_normal((R, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    d = S[None, :] - p
    eta = np.arccos(np.clip(np.sum(d * a, 1) / np.linalg.norm(d, axis=1), -1, 1))
    bkg = rng.uniform(size=R) > frac_src
    eta[bkg] = np.arccos(rng.uniform(-1, 1, bkg.sum()))
    lo, hi = np.log(np.radians(deta_deg))
    deta = np.exp(rng.uniform(lo, hi, R))
    rings = {k: v.astype(np.float32) for k, v in
             (("ax", a[:, 0]), ("ay", a[:, 1]), ("az", a[:, 2]), ("eta", eta), ("deta", deta))}
    rings["valid"] = np.ones(R, np.uint8)
    return rings, p.astype(np.float32)


def rings_dev(r):
    out = {k: dev(r[k]) for k in ("ax", "ay", "az", "eta", "deta")}
    out["valid"] = dev(r["valid"], np.uint8)
    return out


def fp32_bound(rings, apex, vox, idx):
    """Per voxel, the sum over rings of |d term / d theta| times the FP32
    error of theta: the rounding of d = v - p (2^-24 |v|, |p| per component,
    turned by 1/|d| into an angle) plus the far-field pair's own (3e-7 rad)."""
    a = np.stack([rings["ax"], rings["ay"], rings["az"]], 1).astype(np.float64)
    p = apex.astype(np.float64)
    out = np.zeros(idx.size)
    for q, j in enumerate(idx):
        v = np.array([vox[0][j], vox[1][j], vox[2][j]], np.float64)
        d = v[None, :] - p
        nd = np.linalg.norm(d, axis=1)
        th = np.arctan2(np.linalg.norm(np.cross(d, a), axis=1), np.sum(d * a, 1))
        r = (th - rings["eta"]) / rings["deta"]
        dth = 2.0 ** -23 * (np.abs(v).max() + np.abs(p).max(1)) / nd + 3e-7
        out[q] = np.sum(np.abs(r) / rings["deta"] * np.exp(-0.5 * r * r) * dth)
    return out


def check_image(img, want, bound):
    tol = 1e-5 * np.maximum(want, 1e-3 * want.max()) + bound
    bad = np.abs(img - want) > tol
    assert not bad.any(), (np.flatnonzero(bad)[:5], img[bad][:5], want[bad][:5])


@pytest.mark.parametrize("shape", ["cube", "cylinder", "sphere"])
def test_universe_bit_exact(cc, shape):
    for n, pitch, c in ((1, 1.0, (0, 0, 0)), (7, 0.37, (1.5, -2.25, 20.0)), (64, 0.3125, (0, 0, 20.0))):
        got = cc.voxel_universe(shape, n, pitch, c)
        torch.cuda.synchronize()
        want = oracle.universe(shape, n, np.float32(pitch), center=tuple(np.float32(v) for v in c))
        for g, w in zip(got, want):
            np.testing.assert_array_equal(g.cpu().numpy(), w.astype(np.float32))


def test_ring_apex_bit_exact(cc):
    ev = synth.simulate_events(n_src=3000, n_bkg=6000, seed=31)
    p = cc.Params()
    n = dev(ev["n"], np.uint8)
    x, y, z, e = (dev(ev[k]) for k in "xyze")
    rings = cc.rings_from_events(n, x, y, z, e, p)
    apex = cc.ring_apex(n, x, y, z, rings)
    torch.cuda.synchronize()
    r_or = oracle.rings_from_events(ev, p.sigma_e_frac, p.sigma_pos_cm, p.deta_min, p.deta_max)
    want = oracle.ring_apex({k: ev[k] for k in ("n", "x", "y", "z")}, r_or).astype(np.float32)
    got = np.stack([t.cpu().numpy() for t in apex], 1)
    # the ordering is bit-exact, so every apex is the oracle's, bit for bit
    np.testing.assert_array_equal(rings["valid"].cpu().numpy(), r_or["valid"])
    np.testing.assert_array_equal(rings["perm"].cpu().numpy(), r_or["perm"])
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("shape,R,kcut", [("cube", 3000, 0.0), ("sphere", 20000, 0.0),
                                          ("cylinder", 129, 0.0), ("cube", 7000, 5.0)])
def test_image_matches_oracle(cc, shape, R, kcut):
    rng = np.random.default_rng(R)
    S = np.array([1.3, -0.7, 20.2])
    rings, apex = near_rings(rng, R, S)
    vox = cc.voxel_universe(shape, 24, 0.8, (0.0, 0.0, 20.0))
    vnp = tuple(v.astype(np.float32) for v in oracle.universe(shape, 24, 0.8, (0.0, 0.0, 20.0)))
    p = cc.Params(k_cut=kcut)
    img, am, st = cc.backproject(rings_dev(rings), tuple(dev(apex[:, c]) for c in range(3)), vox, p)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    img = img.cpu().numpy()
    idx = np.arange(0, img.size, 3)
    if kcut == 0:
        want = oracle.backproject(rings, apex, vnp, idx=idx)
        check_image(img[idx], want, fp32_bound(rings, apex, vnp, idx))
    else:   # terms at |r| near the cut may fall on either side: bracket them
        lo = oracle.backproject(rings, apex, vnp, idx=idx, k_cut=kcut * (1 - 1e-4))
        hi = oracle.backproject(rings, apex, vnp, idx=idx, k_cut=kcut * (1 + 1e-4))
        b = fp32_bound(rings, apex, vnp, idx) + 1e-5 * np.maximum(hi, 1e-3 * hi.max())
        assert ((img[idx] >= lo - b) & (img[idx] <= hi + b)).all()
    j = int(am.item())                      # the argmax is the image's first maximum
    assert img[j] == img.max() and (img[:j] < img[j]).all()


def test_voxels_in_any_order_give_the_same_image(cc):
    """The sweep takes the voxels in their Morton order, found from the
    coordinates, so a shuffled voxel list (positions all distinct) gives the
    same image, permuted, bit for bit; and it satisfies the parity rule."""
    rng = np.random.default_rng(31)
    S = np.array([1.3, -0.7, 20.2])
    rings, apex = near_rings(rng, 3000, S, deta_deg=(0.5, 20.0))
    vnp = tuple(v.astype(np.float32) for v in oracle.universe("sphere", 24, 0.8, (0.0, 0.0, 20.0)))
    V = vnp[0].size
    sh = rng.permutation(V)
    rd = rings_dev(rings)
    ap = tuple(dev(apex[:, c]) for c in range(3))
    img, am, st = cc.backproject(rd, ap, tuple(dev(v) for v in vnp))
    img_s, am_s, st_s = cc.backproject(rd, ap, tuple(dev(v[sh]) for v in vnp))
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(st_s.item()) == 0
    img, img_s = img.cpu().numpy(), img_s.cpu().numpy()
    np.testing.assert_array_equal(img_s, img[sh])
    j = int(am_s.item())                    # the first maximum of the shuffled list
    assert img_s[j] == img_s.max() and (img_s[:j] < img_s[j]).all()
    idx = np.arange(0, V, 5)
    want = oracle.backproject(rings, apex, vnp, idx=idx)
    check_image(img[idx], want, fp32_bound(rings, apex, vnp, idx))


def test_planted_source_voxel_and_invalid_rings(cc):
    rng = np.random.default_rng(4)
    n, pitch = 32, 0.5
    vox = cc.voxel_universe("cube", n, pitch, (0.0, 0.0, 20.0))
    vnp = oracle.universe("cube", n, pitch, (0.0, 0.0, 20.0))
    j_src = 12345
    S = np.array([vnp[0][j_src], vnp[1][j_src], vnp[2][j_src]], np.float64)
    rings, apex = near_rings(rng, 5000, S, frac_src=1.0, deta_deg=(1.0, 1.0))
    rings["valid"][::7] = 0
    rings["deta"][3::11] = np.nan                  # dropped as non-finite
    img, am, st = cc.backproject(rings_dev(rings), tuple(dev(apex[:, c]) for c in range(3)), vox)
    torch.cuda.synchronize()
    kept = (rings["valid"] == 1) & np.isfinite(rings["deta"])
    assert int(am.item()) == j_src
    assert abs(float(img[j_src].item()) - kept.sum()) < kept.sum() * 2e-5


def test_far_field_limit_matches_the_sky_sweep(cc):
    """Every apex at one point P: the image along rays from P is the far-field
    map; voxels placed at P + 1000 c_j reproduce the sky map of the same rings
    within FP32 rounding."""
    rings_np, s, _ = synth.rings_burst(n=4000, seed=8)
    rings = {k: np.asarray(rings_np[k], np.float32) for k in ("ax", "ay", "az", "eta", "deta")}
    rings["valid"] = np.ones(4000, np.uint8)
    g = oracle.grid_fibonacci(3072)
    P = np.array([0.25, -0.5, 0.125])
    vox_np = tuple((P[c] + 1000.0 * g[c]).astype(np.float32) for c in range(3))
    apex = np.tile(P.astype(np.float32), (4000, 1))
    img, _, _ = cc.backproject(rings_dev(rings), tuple(dev(apex[:, c]) for c in range(3)),
                               tuple(dev(v) for v in vox_np))
    torch.cuda.synchronize()
    idx = np.arange(0, 3072, 5)
    want = oracle.backproject(rings, apex, vox_np, idx=idx)
    check_image(img.cpu().numpy()[idx], want, fp32_bound(rings, apex, vox_np, idx))
