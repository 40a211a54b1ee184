"""Oracle of the learned ring filter: ring features, the MLP
16 -> 128 -> 128 -> 128 -> 2 (ReLU), its loss and its gradients, in numpy FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The GPU keeps weights,
inputs and activations in BF16 and accumulates in FP32; ``round_points=True``
rounds to BF16 at exactly the points where the GPU does, so that the two can be
compared to FP32-accumulation accuracy.  ``round_points=False`` is the plain
FP64 network, pinned against finite differences.

Network (reading of the learned ring filter): out = (z, v) with z the
source/background logit and v = log of the predicted ring width.  Loss per
ring (mean over the batch, invalid rings weigh 0):
    BCE(z, y) + y (v + r^2 exp(-2 v) / 2)
with y = 1 for a source ring and r its angular residual to the true source
(the Gaussian negative log-likelihood of the residual for width exp(v)).

Parameter layout (flat FP32, 35,458 values): W1[128,16] b1[128] W2[128,128]
b2[128] W3[128,128] b3[128] W4[2,128] b4[2].
"""
from __future__ import annotations

import math

import numpy as np

import oracle

SIZES = [(128, 16), (128, 128), (128, 128), (2, 128)]
N_FEATURES = 16
N_PARAMS = sum(o * i + o for o, i in SIZES)


def unpack(p):
    out, off = [], 0
    for o, i in SIZES:
        W = p[off:off + o * i].reshape(o, i)
        off += o * i
        b = p[off:off + o]
        off += o
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases, float32."""
    rng = np.random.default_rng(seed)
    layers = []
    for o, i in SIZES:
        lim = math.sqrt(6.0 / i)
        layers.append((rng.uniform(-lim, lim, (o, i)), np.zeros(o)))
    return pack(layers).astype(np.float32)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    r = np.where(np.isnan(a), u.astype(np.uint32) | 0x400000, r)
    return r.view(np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# features
# --------------------------------------------------------------------------
def features(ev, rings, sigma_pos_cm=1.0):
    """16 features per ring from its event and its (oracle) ring:
    eta/pi, cos eta, sin eta, log(deta)/4, [k=2], [k=3], [k=4],
    log(E0/500 keV), E1/E0, E_2nd/E0, E_last/E0, log(|x1-x2|/5 cm), a_z,
    z1/30 cm, z2/30 cm, deta_G/deta (the share of the width from positions).
    Invalid rings get zeros."""
    import itertools
    n = ev["n"].astype(np.int64)
    N = n.size
    perms = {k: list(itertools.permutations(range(k))) for k in (2, 3, 4)}
    x, y, z, e = (np.asarray(ev[c], np.float64) for c in "xyze")
    F = np.zeros((N, N_FEATURES))
    for i in range(N):
        if not rings["valid"][i]:
            continue
        k = int(n[i])
        o = perms[k][rings["perm"][i]]
        f, s, l = o[0], o[1], o[-1]
        e0 = sum(e[j, i] for j in range(k))
        d = np.array([x[f, i] - x[s, i], y[f, i] - y[s, i], z[f, i] - z[s, i]])
        L = math.sqrt(d @ d)
        eta, deta = rings["eta"][i], rings["deta"][i]
        F[i] = [eta / math.pi, math.cos(eta), math.sin(eta), math.log(deta) / 4.0,
                k == 2, k == 3, k == 4, math.log(e0 / 500.0), e[f, i] / e0,
                e[s, i] / e0, e[l, i] / e0, math.log(L / 5.0), rings["az"][i],
                z[f, i] / 30.0, z[s, i] / 30.0,
                math.sqrt(2.0) * sigma_pos_cm / L / deta]
    return F


# --------------------------------------------------------------------------
# network
# --------------------------------------------------------------------------
def forward(p, X, round_points=True):
    """Returns (out [B,2], activations) with activations = [A0, H1, H2, H3]
    (inputs of each layer) and pre-activations [P1, P2, P3]."""
    r = bf16 if round_points else (lambda a: np.asarray(a, np.float64))
    L = unpack(np.asarray(p, np.float64))
    A = [r(X)]
    P = []
    for li, (W, b) in enumerate(L):
        z = A[-1] @ r(W).T + b
        if li < 3:
            P.append(z)
            A.append(r(np.maximum(z, 0.0)))
        else:
            out = z
    return out, A, P


def loss(out, y, res, w):
    z, v = out[:, 0], out[:, 1]
    bce = np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))
    nll = y * (v + 0.5 * res * res * np.exp(-2.0 * v))
    return float(np.sum(w * (bce + nll)) / len(z))


def loss_and_grad(p, X, y, res, w, round_points=True):
    """Loss and its gradient with respect to the flat parameters."""
    r = bf16 if round_points else (lambda a: np.asarray(a, np.float64))
    B = X.shape[0]
    out, A, P = forward(p, X, round_points)
    z, v = out[:, 0], out[:, 1]
    sig = 1.0 / (1.0 + np.exp(-z))
    d_out = np.zeros_like(out)
    d_out[:, 0] = w * (sig - y) / B
    d_out[:, 1] = w * y * (1.0 - res * res * np.exp(-2.0 * v)) / B
    L = unpack(np.asarray(p, np.float64))
    grads = [None] * 4
    dP = r(d_out)
    for li in range(3, -1, -1):
        W, _ = L[li]
        grads[li] = (dP.T @ A[li], dP.sum(0))
        if li > 0:
            dA = dP @ r(W)
            dP = r(np.where(A[li] > 0, dA, 0.0))     # ReLU gate: the layer's input > 0
    return loss(out, y, res, w), pack(grads)


def apply_filter(out, valid, deta, tau, deta_min, deta_max):
    """Rings kept when sigma(z) >= tau; their width becomes exp(v) clamped."""
    z, v = out[:, 0], out[:, 1]
    keep = (valid == 1) & (1.0 / (1.0 + np.exp(-z)) >= tau)
    return keep.astype(np.uint8), np.clip(np.exp(v), deta_min, deta_max)


def residuals(rings, source):
    a = np.stack([rings["ax"], rings["ay"], rings["az"]], 1).astype(np.float64)
    return np.array([oracle.angle(ai, source) for ai in a]) - rings["eta"]
