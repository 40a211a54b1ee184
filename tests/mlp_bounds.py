"""Element-wise error bounds of the GPU's ring-filter network against the
oracle (oracle/mlp.py with BF16 rounding points), derived from the
arithmetic.

The GPU and the oracle see the same BF16 inputs and weights.  They differ in
two ways:
  * accumulation: the GPU sums K products (each exact in FP32: BF16 x BF16)
    in FP32; any order of n additions errs by at most gamma_n sum |terms|,
    gamma_n = n u / (1 - n u), with u = 2^-23 (one FP32 ulp per addition, so
    that adders that truncate are covered too);
  * rounding to BF16 at the same points (hidden activations, backward
    signals): where the FP32 value lies within its bound of a BF16 rounding
    boundary, the two may round apart by one BF16 ulp.  The bound of a
    rounded value is the widest BF16 step over the interval its input can
    take; it is propagated into every later product (|W| times the
    operand's bound), and a ReLU gate whose input can change sign there
    passes up to the whole value.
Every bound is per element; the tests compare every element against it.
"""
import numpy as np

from oracle import mlp

U = 2.0 ** -23


def gamma(n):
    return n * U / (1.0 - n * U)


def bf16_step(x, dx):
    """Largest |bf16(x') - bf16(x)| over |x' - x| <= dx (bf16 is monotone)."""
    a = mlp.bf16(x)
    return np.maximum(mlp.bf16(x + dx) - a, a - mlp.bf16(x - dx))


def relu_bf16_step(z, dz):
    a = mlp.bf16(np.maximum(z, 0.0))
    return np.maximum(mlp.bf16(np.maximum(z + dz, 0.0)) - a,
                      a - mlp.bf16(np.maximum(z - dz, 0.0)))


def forward_bounds(p, X):
    """(want, bound, hidden activations, their bounds, output bound) of the
    forward pass: want = the oracle's outputs; bound = element-wise bound on
    |GPU - oracle|.  Each layer is K products plus the FP32 bias, which the
    GPU folds into the accumulator as three BF16 pieces (a K = 16 product:
    n = K + 16 accumulations, and 2^-23 |b| for the pieces' own rounding)."""
    out, A, P = mlp.forward(p, X, round_points=True)
    layers = mlp.unpack(np.asarray(p, np.float64))
    dA = [np.zeros_like(A[0])]
    dz = None
    for li, (W, b) in enumerate(layers):
        Wr = np.abs(mlp.bf16(W))
        terms = np.abs(A[li]) @ Wr.T + np.abs(b)
        dz = gamma(W.shape[1] + 16) * terms + dA[li] @ Wr.T + U * np.abs(b)
        if li < 3:
            dA.append(relu_bf16_step(P[li], dz))
    return out, dz, A, dA


def bw_accumulations(rows, sms):
    """Additions behind one weight or bias gradient in the GPU's backward
    pass on `sms` SMs: each CTA sums its own rows (tpc 128-row tiles, the
    tiles spread over at most min(sms, 256) CTAs), then the CTAs' partials
    are summed in order.  With sms = 1 it bounds a plain sequential sum."""
    tiles = max(1, -(-rows // 128))
    cap = max(1, min(sms, 256))
    tpc = -(-tiles // cap)
    ncta = -(-tiles // tpc)
    return tpc * 128 + ncta


def grad_bounds(p, X, y, res, w, sms=1):
    """(want_grad, bound) for the flat gradient: the GPU's backward pass from
    its own forward outputs (bounded by forward_bounds), through
      d_out = w (sigmoid(z) - y) / B, w y (1 - r^2 e^{-2v}) / B in FP32
      (sigmoid' <= 1/4; expf within 2 ulp; 10 roundings of the largest
      magnitude involved, generously),
      dP = bf16(d_out), then per layer dW = dP^T A and db = column sums of
      dP (per CTA over its rows, then over the CTAs: bw_accumulations), and
      dP_prev = bf16(relu gate of (dP W)) (n = K).
    """
    B = X.shape[0]
    _, want = mlp.loss_and_grad(p, X, y, res, w, round_points=True)
    out, dz_out, A, dA = forward_bounds(p, X)
    z, v = out[:, 0], out[:, 1]
    dzz, dvv = dz_out[:, 0], dz_out[:, 1]
    sig = 1.0 / (1.0 + np.exp(-z))
    d0 = w * (sig - y) / B
    e2v = np.exp(-2.0 * v)
    d1 = w * y * (1.0 - res * res * e2v) / B
    dd0 = w * (0.25 * dzz + 10 * U * (sig + np.abs(sig - y))) / B
    dd1 = w * y * (2.0 * res * res * np.exp(-2.0 * (v - dvv)) * dvv
                   + 10 * U * (1.0 + res * res * np.exp(-2.0 * (v - dvv)))) / B
    d_out = np.stack([d0, d1], 1)
    dP = mlp.bf16(d_out)
    ddP = bf16_step(d_out, np.stack([dd0, dd1], 1))
    layers = mlp.unpack(np.asarray(p, np.float64))
    n_w = n_b = bw_accumulations(B, sms)
    gb = [None] * 4
    for li in range(3, -1, -1):
        W, _ = layers[li]
        gW = gamma(n_w) * (np.abs(dP).T @ np.abs(A[li])) + ddP.T @ np.abs(A[li]) \
            + np.abs(dP).T @ dA[li] + ddP.T @ dA[li]
        gbias = gamma(n_b) * np.abs(dP).sum(0) + ddP.sum(0)
        gb[li] = (gW, gbias)
        if li > 0:
            Wr = mlp.bf16(W)
            dAv = dP @ Wr
            ddA = gamma(W.shape[0]) * (np.abs(dP) @ np.abs(Wr)) + ddP @ np.abs(Wr)
            gate = A[li] > 0
            unsure = (gate & (A[li] - dA[li] <= 0)) | (~gate & (dA[li] > 0))
            masked = np.where(gate, dAv, 0.0)
            dmask = np.where(unsure, np.abs(dAv) + ddA, np.where(gate, ddA, 0.0))
            dP = mlp.bf16(masked)
            ddP = bf16_step(masked, dmask)
    return want, mlp.pack(gb)


# --------------------------------------------------------------------------
# Stage by stage: each stage of the GPU's step checked on the GPU's own
# inputs to it (its activations and backward signals, kept by
# cc_mlp_grad_trace), so that no error is inherited from an earlier stage.
# Every element must lie in the interval the stage's own arithmetic allows:
# BF16 outputs within [bf16(v - d), bf16(v + d)] (one rounding apart at
# most, and only where v lies within d of a rounding boundary), FP32 outputs
# within d, with v the stage in FP64 and d its FP32 accumulation bound.
# --------------------------------------------------------------------------
def in_bf16_interval(got, v, d, relu=False):
    f = (lambda t: np.maximum(t, 0.0)) if relu else (lambda t: t)
    lo, hi = mlp.bf16(f(v - d)), mlp.bf16(f(v + d))
    return (got >= lo) & (got <= hi), lo != hi


def check_layer(a_in, W, b, got, relu):
    """One forward layer: got = bf16(relu(a_in W^T + b)) (hidden) or
    a_in W^T + b in FP32 (output).  Returns (ok mask, ambiguous mask)."""
    Wr = mlp.bf16(W)
    v = a_in @ Wr.T + b
    d = gamma(W.shape[1] + 16) * (np.abs(a_in) @ np.abs(Wr).T + np.abs(b)) + U * np.abs(b)
    if relu:
        return in_bf16_interval(got, v, d, relu=True)
    return np.abs(got - v) <= d, np.zeros(got.shape, bool)


def check_dout(out, y, res, w, got):
    """d(loss)/d(out) from the GPU's outputs, in FP32 then BF16."""
    B = out.shape[0]
    z, v = out[:, 0], out[:, 1]
    sig = 1.0 / (1.0 + np.exp(-z))
    e2v = np.exp(-2.0 * v)
    d0 = w * (sig - y) / B
    d1 = w * y * (1.0 - res * res * e2v) / B
    dd0 = w * 10 * U * (sig + np.abs(sig - y)) / B
    dd1 = w * y * 10 * U * (1.0 + res * res * e2v) / B
    return in_bf16_interval(got, np.stack([d0, d1], 1), np.stack([dd0, dd1], 1))


def check_signal(sig_in, W, gate, got):
    """One backward step: got = bf16((sig_in W) where gate > 0), K = sig_in's
    width."""
    Wr = mlp.bf16(W)
    v = np.where(gate > 0, sig_in @ Wr, 0.0)
    d = np.where(gate > 0, gamma(W.shape[0]) * (np.abs(sig_in) @ np.abs(Wr)), 0.0)
    return in_bf16_interval(got, v, d)


def check_weight_grad(sig, a_in, gW, gb, sms=1):
    """dW = sig^T a_in over the rows and db = column sums of sig, each summed
    per CTA then over the CTAs."""
    B = sig.shape[0]
    n_w = n_b = bw_accumulations(B, sms)
    vW = sig.T @ a_in
    dW = gamma(n_w) * (np.abs(sig).T @ np.abs(a_in))
    vb = sig.sum(0)
    db = gamma(n_b) * np.abs(sig).sum(0)
    return (np.abs(gW - vW) <= dW), (np.abs(gb - vb) <= db)
