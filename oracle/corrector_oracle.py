"""FP64 numpy oracle of the learned residual corrector (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use it.  It
shares no code with the CUDA library.

The corrector refines one coarse exponential step (Lawson4, eq. lawson4) of
the periodic CGL equation: u_{n+1} = C(u_n) + N(x), where x stacks 9 planes
(Re, Im of C(u_n); Re, Im of u_n; the parameters a1, b1, a2, a3, b3 as
constant planes) and N is a stack of 3x3 convolutions with circular padding
(the periodic boundary), ReLU between layers, 2 output planes (Re, Im of the
correction).  Weights are used in BF16 in the forward pass (rounded to
nearest even from FP32 masters) with FP32/FP64 accumulation; training
minimises the mean squared difference to the fine result with Adam.

Layouts: activations (B, C, H, W), W fastest; weights (Cout, Cin, 3, 3);
tap (di, dj) reads x[(i + di - 1) mod H, (j + dj - 1) mod W].
"""
from __future__ import annotations

import numpy as np

IN_CHANNELS = 9
OUT_CHANNELS = 2


def layer_shapes(hidden: int = 32, layers: int = 6):
    """(cin, cout, relu) per layer: 9 -> hidden, (layers-2) x hidden -> hidden, hidden -> 2."""
    shapes = [(IN_CHANNELS, hidden, True)]
    shapes += [(hidden, hidden, True)] * (layers - 2)
    shapes += [(hidden, OUT_CHANNELS, False)]
    return shapes


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float32: keep the top 16 bits of the binary32 pattern after adding
    0x7FFF + (bit 16 of the pattern)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    out = (rounded & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out)


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[b, o, i, j] = bias[o] + sum_{c, di, dj} w[o, c, di, dj] x[b, c, i+di-1, j+dj-1]
    with indices taken modulo H, W (circular padding)."""
    B, C, H, W = x.shape
    y = np.zeros((B, w.shape[0], H, W), dtype=np.float64)
    for di in range(3):
        for dj in range(3):
            xs = np.roll(x, shift=(1 - di, 1 - dj), axis=(2, 3))
            y += np.einsum("oc,bchw->bohw", w[:, :, di, dj].astype(np.float64), xs)
    return y + b.astype(np.float64)[None, :, None, None]


def conv3x3_adjoint(dy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 in x: dx[b, c, m, n] = sum_{o, di, dj} w[o, c, di, dj] dy[b, o, m-di+1, n-dj+1]."""
    B, O, H, W = dy.shape
    dx = np.zeros((B, w.shape[1], H, W), dtype=np.float64)
    for di in range(3):
        for dj in range(3):
            t = np.einsum("oc,bohw->bchw", w[:, :, di, dj].astype(np.float64), dy)
            dx += np.roll(t, shift=(di - 1, dj - 1), axis=(2, 3))
    return dx


def conv3x3_weight_grad(x: np.ndarray, dy: np.ndarray):
    """dw[o, c, di, dj] = sum_{b, i, j} dy[b, o, i, j] x[b, c, i+di-1, j+dj-1];  db[o] = sum dy[b, o]."""
    O, C = dy.shape[1], x.shape[1]
    dw = np.zeros((O, C, 3, 3))
    for di in range(3):
        for dj in range(3):
            xs = np.roll(x, shift=(1 - di, 1 - dj), axis=(2, 3))
            dw[:, :, di, dj] = np.einsum("bohw,bchw->oc", dy, xs)
    return dw, dy.sum(axis=(0, 2, 3))


def features(coarse: np.ndarray, un: np.ndarray, params: np.ndarray) -> np.ndarray:
    """x (B, 9, H, W) from complex coarse results and states (B, H, W) and
    parameters (B, 5) = (a1, b1, a2, a3, b3)."""
    B, H, W = coarse.shape
    x = np.empty((B, IN_CHANNELS, H, W))
    x[:, 0], x[:, 1] = coarse.real, coarse.imag
    x[:, 2], x[:, 3] = un.real, un.imag
    x[:, 4:9] = np.asarray(params, dtype=np.float64)[:, :, None, None]
    return x


def forward(weights, x, round_weights=True, round_acts=False):
    """weights: list of (w, b) FP32 masters.  Returns the activations
    [x, a_1, ..., a_L] (a_L = last convolution, no ReLU) using BF16-rounded w
    (unrounded when round_weights is False) and, with round_acts, each
    convolution's input rounded to BF16 as well (the operands of a BF16
    tensor-core convolution; the activations kept are the unrounded sums).
    The correction is N(x) = out_scale * a_L."""
    acts = [x]
    for l, (w, b) in enumerate(weights):
        inp = bf16_round(acts[-1]) if round_acts else acts[-1]
        y = conv3x3(inp, bf16_round(w) if round_weights else w, b)
        if l < len(weights) - 1:
            y = np.maximum(y, 0.0)
        acts.append(y)
    return acts


def loss_and_grads(weights, x, coarse, target, round_weights=True, out_scale=1.0, round_acts=False):
    """Mean squared difference between C(u_n) + N(x), N(x) = out_scale * a_L,
    and the fine result over all B x 2 x H x W real values, measured in units
    of out_scale (i.e. the mean of ((C + N - F) / out_scale)^2; out_scale may
    hold one value per sample); gradients by
    backpropagation (BF16 weights in the forward pass, gradients taken with
    respect to those weights; with round_acts the incoming gradient of each
    input-gradient convolution is rounded to BF16 too, and so are both
    operands of each weight-gradient product -- the operand precision of a
    BF16 tensor-core implementation).  Returns (loss, grads, N(x))."""
    acts = forward(weights, x, round_weights, round_acts)
    # out_scale: one number, or one per sample (shape (B,) or broadcastable to it)
    s = np.reshape(np.asarray(out_scale, dtype=np.float64), (-1,))
    s = s if s.size > 1 else s[:1]
    s4, s3 = s[:, None, None, None], s[:, None, None]
    out = s4 * acts[-1]
    pred_re = coarse.real + out[:, 0]
    pred_im = coarse.imag + out[:, 1]
    r_re, r_im = (pred_re - target.real) / s3, (pred_im - target.imag) / s3
    count = out.size
    loss = float((np.sum(r_re * r_re) + np.sum(r_im * r_im)) / count)
    dy = np.stack([2 * r_re / count, 2 * r_im / count], axis=1)
    grads = [None] * len(weights)
    for l in reversed(range(len(weights))):
        w, b = weights[l]
        if l < len(weights) - 1:
            dy = dy * (acts[l + 1] > 0)
        if round_acts:
            dw, db = conv3x3_weight_grad(bf16_round(acts[l]).astype(np.float64), bf16_round(dy).astype(np.float64))
        else:
            dw, db = conv3x3_weight_grad(acts[l], dy)
        grads[l] = (dw, db)
        if l > 0:
            dy = conv3x3_adjoint(bf16_round(dy) if round_acts else dy, bf16_round(w) if round_weights else w)
    return loss, grads, out


def adam_step(param, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), bias-corrected, step t >= 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v


def flatten(weights):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in weights]).astype(np.float32)


def unflatten(flat, shapes):
    out, k = [], 0
    for cin, cout, _ in shapes:
        nw = cout * cin * 9
        w = np.asarray(flat[k:k + nw], dtype=np.float32).reshape(cout, cin, 3, 3)
        k += nw
        b = np.asarray(flat[k:k + cout], dtype=np.float32)
        k += cout
        out.append((w, b))
    return out
