"""Pins of the corrector oracle: convolution and its adjoint against direct
definitions, weight gradients and full backpropagation against finite
differences, BF16 rounding against a library conversion, Adam by hand."""
import numpy as np
import pytest

from oracle import corrector_oracle as C


def direct_conv(x, w, b):
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    y = np.zeros((B, Co, H, W))
    for bb in range(B):
        for o in range(Co):
            for i in range(H):
                for j in range(W):
                    s = b[o]
                    for c in range(Ci):
                        for di in range(3):
                            for dj in range(3):
                                s += w[o, c, di, dj] * x[bb, c, (i + di - 1) % H, (j + dj - 1) % W]
                    y[bb, o, i, j] = s
    return y


def test_conv_matches_direct_definition():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 5, 4))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(C.conv3x3(x, w, b), direct_conv(x, w, b), rtol=1e-12, atol=1e-12)


def test_adjoint_identity():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 6, 5))
    y = rng.standard_normal((2, 4, 6, 5))
    w = rng.standard_normal((4, 3, 3, 3))
    lhs = np.sum(C.conv3x3(x, w, np.zeros(4)) * y)
    rhs = np.sum(x * C.conv3x3_adjoint(y, w))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_weight_grad_matches_direct_definition():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 2, 4, 5))
    dy = rng.standard_normal((2, 3, 4, 5))
    dw, db = C.conv3x3_weight_grad(x, dy)
    for o in range(3):
        for c in range(2):
            for di in range(3):
                for dj in range(3):
                    ref = sum(dy[b, o, i, j] * x[b, c, (i + di - 1) % 4, (j + dj - 1) % 5]
                              for b in range(2) for i in range(4) for j in range(5))
                    assert dw[o, c, di, dj] == pytest.approx(ref, rel=1e-12)
    np.testing.assert_allclose(db, dy.sum(axis=(0, 2, 3)))


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    shapes = C.layer_shapes(hidden=4, layers=3)
    weights = [(rng.standard_normal((co, ci, 3, 3)) * 0.3, rng.standard_normal(co) * 0.1) for ci, co, _ in shapes]
    B, H, W = 2, 5, 6
    coarse = rng.standard_normal((B, H, W)) + 1j * rng.standard_normal((B, H, W))
    un = rng.standard_normal((B, H, W)) + 1j * rng.standard_normal((B, H, W))
    target = coarse + 0.1 * (rng.standard_normal((B, H, W)) + 1j * rng.standard_normal((B, H, W)))
    x = C.features(coarse, un, rng.standard_normal((B, 5)))
    loss, grads, _ = C.loss_and_grads(weights, x, coarse, target, round_weights=False)
    h = 1e-6
    for l in range(len(weights)):
        w, b = weights[l]
        for idx in [(0, 0, 1, 1), (w.shape[0] - 1, w.shape[1] - 1, 2, 0)]:
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            lp = C.loss_and_grads(weights[:l] + [(wp, b)] + weights[l + 1:], x, coarse, target, False)[0]
            lm = C.loss_and_grads(weights[:l] + [(wm, b)] + weights[l + 1:], x, coarse, target, False)[0]
            assert grads[l][0][idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)
        bp, bm = b.copy(), b.copy()
        bp[0] += h
        bm[0] -= h
        lp = C.loss_and_grads(weights[:l] + [(w, bp)] + weights[l + 1:], x, coarse, target, False)[0]
        lm = C.loss_and_grads(weights[:l] + [(w, bm)] + weights[l + 1:], x, coarse, target, False)[0]
        assert grads[l][1][0] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)


def test_bf16_rounding():
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 3.14159, 1e-30, 65504.0], dtype=np.float32)
    got = C.bf16_round(vals)
    assert got[0] == 1.0
    assert got[1] == 1.0              # halfway, ties to even
    assert got[2] == 1 + 2 ** -6      # halfway, ties to even (upwards here)
    torch = pytest.importorskip("torch")
    ref = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(got, ref)


def test_adam_step_by_hand():
    p, g = np.array([1.0]), np.array([0.5])
    p1, m, v = C.adam_step(p, g, np.zeros(1), np.zeros(1), 1, lr=0.1)
    # first step: mhat = g, vhat = g^2 -> p - lr * g / (|g| + eps)
    assert p1[0] == pytest.approx(1.0 - 0.1 * 0.5 / (0.5 + 1e-8))
    assert m[0] == pytest.approx(0.05) and v[0] == pytest.approx(0.00025)


def test_features_layout():
    coarse = np.array([[[1 + 2j]]])
    un = np.array([[[3 - 4j]]])
    x = C.features(coarse, un, np.array([[5, 6, 7, 8, 9]]))
    np.testing.assert_array_equal(x[0, :, 0, 0], [1, 2, 3, -4, 5, 6, 7, 8, 9])


def test_flatten_roundtrip():
    shapes = C.layer_shapes(hidden=4, layers=3)
    rng = np.random.default_rng(5)
    ws = [(rng.standard_normal((co, ci, 3, 3)).astype(np.float32), rng.standard_normal(co).astype(np.float32))
          for ci, co, _ in shapes]
    back = C.unflatten(C.flatten(ws), shapes)
    for (a, b), (c, d) in zip(ws, back):
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(b, d)
