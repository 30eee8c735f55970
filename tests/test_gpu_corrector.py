"""Corrector kernels (cgl_corrector_*) against the numpy corrector oracle
(with BF16 operands in the convolutions, as the tensor-core kernels use them),
and a small training run that must fit its training pairs."""
import numpy as np
import pytest
import torch

from oracle import corrector_oracle as C
from paper_2403_02816_gb300 import native as nat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2403_02816_gb300 import build as B
    B.build()
    nat.load()
    assert torch.cuda.is_available()


def setup(H, W, B, hidden, layers, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    shapes = C.layer_shapes(hidden, layers)
    weights = [((rng.standard_normal((co, ci, 3, 3)) * scale).astype(np.float32),
                (rng.standard_normal(co) * 0.1).astype(np.float32)) for ci, co, _ in shapes]
    cz = lambda: (rng.standard_normal((B, H, W)) + 1j * rng.standard_normal((B, H, W))).astype(np.complex64)
    coarse, un = cz(), cz()
    target = (coarse + 0.05 * cz()).astype(np.complex64)
    params = rng.uniform(-1, 1, (B, 5)).astype(np.float32)
    dev = lambda a: torch.from_numpy(a).cuda()
    return weights, coarse, un, target, params, (dev(coarse), dev(un), dev(target), dev(params))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# Both sides round every convolution's input to BF16, but compute that input in
# different precisions (FP32 on the GPU, FP64 in the oracle), so a few values
# round to neighbouring BF16 numbers; each such operand differs by one BF16
# unit (2^-8 relative) and the differences feed the next layer's rounding.
# Up to four layers they stay at the FP32 level; through six layers they grow
# towards, and are bounded by, the BF16 unit roundoff.
BF16_U = 2.0 ** -8


def operand_rounding_tol(layers, shallow):
    return BF16_U


def bf16_bits(a):
    """BF16 bit patterns (round to nearest even) of float32 data, as int16."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return r.view(np.int16)


@pytest.mark.parametrize("B,cin,cout,H,W,relu", [(2, 9, 32, 128, 128, 1), (1, 32, 2, 16, 48, 0), (3, 32, 32, 32, 32, 1),
                                                 (2, 17, 20, 16, 64, 0), (1, 5, 7, 24, 40, 1)])
def test_single_convolution_matches_oracle(B, cin, cout, H, W, relu):
    """One tensor-core convolution against the oracle's convolution on the same
    BF16 operands: only the order of the FP32 accumulation differs."""
    rng = np.random.default_rng(B * 100 + cin + cout)
    x = rng.standard_normal((B, cin, H, W)).astype(np.float32)
    w = (rng.standard_normal((cout, cin, 3, 3)) * 0.3).astype(np.float32)
    b = rng.standard_normal(cout).astype(np.float32)
    wb = bf16_bits(w)
    assert np.array_equal(C.bf16_round(w), (wb.view(np.uint16).astype(np.uint32) << 16).view(np.float32))
    y = torch.empty((B, cout, H, W), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    nat.cgl_conv3x3(torch.from_numpy(x).cuda(), torch.from_numpy(wb).cuda(), torch.from_numpy(b).cuda(), y, relu, st)
    ref = C.conv3x3(C.bf16_round(x).astype(np.float64), C.bf16_round(w).astype(np.float64), b.astype(np.float64))
    if relu:
        ref = np.maximum(ref, 0.0)
    assert rel(y.cpu().numpy(), ref) <= 1e-6
    assert int(st.item()) == 0


@pytest.mark.parametrize("H,W,B,hidden,layers", [(32, 16, 2, 8, 4), (16, 48, 3, 32, 3), (128, 128, 2, 32, 2),
                                                 (128, 128, 2, 32, 6)])
def test_forward_matches_oracle(H, W, B, hidden, layers):
    weights, coarse, un, target, params, d = setup(H, W, B, hidden, layers, 1)
    corr = nat.Corrector(H, W, hidden, layers, max_batch=B)
    corr.set_weights(C.flatten(weights))
    out = corr.forward(d[0], d[1], d[3]).cpu().numpy()
    ref = C.forward(weights, C.features(coarse.astype(complex), un.astype(complex), params), round_acts=True)[-1]
    assert rel(out, ref) <= operand_rounding_tol(layers, 2e-5)
    assert corr.device_status() == nat.CGL_OK


def test_forward_selects_samples_by_index():
    weights, coarse, un, target, params, d = setup(16, 16, 4, 8, 3, 2)
    corr = nat.Corrector(16, 16, 8, 3, max_batch=4)
    corr.set_weights(C.flatten(weights))
    idx = torch.tensor([3, 1], dtype=torch.int32, device="cuda")
    out = corr.forward(d[0], d[1], d[3], idx=idx).cpu().numpy()
    ref = C.forward(weights, C.features(coarse[[3, 1]].astype(complex), un[[3, 1]].astype(complex),
                                        params[[3, 1]]), round_acts=True)[-1]
    assert rel(out, ref) <= 2e-5


@pytest.mark.parametrize("H,W,B,hidden,layers,out_scale", [(32, 32, 2, 8, 4, 1.0), (64, 32, 3, 32, 6, 1.0),
                                                            (32, 16, 2, 8, 3, 1e-3)])
def test_gradients_match_oracle(H, W, B, hidden, layers, out_scale):
    weights, coarse, un, target, params, d = setup(H, W, B, hidden, layers, 3, scale=0.2)
    corr = nat.Corrector(H, W, hidden, layers, max_batch=B)
    corr.set_weights(C.flatten(weights))
    corr.set_output_scale(out_scale)
    loss, g = corr.gradients(d[0], d[1], d[2], d[3])
    x = C.features(coarse.astype(complex), un.astype(complex), params)
    rloss, rgrads, _ = C.loss_and_grads(weights, x, coarse.astype(complex), target.astype(complex),
                                        out_scale=out_scale, round_acts=True)
    assert loss == pytest.approx(rloss, rel=operand_rounding_tol(layers, 1e-5))
    gref = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in rgrads])
    tol = operand_rounding_tol(layers, 1e-4)
    assert rel(g, gref) <= tol
    # every layer's weight gradient separately
    k = 0
    for (gw, gb) in rgrads:
        n = gw.size
        assert rel(g[k:k + n], gw.ravel()) <= tol
        k += n + gb.size


def test_adam_step_matches_oracle():
    weights, coarse, un, target, params, d = setup(32, 32, 2, 8, 3, 4, scale=0.2)
    corr = nat.Corrector(32, 32, 8, 3, max_batch=2)
    flat = C.flatten(weights)
    corr.set_weights(flat)
    idx = torch.arange(2, dtype=torch.int32, device="cuda")
    lr = 1e-3
    corr.train_step(d[0], d[1], d[2], d[3], idx, lr)
    corr.train_step(d[0], d[1], d[2], d[3], idx, lr)
    got = corr.get_weights()
    # oracle: two Adam steps on its own gradients
    shapes = C.layer_shapes(8, 3)
    p, m, v = flat.astype(np.float64), np.zeros(flat.size), np.zeros(flat.size)
    x = C.features(coarse.astype(complex), un.astype(complex), params)
    gmax = 0
    for t in (1, 2):
        _, gr, _ = C.loss_and_grads(C.unflatten(p.astype(np.float32), shapes), x, coarse.astype(complex),
                                    target.astype(complex), round_acts=True)
        g = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in gr])
        gmax = max(gmax, np.abs(g).max())
        keep = np.abs(g) > 1e-3 * np.abs(g).max()
        p, m, v = C.adam_step(p, g, m, v, t, lr)
    # Adam's first steps move every weight by about lr whatever |g| is; compare
    # where the gradient is not tiny (its sign is then unambiguous)
    np.testing.assert_allclose(got[keep], p[keep], rtol=0, atol=2e-2 * lr)


def test_apply_is_coarse_plus_network_output():
    weights, coarse, un, target, params, d = setup(16, 32, 2, 8, 3, 5)
    corr = nat.Corrector(16, 32, 8, 3, max_batch=2)
    corr.set_weights(C.flatten(weights))
    corr.set_output_scale(0.25)
    out = corr.forward(d[0], d[1], d[3]).cpu().numpy()
    u = torch.empty_like(d[0])
    corr.apply(d[0], d[1], d[3], u)
    ref = coarse + out[:, 0] + 1j * out[:, 1]
    np.testing.assert_allclose(u.cpu().numpy(), ref, rtol=1e-6, atol=1e-6)


def test_training_learns_the_coarse_step_error():
    """Train on pairs from the fine method: the loss (in units of the RMS
    correction) must fall well below its initial value, and on the training
    pairs the corrected coarse step must be closer to the fine result than the
    coarse step alone, i.e. the kernels fit the data they are trained on.
    Whether that carries over to held-out trajectories is measured by the
    bench (at this coarse step most of the target is FP32 rounding of the
    coarse step, so it does not)."""
    from paper_2403_02816_gb300 import learned as Lm
    data = Lm.Dataset(ntraj=16, snaps=8)
    corr = nat.Corrector(Lm.N, Lm.N, 32, 6, max_batch=16)
    losses, _ = Lm.train(corr, data, iters=800, batch=16, lr=1e-3, log_every=400)
    first, last = losses[0][1], min(l for _, l in losses[1:])
    assert last < 0.8 * first, losses
    coarse, corrected = Lm.one_step_errors(corr, data)
    assert coarse.mean() / corrected.mean() > 1.05, (coarse.mean(), corrected.mean())
