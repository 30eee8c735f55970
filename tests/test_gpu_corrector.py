"""Corrector kernels (cgl_corrector_*) against the numpy corrector oracle, and
a small training run that must improve the coarse step on held-out data."""
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


@pytest.mark.parametrize("H,W,B,hidden,layers", [(32, 16, 2, 8, 4), (16, 48, 3, 32, 3), (128, 128, 2, 32, 6)])
def test_forward_matches_oracle(H, W, B, hidden, layers):
    weights, coarse, un, target, params, d = setup(H, W, B, hidden, layers, 1)
    corr = nat.Corrector(H, W, hidden, layers, max_batch=B)
    corr.set_weights(C.flatten(weights))
    out = corr.forward(d[0], d[1], d[3]).cpu().numpy()
    ref = C.forward(weights, C.features(coarse.astype(complex), un.astype(complex), params))[-1]
    assert rel(out, ref) <= 1e-5


def test_forward_selects_samples_by_index():
    weights, coarse, un, target, params, d = setup(16, 16, 4, 8, 3, 2)
    corr = nat.Corrector(16, 16, 8, 3, max_batch=4)
    corr.set_weights(C.flatten(weights))
    idx = torch.tensor([3, 1], dtype=torch.int32, device="cuda")
    out = corr.forward(d[0], d[1], d[3], idx=idx).cpu().numpy()
    ref = C.forward(weights, C.features(coarse[[3, 1]].astype(complex), un[[3, 1]].astype(complex),
                                        params[[3, 1]]))[-1]
    assert rel(out, ref) <= 1e-5


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
                                        out_scale=out_scale)
    assert loss == pytest.approx(rloss, rel=1e-5)
    gref = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in rgrads])
    assert rel(g, gref) <= 1e-4
    # every layer's weight gradient separately
    k = 0
    for (gw, gb) in rgrads:
        n = gw.size
        assert rel(g[k:k + n], gw.ravel()) <= 1e-4
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
                                    target.astype(complex))
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
