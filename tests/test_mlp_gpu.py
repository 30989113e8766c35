"""GPU tests of the warm-start network kernels against the FP64 reference
(oracle/mlp.py) with the same BF16 operand rounding: features (exact),
forward, loss and gradient (the gradient check), Adam, determinism, and a
short training run that lowers the loss."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as M
from paper_2503_08264_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_08264_gb300 import build
    build.build()


def _case(n, seed):
    rng = np.random.default_rng(seed)
    model = S.hier_logistic(M=n, N=5, seed=seed)
    x, y = model.levels[1].x, model.levels[1].y
    m = rng.standard_normal((n, 18)) * 0.7
    s = rng.uniform(0.2, 1.2, (n, 18))
    target = np.stack([m, s], 1).astype(np.float32)            # [n, 2, D]
    return x, y, target


def _ws(seed=0, scale=1.0):
    from paper_2503_08264_gb300.warmstart import WarmStart
    p = S.mlp_init(seed)
    return WarmStart(params=p * scale), p


@pytest.mark.parametrize("n", [1, 45, 200])
def test_features_forward_loss_and_gradient_match_reference(n):
    x, y, target = _case(n, seed=100 + n)
    ws, p = _ws(seed=n)
    f = ws.features(torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda())
    f_ref = M.features(x, y)
    np.testing.assert_array_equal(f.cpu().numpy(), f_ref.astype(np.float32))
    out = ws.forward(f).cpu().numpy()
    o_ref, _ = M.forward(p.astype(np.float64), f_ref, bf16=True)
    np.testing.assert_allclose(out, o_ref, rtol=2e-5, atol=2e-5 * np.abs(o_ref).max())
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = ws.loss_grad(f, torch.as_tensor(target).cuda(), loss).cpu().numpy()
    l_ref, g_ref = M.loss_grad(p.astype(np.float64), f_ref, target[:, 0].astype(np.float64),
                               target[:, 1].astype(np.float64), bf16=True)
    assert abs(loss.item() - l_ref) <= 1e-5 * abs(l_ref)
    gs = np.abs(g_ref).max()
    err = np.abs(g - g_ref).max() / gs
    print(f"n={n}: loss {loss.item():.6f} vs {l_ref:.6f}, gradient max error {err:.2e} of max |g|")
    assert err < 1e-4
    # per-layer check: every block of the flat layout is close, not only the largest
    off = 0
    for i, o in zip(M.SIZES[:-1], M.SIZES[1:]):
        for sz in (o * i, o):
            blk, ref = g[off:off + sz], g_ref[off:off + sz]
            assert np.abs(blk - ref).max() <= 1e-4 * max(np.abs(ref).max(), 1e-3 * gs)
            off += sz


def test_adam_step_matches_reference_and_gradient_is_deterministic():
    x, y, target = _case(300, seed=7)
    ws, p = _ws(seed=3)
    f = ws.features(torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda())
    t = torch.as_tensor(target).cuda()
    g1 = ws.loss_grad(f, t).clone()
    g2 = ws.loss_grad(f, t).clone()
    assert torch.equal(g1, g2)
    theta = ws.params.double().cpu().numpy()
    m0, v0 = np.zeros_like(theta), np.zeros_like(theta)
    ref, mr, vr = theta, m0, v0
    gg = g1.double().cpu().numpy()
    for step in (1, 2):
        ws.grad.copy_(g1)
        ws.step(lr=1e-3)
        ref, mr, vr = M.adam(ref, gg, mr, vr, t=step, lr=1e-3)
    np.testing.assert_allclose(ws.params.cpu().numpy(), ref, rtol=0, atol=2e-6)
    np.testing.assert_allclose(ws.m.cpu().numpy(), mr, rtol=1e-6, atol=1e-12)


def test_training_lowers_the_loss():
    x, y, _ = _case(2048, seed=11)
    # targets a smooth function of the features, so a network can fit them
    f_ref = M.features(x, y)
    m = np.tanh(f_ref[:, :18] - 0.5 * f_ref[:, 18:36])
    s = np.exp(-0.3 * f_ref[:, 36:37] / 5.0) * np.ones((1, 18))
    target = torch.as_tensor(np.stack([m, s], 1).astype(np.float32)).cuda()
    ws, _ = _ws(seed=5)
    f = ws.features(torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda())
    hist = ws.train(f, target, epochs=30, batch=256, lr=3e-3)
    print("loss per epoch", [round(h, 4) for h in hist[::5]], hist[-1])
    assert hist[-1] < 0.2 * hist[0]
