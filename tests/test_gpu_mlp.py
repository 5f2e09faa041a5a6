"""Cost-model kernels (pv_mlp_forward / backward / adam) against the fp64
reference: forward outputs and gradients within a relative 1e-4 (fp32
arithmetic over sums of up to thousands of terms), Adam exactly as defined,
and training on the GPU reduces the loss as the reference does."""
import ctypes

import numpy as np
import pytest

from oracle import mlp_ref
from paper_1709_00700_gb300 import pv

pytestmark = pytest.mark.gpu
H = 64


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def ctx():
    c = pv.Context(0)
    yield c
    c.close()


def _case(B, F, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, F))
    t = rng.normal(size=B)
    mu, sigma = X.mean(0), X.std(0) + 0.1
    p = mlp_ref.init(F, H, seed=seed) + rng.normal(0, 0.02, mlp_ref.n_params(F, H))
    return X, t, mu, sigma, p


@pytest.mark.parametrize("B,F", [(1, 1), (7, 5), (130, 20), (5000, 31), (64, 64)])
def test_forward_and_backward_match_reference(ctx, B, F):
    import torch
    X, t, mu, sigma, p = _case(B, F, B + F)
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")  # noqa: E731
    dp, dX, dmu, dsig, dt = dev(p), dev(X), dev(mu), dev(sigma), dev(t)
    y = torch.empty(B, device="cuda")
    act = torch.empty(B * 2 * H, device="cuda")
    dz = torch.empty(B * (2 * H + 1), device="cuda")
    grad = torch.empty(len(p), device="cuda")
    loss = torch.empty(1, device="cuda")
    lib = ctx.lib
    assert lib.pv_mlp_forward(ctx.h, _ptr(dp), _ptr(dX), _ptr(dmu), _ptr(dsig), B, F, _ptr(y), _ptr(act)) == 0
    assert lib.pv_mlp_backward(ctx.h, _ptr(dp), _ptr(dX), _ptr(dmu), _ptr(dsig), _ptr(act), _ptr(y), _ptr(dt), B, F,
                               _ptr(dz), _ptr(grad), _ptr(loss)) == 0
    ctx.stream.synchronize()
    # the reference sees the same fp32-rounded inputs
    r = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731
    yr, cache = mlp_ref.forward(r(p), r(X), r(mu), r(sigma), H)
    gr = mlp_ref.backward(r(p), cache, yr, r(t), H)
    assert np.allclose(y.cpu().numpy(), yr, rtol=1e-4, atol=1e-4 * np.abs(yr).max())
    g = grad.cpu().numpy()
    scale = np.abs(gr).max()
    assert np.allclose(g, gr, rtol=1e-3, atol=1e-4 * scale), np.abs(g - gr).max() / scale
    assert abs(loss.item() - mlp_ref.loss(yr, r(t))) <= 1e-4 * max(1.0, mlp_ref.loss(yr, r(t)))


def test_adam_matches_reference(ctx):
    import torch
    rng = np.random.default_rng(9)
    n = 10_000
    p, g, m, v = (rng.normal(size=n) for _ in range(4))
    v = np.abs(v)
    dp, dg, dm, dv = (torch.tensor(a, dtype=torch.float32, device="cuda") for a in (p, g, m, v))
    assert ctx.lib.pv_mlp_adam(ctx.h, _ptr(dp), _ptr(dg), _ptr(dm), _ptr(dv), n, 1e-3, 0.9, 0.999, 1e-8, 7) == 0
    ctx.stream.synchronize()
    r = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731
    p1, m1, v1 = mlp_ref.adam_step(r(p), r(g), r(m), r(v), 7, lr=1e-3)
    assert np.allclose(dp.cpu().numpy(), p1, rtol=1e-5, atol=1e-6)
    assert np.allclose(dm.cpu().numpy(), m1, rtol=1e-5, atol=1e-6)
    assert np.allclose(dv.cpu().numpy(), v1, rtol=1e-5, atol=1e-6)


def test_gpu_training_reduces_loss(ctx):
    import torch
    from paper_1709_00700_gb300 import costmodel
    rng = np.random.default_rng(3)
    B, F = 2048, 12
    X = rng.normal(size=(B, F))
    t = np.maximum(X @ rng.normal(size=F), 0.0) - 0.5 * X[:, 0]
    net = costmodel.Net(ctx, F, seed=4)
    net.fit_standardisation(X)
    l0 = net.loss(X, t)
    hist = net.train(X, t, epochs=400, lr=3e-3, batch=B)
    assert net.loss(X, t) < 0.05 * l0
    assert hist[-1] < hist[0]
