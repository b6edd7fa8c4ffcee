"""Adjoint gradient of the held-out MSE (krr_grad) against the FP64 oracle and central
finite differences, and the derivative kernel product it relies on (needs a GB300).

Tolerance: 1e-4 relative, as for the solution alpha.
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import krr_oracle as O

pytestmark = pytest.mark.gpu


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.mark.parametrize("n,m,d", [(1500, 300, 10), (777, 131, 3)])
def test_dsigma_product_vs_oracle(n, m, d):
    from paper_1905_10587_gb300.api import KRR
    rng = np.random.Generator(np.random.PCG64(n))
    X = rng.normal(size=(n, d)).astype(np.float32)
    Xv = rng.normal(size=(m, d)).astype(np.float32)
    v = rng.normal(size=n).astype(np.float32)
    sigma = 2.0
    ctx = KRR()
    got = ctx.kmvm_dsigma(_t(Xv), _t(X), _t(v), sigma).cpu().numpy()
    D = O.sqdist(Xv, X)
    ref = (np.exp(-D / (2 * sigma ** 2)) * D / sigma ** 2) @ v.astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    # square case, rows = columns
    got2 = ctx.kmvm_dsigma(_t(X), _t(X), _t(v), sigma).cpu().numpy()
    D2 = O.sqdist(X, X)
    ref2 = (np.exp(-D2 / (2 * sigma ** 2)) * D2 / sigma ** 2) @ v.astype(np.float64)
    assert np.linalg.norm(got2 - ref2) / np.linalg.norm(ref2) <= 1e-5


def _gradient_case():
    p = synth.gradient(n=2000, m=400, k=150)
    return p


@pytest.mark.parametrize("precision", [0, 1])
def test_grad_vs_fp64_oracle(precision):
    from paper_1905_10587_gb300.api import KRR
    p = _gradient_case()
    ctx = KRR(precision=precision)
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=3)
    loss, ds, db, dy = ctx.grad(_t(p.Y[:, 0]), _t(p.Xval), _t(p.yval), tol=1e-9)
    L, gs, gb, gy = O.grad_val_mse(p.X, p.Y[:, 0], p.Xval, p.yval, p.sigma, p.beta)
    assert loss == pytest.approx(L, rel=1e-4)
    assert ds == pytest.approx(gs, rel=1e-4)
    assert db == pytest.approx(gb, rel=1e-4)
    dy = dy.cpu().numpy()
    assert np.linalg.norm(dy - gy) / np.linalg.norm(gy) <= 1e-4


def test_grad_vs_central_differences_of_gpu_loss():
    from paper_1905_10587_gb300.api import KRR
    p = _gradient_case()
    X, y, Xv, yv = _t(p.X), _t(p.Y[:, 0]), _t(p.Xval), _t(p.yval)

    def loss_at(sigma, beta, yy=y):
        c = KRR()
        c.build(X, sigma, beta, p.k, seed=3)
        out = c.grad(yy, Xv, yv, tol=1e-10)
        c.close()
        return out

    L0, ds, db, dy = loss_at(p.sigma, p.beta)
    h = 1e-3
    fd_s = (loss_at(p.sigma * math.exp(h), p.beta)[0] - loss_at(p.sigma * math.exp(-h), p.beta)[0]) / (2 * h)
    fd_b = (loss_at(p.sigma, p.beta * math.exp(h))[0] - loss_at(p.sigma, p.beta * math.exp(-h))[0]) / (2 * h)
    u = synth.rademacher_unit(p.n, 5)
    du = torch.from_numpy(u).to("cuda", torch.float32)
    hy = 1e-2
    fd_y = (loss_at(p.sigma, p.beta, y + hy * du)[0] - loss_at(p.sigma, p.beta, y - hy * du)[0]) / (2 * hy)
    assert ds == pytest.approx(fd_s, rel=1e-4)
    assert db == pytest.approx(fd_b, rel=1e-4)
    assert float(dy.cpu().numpy() @ u) == pytest.approx(fd_y, rel=1e-3)


def test_autograd_function_matches_grad():
    from paper_1905_10587_gb300.api import KRR, validation_loss
    p = _gradient_case()
    X, Xv, yv = _t(p.X), _t(p.Xval), _t(p.yval)
    y = _t(p.Y[:, 0]).requires_grad_(True)
    ls = torch.tensor(math.log(p.sigma), dtype=torch.float64, device="cuda", requires_grad=True)
    lb = torch.tensor(math.log(p.beta), dtype=torch.float64, device="cuda", requires_grad=True)
    L = validation_loss(y, ls, lb, X, Xv, yv, p.k, 3, 1e-9)
    L.backward()
    ctx = KRR()
    ctx.build(X, p.sigma, p.beta, p.k, seed=3)
    loss, ds, db, dy = ctx.grad(y.detach(), Xv, yv, tol=1e-9)
    assert float(L.detach()) == pytest.approx(loss, rel=1e-9)
    # two builds, each solved to a 1e-9 residual: the adjoint carries that residual times
    # the condition of K + beta I into the gradient, about 1e-6 here (the oracle and
    # finite-difference tests hold the gradient itself to 1e-4)
    assert float(ls.grad) == pytest.approx(ds, rel=1e-5)
    assert float(lb.grad) == pytest.approx(db, rel=1e-5)
    # two separate builds (sigma = exp(log sigma) differs in the last bit), each solved to 1e-9
    gy, ref = y.grad.double().cpu().numpy(), dy.cpu().numpy()
    assert np.linalg.norm(gy - ref) / np.linalg.norm(ref) <= 1e-5
