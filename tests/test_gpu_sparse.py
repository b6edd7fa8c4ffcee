"""Algorithm 2 (sparse anchor selection) on the GPU against the oracle (needs a GB300).

The draws are integer and sign work, so they must match the oracle's Philox draws
exactly; the sketch entries are FP32 sums of r kernel terms, held to 1e-5 of the sum
of their magnitudes; a build on the sparse sketch must give a preconditioner with which
the solve meets the 1e-6 residual, and anchors as good as the oracle's (within 2x in
the spectral norm of K - K~).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import krr_oracle as O

pytestmark = pytest.mark.gpu


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.mark.parametrize("seed,l,r,n", [(0, 1, 1, 1), (7, 105, 8, 2000), (2 ** 40 + 3, 33, 5, 1_000_000),
                                        (12, 1005, 16, 100_000)])
def test_sparse_draws_match_oracle_exactly(seed, l, r, n):
    from paper_1905_10587_gb300.api import KRR
    R, S = KRR().sparse_draw(seed, l, r, n)
    R_or, v_or = O.sparse_draw(seed, l, r, n)
    assert np.array_equal(R.cpu().numpy().astype(np.int64), R_or)
    assert np.array_equal(S.cpu().numpy().astype(np.float64), v_or)


@pytest.mark.parametrize("n,d,l,r", [(1, 3, 1, 1), (777, 4, 37, 8), (4099, 13, 70, 16), (300, 64, 9, 3)])
def test_sparse_sketch_matches_oracle(n, d, l, r):
    from paper_1905_10587_gb300.api import KRR
    rng = np.random.Generator(np.random.PCG64(n + d))
    X = rng.uniform(-2, 2, size=(n, d)).astype(np.float32)
    sigma = 0.4 * np.sqrt(d)
    Y = KRR().sparse_sketch(_t(X), sigma, l, r, seed=21).cpu().numpy().astype(np.float64)
    R, v = O.sparse_draw(21, l, r, n)
    ref = O.sparse_sketch(X, sigma, R, v)
    mag = O.sparse_sketch(X, sigma, R, np.abs(v))       # sum of |terms| per entry
    assert np.all(np.abs(Y - ref) <= 1e-5 * mag + 1e-30)


def test_build_on_sparse_sketch_solves_small_config():
    from paper_1905_10587_gb300.api import KRR
    p = synth.small(n=1000, k=50)
    ctx = KRR(sparse_r=8)
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=5)
    S = ctx.anchors().cpu().numpy()
    Kfull = O.kernel_matrix(p.X, p.X, p.sigma)
    err_gpu = np.linalg.norm(Kfull - O.Nystrom(p.X, S, p.sigma, p.beta).ktilde(), 2)
    S_or = O.sparse_anchor_selection(p.X, p.sigma, p.k, p.l, 8, seed=5)
    err_or = np.linalg.norm(Kfull - O.Nystrom(p.X, S_or, p.sigma, p.beta).ktilde(), 2)
    assert err_gpu <= 2.0 * err_or
    a, info = ctx.solve(_t(p.Y), tol=1e-6)
    res = np.linalg.norm(O.residual(p.X, a.cpu().numpy(), p.Y, p.sigma, p.beta)) / np.linalg.norm(p.Y)
    assert res <= 1e-6


def test_sparse_r_option_is_validated():
    from paper_1905_10587_gb300.api import KRR, KRRError
    with pytest.raises(KRRError):
        KRR(sparse_r=-1)
