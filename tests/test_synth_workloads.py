"""The seeded synthetic workloads match their stated recipes (shapes, parameters,
distributions) and are reproducible; every GPU parity test and the bench draw from them."""
import numpy as np

import synth


def test_small_recipe():
    p = synth.small()
    assert p.X.shape == (2000, 4) and p.Y.shape == (2000, 1)
    assert p.X.dtype == np.float32 and p.Y.dtype == np.float32
    assert (p.sigma, p.beta, p.k) == (0.5, 1e-2, 100)
    assert p.X.min() >= 0.0 and p.X.max() <= 1.0
    resid = p.Y[:, 0] - np.sin(2 * np.pi * p.X.astype(np.float64).sum(1))
    assert abs(resid.std() - 0.01) < 0.002           # N(0, 0.01^2) noise


def test_mixture_recipe_is_the_bench_workload():
    p = synth.mixture(n=20000)
    assert p.X.shape == (20000, 8)
    assert (p.sigma, p.beta) == (1.0, 1e-3) and p.k == 1000
    X = p.X.astype(np.float64)
    f = np.linalg.norm(X, axis=1) * np.cos(X[:, 0])
    assert abs((p.Y[:, 0] - f).std() - 0.05) < 0.005  # N(0, 0.05^2) noise
    q = synth.mixture(n=20000)
    assert np.array_equal(p.X, q.X) and np.array_equal(p.Y, q.Y)
    assert not np.array_equal(synth.mixture(n=200, seed=1001).X, synth.mixture(n=200).X)


def test_cube_recipe():
    p = synth.cube3d(n=5000, nrhs=16)
    assert p.X.shape == (5000, 3) and p.Y.shape == (5000, 16)
    assert (p.sigma, p.beta, p.k) == (0.8, 1e-4, 2000)
    assert p.X.min() >= 0.0 and p.X.max() <= 10.0
    extra = p.Y[:, 1:].astype(np.float64)            # the extra columns are N(0, 1)
    assert abs(extra.mean()) < 0.05 and abs(extra.std() - 1.0) < 0.05


def test_batched_recipe():
    probs = synth.batched()
    assert len(probs) == 64
    ns = np.array([p.n for p in probs])
    ds = np.array([p.d for p in probs])
    assert ns.min() >= 1000 and ns.max() <= 50000
    assert ds.min() >= 2 and ds.max() <= 16
    for p in probs:
        assert p.Y.shape == (p.n, 8)
        assert p.sigma == np.float64(np.sqrt(p.d)) and p.beta == 1e-3
        assert p.k == min(500, p.n // 10)
        assert np.abs(p.Y).max() <= 1.0               # y_j = sin(w_j . x)


def test_gradient_recipe():
    p = synth.gradient(n=3000, m=500)
    assert p.X.shape == (3000, 10) and p.Xval.shape == (500, 10) and p.yval.shape == (500,)
    assert (p.sigma, p.beta) == (2.0, 1e-3)
