"""Seeded synthetic workloads for Gaussian kernel ridge regression.

This module only draws inputs: point sets X, targets y and the problem
parameters (sigma, beta, rank k) of the five workloads the solver is measured
on.  It holds none of the method's arithmetic, so both the FP64 oracle and the
CUDA path can take their inputs from here without sharing any computation.

Every array is generated in float64 with NumPy's PCG64 and then rounded to
float32; the float32 values are what both sides receive (the oracle upcasts
them back to float64), so the two see bit-identical data.

Kernel convention: K_ij = exp(-||x_i - x_j||^2 / (2 sigma^2)).  The paper writes
the Gaussian with a width h and exponent -||x-y||^2/h^2 (Section 2.4, Eq. for the
discrete Gauss transform), so h = sqrt(2) * sigma.

Workloads (the paper's datasets are not available; these stand in for them):

* ``small``     n=2000, d=4, X ~ U[0,1]^4, y = sin(2 pi sum x) + N(0, 0.01^2),
                sigma=0.5, beta=1e-2, k=100, one right-hand side.
* ``mixture``   n=100000, d=8, X from a 10-component Gaussian mixture (means
                U[-5,5]^8, isotropic std 1, equal weights),
                y = ||x|| cos(x_1) + N(0, 0.05^2), sigma=1, beta=1e-3, k=1000.
* ``cube3d``    n=1e6, d=3, X ~ U[0,10]^3, y = sum sin(x_i) + N(0, 0.1^2),
                sigma=0.8, beta=1e-4, k=2000, 1 or 16 right-hand sides (the
                extra columns are independent N(0,1)).
* ``cube3d_density_matched``  the cube shrunk to n points at the same density
                (side 10 (n/1e6)^(1/3)) and anchors per volume (k = 2000 n/1e6).
* ``batched``   64 problems, n log-uniform in [1000, 50000], d uniform in
                {2..16}, X ~ N(0,I), 8 right-hand sides y_j = sin(w_j . x) with
                w_j ~ N(0,I), sigma=sqrt(d), beta=1e-3, k=min(500, n/10).
* ``gradient``  2e5 training + 2e4 held-out points, d=10, X ~ N(0,I),
                y = tanh(a . x) + N(0, 0.1^2), a ~ N(0, I/10), sigma=2,
                beta=1e-3, k=1500.

The low-dimensional cube stands in for the paper's 3-D synthetic field
experiment (Section 5.2) and the mixture / gradient workloads for its
higher-dimensional regression datasets (Section 5.3), at smaller d.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = ["Problem", "small", "mixture", "cube3d", "cube3d_density_matched", "batched", "gradient",
           "WORKLOADS", "rademacher_unit"]


@dataclass
class Problem:
    """One KRR problem: points, targets and method parameters.

    X is (n, d) float32 C-contiguous; Y is (n, nrhs) float32 (nrhs columns);
    Xval / yval are the held-out set when the workload has one.
    """
    name: str
    X: np.ndarray
    Y: np.ndarray
    sigma: float
    beta: float
    k: int
    oversample: int = 5
    tol: float = 1e-6
    Xval: np.ndarray | None = None
    yval: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]

    @property
    def nrhs(self) -> int:
        return self.Y.shape[1]

    @property
    def l(self) -> int:
        return self.k + self.oversample


def _f32(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def small(seed: int = 0, n: int = 2000, k: int = 100) -> Problem:
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.uniform(0.0, 1.0, size=(n, 4))
    y = np.sin(2.0 * np.pi * X.sum(axis=1)) + rng.normal(0.0, 0.01, size=n)
    return Problem("small", _f32(X), _f32(y[:, None]), 0.5, 1e-2, min(k, n))


def mixture(seed: int = 1000, n: int = 100_000, k: int = 1000) -> Problem:
    rng = np.random.Generator(np.random.PCG64(seed))
    d, comps = 8, 10
    means = rng.uniform(-5.0, 5.0, size=(comps, d))
    lab = rng.integers(0, comps, size=n)
    X = means[lab] + rng.normal(0.0, 1.0, size=(n, d))
    y = np.linalg.norm(X, axis=1) * np.cos(X[:, 0]) + rng.normal(0.0, 0.05, size=n)
    return Problem("mixture", _f32(X), _f32(y[:, None]), 1.0, 1e-3, min(k, n))


def cube3d(seed: int = 2000, n: int = 1_000_000, nrhs: int = 1, k: int = 2000,
           side: float = 10.0) -> Problem:
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.uniform(0.0, side, size=(n, 3))
    y = np.sin(X).sum(axis=1) + rng.normal(0.0, 0.1, size=n)
    cols = [y]
    for _ in range(nrhs - 1):
        cols.append(rng.normal(0.0, 1.0, size=n))
    return Problem("cube3d", _f32(X), _f32(np.stack(cols, axis=1)), 0.8, 1e-4, min(k, n))


def cube3d_density_matched(n: int, seed: int = 2000, nrhs: int = 1) -> Problem:
    """The cube workload shrunk to n points at the same density (10^6 points per 10^3
    volume: side 10 (n / 10^6)^(1/3)) and the same anchors per volume (k = 2000 n / 10^6),
    so the kernel's neighbour counts, its spectrum per unit volume and the preconditioner's
    coverage match the full-size problem."""
    side = 10.0 * (n / 1e6) ** (1.0 / 3.0)
    k = max(1, int(round(2000 * n / 1e6)))
    p = cube3d(seed=seed, n=n, nrhs=nrhs, k=k, side=side)
    p.name = "cube3d_density_matched"
    return p


def batched(seed: int = 3000, nprob: int = 64, n_lo: int = 1000, n_hi: int = 50_000,
            nrhs: int = 8) -> list[Problem]:
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=nprob)).astype(np.int64)
    ds = rng.integers(2, 17, size=nprob)
    probs = []
    for p in range(nprob):
        n, d = int(ns[p]), int(ds[p])
        X = rng.normal(0.0, 1.0, size=(n, d))
        W = rng.normal(0.0, 1.0, size=(nrhs, d))
        Y = np.sin(X @ W.T)
        probs.append(Problem(f"batched[{p}]", _f32(X), _f32(Y), float(np.sqrt(d)), 1e-3,
                             int(min(500, n // 10))))
    return probs


def gradient(seed: int = 4000, n: int = 200_000, m: int = 20_000, k: int = 1500) -> Problem:
    rng = np.random.Generator(np.random.PCG64(seed))
    d = 10
    a = rng.normal(0.0, np.sqrt(0.1), size=d)
    X = rng.normal(0.0, 1.0, size=(n, d))
    Xv = rng.normal(0.0, 1.0, size=(m, d))
    y = np.tanh(X @ a) + rng.normal(0.0, 0.1, size=n)
    yv = np.tanh(Xv @ a) + rng.normal(0.0, 0.1, size=m)
    return Problem("gradient", _f32(X), _f32(y[:, None]), 2.0, 1e-3, min(k, n),
                   Xval=_f32(Xv), yval=_f32(yv))


def rademacher_unit(n: int, seed: int) -> np.ndarray:
    """A seeded unit-norm direction with +-1/sqrt(n) entries (for directional FD checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.integers(0, 2, size=n) * 2 - 1) / np.sqrt(n)


WORKLOADS = {"small": small, "mixture": mixture, "cube3d": cube3d,
             "batched": batched, "gradient": gradient}
