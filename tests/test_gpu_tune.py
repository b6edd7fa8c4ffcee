"""krr_autotune on the GPU: the tuned split count and P.V form are stored under the
configuration's key, and products that take them still match the oracle."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import krr_oracle as O

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32)


@pytest.mark.parametrize("precision,nrhs", [(1, 16), (1, 1), (0, 4)])
def test_autotune_then_tuned_products_match_the_oracle(precision, nrhs):
    from paper_1905_10587_gb300 import api
    api.tune_clear()
    p = synth.mixture(n=20000, k=200)
    X = _t(p.X)
    rng = np.random.Generator(np.random.PCG64(4))
    V = rng.normal(size=(p.n, nrhs)).astype(np.float32)
    ctx = api.KRR(precision=precision)
    ctx.build(X, p.sigma, p.beta, p.k, seed=1)
    splits, pv, ms = ctx.autotune(nrhs=nrhs, reps=2)
    assert splits >= 1 and ms > 0
    width = 64 if precision == 1 else 8
    key = f"form={precision} w={width} r={nrhs} lg={int(math.floor(math.log2(p.n)))}"
    assert api.tune_get(key) == (splits, pv, pytest.approx(ms))
    tuned = api.KRR(precision=precision, autotune=1)
    Q = tuned.kmvm(X, X, _t(V), p.sigma, p.beta).cpu().numpy()
    rows = rng.choice(p.n, 128, replace=False)
    ref = O.kmvm(p.X, V.astype(np.float64), p.sigma, p.beta, rows=rows)
    rel = np.linalg.norm(Q[rows] - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rel.max() <= 1e-5
    api.tune_clear()
