"""Batched solves (krr_batch_solve) of independent problems of uneven n and d against the
FP64 dense solve of each (needs a GB300)."""
import numpy as np
import pytest
import torch

import synth
from oracle import krr_oracle as O

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32)


@pytest.mark.parametrize("workers", [1, 4])
def test_batch_solve_matches_dense(workers):
    from paper_1905_10587_gb300 import api
    probs = synth.batched(seed=77, nprob=6, n_lo=300, n_hi=2500, nrhs=3)
    args = [(_t(p.X), _t(p.Y), p.sigma, p.beta, max(1, p.k)) for p in probs]
    alphas, infos, stats = api.batch_solve(args, tol=1e-7, seed=5, workers=workers)
    assert all(s == 0 for s in stats)
    for p, a, inf in zip(probs, alphas, infos):
        a = a.cpu().numpy()
        ref = O.solve_dense(p.X, p.Y.astype(np.float64), p.sigma, p.beta)
        rel = np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert rel.max() <= 1e-4, (p.name, rel)
        r = O.residual(p.X, a, p.Y, p.sigma, p.beta)
        rr = np.linalg.norm(r, axis=0) / np.linalg.norm(p.Y.astype(np.float64), axis=0)
        assert rr.max() <= 1e-7 * 1.01
        assert max(inf["rel_residual"]) <= 1e-7


def test_batch_solve_rejects_bad_problem():
    from paper_1905_10587_gb300 import api
    from paper_1905_10587_gb300.api import KRRError
    X = _t(np.zeros((10, 2)))
    Y = _t(np.ones((10, 1)))
    with pytest.raises(KRRError):
        api.batch_solve([(X, Y, 1.0, -1.0, 3)])
