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


# ------------------------------------------------------------------ grouped (lockstep) form
def _check(p, a, tol):
    a = a.cpu().numpy()
    a = a[:, None] if a.ndim == 1 else a
    ref = O.solve_dense(p.X, p.Y.astype(np.float64), p.sigma, p.beta)
    rel = np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)
    r = O.residual(p.X, a, p.Y, p.sigma, p.beta)
    rr = np.linalg.norm(r, axis=0) / np.linalg.norm(p.Y.astype(np.float64), axis=0)
    return rel.max(), rr.max()


@pytest.mark.parametrize("precision,nrhs", [(1, 3), (0, 3), (1, 8)])
def test_grouped_batch_solve_matches_dense(precision, nrhs):
    # every step of the lockstep recurrence is one launch over all problems; three
    # right-hand sides run as product chunks of 2 + 1 and Woodbury passes of 2 + 1
    from paper_1905_10587_gb300 import api
    probs = synth.batched(seed=78, nprob=7, n_lo=300, n_hi=3000, nrhs=nrhs)
    args = [(_t(p.X), _t(p.Y), p.sigma, p.beta, max(1, p.k)) for p in probs]
    alphas, infos, stats = api.batch_solve(args, tol=1e-7, seed=5, workers=4, grouped=True,
                                           precision=precision)
    assert all(s == 0 for s in stats), stats
    for p, a, inf in zip(probs, alphas, infos):
        rel, rr = _check(p, a, 1e-7)
        assert rel <= 1e-4, (p.name, rel)
        assert rr <= 1e-7 * 1.01, (p.name, rr)
        assert max(inf["rel_residual"]) <= 1e-7
        assert inf["iters"] > 0 and inf["mvm_count"] >= inf["iters"]


def test_grouped_batch_mixes_tensor_core_and_wide_problems():
    # d = 20 has no tensor-core features: that problem's product runs on its own inside the
    # lockstep loop while the others go through the grouped tensor-core launch
    from paper_1905_10587_gb300 import api
    rng = np.random.Generator(np.random.PCG64(90))
    probs = synth.batched(seed=79, nprob=4, n_lo=500, n_hi=2000, nrhs=2)
    X = rng.normal(size=(1200, 20)).astype(np.float32)
    Y = np.sin(X[:, :2].astype(np.float64)).astype(np.float32)
    probs.append(synth.Problem("wide", X, Y, float(np.sqrt(20)), 1e-3, 120))
    args = [(_t(p.X), _t(p.Y), p.sigma, p.beta, p.k) for p in probs]
    alphas, infos, stats = api.batch_solve(args, tol=1e-7, seed=2, grouped=True, precision=1)
    assert all(s == 0 for s in stats), stats
    assert [i["product_form"] for i in infos] == [1, 1, 1, 1, 0]
    for p, a in zip(probs, alphas):
        rel, rr = _check(p, a, 1e-7)
        assert rel <= 1e-4 and rr <= 1e-7 * 1.01, (p.name, rel, rr)


def test_grouped_matches_one_by_one_on_larger_batch():
    # 16 problems up to n = 12000 with 8 right-hand sides: both batch forms reach the
    # tolerance and agree with each other well inside it
    from paper_1905_10587_gb300 import api
    probs = synth.batched(seed=80, nprob=16, n_lo=1000, n_hi=12000, nrhs=8)
    args = [(_t(p.X), _t(p.Y), p.sigma, p.beta, max(1, p.k)) for p in probs]
    a1, i1, s1 = api.batch_solve(args, tol=1e-6, seed=3, grouped=False, precision=1)
    a2, i2, s2 = api.batch_solve(args, tol=1e-6, seed=3, grouped=True, precision=1)
    assert all(s == 0 for s in s1) and all(s == 0 for s in s2)
    for p, x, y, f in zip(probs, a1, a2, i2):
        assert max(f["rel_residual"]) <= 1e-6
        d = (torch.linalg.norm(x - y, dim=0) / torch.linalg.norm(x, dim=0)).max().item()
        assert d <= 1e-3, (p.name, d)


def test_grouped_escalates_a_breakdown_in_place():
    # tight clusters spread over a wide box make the FP32 expansion indefinite: the grouped
    # recurrence of that problem breaks down, drops its unverified correction and goes on in
    # the exact-difference form inside the group; the other problem converges beside it
    from paper_1905_10587_gb300 import api
    rng = np.random.Generator(np.random.PCG64(5))
    centres = rng.uniform(0.0, 150.0, size=(40, 3))
    Xc = (centres[:, None, :] + rng.normal(0.0, 0.02, size=(40, 75, 3))).reshape(-1, 3).astype(np.float32)
    yc = (np.sin(Xc.astype(np.float64)).sum(axis=1) + rng.normal(0.0, 0.01, size=Xc.shape[0]))
    hard = synth.Problem("clusters", Xc, yc.astype(np.float32)[:, None], 1.0, 1e-3, 40)
    easy = synth.small(n=1500, k=100)
    probs = [hard, easy]
    args = [(_t(p.X), _t(p.Y), p.sigma, p.beta, p.k) for p in probs]
    alphas, infos, stats = api.batch_solve(args, tol=1e-6, seed=2, grouped=True, precision=1)
    assert all(s == 0 for s in stats), stats
    assert infos[0]["product_form"] == 2          # finished in the exact-difference form
    for p, a in zip(probs, alphas):
        _, rr = _check(p, a, 1e-6)
        assert rr <= 1e-6 * 1.01, (p.name, rr)


def test_grouped_stalled_product_reports_timeout():
    from paper_1905_10587_gb300 import _lib, api
    from paper_1905_10587_gb300.api import KRRError
    probs = synth.batched(seed=81, nprob=3, n_lo=500, n_hi=1500, nrhs=2)
    args = [(_t(p.X), _t(p.Y), p.sigma, p.beta, max(1, p.k)) for p in probs]
    with pytest.raises(KRRError) as ei:
        api.batch_solve(args, tol=1e-6, grouped=True, precision=1, wait_limit_log2=20, test_stall_copies=1)
    assert ei.value.code == _lib.KRR_E_TIMEOUT
