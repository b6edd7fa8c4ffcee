"""Failure detection on the GPU without a fault: the bounded device waits.

Every mbarrier wait in the tensor-core product gives up after a cycle limit, sets an
error word, drains what it issued and returns.  The test option test_stall_copies makes
the product's copy producer issue nothing, so no copy or MMA is ever in flight and
every consumer wait runs out; with wait_limit_log2 = 20 (about 0.5 ms per wait) the call
returns KRR_E_TIMEOUT quickly.  The context (and the device) must stay usable.
"""
import numpy as np
import pytest
import torch

from oracle import krr_oracle as O

pytestmark = pytest.mark.gpu


def _case(n=3000, d=6, nrhs=2, seed=31):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.uniform(-1, 1, size=(n, d)).astype(np.float32)
    V = rng.normal(size=(n, nrhs)).astype(np.float32)
    return X, V


@pytest.mark.parametrize("nrhs", [1, 2, 16])
def test_stalled_tensor_core_product_times_out_and_reports_it(nrhs):
    # nrhs = 1 runs the V-folded product, nrhs = 16 the one with P.V on the tensor cores
    # (each its own kernel and waits)
    from paper_1905_10587_gb300 import _lib
    from paper_1905_10587_gb300.api import KRR, KRRError
    X, V = _case(nrhs=nrhs)
    Xd, Vd = torch.from_numpy(X).cuda(), torch.from_numpy(V).cuda()
    ctx = KRR(precision=1, wait_limit_log2=20, test_stall_copies=1)
    with pytest.raises(KRRError) as ei:
        ctx.kmvm(Xd, Xd, Vd, 0.7, 1e-3)
    assert ei.value.code == _lib.KRR_E_TIMEOUT
    assert "timed out" in str(ei.value)
    # the device is still usable: a normal tensor-core product afterwards is correct
    torch.cuda.synchronize()
    Q = KRR(precision=1).kmvm(Xd, Xd, Vd, 0.7, 1e-3).cpu().numpy()
    ref = O.kmvm(X, V.astype(np.float64), 0.7, 1e-3)
    rel = np.linalg.norm(Q - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rel.max() <= 1e-5


def test_stalled_product_inside_a_solve_is_reported():
    # the solver reads the error word with the CG scalars and stops with KRR_E_TIMEOUT
    import synth
    from paper_1905_10587_gb300 import _lib
    from paper_1905_10587_gb300.api import KRR, KRRError
    p = synth.small(n=900, k=40)
    X = torch.from_numpy(p.X).cuda()
    Y = torch.from_numpy(p.Y).cuda()
    ctx = KRR(precision=1, wait_limit_log2=20, test_stall_copies=1)
    ctx.build(X, p.sigma, p.beta, p.k, seed=1)     # the sketch does not stall
    with pytest.raises(KRRError) as ei:
        ctx.solve(Y, tol=1e-6)
    assert ei.value.code == _lib.KRR_E_TIMEOUT


def test_wait_options_are_validated():
    from paper_1905_10587_gb300.api import KRR, KRRError
    for bad in (dict(wait_limit_log2=5), dict(wait_limit_log2=41), dict(test_stall_copies=2)):
        with pytest.raises(KRRError):
            KRR(**bad)
