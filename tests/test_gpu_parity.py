"""CUDA path vs the FP64 oracle on the same seeded inputs (needs a GB300).

Tolerances: kernel products <= 1e-5 relative (norm-wise per column), the final
solve residual <= 1e-6 relative measured by the oracle's FP64 product, and alpha
within 1e-4 relative of the dense FP64 solve wherever the dense solve fits.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import krr_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    from paper_1905_10587_gb300.api import KRR
    return KRR


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _relcols(got, ref):
    got = np.atleast_2d(np.asarray(got, dtype=np.float64).T).T
    ref = np.atleast_2d(np.asarray(ref, dtype=np.float64).T).T
    return np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)


# ------------------------------------------------------------------ kernel products
@pytest.mark.parametrize("n,d,nrhs,beta", [(2000, 4, 1, 1e-2), (1, 3, 1, 0.5), (127, 2, 3, 0.0),
                                            (1000, 8, 16, 1e-3), (777, 13, 5, 0.1),
                                            (300, 20, 2, 0.0), (130, 64, 1, 1.0)])
def test_kmvm_square(K, n, d, nrhs, beta):
    rng = np.random.Generator(np.random.PCG64(n + d))
    X = rng.uniform(-2, 2, size=(n, d)).astype(np.float32)
    V = rng.normal(size=(n, nrhs)).astype(np.float32)
    sigma = 0.3 * np.sqrt(d)
    ctx = K()
    Q = ctx.kmvm(_t(X), _t(X), _t(V), sigma, beta).cpu().numpy()
    ref = O.kmvm(X, V.astype(np.float64), sigma, beta)
    assert _relcols(Q, ref).max() <= 1e-5


def test_kmvm_rectangular_and_small_config(K):
    p = synth.small()
    rng = np.random.Generator(np.random.PCG64(5))
    Xt = rng.uniform(0, 1, size=(333, 4)).astype(np.float32)
    V = p.Y
    ctx = K()
    Q = ctx.kmvm(_t(Xt), _t(p.X), _t(V), p.sigma).cpu().numpy()
    ref = O.kmvm_rect(Xt, p.X, V.astype(np.float64), p.sigma)
    assert _relcols(Q, ref).max() <= 1e-5
    Q2 = ctx.kmvm(_t(p.X), _t(p.X), _t(V), p.sigma, p.beta).cpu().numpy()
    assert _relcols(Q2, O.kmvm(p.X, V, p.sigma, p.beta)).max() <= 1e-5


def test_kmvm_full_size_sampled_rows(K):
    p = synth.mixture()
    ctx = K()
    Q = ctx.kmvm(_t(p.X), _t(p.X), _t(p.Y), p.sigma, p.beta).cpu().numpy()
    rows = np.random.Generator(np.random.PCG64(9)).choice(p.n, 256, replace=False)
    ref = O.kmvm(p.X, p.Y.astype(np.float64), p.sigma, p.beta, rows=rows)
    assert _relcols(Q[rows], ref).max() <= 1e-5


def test_residual_hp_fp64(K):
    p = synth.small(n=700)
    rng = np.random.Generator(np.random.PCG64(3))
    A = rng.normal(size=(p.n, 2))
    Y = np.concatenate([p.Y, p.Y * 0.5], axis=1).astype(np.float32)
    ctx = K()
    R = ctx.residual_hp(_t(p.X), _t(Y), _t(A, torch.float64), p.sigma, p.beta).cpu().numpy()
    ref = O.residual(p.X, A, Y, p.sigma, p.beta)
    assert np.abs(R - ref).max() <= 1e-12 * np.abs(ref).max() + 1e-13


@pytest.mark.parametrize("d,nrhs", [(3, 1), (8, 2), (10, 1), (16, 3)])
def test_residual_float_float_vs_fp64(K, d, nrhs):
    # the float-float residual against the oracle, scaled by the condition of each sum
    rng = np.random.Generator(np.random.PCG64(d))
    n = 900
    X = rng.normal(size=(n, d)).astype(np.float32) * 2 + 5
    A = rng.normal(size=(n, nrhs)) * 100
    Y = rng.normal(size=(n, nrhs)).astype(np.float32)
    sigma, beta = 0.4 * np.sqrt(d), 1e-3
    ctx = K()
    R = ctx.residual_hp(_t(X), _t(Y), _t(A, torch.float64), sigma, beta, mode="ff").cpu().numpy()
    ref = O.residual(X, A, Y, sigma, beta)
    cond = O.kmvm(X, np.abs(A), sigma, 0.0) + beta * np.abs(A) + np.abs(Y)
    assert np.all(np.abs(R - ref) <= 2e-11 * cond)
    R64 = ctx.residual_hp(_t(X), _t(Y), _t(A, torch.float64), sigma, beta).cpu().numpy()
    assert np.all(np.abs(R - R64) <= 2e-11 * cond)


def test_solve_with_fp64_residual_mode(K):
    p = synth.small(n=600, k=40)
    ctx = K(residual=1)
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=1)
    alpha, info = ctx.solve(_t(p.Y), tol=1e-8)
    ref = O.solve_dense(p.X, p.Y.astype(np.float64), p.sigma, p.beta)
    assert np.linalg.norm(alpha.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5


# ------------------------------------------------------------------ tensor-core product
def test_tc_descriptor_known_answer():
    from paper_1905_10587_gb300 import api
    bad, err = api.tc_selftest(0)
    assert bad == 0 and err == 0.0
    bad1, _ = api.tc_selftest(1)   # the swapped stride convention must be detected
    assert bad1 > 0
    bad2, err2 = api.tc_selftest(2)   # 128-byte swizzled layout, K = 64 in four steps
    assert bad2 == 0 and err2 == 0.0
    bad3, _ = api.tc_selftest(3)   # the same data through an unswizzled descriptor
    assert bad3 > 0
    bad4, err4 = api.tc_selftest(4)   # FP16, A from tensor memory (the P.V step)
    assert bad4 == 0 and err4 == 0.0


@pytest.mark.parametrize("n,d,nrhs,beta", [(2000, 4, 1, 1e-2), (1, 3, 1, 0.5), (127, 2, 3, 0.0),
                                            (1000, 8, 16, 1e-3), (777, 13, 5, 0.1),
                                            (300, 16, 2, 0.0), (4099, 3, 1, 1e-4)])
def test_kmvm_tensor_core_square(K, n, d, nrhs, beta):
    rng = np.random.Generator(np.random.PCG64(n + d))
    X = rng.uniform(-2, 2, size=(n, d)).astype(np.float32)
    V = rng.normal(size=(n, nrhs)).astype(np.float32)
    sigma = 0.3 * np.sqrt(d)
    ctx = K(precision=1)
    Q = ctx.kmvm(_t(X), _t(X), _t(V), sigma, beta).cpu().numpy()
    ref = O.kmvm(X, V.astype(np.float64), sigma, beta)
    assert _relcols(Q, ref).max() <= 1e-5


@pytest.mark.parametrize("nr,nc,d,nrhs,scaled", [(3000, 3000, 3, 16, False), (2500, 4099, 8, 8, False),
                                                  (1000, 777, 13, 16, True), (5000, 5000, 16, 8, True),
                                                  (1, 300, 4, 16, False), (4099, 4099, 8, 1, False),
                                                  (3000, 2000, 5, 4, True), (700, 700, 2, 2, False)])
def test_kmvm_tensor_core_pv_on_tensor_cores(K, nr, nc, d, nrhs, scaled):
    # P V contracted on the tensor cores (FP16 hi + lo parts of P and of the per-column
    # rescaled V; the default for blocks of 8 or 16 right-hand sides, tc_pv = 2 for fewer):
    # several column tiles and splits, a ragged tail, rectangular shapes, columns spanning
    # 10^-30 .. 10^25 and a zero column
    rng = np.random.Generator(np.random.PCG64(nr + 7 * nc + d))
    Xc = rng.uniform(-2, 2, size=(nc, d)).astype(np.float32)
    Xr = Xc[:nr] if nr <= nc else rng.uniform(-2, 2, size=(nr, d)).astype(np.float32)
    if nr != nc:
        Xr = Xr + np.float32(0.05)
    V = rng.normal(size=(nc, nrhs)).astype(np.float32)
    if scaled:
        V *= (10.0 ** np.linspace(-30, 25, nrhs)).astype(np.float32)
        V[:, nrhs - 2] = 0.0
    sigma = 0.3 * np.sqrt(d)
    beta = 1e-3 if nr == nc else 0.0
    V64 = V.astype(np.float64)
    ref = O.kmvm(Xc, V64, sigma, beta) if nr == nc else O.kmvm_rect(Xr, Xc, V64, sigma)
    mag = O.kmvm_rect(Xr, Xc, np.abs(V64), sigma)                 # sum of |terms|
    if nr == nc:
        mag += beta * np.abs(V64)
    nz = np.abs(V).max(axis=0) > 0
    Qs = {}
    on = 1 if nrhs >= 8 else 2
    for tc_pv in (on, 0):
        Q = K(precision=1, tc_pv=tc_pv).kmvm(_t(Xr), _t(Xc), _t(V), sigma, beta).cpu().numpy()
        assert np.all(Q[:, ~nz] == 0.0)
        if nr >= 64:   # (one row that cancels has no meaningful column norm)
            assert _relcols(Q[:, nz], ref[:, nz]).max() <= 1e-5
        assert (np.abs(Q[:, nz] - ref[:, nz]) / mag[:, nz]).max() <= 3e-5
        Qs[tc_pv] = Q
    # both forms share the exponents; the P V arithmetic alone (FP16 hi + lo parts, 22
    # bits, against FP32 products) moves every output by a few 2^-22 of its |terms| at most
    assert (np.abs(Qs[on][:, nz] - Qs[0][:, nz]) / mag[:, nz]).max() <= 3e-6


def test_kmvm_tensor_core_square_full_size_sampled_rows(K):
    # the bench workload itself (mixture, n = 10^5, d = 8) in the tensor-core form the
    # bench times: 256 sampled rows of (K + beta I) V against the oracle, for y and for
    # an N(0,1) column (the random column cancels more)
    p = synth.mixture()
    rng = np.random.Generator(np.random.PCG64(19))
    V = np.concatenate([p.Y, rng.normal(size=(p.n, 1)).astype(np.float32)], axis=1)
    ctx = K(precision=1)
    Q = ctx.kmvm(_t(p.X), _t(p.X), _t(V), p.sigma, p.beta).cpu().numpy()
    rows = rng.choice(p.n, 256, replace=False)
    ref = O.kmvm(p.X, V.astype(np.float64), p.sigma, p.beta, rows=rows)
    assert _relcols(Q[rows], ref).max() <= 1e-5


def test_kmvm_tensor_core_rectangular_full_size(K):
    p = synth.mixture()
    rng = np.random.Generator(np.random.PCG64(6))
    Xt = p.X[rng.choice(p.n, 3000, replace=False)] + 0.1
    ctx = K(precision=1)
    Q = ctx.kmvm(_t(Xt), _t(p.X), _t(p.Y), p.sigma).cpu().numpy()
    rows = rng.choice(len(Xt), 200, replace=False)
    ref = O.kmvm_rect(Xt[rows], p.X, p.Y.astype(np.float64), p.sigma)
    assert _relcols(Q[rows], ref).max() <= 1e-5


def test_tensor_core_sketch_close_to_fp32_sketch(K):
    # the build's BF16 tensor-core sketch against the FP32 sketch of the same Omega
    p = synth.mixture(n=3000, k=200)
    ctx = K(precision=1)
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=9)
    S_tc = ctx.anchors().cpu().numpy()
    ctx0 = K(precision=0)
    ctx0.build(_t(p.X), p.sigma, p.beta, p.k, seed=9)
    S_32 = ctx0.anchors().cpu().numpy()
    Kfull = O.kernel_matrix(p.X, p.X, p.sigma)
    e_tc = np.linalg.norm(Kfull - O.Nystrom(p.X, S_tc, p.sigma, p.beta).ktilde(), 2)
    e_32 = np.linalg.norm(Kfull - O.Nystrom(p.X, S_32, p.sigma, p.beta).ktilde(), 2)
    assert e_tc <= 1.5 * e_32


def test_tensor_core_sketch_vs_oracle(K):
    # BF16 kernel values and Omega each round at 2^-9 relative, so every term of
    # Y_ia = sum_j K_ij Omega_aj is off by at most ~2^-8 of |K_ij Omega_aj|; bound each
    # entry by 2^-7 times the sum of absolute terms
    p = synth.small(n=1500)
    l = 300
    ctx = K(precision=1)
    Y = ctx.sketch(_t(p.X), p.sigma, l, seed=11).cpu().numpy()
    Om = O.omega(11, l, p.n)
    ref = O.sketch(p.X, p.sigma, Om)
    cond = O.sketch(p.X, p.sigma, np.abs(Om))
    assert np.all(np.abs(Y - ref) <= 2.0 ** -7 * cond)


def test_solve_tensor_core_vs_dense(K):
    p = synth.small()
    ctx = K(precision=1)
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=1)
    alpha, info = ctx.solve(_t(p.Y), tol=p.tol)
    a = alpha.cpu().numpy()
    ref = O.solve_dense(p.X, p.Y.astype(np.float64), p.sigma, p.beta)
    r = O.residual(p.X, a, p.Y, p.sigma, p.beta)
    assert np.linalg.norm(r) / np.linalg.norm(p.Y) <= 1e-6
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) <= 1e-4


# ------------------------------------------------------------------ Algorithm 1
def test_omega_matches_oracle_generator(K):
    ctx = K()
    l, n, seed = 7, 1000, 123456789012345
    Om = ctx.omega(seed, l, n).cpu().numpy()
    ref = O.omega(seed, l, n)
    np.testing.assert_allclose(Om, ref.T, rtol=0, atol=2e-5)


def test_sketch_matches_oracle(K):
    p = synth.small(n=600)
    l = 25
    ctx = K()
    Y = ctx.sketch(_t(p.X), p.sigma, l, seed=11).cpu().numpy()
    ref = O.sketch(p.X, p.sigma, O.omega(11, l, p.n))
    assert _relcols(Y, ref).max() <= 1e-5


def test_qrcp_pivots_on_shared_sketch(K):
    p = synth.small(n=1500)
    l, k = 40, 35
    Y = O.sketch(p.X, p.sigma, O.omega(3, l, p.n)).astype(np.float32)
    ctx = K()
    piv, rd = ctx.qrcp(_t(Y), k)
    piv, rd = piv.cpu().numpy(), rd.cpu().numpy()
    # pivots are argmax decisions taken in FP32: replay the GPU's sequence through the
    # FP64 greedy rule; every choice must be maximal up to FP32 rounding of the residuals
    got, best = O.qrcp_replay(Y.T.astype(np.float64), piv)
    tol = 1e-5 * best[0]
    assert len(set(piv.tolist())) == k
    assert np.all(got >= best - tol)
    np.testing.assert_allclose(rd, got, rtol=0, atol=tol)
    # where the FP64 rule has a clear winner, the choice is unique and must agree
    ref_p, _, gap = O.qrcp_greedy(Y.T.astype(np.float64), k)
    upto = int(np.argmax(gap < 1e-3)) if np.any(gap < 1e-3) else k
    assert np.array_equal(piv[:upto], ref_p[:upto])


def test_qrcp_pivots_across_panels(K):
    # three panels of the blocked pivoted QR (l = 100, k = 90) on rows with a decaying
    # spectrum: the GPU's pivots replayed through the FP64 greedy rule are maximal within
    # FP32 rounding, |R_jj| match, and agree with the FP64 choice wherever it is clear
    rng = np.random.Generator(np.random.PCG64(17))
    l, n, k = 100, 5000, 90
    Y = (rng.normal(size=(n, l)) @ np.diag(np.logspace(0, -4, l))).astype(np.float32)
    ctx = K()
    piv, rd = ctx.qrcp(_t(Y), k)
    piv, rd = piv.cpu().numpy(), rd.cpu().numpy()
    got, best = O.qrcp_replay(Y.T.astype(np.float64), piv)
    tol = 1e-5 * best[0]
    assert len(set(piv.tolist())) == k
    assert np.all(got >= best - tol)
    np.testing.assert_allclose(rd, got, rtol=0, atol=tol)
    ref_p, _, gap = O.qrcp_greedy(Y.T.astype(np.float64), k)
    upto = int(np.argmax(gap < 1e-3)) if np.any(gap < 1e-3) else k
    assert np.array_equal(piv[:upto], ref_p[:upto])


def _kahan(n, c):
    s = np.sqrt(1 - c * c)
    return np.diag(s ** np.arange(n)) @ (np.eye(n) + np.triu(-c * np.ones((n, n)), 1))


def test_strong_rrqr_on_kahan_matrix(K):
    # Kahan's matrix (30 x 30, c = 0.285; columns scaled by 1 - 1e-4 j so that pivoting keeps
    # their order in FP32): pivoted QR leaves max |R11^{-1} R12| = 318 and r_nn = 0.29 while
    # sigma_n / sigma_1 = 1e-4.  The GPU's strong RRQR (f = 2) must swap, end with the
    # Gu-Eisenstat measure within f, and its pivots must reveal the rank in FP64: the
    # oracle's QR of the permuted matrix has |R11^{-1} R12| <= f and a trailing |r_nn| within
    # sigma_n sqrt(1 + f^2 k (n - k))
    import scipy.linalg as sla
    n, k, f = 30, 29, 2.0
    A = _kahan(n, 0.285) @ np.diag(1 - 1e-4 * np.arange(n))
    Y = A.T.astype(np.float32)                     # rows of Y = columns of A (points)
    ctx = K()
    piv0, _ = ctx.qrcp(_t(Y), k)
    assert np.array_equal(piv0.cpu().numpy(), np.arange(k))
    piv, rd, swaps, rho = ctx.strong_rrqr(_t(Y), k, f)
    piv = piv.cpu().numpy()
    print(f"Kahan: {swaps} swaps, rho {rho:.3f}")
    assert swaps >= 1 and rho <= f * (1 + 1e-3)
    assert len(set(piv.tolist())) == k
    rest = np.setdiff1d(np.arange(n), piv)
    A64 = Y.T.astype(np.float64)
    R = np.linalg.qr(A64[:, np.concatenate([piv, rest])], mode="r")
    W = sla.solve_triangular(R[:k, :k], R[:k, k:])
    assert np.abs(W).max() <= f * (1 + 1e-2)
    sig = np.linalg.svd(A64, compute_uv=False)
    assert abs(R[-1, -1]) <= sig[-1] * np.sqrt(1 + f * f * k * (n - k)) * (1 + 1e-2)
    np.testing.assert_allclose(rd.cpu().numpy(), np.abs(np.diag(R)[:k]), rtol=1e-3)


def test_strong_rrqr_on_a_kernel_sketch_keeps_the_pivots(K):
    # Section 3's remark: on a Gaussian kernel sketch pivoted QR already meets the strong
    # conditions with f = 2, so the strong RRQR makes no swap and keeps the pivots; a build
    # with strong_f = 2 ends within f (its FP32 sketch of 105 projections for 100 anchors
    # may need a swap near the end of R11) and solves as usual
    p = synth.small(n=1500)
    l, k = 40, 35
    Y = O.sketch(p.X, p.sigma, O.omega(3, l, p.n)).astype(np.float32)
    ctx = K()
    piv0, _ = ctx.qrcp(_t(Y), k)
    piv, _, swaps, rho = ctx.strong_rrqr(_t(Y), k, 2.0)
    assert swaps == 0 and rho <= 2.0
    assert np.array_equal(piv.cpu().numpy(), piv0.cpu().numpy())
    q = synth.small()
    ctx2 = K(strong_f=2.0)
    ctx2.build(_t(q.X), q.sigma, q.beta, q.k, seed=1)
    sw, rho2 = ctx2.anchor_stats()
    print(f"build with strong RRQR: {sw} swaps, rho {rho2:.3f}")
    assert 0.0 < rho2 <= 2.0 * (1 + 1e-3)
    alpha, info = ctx2.solve(_t(q.Y), tol=q.tol)
    r = O.residual(q.X, alpha.cpu().numpy(), q.Y, q.sigma, q.beta)
    assert np.linalg.norm(r) / np.linalg.norm(q.Y) <= 1e-6


def test_qrcp_pivots_distinct_gaps(K):
    # columns with well separated norms along orthogonal directions: a unique order
    rng = np.random.Generator(np.random.PCG64(4))
    l, n, k = 24, 3000, 20
    Q, _ = np.linalg.qr(rng.normal(size=(l, l)))
    Y = (rng.normal(size=(n, l)) * 1e-3).astype(np.float64)
    rows = rng.choice(n, k, replace=False)
    for j, i in enumerate(rows):
        Y[i] = Q[:, j] * (10.0 - 0.4 * j)
    Y = Y.astype(np.float32)
    ctx = K()
    piv, rd = ctx.qrcp(_t(Y), k)
    assert np.array_equal(piv.cpu().numpy(), rows)
    ref_p, ref_n, _ = O.qrcp_greedy(Y.T.astype(np.float64), k)
    assert np.array_equal(ref_p, rows)
    np.testing.assert_allclose(rd.cpu().numpy(), ref_n, rtol=1e-5)


# ------------------------------------------------------------------ Algorithms 3-4
def test_precond_apply_matches_oracle_with_shared_anchors(K):
    p = synth.small(n=1200, k=60)
    ctx = K()
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=5)
    S = ctx.anchors().cpu().numpy()
    assert len(S) == p.k
    M = O.Nystrom(p.X, S, p.sigma, p.beta)
    x = np.random.Generator(np.random.PCG64(2)).normal(size=(p.n, 2)).astype(np.float32)
    z = ctx.apply_precond(_t(x)).cpu().numpy().astype(np.float64)
    ref = np.stack([M.apply(x[:, 0]), M.apply(x[:, 1])], axis=1)
    # Backward error.  The GPU stores F = C L1^{-T} in FP32 (kernel values within 4u,
    # u = 2^-24, L1^{-T} rounded once, k-term FP32 sums) and forms z = (x - F v) / beta
    # with a k-term FP32 sum and one FP32 subtraction; the k x k solves are FP64.  To first
    # order z is then the exact Woodbury apply of F^ = F + E with ||E|| <= (k + 5) u ||F||,
    # perturbed by the F v sum: (K~ + beta I) z - x has norm at most
    #   eta (||K~|| + beta) ||z||,   eta = (2 (k + 5) + (k + 2)) u,
    # against the oracle's K~ on the same anchors (Eq. (7)).
    Kt = M.ktilde()
    nrmA = np.linalg.norm(Kt, 2) + p.beta
    k = len(S)
    eta = (2 * (k + 5) + (k + 2)) * 2.0 ** -24
    res = Kt @ z + p.beta * z - x
    back = np.linalg.norm(res, axis=0) / (nrmA * np.linalg.norm(z, axis=0))
    print(f"apply backward error {back.max():.3e} (bound {eta:.3e})")
    assert back.max() <= eta
    # Forward error follows: ||z - z*|| / ||z*|| <= cond(K~ + beta I) eta, with
    # cond = (||K~|| + beta) / beta (the u ||K~|| / beta scale of an FP32 apply).
    fwd = _relcols(z, ref).max()
    print(f"apply forward error {fwd:.3e} (bound {nrmA / p.beta * eta:.3e})")
    assert fwd <= nrmA / p.beta * eta


def test_anchor_quality_close_to_oracle(K):
    p = synth.small(n=1000, k=50)
    ctx = K()
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=5)
    S = ctx.anchors().cpu().numpy()
    Kfull = O.kernel_matrix(p.X, p.X, p.sigma)
    err_gpu = np.linalg.norm(Kfull - O.Nystrom(p.X, S, p.sigma, p.beta).ktilde(), 2)
    S_or = O.anchor_selection(p.X, p.sigma, p.k, p.l, seed=5)
    err_or = np.linalg.norm(Kfull - O.Nystrom(p.X, S_or, p.sigma, p.beta).ktilde(), 2)
    assert err_gpu <= 2.0 * err_or


@pytest.mark.parametrize("sparse_r", [0, 8])
def test_gpu_anchors_meet_the_corollary_condition_bound(K, sparse_r):
    # the anchors the GPU picks (Algorithm 1 or 2) precondition K + beta I below the
    # Corollary 4.10 bound 1 + 2 lambda_{k+1} sqrt(4k(n-k)+1) / beta, and far below
    # the unpreconditioned condition number
    p = synth.small(n=800, k=40)
    ctx = K(sparse_r=sparse_r)
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=4)
    S = ctx.anchors().cpu().numpy()
    Kf = O.kernel_matrix(p.X, p.X, p.sigma)
    lam = np.linalg.eigvalsh(Kf)[::-1]
    mu = O.preconditioned_spectrum(Kf, O.Nystrom(p.X, S, p.sigma, p.beta).ktilde(), p.beta)
    cond = mu.max() / mu.min()
    assert cond <= O.cond_bound_id(lam[len(S)], len(S), p.n, p.beta)
    assert cond < 0.1 * (lam[0] + p.beta) / (lam[-1] + p.beta)


def test_condition_estimate_from_pcg_coefficients(K):
    # Section 5.1's quantity from the solve: the extreme Ritz values of the Lanczos
    # tridiagonal that column 0's CG coefficients define bound the spectrum from inside, so
    # the estimate is at most the exact condition number (oracle, FP64 generalized
    # eigenvalues on the same anchors) and, after enough steps, close to it; with
    # no_precond it estimates cond(K + beta I) itself
    p = synth.small(n=1000, k=40)
    ctx = K(inner_tol=1e-6)
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=4)
    S = ctx.anchors().cpu().numpy()
    _, info = ctx.solve(_t(p.Y), tol=1e-7)
    Kf = O.kernel_matrix(p.X, p.X, p.sigma)
    mu = O.preconditioned_spectrum(Kf, O.Nystrom(p.X, S, p.sigma, p.beta).ktilde(), p.beta)
    exact = mu.max() / mu.min()
    print(f"preconditioned: estimate {info['cond_estimate']:.4g} ({info['lanczos_steps']} steps), "
          f"exact {exact:.4g}")
    assert info["lanczos_steps"] >= 10
    assert info["cond_estimate"] <= exact * (1 + 1e-6)
    assert info["cond_estimate"] >= 0.5 * exact
    ctx2 = K(no_precond=1, inner_tol=1e-6, max_iter=20000)
    ctx2.build(_t(p.X), p.sigma, p.beta, p.k, seed=4)
    _, info2 = ctx2.solve(_t(p.Y), tol=1e-7, allow_noconv=True)
    lam = np.linalg.eigvalsh(Kf)
    exact2 = (lam[-1] + p.beta) / (lam[0] + p.beta)
    print(f"plain CG: estimate {info2['cond_estimate']:.4g} ({info2['lanczos_steps']} steps), "
          f"exact {exact2:.4g}")
    assert info2["cond_estimate"] <= exact2 * (1 + 1e-6)
    assert info2["cond_estimate"] >= 0.1 * exact2
    assert info2["cond_estimate"] > 10 * info["cond_estimate"]


# ------------------------------------------------------------------ Algorithm 5
def test_solve_small_config_vs_dense(K):
    p = synth.small()
    ctx = K()
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=1)
    alpha, info = ctx.solve(_t(p.Y), tol=p.tol)
    a = alpha.cpu().numpy()
    ref = O.solve_dense(p.X, p.Y.astype(np.float64), p.sigma, p.beta)
    r = O.residual(p.X, a, p.Y, p.sigma, p.beta)
    assert np.linalg.norm(r) / np.linalg.norm(p.Y) <= 1e-6
    assert info["rel_residual"][0] <= 1e-6
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) <= 1e-4


def test_solve_multi_rhs_and_predict(K):
    p = synth.small(n=900, k=60)
    rng = np.random.Generator(np.random.PCG64(8))
    Y = np.concatenate([p.Y, rng.normal(size=(p.n, 2))], axis=1).astype(np.float32)
    ctx = K()
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=2)
    alpha, info = ctx.solve(_t(Y), tol=1e-6)
    a = alpha.cpu().numpy()
    ref = O.solve_dense(p.X, Y.astype(np.float64), p.sigma, p.beta)
    assert _relcols(a, ref).max() <= 1e-4
    Xt = rng.uniform(0, 1, size=(200, 4)).astype(np.float32)
    a32 = a.astype(np.float32).astype(np.float64)
    f = ctx.predict(_t(Xt), alpha.float()).cpu().numpy()
    fref = O.predict(Xt, p.X, a32, p.sigma)
    # FP32 sums with cancellation: bound by the condition of each sum, sum_j K_ij |alpha_j|
    cond = O.predict(Xt, p.X, np.abs(a32), p.sigma)
    assert np.all(np.abs(f - fref) <= 1e-5 * cond)


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_full_size_mixture_sampled_residual(K, precision):
    p = synth.mixture()
    ctx = K(precision=precision)
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=1)
    alpha, info = ctx.solve(_t(p.Y), tol=p.tol)
    a = alpha.cpu().numpy()
    rows = np.random.Generator(np.random.PCG64(4)).choice(p.n, 512, replace=False)
    r = O.residual(p.X, a, p.Y, p.sigma, p.beta, rows=rows)
    # sampled estimate of ||r|| / ||y||
    assert np.linalg.norm(r) / np.linalg.norm(p.Y[rows]) <= 2e-6
    assert info["rel_residual"][0] <= 1e-6


def test_pcg_iterations_match_fp64_oracle(K):
    # one sweep to 1e-4: the FP32 path must converge about as fast as the FP64 PCG of
    # Algorithm 5 with the same anchors (an inexact preconditioner shows up here first)
    p = synth.mixture(n=5000, k=500)
    ctx = K(inner_tol=1e-4)
    ctx.build(_t(p.X), p.sigma, p.beta, p.k, seed=1)
    S = ctx.anchors().cpu().numpy()
    alpha, info = ctx.solve(_t(p.Y), tol=1e-4)
    A = O.kernel_matrix(p.X, p.X, p.sigma) + p.beta * np.eye(p.n)
    M = O.Nystrom(p.X, S, p.sigma, p.beta)
    _, it = O.pcg(lambda v: A @ v, p.Y[:, 0].astype(np.float64), M.apply, tol=1e-4,
                  replace_every=10 ** 9)
    assert info["iters"] <= int(1.2 * it) + 2
    # to 1e-6 with reliable updates: the replacements must not restart the recurrence.
    # An FP32 recurrence loses CG's superlinear tail: emulating the FP32 product,
    # preconditioner or vectors (each alone) turns 81 FP64 iterations into 105-117 at
    # n = 1e4 on this workload, so the bound allows 1.5x.
    ctx2 = K()
    ctx2.build(_t(p.X), p.sigma, p.beta, p.k, seed=1)
    _, info2 = ctx2.solve(_t(p.Y), tol=1e-6)
    _, it6 = O.pcg(lambda v: A @ v, p.Y[:, 0].astype(np.float64), M.apply, tol=1e-6,
                   replace_every=10 ** 9)
    assert info2["iters"] <= int(1.5 * it6) + 2


# ------------------------------------------------------------------ edge cases
def test_rank_deficient_points_drop_anchors(K):
    base = np.random.Generator(np.random.PCG64(1)).uniform(0, 1, size=(12, 2))
    X = np.repeat(base, 40, axis=0).astype(np.float32)
    y = np.sin(X.sum(1)).astype(np.float32)
    ctx = K()
    ctx.build(_t(X), 0.3, 0.1, 30, seed=3)
    S = ctx.anchors().cpu().numpy()
    assert len(S) <= 12
    alpha, info = ctx.solve(_t(y), tol=1e-8)
    r = O.residual(X, alpha.cpu().numpy(), y, 0.3, 0.1)
    assert np.linalg.norm(r) / np.linalg.norm(y) <= 1e-8


def test_tiny_problem_k_equals_n(K):
    X = np.array([[0.0], [1.0], [2.5]], dtype=np.float32)
    y = np.array([1.0, -2.0, 0.5], dtype=np.float32)
    ctx = K()
    ctx.build(_t(X), 0.7, 0.05, 3, seed=0)
    alpha, _ = ctx.solve(_t(y), tol=1e-10)
    np.testing.assert_allclose(alpha.cpu().numpy(), O.solve_dense(X, y, 0.7, 0.05), rtol=1e-8)


def test_bad_arguments_raise(K):
    from paper_1905_10587_gb300.api import KRRError
    ctx = K()
    X = torch.zeros((10, 2), device="cuda")
    with pytest.raises(KRRError):
        ctx.build(X, -1.0, 0.1, 3)
    with pytest.raises(KRRError):
        ctx.build(X, 1.0, 0.0, 3)
    with pytest.raises(KRRError):
        ctx.build(X, 1.0, 0.1, 11)
    with pytest.raises(KRRError):
        ctx.solve(torch.zeros(10, device="cuda"))
    with pytest.raises(KRRError):
        ctx.kmvm(X, X[:5], torch.zeros(5, device="cuda"), 1.0, beta=0.1)
