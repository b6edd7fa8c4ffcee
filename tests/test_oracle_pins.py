"""Pins for the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula and compares it with itself: each
check goes through a different route (brute force, a closed form, a textbook
identity, a published known-answer vector, a printed worked example, an
invariant proved in the paper).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.stats as st

from oracle import krr_oracle as O
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pts(n, d, seed, scale=1.0):
    return np.random.Generator(np.random.PCG64(seed)).uniform(0, scale, size=(n, d))


# -------------------------------------------------------------- kernel matrix
def test_kernel_matrix_symmetric_unit_diag_psd():
    X = _pts(120, 3, 1)
    K = O.kernel_matrix(X, X, 0.3)
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 1.0)
    lam = np.linalg.eigvalsh(K)
    assert lam.min() >= -120 * np.finfo(float).eps * lam.max()


def test_kernel_two_points_closed_form():
    # K = [[1, e^{-delta^2/(2 sigma^2)}], [., 1]] for two points at distance delta
    X = np.array([[0.0, 0.0], [0.3, 0.4]])          # delta = 0.5
    K = O.kernel_matrix(X, X, 0.25)
    assert K[0, 1] == pytest.approx(math.exp(-0.25 / (2 * 0.0625)), rel=1e-15)


def test_kernel_translation_invariant():
    X = _pts(50, 4, 2)
    sh = np.array([3.0, -7.0, 11.0, 0.5])
    np.testing.assert_allclose(O.kernel_matrix(X, X, 0.7), O.kernel_matrix(X + sh, X + sh, 0.7),
                               rtol=0, atol=1e-13)


def test_h_convention_matches_paper_gauss_transform():
    # paper: exp(-||x-y||^2/h^2) with h = sqrt(2) sigma
    x, y, sigma = np.array([[0.1, 0.2]]), np.array([[0.5, -0.3]]), 0.4
    h = math.sqrt(2) * sigma
    assert O.kernel_matrix(x, y, sigma)[0, 0] == pytest.approx(
        math.exp(-((0.4) ** 2 + 0.5 ** 2) / h ** 2), rel=1e-15)


def test_kmvm_brute_force_loops():
    rng = np.random.Generator(np.random.PCG64(3))
    X = rng.normal(size=(7, 3))
    V = rng.normal(size=(7, 2))
    sigma, beta = 0.9, 0.25
    ref = np.zeros((7, 2))
    for i in range(7):
        for j in range(7):
            dd = sum((X[i, c] - X[j, c]) ** 2 for c in range(3))
            for r in range(2):
                ref[i, r] += math.exp(-dd / (2 * sigma * sigma)) * V[j, r]
        ref[i] += beta * V[i]
    np.testing.assert_allclose(O.kmvm(X, V, sigma, beta), ref, rtol=1e-14, atol=1e-14)
    rows = np.array([5, 0, 3])
    np.testing.assert_allclose(O.kmvm(X, V, sigma, beta, rows=rows), ref[rows], rtol=1e-14)
    # the C helper (every host core) against the same loops
    np.testing.assert_allclose(O.kmvm_c(X, V, sigma, beta), ref, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(O.kmvm_c(X, V, sigma, beta, rows=rows), ref[rows], rtol=1e-14)
    np.testing.assert_allclose(O.kmvm_c(X, V[:, 0], sigma, 0.0), ref[:, 0] - beta * V[:, 0],
                               rtol=1e-13, atol=1e-14)


def test_kmvm_c_helper_is_thread_count_independent():
    # each output row is summed by one thread in index order: results are bitwise
    # identical for any thread count (the helper is run in a child with 1 and 3 threads)
    import subprocess
    import sys
    code = ("import sys, numpy as np; sys.path.insert(0, %r); from oracle import krr_oracle as O; "
            "rng = np.random.Generator(np.random.PCG64(8)); X = rng.normal(size=(600, 4)); "
            "V = rng.normal(size=(600, 2)); sys.stdout.write(O.kmvm_c(X, V, 0.7, 0.1).tobytes().hex())")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        outs.append(subprocess.run([sys.executable, "-c", code % root], env=env, check=True,
                                   capture_output=True, text=True).stdout)
    assert outs[0] == outs[1] and len(outs[0]) == 600 * 2 * 16


def test_kmvm_rect_brute_force():
    rng = np.random.Generator(np.random.PCG64(4))
    A, B, v = rng.normal(size=(5, 2)), rng.normal(size=(9, 2)), rng.normal(size=9)
    ref = [sum(math.exp(-((A[i] - B[j]) ** 2).sum() / 2.0) * v[j] for j in range(9)) for i in range(5)]
    np.testing.assert_allclose(O.kmvm_rect(A, B, v, 1.0), ref, rtol=1e-14)


# ----------------------------------------------------------------- solve
def test_solve_dense_residual_and_limits():
    p = synth.small(n=300)
    a = O.solve_dense(p.X, p.Y, p.sigma, p.beta)
    r = O.residual(p.X, a, p.Y, p.sigma, p.beta)
    assert np.linalg.norm(r) / np.linalg.norm(p.Y) < 1e-12
    # beta -> infinity: alpha -> y / beta
    big = 1e9
    a2 = O.solve_dense(p.X, p.Y, p.sigma, big)
    np.testing.assert_allclose(a2 * big, p.Y.astype(float), rtol=1e-5, atol=1e-6)
    # one point: alpha = y / (1 + beta)
    a1 = O.solve_dense(np.zeros((1, 2)), np.array([3.0]), 1.0, 0.5)
    assert a1[0] == pytest.approx(2.0, rel=1e-15)


def test_predict_at_training_points_is_y_minus_beta_alpha():
    # (K + beta I) alpha = y  =>  f(x_i) = (K alpha)_i = y_i - beta alpha_i
    p = synth.small(n=250)
    a = O.solve_dense(p.X, p.Y[:, 0], p.sigma, p.beta)
    f = O.predict(p.X, p.X, a, p.sigma)
    np.testing.assert_allclose(f, p.Y[:, 0] - p.beta * a, rtol=0, atol=1e-9)


# ------------------------------------------------------------ random matrix
def test_philox_known_answer_vectors():
    rows = [ln.split() for ln in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = O.philox4x32_10(*v[0:4], v[4], v[5])
        assert [int(o) for o in out] == v[6:10]


def test_omega_counter_layout():
    # entry (0,0) with seed 0 is Box-Muller of the first two words of Philox(0; 0)
    r0, r1 = 0x6627e8d5, 0xe169c58d
    u1 = ((r0 >> 8) + 1) / 2 ** 24
    u2 = (r1 >> 8) / 2 ** 24
    om = O.omega(0, 3, 2)
    assert om[0, 0] == pytest.approx(math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2), rel=1e-14)
    assert om[1, 0] == pytest.approx(math.sqrt(-2 * math.log(u1)) * math.sin(2 * math.pi * u2), rel=1e-14)
    # the second column uses counter word 0 = 1
    w = O.philox4x32_10(1, 0, 0, 0, 0, 0)
    u1 = ((int(w[0]) >> 8) + 1) / 2 ** 24
    u2 = (int(w[1]) >> 8) / 2 ** 24
    assert om[0, 1] == pytest.approx(math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2), rel=1e-14)


def test_omega_is_standard_normal():
    om = O.omega(12345, 8, 20000)
    flat = om.ravel()
    assert abs(flat.mean()) < 0.02
    assert abs(flat.var() - 1.0) < 0.02
    assert st.kstest(flat, "norm").pvalue > 1e-3
    C = np.corrcoef(om)
    assert np.abs(C - np.eye(8)).max() < 0.05
    assert not np.array_equal(O.omega(1, 2, 10), O.omega(2, 2, 10))


# --------------------------------------------------------------- pivoted QR
def test_qrcp_matches_greedy_rule():
    rng = np.random.Generator(np.random.PCG64(7))
    A = rng.normal(size=(12, 60)) * rng.uniform(0.1, 3, size=60)
    p_lapack, rd = O.qrcp(A, 10)
    p_greedy, nrm, gap = O.qrcp_greedy(A, 10)
    upto = np.argmax(gap < 1e-8) if np.any(gap < 1e-8) else len(gap)
    assert upto >= 5
    assert np.array_equal(p_lapack[:upto], p_greedy[:upto])
    np.testing.assert_allclose(rd[:upto], nrm[:upto], rtol=1e-10)


def test_qrcp_replay_of_greedy_pivots_is_maximal():
    rng = np.random.Generator(np.random.PCG64(17))
    A = rng.normal(size=(9, 40))
    piv, nrm, _ = O.qrcp_greedy(A, 8)
    got, best = O.qrcp_replay(A, piv)
    np.testing.assert_allclose(got, best, rtol=1e-12)
    np.testing.assert_allclose(got, nrm, rtol=1e-12)
    # a non-greedy sequence is caught
    bad = piv.copy()
    bad[2], bad[5] = bad[5], bad[2]
    g2, b2 = O.qrcp_replay(A, bad)
    assert g2[2] < b2[2] * (1 - 1e-6)


def test_qrcp_picks_largest_then_orthogonal():
    # columns e1*5, e1*4 (parallel to the first), e2*3: pivots 0 then 2
    A = np.array([[5.0, 4.0, 0.0], [0.0, 0.0, 3.0]])
    p, rd = O.qrcp(A, 2)
    assert list(p) == [0, 2]
    np.testing.assert_allclose(rd, [5.0, 3.0])


# ------------------------------------------------------ Nystrom / Woodbury
def _nys_case(n=160, k=20, seed=5):
    X = _pts(n, 2, seed)
    S = O.anchor_selection(X, 0.3, k, k + 5, seed=11)
    return X, S, O.Nystrom(X, S, 0.3, 1e-2)


def test_woodbury_apply_equals_dense_inverse():
    X, S, M = _nys_case()
    K = O.kernel_matrix(X, X, 0.3)
    C = K[:, S]
    Kt = C @ np.linalg.pinv(K[np.ix_(S, S)], rcond=1e-13) @ C.T   # independent route
    x = np.random.Generator(np.random.PCG64(1)).normal(size=len(X))
    ref = np.linalg.solve(Kt + 1e-2 * np.eye(len(X)), x)
    np.testing.assert_allclose(M.apply(x), ref, rtol=1e-8, atol=1e-8 * np.abs(ref).max())


def test_nystrom_schur_and_spectrum_bounds():
    X, S, M = _nys_case()
    K = O.kernel_matrix(X, X, 0.3)
    Kt = M.ktilde()
    E = K - Kt
    lam = np.linalg.eigvalsh((E + E.T) / 2)
    assert lam.min() > -1e-10                    # Lemma 4.2: K - K~ >= 0
    nrmE = lam.max()
    mu = O.preconditioned_spectrum(K, Kt, 1e-2)  # Theorem 4.5 proof
    assert mu.min() > 1 - 1e-8
    assert mu.max() < 1 + nrmE / 1e-2 + 1e-6
    lk1 = np.linalg.eigvalsh(K)[::-1][len(S)]
    assert mu.max() / mu.min() <= O.cond_bound_id(lk1, len(S), len(X), 1e-2)


def test_all_points_as_anchors_gives_exact_inverse():
    X = _pts(40, 2, 9)
    M = O.Nystrom(X, np.arange(40), 0.2, 0.05)
    A = O.kernel_matrix(X, X, 0.2) + 0.05 * np.eye(40)
    x = np.arange(40.0)
    np.testing.assert_allclose(A @ M.apply(x), x, rtol=1e-6, atol=1e-6)


def test_rank_deficient_data_converges_in_one_step():
    # n points at only k distinct locations: rank(K) = k, K~ = K, PCG converges at once
    base = _pts(6, 2, 3)
    X = np.repeat(base, 10, axis=0)
    y = np.random.Generator(np.random.PCG64(2)).normal(size=60)
    a, it, S, M = O.solve_krr(X, y, 0.4, 0.1, k=6, seed=4, tol=1e-10)
    assert len(set(map(tuple, X[S]))) == 6
    assert it <= 2
    np.testing.assert_allclose(a, O.solve_dense(X, y, 0.4, 0.1), rtol=1e-8, atol=1e-9)


def test_svd_preconditioner_condition_number_remark():
    # best rank-k approximation => cond = 1 + lambda_{k+1}/beta exactly (Section 4 remark)
    X = _pts(90, 2, 8)
    K = O.kernel_matrix(X, X, 0.25)
    lam, V = np.linalg.eigh(K)
    lam, V = lam[::-1], V[:, ::-1]
    k, beta = 12, 0.03
    Kk = (V[:, :k] * lam[:k]) @ V[:, :k].T
    mu = O.preconditioned_spectrum(K, Kk, beta)
    assert mu.max() / mu.min() == pytest.approx(1 + lam[k] / beta, rel=1e-8)


# ------------------------------------------------------------------- PCG
def test_pcg_equals_dense_cholesky():
    p = synth.small(n=400, k=40)
    y = p.Y[:, 0].astype(float)
    a, it, S, M = O.solve_krr(p.X, y, p.sigma, p.beta, p.k, seed=7, tol=1e-12)
    ref = O.solve_dense(p.X, y, p.sigma, p.beta)
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < 1e-8
    # and the preconditioner helps: plain CG needs more iterations
    A = O.kernel_matrix(p.X, p.X, p.sigma) + p.beta * np.eye(p.n)
    _, it0 = O.pcg(lambda v: A @ v, y, None, tol=1e-12)
    assert it < it0


def test_pcg_textbook_on_spd_matrix():
    rng = np.random.Generator(np.random.PCG64(0))
    B = rng.normal(size=(30, 30))
    A = B @ B.T + 30 * np.eye(30)
    b = rng.normal(size=30)
    x, it = O.pcg(lambda v: A @ v, b, tol=1e-13)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10)
    assert it <= 30 + 5


# --------------------------------------------------------------- gradient
def test_gradient_matches_central_differences():
    rng = np.random.Generator(np.random.PCG64(21))
    n, m, d = 150, 40, 3
    X, Xv = rng.normal(size=(n, d)), rng.normal(size=(m, d))
    y, yv = np.sin(X.sum(1)), np.sin(Xv.sum(1))
    sigma, beta = 1.3, 0.05
    L, gs, gb, gy = O.grad_val_mse(X, y, Xv, yv, sigma, beta)
    assert L == pytest.approx(O.val_mse(X, y, Xv, yv, sigma, beta), rel=1e-12)
    h = 1e-4
    fd_s = (O.val_mse(X, y, Xv, yv, sigma * math.exp(h), beta)
            - O.val_mse(X, y, Xv, yv, sigma * math.exp(-h), beta)) / (2 * h)
    fd_b = (O.val_mse(X, y, Xv, yv, sigma, beta * math.exp(h))
            - O.val_mse(X, y, Xv, yv, sigma, beta * math.exp(-h))) / (2 * h)
    u = synth.rademacher_unit(n, 5)
    fd_y = (O.val_mse(X, y + h * u, Xv, yv, sigma, beta)
            - O.val_mse(X, y - h * u, Xv, yv, sigma, beta)) / (2 * h)
    assert gs == pytest.approx(fd_s, rel=1e-6)
    assert gb == pytest.approx(fd_b, rel=1e-6)
    assert gy @ u == pytest.approx(fd_y, rel=1e-6)


# ------------------------------------------------------------- theory helpers
def test_corollary_worked_examples():
    rows = [ln.split() for ln in open(os.path.join(GOLD, "tradeoff_examples.txt"))
            if ln.strip() and not ln.startswith("#")]
    for kind, h, n, beta, xi, d, q, exp in rows:
        h, n, beta, xi, d, q = float(h), float(n), float(beta), float(xi), int(d), float(q)
        if kind == "gamma":
            # the remark prints gamma to two decimals, truncated (3.346 -> 3.34)
            g = O.tradeoff_gamma(h, n, beta, xi, Mbar=n)
            assert 0.0 <= g - float(exp) < 0.01
        else:
            assert O.tradeoff_rank([q] * d, h, n, beta, xi, Mbar=n) == eval(exp)


def test_numerical_rank_helper_matches_corollary_proof():
    # Eq. (26): with delta = beta (xi - 1) / (Mbar n) (taking ||K|| = n), the
    # theorem's gamma equals the corollary's, so the two rank formulas agree.
    # (The theorem's bound is used as a formula only: on measured kernels it can be
    # exceeded, e.g. 63 > 49 for 600 points in [0,2]^2, h = 0.707, delta = 1e-6.)
    h, n, beta, xi, Mbar = 0.9, 1e5, 1e-3, 10.0, 1e5
    delta = beta * (xi - 1) / (Mbar * n)
    for q in ([1.0, 2.0], [0.5, 0.5, 3.0]):
        assert O.numerical_rank_bound(q, h, delta) == O.tradeoff_rank(q, h, n, beta, xi, Mbar)


def test_cond_bound_id_hand_worked_values():
    # Corollary 4.10: cond <= 1 + 2 lambda_{k+1} sqrt(4k(n-k)+1) / beta, worked by hand.
    # k=1, n=2, lambda=0.5, beta=1: sqrt(4*1*1+1) = sqrt(5), so 1 + 2*0.5*sqrt(5) = 1 + sqrt(5)
    assert O.cond_bound_id(0.5, 1, 2, 1.0) == pytest.approx(1.0 + math.sqrt(5.0), rel=1e-15)
    # k=2, n=4, lambda=0.25, beta=0.5: sqrt(4*2*2+1) = sqrt(17); 1 + 2*0.25*sqrt(17)/0.5
    assert O.cond_bound_id(0.25, 2, 4, 0.5) == pytest.approx(1.0 + math.sqrt(17.0), rel=1e-15)
    # k=3, n=10, lambda=1e-3, beta=1e-2: sqrt(4*3*7+1) = sqrt(85) = 9.2195...; 1 + 0.2 sqrt(85)
    assert O.cond_bound_id(1e-3, 3, 10, 1e-2) == pytest.approx(2.8439088914585776, rel=1e-14)
    # Remark 4.8: at k = n/2 the factor is sqrt(n^2+1), and the corollary's last line
    # (sqrt(4k(n-k)+1) <= n+1) bounds every k
    n, lam, beta = 6, 0.3, 0.7
    assert O.cond_bound_id(lam, 3, n, beta) == pytest.approx(1 + 2 * lam * math.sqrt(37.0) / beta)
    for k in range(0, n + 1):
        assert O.cond_bound_id(lam, k, n, beta) <= 1 + 2 * lam * (n + 1) / beta


def test_cond_bound_id_holds_for_two_points():
    # two points at distance delta: K = [[1, e], [e, 1]], e = exp(-delta^2 / (2 sigma^2)),
    # eigenvalues 1 + e and 1 - e.  One anchor (the first point) gives K~ = C C^T with
    # C = (1, e): K~ = [[1, e], [e, e^2]].  det((K + beta I) - mu (K~ + beta I)) factors as
    # (1 - mu) [(1 + beta)(1 + beta - mu (e^2 + beta)) - e^2 (1 - mu)], so the preconditioned
    # eigenvalues are 1 and ((1 + beta)^2 - e^2) / (beta (1 + beta + e^2)).
    sigma, beta = 1.0, 0.1
    for delta in (0.3, 1.0, 2.5):
        e = math.exp(-delta * delta / (2 * sigma * sigma))
        X = np.array([[0.0], [delta]])
        K = O.kernel_matrix(X, X, sigma)
        Kt = O.Nystrom(X, np.array([0]), sigma, beta).ktilde()
        mu = O.preconditioned_spectrum(K, Kt, beta)
        mu2 = ((1 + beta) ** 2 - e * e) / (beta * (1 + beta + e * e))
        assert mu.min() == pytest.approx(1.0, rel=1e-12)
        assert mu.max() == pytest.approx(mu2, rel=1e-12)
        assert mu.max() / mu.min() <= O.cond_bound_id(1 - e, 1, 2, beta)


def test_iteration_estimates_hand_worked_values():
    # Eq. (31): i = -sqrt(lambda_1) ln(delta) / (2 sqrt(beta)).
    # lambda_1 = 100, beta = 1, delta = e^-2: -10 * (-2) / 2 = 10
    assert O.iters_unpreconditioned(100.0, 1.0, math.exp(-2.0)) == pytest.approx(10.0, rel=1e-14)
    # lambda_1 = 1e4, beta = 1e-2, delta = e^-3: -100 * (-3) / (2 * 0.1) = 1500
    assert O.iters_unpreconditioned(1e4, 1e-2, math.exp(-3.0)) == pytest.approx(1500.0, rel=1e-14)
    # Eq. (33): i = ln(delta) / ln((sqrt(beta + M lam) - sqrt(beta)) / (sqrt(beta + M lam) + sqrt(beta))).
    # M lam = 8, beta = 1: sqrt(9) = 3, ratio (3-1)/(3+1) = 1/2; delta = 2^-10 gives 10
    assert O.iters_preconditioned(8.0, 1.0, 1.0, 2.0 ** -10) == pytest.approx(10.0, rel=1e-14)
    # M = 3, lam = 8, beta = 1: sqrt(25) = 5, ratio 4/6 = 2/3; delta = (2/3)^7 gives 7
    assert O.iters_preconditioned(3.0, 8.0, 1.0, (2.0 / 3.0) ** 7) == pytest.approx(7.0, rel=1e-13)
    # M lam = 3, beta = 1: sqrt(4) = 2, ratio 1/3; delta = 3^-5 gives 5 (the beta scale
    # cancels: beta = 4, M lam = 12 gives the same)
    assert O.iters_preconditioned(1.0, 3.0, 1.0, 3.0 ** -5) == pytest.approx(5.0, rel=1e-13)
    assert O.iters_preconditioned(2.0, 6.0, 4.0, 3.0 ** -5) == pytest.approx(5.0, rel=1e-13)
    # Eq. (34)'s small-M-lambda limit: the ratio of Eq. (33) tends to M lam / (4 beta)
    x = 1e-7
    assert O.iters_preconditioned(1.0, x, 1.0, 1e-6) == pytest.approx(
        math.log(1e-6) / math.log(x / 4.0), rel=1e-6)


def test_iteration_estimates_are_consistent():
    # Eq. (33) with M lambda -> large recovers the unpreconditioned estimate's order
    e1 = O.iters_unpreconditioned(1e4, 1e-2, 1e-6)
    e2 = O.iters_preconditioned(1.0, 1e4, 1e-2, 1e-6)
    assert e2 == pytest.approx(e1, rel=0.05)
    assert O.iters_preconditioned(1.0, 1e-3, 1e-2, 1e-6) < e2


# ------------------------------------------------ Algorithm 2 (sparse anchors)
def test_sparse_draw_is_uniform_rademacher_and_deterministic():
    n = 1000
    R, v = O.sparse_draw(77, 400, 50, n)
    assert R.shape == (400, 50) and v.shape == (400, 50)
    assert R.min() >= 0 and R.max() < n
    assert set(np.unique(v)) == {-1.0, 1.0}
    # indices uniform on {0..n-1}: chi-square over 10 equal bins, signs fair
    counts = np.bincount(R.ravel() * 10 // n, minlength=10)
    assert st.chisquare(counts).pvalue > 1e-3
    assert abs(v.mean()) < 0.02
    R2, v2 = O.sparse_draw(77, 400, 50, n)
    assert np.array_equal(R, R2) and np.array_equal(v, v2)
    assert not np.array_equal(O.sparse_draw(78, 4, 5, n)[0], O.sparse_draw(77, 4, 5, n)[0])


def test_sparse_draw_word_layout():
    # entry (i, m) = (2, 3): Philox counter (2, 3, tag, 0), key (seed, 0); index is the
    # high 32 bits of r0 * n, sign from the top bit of r1
    w = O.philox4x32_10(2, 3, O.SPARSE_TAG, 0, 5, 0)
    R, v = O.sparse_draw(5, 4, 6, 999)
    assert R[2, 3] == (int(w[0]) * 999) // 2 ** 32
    assert v[2, 3] == (1.0 if int(w[1]) < 2 ** 31 else -1.0)


def test_sparse_sketch_brute_force():
    X = _pts(23, 3, 31, scale=2.0)
    R, v = O.sparse_draw(9, 6, 4, 23)
    sigma = 0.7
    Y = O.sparse_sketch(X, sigma, R, v)
    for i in range(6):
        for j in range(23):
            s = 0.0
            for m in range(4):
                d2 = sum((X[j, c] - X[R[i, m], c]) ** 2 for c in range(3))
                s += math.exp(-d2 / (2 * sigma * sigma)) * v[i, m]
            assert Y[j, i] == pytest.approx(s, rel=1e-12, abs=1e-15)


def test_sparse_anchors_pick_one_point_per_cluster():
    # k distinct points, each repeated: K has rank k, every projection column lies in its
    # span, and the pivoted QR must return k points from k different clusters
    rng = np.random.Generator(np.random.PCG64(3))
    centres = rng.uniform(0, 6, size=(5, 2))
    X = np.repeat(centres, 30, axis=0)
    S = O.sparse_anchor_selection(X, 1.0, 5, 12, 4, seed=11)
    groups = S // 30
    assert len(set(groups.tolist())) == 5


def test_sparse_anchors_are_comparable_to_gaussian_ones():
    # same k: the Nystrom error of the sparse ID stays within a small factor of Algorithm 1's
    # and well below that of anchors drawn uniformly at random
    X = _pts(600, 2, 5, scale=3.0)
    sigma, k = 0.5, 40
    K = O.kernel_matrix(X, X, sigma)

    def err(S):
        C = K[:, S]
        return np.linalg.norm(K - C @ np.linalg.pinv(K[np.ix_(S, S)]) @ C.T, 2)

    e_sparse = err(O.sparse_anchor_selection(X, sigma, k, k + 5, 8, seed=2))
    e_gauss = err(O.anchor_selection(X, sigma, k, k + 5, seed=2))
    e_random = err(np.random.Generator(np.random.PCG64(0)).choice(600, k, replace=False))
    assert e_sparse <= 2 * e_gauss          # 1.69 vs 1.85 here
    assert e_sparse <= 0.5 * e_random       # uniformly random anchors: 7.1


def test_condition_table_falls_with_k_and_meets_the_corollary():
    # Section 5.1's experiment on a small synthetic set: preconditioning lowers the
    # condition number, more anchors lower it further, and each value sits under the
    # Corollary 4.10 bound
    X = _pts(400, 2, 9, scale=2.0)
    rows = O.condition_table(X, 0.4, 1e-2, (10, 30, 60), seed=1)
    conds = [r["cond"] for r in rows]
    assert conds[0] > conds[1] > conds[2] > conds[3] >= 1.0
    for r in rows[1:]:
        assert r["cond"] <= r["bound"]


# ------------------------------------------------------------- strong RRQR
def _kahan(n, c):
    s = math.sqrt(1 - c * c)
    return np.diag(s ** np.arange(n)) @ (np.eye(n) + np.triu(-c * np.ones((n, n)), 1))


def test_strong_rrqr_reveals_the_kahan_matrix_rank_where_pivoted_qr_does_not():
    # Kahan's matrix (columns scaled by 1 - 1e-10 j so that pivoting keeps their order):
    # pivoted QR leaves r_nn near 2e-2 while sigma_n is 1e-11; strong RRQR with f = 2
    # must bring the trailing block under sigma_n sqrt(1 + f^2 k (n - k)) (Gu-Eisenstat)
    n, k, f = 90, 89, 2.0
    A = _kahan(n, 0.285) @ np.diag(1 - 1e-10 * np.arange(n))
    sig = np.linalg.svd(A, compute_uv=False)
    R0, P0 = sla.qr(A, mode="r", pivoting=True)
    bound = sig[-1] * math.sqrt(1 + f * f * k * (n - k))
    assert abs(R0[-1, -1]) > 1e6 * bound
    perm, swaps = O.strong_rrqr(A, k, f)
    assert swaps >= 1
    R = np.linalg.qr(A[:, perm], mode="r")
    assert abs(R[-1, -1]) <= bound * (1 + 1e-6)


def test_strong_rrqr_meets_its_bounds_on_a_sketch():
    # on a Gaussian sketch of a kernel matrix: |R11^{-1} R12| <= f and the singular values
    # of R11 and R22 within sqrt(1 + f^2 k (n - k)) of those of A
    X = _pts(120, 2, 12, scale=2.0)
    A = O.sketch(X, 0.5, O.omega(3, 25, 120)).T          # l x n, columns = points
    k, f = 20, 2.0
    perm, _ = O.strong_rrqr(A, k, f)
    R = np.linalg.qr(A[:, perm], mode="r")
    W = sla.solve_triangular(R[:k, :k], R[:k, k:])
    assert np.abs(W).max() <= f * (1 + 1e-9)
    n = A.shape[1]
    fac = math.sqrt(1 + f * f * k * (n - k))
    sA = np.linalg.svd(A, compute_uv=False)
    s11 = np.linalg.svd(R[:k, :k], compute_uv=False)
    s22 = np.linalg.svd(R[k:, k:], compute_uv=False)
    assert np.all(s11 >= sA[:k] / fac * (1 - 1e-9))
    assert np.all(s22[:len(sA) - k] <= sA[k:k + len(s22)] * fac * (1 + 1e-9) + 1e-14)


def test_pivoted_qr_of_kernel_sketches_already_meets_strong_rrqr():
    # Section 3's remark (pivoted QR works in practice): on Gaussian kernel sketches the
    # pivoted QR's first k columns already satisfy the strong RRQR conditions with f = 2,
    # so no swap is needed and the ID bound of Eq. (4) holds for the GPU's pivot rule
    for seed, (n, d, sigma, l, k) in enumerate([(120, 2, 0.5, 25, 20), (600, 4, 0.5, 105, 100)]):
        X = np.random.Generator(np.random.PCG64(seed)).uniform(0, 2, size=(n, d))
        A = O.sketch(X, sigma, O.omega(3, l, n)).T
        _, swaps = O.strong_rrqr(A, k, 2.0)
        assert swaps == 0
