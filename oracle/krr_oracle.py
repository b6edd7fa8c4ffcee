"""FP64 CPU oracle for preconditioned Gaussian kernel ridge regression.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
CPU-baseline leg of the benchmark may import this module.  The CUDA path never
imports, links or calls it, and it shares no code, table or helper with the
CUDA path; the only common input is the seeded data from ``synth``.

Everything here is plain NumPy / SciPy in float64 (plus one C helper, kmvm64.c, that
evaluates the kernel product's definition on every host core for the CPU baseline),
written to be checked by eye
against the paper (Shabat, Choshen, Ben-Or, Carmel, "Fast and Accurate Gaussian
Kernel Ridge Regression Using Matrix Decompositions for Preconditioning",
arXiv 1905.10587).  Library primitives used as single steps: numpy matmul,
numpy.linalg.eigh, scipy.linalg.cholesky / cho_solve / solve_triangular and
scipy.linalg.qr with column pivoting (LAPACK dgeqp3).

Kernel convention: K_ij = exp(-||x_i - x_j||^2 / (2 sigma^2)).  The paper's
Gaussian is exp(-||x - y||^2 / h^2) (Eq. of the discrete Gauss transform,
Section 2.4), so h = sqrt(2) sigma.  Parameters named ``h`` below are the
paper's width; everything else takes sigma.

Readings where the paper is silent or garbled (all listed in the design notes):
  * Algorithm 1 declares Omega as l x n and applies the transform along n, so
    the sketch is Y = K Omega^T (n x l) and the pivoted QR runs on Y^T (l x n).
  * Oversampling l = k + 5 (the paper's experiments, Section 5.1).
  * U^(1/2) is built from an EVD of K_SS = U^(-1), truncated at
    tau = k * eps64 * lambda_max, so that U = K_SS^+ (Section 2.2 defines the
    Nystrom U through a pseudo-inverse).
  * The Cholesky factor of Eq. (10) is taken upper triangular so that
    L^T L equals the printed product.
  * Algorithm 3, step 4 is read as Y = C U^(1/2) (n x k), the only order
    consistent with Eq. (10).
  * CG is the textbook preconditioned CG; the true residual replaces the
    recursive one every 50 iterations.
  * The random test matrix is drawn with Philox4x32-10 (Salmon et al., SC'11)
    and Box-Muller, defined in ``omega`` below; the CUDA path implements the
    same published generator independently.
  * Algorithm 2's "set R of r values chosen randomly" is drawn with replacement
    (independent uniform indices, ``sparse_draw``); the paper gives no r.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

EPS64 = np.finfo(np.float64).eps


# ----------------------------------------------------------------------------
# Kernel matrix and its products (Section 1, Eq. (1) and Remark 1.1; Section 2.4)
# ----------------------------------------------------------------------------
def sqdist(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Pairwise squared distances ||a_i - b_j||^2 from explicit differences."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    D = np.zeros((A.shape[0], B.shape[0]))
    for c in range(A.shape[1]):
        diff = A[:, c][:, None] - B[:, c][None, :]
        D += diff * diff
    return D


def kernel_matrix(A: np.ndarray, B: np.ndarray, sigma: float) -> np.ndarray:
    """K_ij = exp(-||a_i - b_j||^2 / (2 sigma^2)) (Remark 1.1; Eq. (6) with h^2 = 2 sigma^2)."""
    return np.exp(-sqdist(A, B) / (2.0 * sigma * sigma))


def kmvm(X: np.ndarray, V: np.ndarray, sigma: float, beta: float = 0.0,
         rows: np.ndarray | None = None, block: int = 16) -> np.ndarray:
    """(K + beta I) V, restricted to ``rows`` if given (the discrete Gauss transform, Eq. (6)).

    Rows are evaluated a few at a time straight from the definition, so this
    works at any n without forming K.  V is (n, nrhs) or (n,).
    """
    X = np.asarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V2 = V[:, None] if vec else V
    idx = np.arange(X.shape[0]) if rows is None else np.asarray(rows)
    out = np.empty((idx.size, V2.shape[1]))
    for s in range(0, idx.size, block):
        r = idx[s:s + block]
        out[s:s + len(r)] = kernel_matrix(X[r], X, sigma) @ V2 + beta * V2[r]
    return out[:, 0] if vec else out


_CLIB = None


def _clib():
    """The oracle's C helper (kmvm64.c, FP64, OpenMP over rows), built on first use."""
    global _CLIB
    if _CLIB is None:
        import ctypes as C
        from . import build_c
        lib = C.CDLL(build_c.build())
        lib.oracle_kmvm.restype = None
        lib.oracle_kmvm.argtypes = [C.c_void_p, C.c_longlong, C.c_int, C.c_void_p, C.c_int,
                                    C.c_double, C.c_double, C.c_void_p, C.c_longlong, C.c_void_p]
        lib.oracle_threads.restype = C.c_int
        _CLIB = lib
    return _CLIB


def oracle_threads() -> int:
    """Threads the C helper's OpenMP loops use."""
    return int(_clib().oracle_threads())


def kmvm_c(X: np.ndarray, V: np.ndarray, sigma: float, beta: float = 0.0,
           rows: np.ndarray | None = None) -> np.ndarray:
    """(K + beta I) V on ``rows`` (all rows if None): the same definition as ``kmvm``
    evaluated by the C helper on every host core (FP64, libm exp, index-order sums)."""
    import ctypes as C
    X = np.ascontiguousarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V2 = np.ascontiguousarray(V[:, None] if vec else V)
    n, d = X.shape
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    m = n if r is None else r.size
    out = np.empty((m, V2.shape[1]))
    _clib().oracle_kmvm(X.ctypes.data, n, d, V2.ctypes.data, V2.shape[1], float(sigma), float(beta),
                        None if r is None else r.ctypes.data, m, out.ctypes.data)
    return out[:, 0] if vec else out


def kmvm_rect(Xr: np.ndarray, Xc: np.ndarray, V: np.ndarray, sigma: float,
              block: int = 64) -> np.ndarray:
    """K(Xr, Xc) V for two point sets (Definition 2.1: FIG(Xc, Xr, h, V))."""
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V2 = V[:, None] if vec else V
    out = np.empty((Xr.shape[0], V2.shape[1]))
    for s in range(0, Xr.shape[0], block):
        out[s:s + block] = kernel_matrix(Xr[s:s + block], Xc, sigma) @ V2
    return out[:, 0] if vec else out


def predict(Xtest: np.ndarray, X: np.ndarray, alpha: np.ndarray, sigma: float) -> np.ndarray:
    """f(x) = sum_j k(x_j, x) alpha_j by brute force (Section 1, Eq. (1))."""
    return kmvm_rect(Xtest, X, alpha, sigma)


def solve_dense(X: np.ndarray, Y: np.ndarray, sigma: float, beta: float) -> np.ndarray:
    """alpha = (K + beta I)^{-1} y by dense Cholesky (Eq. (2))."""
    K = kernel_matrix(X, X, sigma)
    K[np.diag_indices_from(K)] += beta
    c = sla.cho_factor(K, lower=True)
    return sla.cho_solve(c, np.asarray(Y, dtype=np.float64))


def residual(X, alpha, Y, sigma, beta, rows=None) -> np.ndarray:
    """y - (K + beta I) alpha (optionally on a subset of rows)."""
    Y = np.asarray(Y, dtype=np.float64)
    r = np.arange(X.shape[0]) if rows is None else np.asarray(rows)
    return Y[r] - kmvm(X, alpha, sigma, beta, rows=r)


# ----------------------------------------------------------------------------
# Random test matrix: Philox4x32-10 counter-based generator + Box-Muller
# ----------------------------------------------------------------------------
_M0, _M1 = 0xD2511F53, 0xCD9E8D57          # Philox4x32 round multipliers
_W0, _W1 = 0x9E3779B9, 0xBB67AE85          # Philox4x32 key increments (Weyl sequence)
_MASK = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11, Section 3.3).

    Each round: (c0,c1,c2,c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
    the key is bumped by the Weyl constants between rounds.  Arguments are
    arrays (or scalars) of uint32 values; returns four uint64 arrays < 2^32.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64)
    k1 = np.asarray(k1, dtype=np.uint64)
    m = np.uint64(_MASK)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + np.uint64(_W0)) & m
            k1 = (k1 + np.uint64(_W1)) & m
        p0 = np.uint64(_M0) * c0
        p1 = np.uint64(_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & m
        hi1, lo1 = p1 >> np.uint64(32), p1 & m
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def omega(seed: int, l: int, n: int) -> np.ndarray:
    """The l x n Gaussian test matrix of Algorithm 1, step 1 (entries N(0,1)).

    Entry (a, j) comes from Philox4x32-10 with counter (j mod 2^32, j div 2^32,
    a div 2, 0) and key (seed mod 2^32, seed div 2^32).  With r0, r1 the first
    two output words, u1 = ((r0 >> 8) + 1) 2^-24 in (0, 1] and
    u2 = (r1 >> 8) 2^-24 in [0, 1) (both exact in float32), the Box-Muller pair
    sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2) gives rows 2c and 2c+1.
    """
    j = np.arange(n, dtype=np.uint64)
    out = np.empty((l, n))
    k0, k1 = seed & _MASK, (seed >> 32) & _MASK
    for c in range((l + 1) // 2):
        r0, r1, _, _ = philox4x32_10(j & np.uint64(_MASK), j >> np.uint64(32),
                                     np.full(n, c, np.uint64), np.zeros(n, np.uint64), k0, k1)
        u1 = ((r0 >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
        u2 = (r1 >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
        rad = np.sqrt(-2.0 * np.log(u1))
        out[2 * c] = rad * np.cos(2.0 * np.pi * u2)
        if 2 * c + 1 < l:
            out[2 * c + 1] = rad * np.sin(2.0 * np.pi * u2)
    return out


# ----------------------------------------------------------------------------
# Algorithm 1 (AnchorSelection)
# ----------------------------------------------------------------------------
def sketch(X: np.ndarray, sigma: float, Om: np.ndarray) -> np.ndarray:
    """Y = K Omega^T (n x l): Algorithm 1, step 2 (the transform applied to Omega)."""
    return kmvm_rect(X, X, Om.T, sigma)


def qrcp(Yt: np.ndarray, k: int):
    """Column-pivoted QR of Y^T (l x n) (Algorithm 1, step 3; pivoted QR per Section 3 remarks).

    Returns (pivots[:k], |diag R|[:k]) from LAPACK dgeqp3 (Businger-Golub:
    largest remaining column norm, first index on ties).
    """
    R, P = sla.qr(np.asarray(Yt, dtype=np.float64), mode="r", pivoting=True)
    kk = min(k, R.shape[0], R.shape[1])
    return np.asarray(P[:kk], dtype=np.int64), np.abs(np.diag(R)[:kk])


def strong_rrqr(A: np.ndarray, k: int, f: float = 2.0, max_swaps: int = 10_000):
    """Strong rank-revealing QR (Gu and Eisenstat, 1996), the factorization Section 2.3's
    interpolative-decomposition bound (Eq. (4)) assumes: start from the pivoted QR
    and, while some entry of R11^{-1} R12 or some ratio gamma_j(R22) / omega_i(R11)
    exceeds f in the combined measure
        (R11^{-1} R12)_ij^2 + (gamma_j / omega_i)^2 > f^2,
    swap column i of the leading block with column j of the trailing one (gamma_j: norm of
    column j of R22, omega_i: 1 / norm of row i of R11^{-1}).  Each swap multiplies
    |det R11| by more than f, so the loop ends.  Returns (perm, swaps): the first k
    entries of perm are the chosen columns.
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    _, P = sla.qr(A, mode="r", pivoting=True)
    perm = np.asarray(P, dtype=np.int64).copy()
    for swaps in range(max_swaps + 1):
        R = np.linalg.qr(A[:, perm], mode="r")
        R11, R12 = R[:k, :k], R[:k, k:]
        R22 = R[k:, k:]
        W = sla.solve_triangular(R11, R12)
        R11inv = sla.solve_triangular(R11, np.eye(k))
        omega = 1.0 / np.linalg.norm(R11inv, axis=1)
        gamma = np.linalg.norm(R22, axis=0) if R22.size else np.zeros(n - k)
        rho = W ** 2 + (gamma[None, :] / omega[:, None]) ** 2
        i, j = np.unravel_index(int(np.argmax(rho)), rho.shape)
        if rho[i, j] <= f * f or swaps == max_swaps:
            return perm, swaps
        perm[i], perm[k + j] = perm[k + j], perm[i]


def qrcp_greedy(Yt: np.ndarray, k: int):
    """The same pivot rule spelled out: repeatedly take the column with the largest
    residual norm and project it out of all columns (modified Gram-Schmidt).

    Returns (pivots, residual norms at selection, gap), gap[j] being the relative
    margin between the chosen and the runner-up squared norm at step j.
    """
    A = np.array(Yt, dtype=np.float64, copy=True)
    n = A.shape[1]
    chosen = np.zeros(n, dtype=bool)
    piv, nrm, gap = [], [], []
    for _ in range(min(k, A.shape[0], n)):
        s = np.einsum("ij,ij->j", A, A)
        s[chosen] = -1.0
        order = np.argsort(-s, kind="stable")
        p = int(order[0])
        second = s[order[1]] if n > 1 else 0.0
        gap.append((s[p] - max(second, 0.0)) / max(s[p], 1e-300))
        piv.append(p)
        nrm.append(math.sqrt(max(s[p], 0.0)))
        chosen[p] = True
        q = A[:, p] / math.sqrt(s[p])
        A -= np.outer(q, q @ A)
    return np.array(piv, dtype=np.int64), np.array(nrm), np.array(gap)


def qrcp_replay(Yt: np.ndarray, piv: np.ndarray):
    """Replay a given pivot sequence through the greedy rule of ``qrcp_greedy``.

    Returns, per step, the residual norm of the given pivot and the largest
    residual norm among the columns still available, so a caller can check
    that each given choice was (within its own rounding) a maximal one.
    """
    A = np.array(Yt, dtype=np.float64, copy=True)
    chosen = np.zeros(A.shape[1], dtype=bool)
    got, best = [], []
    for p in np.asarray(piv, dtype=np.int64):
        s = np.einsum("ij,ij->j", A, A)
        s[chosen] = -1.0
        got.append(math.sqrt(max(s[p], 0.0)))
        best.append(math.sqrt(max(s.max(), 0.0)))
        chosen[p] = True
        if s[p] > 0.0:
            q = A[:, p] / math.sqrt(s[p])
            A -= np.outer(q, q @ A)
    return np.array(got), np.array(best)


def anchor_selection(X: np.ndarray, sigma: float, k: int, l: int, seed: int):
    """Algorithm 1: Gaussian sketch, pivoted QR on Y^T, S = first k pivots."""
    Om = omega(seed, l, X.shape[0])
    Y = sketch(X, sigma, Om)
    S, _ = qrcp(Y.T, k)
    return S


# ----------------------------------------------------------------------------
# Algorithm 2 (SparseAnchorSelection)
# ----------------------------------------------------------------------------
SPARSE_TAG = 0x53505253   # third Philox counter word of the sparse draws ("SPRS")


def sparse_draw(seed: int, l: int, r: int, n: int):
    """Algorithm 2, steps 3-4: for each projection i a set R of r row indices and a
    Rademacher vector v.

    Entry (i, m) uses Philox4x32-10 with counter (i, m, SPARSE_TAG, 0) and key
    (seed mod 2^32, seed div 2^32); with r0, r1 the first two output words the index
    is floor(r0 n / 2^32) and the sign is +1 if the top bit of r1 is clear, else -1.
    Indices are drawn independently (with replacement): for r << n this is a set
    except for rare repeats, which then count twice.  Returns (R, v), both l x r.
    """
    i = np.repeat(np.arange(l, dtype=np.uint64), r)
    m = np.tile(np.arange(r, dtype=np.uint64), l)
    k0, k1 = seed & _MASK, (seed >> 32) & _MASK
    r0, r1, _, _ = philox4x32_10(i, m, np.full(i.shape, SPARSE_TAG, np.uint64),
                                 np.zeros(i.shape, np.uint64), k0, k1)
    R = ((r0 * np.uint64(n)) >> np.uint64(32)).astype(np.int64).reshape(l, r)
    v = np.where((r1 >> np.uint64(31)) == 0, 1.0, -1.0).reshape(l, r)
    return R, v


def sparse_sketch(X: np.ndarray, sigma: float, R: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Algorithm 2, steps 5-6: Y(:, i) = K(X, X_R) v for each projection i (n x l)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.empty((X.shape[0], R.shape[0]))
    for i in range(R.shape[0]):
        Y[:, i] = kmvm_rect(X, X[R[i]], v[i], sigma)
    return Y


def sparse_anchor_selection(X: np.ndarray, sigma: float, k: int, l: int, r: int, seed: int):
    """Algorithm 2: sparse sketch, pivoted QR on Y^T, S = first k pivots."""
    R, v = sparse_draw(seed, l, r, X.shape[0])
    S, _ = qrcp(sparse_sketch(X, sigma, R, v).T, k)
    return S


# ----------------------------------------------------------------------------
# Algorithm 3 (BuildCholesky) and Algorithm 4 (ApplyPreconditioner)
# ----------------------------------------------------------------------------
class Nystrom:
    """The preconditioner (K~ + beta I)^{-1} of Section 3 for the Nystrom approximation
    K~ = C U C^T on the anchor set S (Algorithms 3 and 4; Eqs. (7) and (10)).

    C = K(X, X_S) holds the anchor columns and U = K_SS^+ (Section 2.2 defines U through
    a pseudo-inverse).  With a symmetric square root U^{1/2} of U and F = C U^{1/2}, K~ is
    F F^T, and the Woodbury identity (Eq. (7)) turns the n x n inverse into a k x k one:
        (F F^T + beta I)^{-1} = (I - F G^{-1} F^T) / beta,   G = beta I + F^T F,
    where G is factored once by Cholesky as L^T L with L upper triangular (Eq. (10)).
    U^{1/2} comes from the eigendecomposition of K_SS, eigenvalues below
    k eps64 lambda_max being treated as zero (so U is the pseudo-inverse).
    """

    def __init__(self, X: np.ndarray, S: np.ndarray, sigma: float, beta: float):
        X = np.asarray(X, dtype=np.float64)
        self.X, self.S, self.sigma, self.beta = X, np.asarray(S), sigma, beta
        XS = X[self.S]
        Kss = kernel_matrix(XS, XS, sigma)                   # K_SS = U^{-1}
        lam, Vec = np.linalg.eigh(Kss)
        keep = lam > len(self.S) * EPS64 * lam.max()
        root = np.zeros_like(lam)
        root[keep] = 1.0 / np.sqrt(lam[keep])
        self.Uhalf = (Vec * root) @ Vec.T                    # U^{1/2}, U = K_SS^+
        self.C = kernel_matrix(X, XS, sigma)                 # C = K(X, X_S)
        F = self.C @ self.Uhalf                              # K~ = F F^T
        G = beta * np.eye(len(self.S)) + self.Uhalf @ (self.C.T @ F)   # beta I + F^T F
        self.L = sla.cholesky(G, lower=False)                # G = L^T L

    def ktilde(self) -> np.ndarray:
        F = self.C @ self.Uhalf
        return F @ F.T

    def apply(self, x: np.ndarray) -> np.ndarray:
        """(K~ + beta I)^{-1} x = (x - F G^{-1} F^T x) / beta, with F^T x = U^{1/2} (C^T x)
        and G^{-1} applied through the two triangular solves of G = L^T L."""
        x = np.asarray(x, dtype=np.float64)
        u = self.Uhalf @ (self.C.T @ x)                      # F^T x
        w = sla.solve_triangular(self.L, u, trans="T", lower=False)
        v = sla.solve_triangular(self.L, w, lower=False)     # G^{-1} F^T x
        return x / self.beta - (self.C @ (self.Uhalf @ v)) / self.beta


# ----------------------------------------------------------------------------
# Algorithm 5 (SolveKRR): preconditioned conjugate gradient
# ----------------------------------------------------------------------------
def pcg(Amul, b: np.ndarray, Minv=None, tol: float = 1e-6, maxiter: int = 10_000,
        replace_every: int = 50):
    """Textbook preconditioned CG for A x = b (Algorithm 5, step 3).

    Stops when ||b - A x|| / ||b|| <= tol (recursive residual, replaced by the
    true one every ``replace_every`` iterations).  Returns (x, iterations).
    """
    b = np.asarray(b, dtype=np.float64)
    Minv = Minv or (lambda v: v)
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0
    z = Minv(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxiter:
        q = Amul(p)
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        it += 1
        if it % replace_every == 0:
            r = b - Amul(x)
        if np.linalg.norm(r) / nb <= tol:
            break
        z = Minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


def solve_krr(X: np.ndarray, y: np.ndarray, sigma: float, beta: float, k: int,
              seed: int, oversample: int = 5, tol: float = 1e-6, maxiter: int = 10_000,
              S: np.ndarray | None = None):
    """Algorithm 5: anchors (Algorithm 1), preconditioner (Algorithm 3), PCG with Algorithm 4.

    Uses a dense K (small n).  Returns (alpha, iterations, anchors, preconditioner).
    """
    X = np.asarray(X, dtype=np.float64)
    if S is None:
        S = anchor_selection(X, sigma, k, k + oversample, seed)
    M = Nystrom(X, S, sigma, beta)
    A = kernel_matrix(X, X, sigma)
    A[np.diag_indices_from(A)] += beta
    alpha, it = pcg(lambda v: A @ v, y, M.apply, tol=tol, maxiter=maxiter)
    return alpha, it, S, M


# ----------------------------------------------------------------------------
# Gradient of the held-out MSE (closed form; the paper has no gradient)
# ----------------------------------------------------------------------------
def grad_val_mse(X, y, Xv, yv, sigma, beta):
    """L = ||K_vt alpha - y_v||^2 / m with alpha = (K + beta I)^{-1} y.

    Returns (L, dL/dlog sigma, dL/dlog beta, dL/dy) from the adjoint:
    g = 2 (f - y_v)/m, lambda = A^{-1} K_vt^T g, dL/dy = lambda,
    dL/dlog beta = -beta lambda^T alpha,
    dL/dlog sigma = g^T (K_vt o D_vt / sigma^2) alpha - lambda^T (K o D / sigma^2) alpha,
    using dK/dlog sigma = K o D / sigma^2 (D = squared distances).
    """
    X = np.asarray(X, dtype=np.float64)
    Xv = np.asarray(Xv, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    yv = np.asarray(yv, dtype=np.float64).reshape(-1)
    D = sqdist(X, X)
    K = np.exp(-D / (2 * sigma * sigma))
    Dv = sqdist(Xv, X)
    Kv = np.exp(-Dv / (2 * sigma * sigma))
    A = K + beta * np.eye(len(y))
    c = sla.cho_factor(A, lower=True)
    alpha = sla.cho_solve(c, y)
    f = Kv @ alpha
    m = len(yv)
    L = float(np.sum((f - yv) ** 2) / m)
    g = 2.0 * (f - yv) / m
    lam = sla.cho_solve(c, Kv.T @ g)
    dlogb = float(-beta * lam @ alpha)
    s2 = sigma * sigma
    dlogs = float(g @ ((Kv * Dv / s2) @ alpha) - lam @ ((K * D / s2) @ alpha))
    return L, dlogs, dlogb, lam


def val_mse(X, y, Xv, yv, sigma, beta) -> float:
    alpha = solve_dense(X, np.asarray(y, dtype=np.float64).reshape(-1), sigma, beta)
    f = kmvm_rect(Xv, X, alpha, sigma)
    return float(np.mean((f - np.asarray(yv, dtype=np.float64).reshape(-1)) ** 2))


# ----------------------------------------------------------------------------
# Theory helpers (Section 4)
# ----------------------------------------------------------------------------
def preconditioned_spectrum(K: np.ndarray, Ktilde: np.ndarray, beta: float) -> np.ndarray:
    """Eigenvalues of (K~ + beta I)^{-1}(K + beta I) as a generalized symmetric problem (Theorem 4.5)."""
    n = K.shape[0]
    return sla.eigh(K + beta * np.eye(n), Ktilde + beta * np.eye(n), eigvals_only=True)


def cond_bound_id(lam_k1: float, k: int, n: int, beta: float) -> float:
    """Corollary 4.10: cond <= 1 + 2 lambda_{k+1} sqrt(4k(n-k)+1) / beta."""
    return 1.0 + 2.0 * lam_k1 * math.sqrt(4.0 * k * (n - k) + 1.0) / beta


def condition_table(X: np.ndarray, sigma: float, beta: float, ks, seed: int = 0, l_extra: int = 5):
    """Section 5.1's experiment on a given point set: cond(K + beta I) and, for each k,
    the condition of the system preconditioned with Algorithm 1's anchors, next to the
    Corollary 4.10 bound.  Returns a list of dicts (k = 0 is the unpreconditioned row)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    K = kernel_matrix(X, X, sigma)
    lam = np.linalg.eigvalsh(K)[::-1]
    rows = [{"k": 0, "cond": (lam[0] + beta) / (max(lam[-1], 0.0) + beta), "bound": None}]
    for k in ks:
        S = anchor_selection(X, sigma, k, k + l_extra, seed)
        mu = preconditioned_spectrum(K, Nystrom(X, S, sigma, beta).ktilde(), beta)
        rows.append({"k": int(k), "cond": float(mu.max() / mu.min()),
                     "bound": cond_bound_id(float(lam[k]), int(k), n, beta)})
    return rows


def numerical_rank_bound(q, h: float, delta: float) -> int:
    """Theorem 4.4: rho_delta <= prod_i (floor(gamma q_i) + 1), gamma = (2/pi) sqrt(h^-2 ln(1/delta))."""
    gamma = (2.0 / math.pi) * math.sqrt(math.log(1.0 / delta) / (h * h))
    return int(np.prod([math.floor(gamma * qi) + 1 for qi in q]))


def tradeoff_gamma(h: float, n: float, beta: float, xi: float, Mbar: float) -> float:
    """The gamma of Corollary 4.6: (2/pi) sqrt(h^-2 ln(Mbar n / (beta (xi - 1))))."""
    return (2.0 / math.pi) * math.sqrt(math.log(Mbar * n / (beta * (xi - 1.0))) / (h * h))


def tradeoff_rank(q, h: float, n: float, beta: float, xi: float, Mbar: float) -> int:
    """Corollary 4.6, Eq. (24): k >= prod_i (floor(q_i gamma) + 1)."""
    g = tradeoff_gamma(h, n, beta, xi, Mbar)
    return int(np.prod([math.floor(qi * g) + 1 for qi in q], dtype=object))


def iters_unpreconditioned(lam1: float, beta: float, delta: float) -> float:
    """Eq. (31): i ~ -sqrt(lambda_1) ln(delta) / (2 sqrt(beta))."""
    return -math.sqrt(lam1) * math.log(delta) / (2.0 * math.sqrt(beta))


def iters_preconditioned(M: float, lam_k1: float, beta: float, delta: float) -> float:
    """Eq. (33): i = ln(delta) / ln((sqrt(beta + M lam) - sqrt(beta)) / (sqrt(beta + M lam) + sqrt(beta)))."""
    a = math.sqrt(beta + M * lam_k1)
    b = math.sqrt(beta)
    return math.log(delta) / math.log((a - b) / (a + b))
