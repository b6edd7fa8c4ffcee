"""Row-sharded PCG across ranks: the collective schedule, checked on CPU with gloo.

The multi-GPU form of the solve (Algorithm 5 with the Algorithm 4 preconditioner) splits
the rows of alpha, r, p, q and z over G ranks; every rank keeps all points.  Per iteration:
  1. all-gather p                      (n x nrhs)   -> the local row block of K p
  2. all-reduce p.q                    (nrhs)       -> step length
  3. all-reduce r.r                    (nrhs)       -> convergence test
  4. all-reduce F^T r  (Woodbury)      (k x nrhs)   -> the k x k solves, replicated
  5. all-reduce r.z                    (nrhs)       -> direction update
The build needs all-reduces of the Gram matrix F^T F (k x k).  Here two gloo ranks run that
schedule with a test-local dense product and the oracle's Nystrom factors restricted to their
rows, and the iterates must equal a single-rank run of the same recurrence (FP64, so equal up
to the summation order of the reductions).
"""
import os
import socket

import numpy as np
import pytest

from oracle import krr_oracle as O

N, D, K_ANCH, SIGMA, BETA, ITERS = 400, 3, 40, 0.6, 1e-1, 12


def _problem():
    rng = np.random.Generator(np.random.PCG64(41))
    X = rng.uniform(0, 2, size=(N, D))
    y = np.sin(X.sum(axis=1)) + rng.normal(0, 0.01, size=N)
    S = O.anchor_selection(X, SIGMA, K_ANCH, K_ANCH + 5, seed=3)
    return X, y, S


def _factors(X, S, rows):
    """Per-rank Woodbury pieces: F_local = C[rows] U^(1/2) and, after an all-reduce of
    F_local^T F_local, the Cholesky factor of G = beta I + F^T F."""
    M = O.Nystrom(X, S, SIGMA, BETA)
    F_local = M.C[rows] @ M.Uhalf
    return F_local


def _pcg_sharded(rank, world, X, y, S, allreduce, allgather):
    """The sharded recurrence; `allreduce(a)` sums a numpy array over ranks in place and
    `allgather(a)` returns the concatenation of every rank's block (row order)."""
    import scipy.linalg as sla
    n = X.shape[0]
    bounds = np.linspace(0, n, world + 1).astype(int)
    rows = np.arange(bounds[rank], bounds[rank + 1])
    K_rows = O.kernel_matrix(X[rows], X, SIGMA)          # local row block of K (stand-in)
    F = _factors(X, S, rows)
    G = F.T @ F
    allreduce(G)                                          # build: Gram matrix over all rows
    G += BETA * np.eye(G.shape[0])
    Lc = sla.cholesky(G, lower=True)

    def apply(r_loc):
        u = F.T @ r_loc
        allreduce(u)                                      # F^T r over all rows
        v = sla.cho_solve((Lc, True), u)                  # replicated k x k solve
        return (r_loc - F @ v) / BETA

    def dot(a, b):
        s = np.array([a @ b])
        allreduce(s)
        return float(s[0])

    x = np.zeros(rows.size)
    r = y[rows].copy()
    z = apply(r)
    p = z.copy()
    rz = dot(r, z)
    hist = []
    for _ in range(ITERS):
        p_full = allgather(p)                             # every rank needs all of p
        q = K_rows @ p_full + BETA * p
        a = rz / dot(p, q)
        x += a * p
        r -= a * q
        hist.append(np.sqrt(dot(r, r)))
        z = apply(r)
        rz_new = dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return allgather(x), np.array(hist)


def _single_rank(X, y, S):
    one = lambda a: a
    return _pcg_sharded(0, 1, X, y, S, one, one)


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def allreduce(a):
        t = torch.from_numpy(a)
        dist.all_reduce(t)
        a[...] = t.numpy()

    def allgather(a):
        n_loc = torch.tensor([a.shape[0]])
        sizes = [torch.zeros_like(n_loc) for _ in range(world)]
        dist.all_gather(sizes, n_loc)
        mx = int(max(s.item() for s in sizes))
        buf = torch.zeros(mx, dtype=torch.float64)
        buf[:a.shape[0]] = torch.from_numpy(a)
        parts = [torch.zeros(mx, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, buf)
        return np.concatenate([p[:int(s.item())].numpy() for p, s in zip(parts, sizes)])

    X, y, S = _problem()
    alpha, hist = _pcg_sharded(rank, world, X, y, S, allreduce, allgather)
    if rank == 0:
        np.save(out + "_alpha.npy", alpha)
        np.save(out + "_hist.npy", hist)
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_row_sharded_pcg_matches_single_rank(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "r")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    alpha2, hist2 = np.load(out + "_alpha.npy"), np.load(out + "_hist.npy")
    X, y, S = _problem()
    alpha1, hist1 = _single_rank(X, y, S)
    np.testing.assert_allclose(hist2, hist1, rtol=1e-7)
    np.testing.assert_allclose(alpha2, alpha1, rtol=1e-7, atol=1e-10)
    # and the recurrence is the oracle's textbook PCG with the same preconditioner
    M = O.Nystrom(X, S, SIGMA, BETA)
    A = O.kernel_matrix(X, X, SIGMA) + BETA * np.eye(N)
    ref, _ = O.pcg(lambda v: A @ v, y, M.apply, tol=0.0, maxiter=ITERS, replace_every=10 ** 9)
    np.testing.assert_allclose(alpha1, ref, rtol=1e-7, atol=1e-10)
