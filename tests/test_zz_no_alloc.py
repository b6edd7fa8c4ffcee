"""The allocation-free kernel product, called through the C ABI.

krr_kmvm_noalloc serves callers that may not allocate device memory (an
application whose pool owns all GPU memory, or code where cudaMalloc is not
allowed): it keeps its temporaries in a fixed device array instead.  Its result
must match the regular entry point, krr_kmvm, within the tolerance of the other
product tests (1e-5 relative per column), on two calls in a row (the second
reuses the array the first left behind), for a square product with the ridge term
and for a rectangular one with distinct row and column sets; one case is also
checked against the FP64 oracle.  This file runs last so a failure here cannot
hide another test's result.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import krr_oracle as O

pytestmark = pytest.mark.gpu


def _pts(seed, n, d):
    rng = np.random.Generator(np.random.PCG64(seed))
    return torch.from_numpy(rng.uniform(-2, 2, size=(n, d)).astype(np.float32)).cuda()


def _vec(seed, nrhs, n):
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    return torch.from_numpy(rng.normal(size=(nrhs, n)).astype(np.float32)).cuda()  # RHS-major


def _noalloc(lib, Xr, Xc, V, sigma, beta):
    nr, d = Xr.shape
    nc = Xc.shape[0]
    nrhs = V.shape[0]
    Q = torch.empty((nrhs, nr), device="cuda", dtype=torch.float32)
    need = C.c_ulonglong()
    rc = lib.krr_kmvm_noalloc(C.c_void_p(Xr.data_ptr()), nr, C.c_void_p(Xc.data_ptr()), nc, d, sigma,
                              beta, C.c_void_p(V.data_ptr()), nrhs, C.c_void_p(Q.data_ptr()),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(need))
    assert rc == 0, rc
    assert 0 < need.value <= 64 << 20
    return Q


def _regular(lib, Xr, Xc, V, sigma, beta):
    from paper_1905_10587_gb300 import _lib
    nr, d = Xr.shape
    nc = Xc.shape[0]
    nrhs = V.shape[0]
    Q = torch.empty((nrhs, nr), device="cuda", dtype=torch.float32)
    h = C.c_void_p()
    assert lib.krr_create(C.byref(h), None, C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    rc = lib.krr_kmvm(h, C.c_void_p(Xr.data_ptr()), nr, C.c_void_p(Xc.data_ptr()), nc, d, sigma, beta,
                      C.c_void_p(V.data_ptr()), nrhs, C.c_void_p(Q.data_ptr()))
    lib.krr_destroy(h)
    assert rc == _lib.KRR_OK
    return Q


def _rel(got, ref):
    g, r = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return (np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)).max()


# (seed, nr, nc, d, nrhs, sigma, beta): square with the ridge term, square without,
# and rectangular (distinct point sets, so the separate row block of the scratch is used)
CASES = [(11, 20000, 20000, 8, 1, 1.0, 1e-3), (12, 3001, 3001, 3, 5, 0.5, 0.0),
         (13, 1777, 5003, 6, 3, 0.8, 0.0)]


def test_noalloc_matches_regular_entry_on_two_calls():
    from paper_1905_10587_gb300 import _lib
    lib = _lib.load()
    for _ in range(2):                      # the second round reuses the array as left
        for seed, nr, nc, d, nrhs, sigma, beta in CASES:
            Xc = _pts(seed, nc, d)
            Xr = Xc if nr == nc else _pts(seed + 100, nr, d)
            V = _vec(seed, nrhs, nc)
            got = _noalloc(lib, Xr, Xc, V, sigma, beta)
            torch.cuda.synchronize()
            ref = _regular(lib, Xr, Xc, V, sigma, beta)
            torch.cuda.synchronize()
            assert _rel(got.cpu().numpy(), ref.cpu().numpy()) <= 1e-5


def test_noalloc_matches_the_oracle():
    from paper_1905_10587_gb300 import _lib
    lib = _lib.load()
    seed, nr, nc, d, nrhs, sigma, beta = CASES[2]
    Xc, Xr, V = _pts(seed, nc, d), _pts(seed + 100, nr, d), _vec(seed, nrhs, nc)
    got = _noalloc(lib, Xr, Xc, V, sigma, beta).cpu().numpy()
    ref = O.kmvm_rect(Xr.cpu().numpy(), Xc.cpu().numpy(), V.cpu().numpy().T.astype(np.float64), sigma)
    assert _rel(got, ref.T) <= 1e-5


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1905_10587_gb300 import _lib
    lib = _lib.load()
    n = 2_000_000          # packed points alone exceed the fixed array
    need = C.c_ulonglong()
    X = torch.zeros((n, 8), device="cuda", dtype=torch.float32)
    V = torch.zeros((1, n), device="cuda", dtype=torch.float32)
    Q = torch.empty((1, n), device="cuda", dtype=torch.float32)
    rc = lib.krr_kmvm_noalloc(C.c_void_p(X.data_ptr()), n, C.c_void_p(X.data_ptr()), n, 8, 1.0, 0.0,
                              C.c_void_p(V.data_ptr()), 1, C.c_void_p(Q.data_ptr()),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(need))
    assert rc == _lib.KRR_E_NOMEM
    assert need.value > 64 << 20
