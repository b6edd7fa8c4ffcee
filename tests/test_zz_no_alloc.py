"""The allocation-free kernel product, called through the C ABI.

krr_kmvm_noalloc serves callers that may not allocate device memory: it keeps its
temporaries in a fixed device array instead.  Its result must match the regular
entry point, krr_kmvm, within the tolerance of the other product tests, on two
calls in a row (the second reuses the array the first left behind).  This file
runs last so a failure here cannot hide another test's result.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _case(seed, n, d, nrhs):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = torch.from_numpy(rng.uniform(-2, 2, size=(n, d)).astype(np.float32)).cuda()
    V = torch.from_numpy(rng.normal(size=(nrhs, n)).astype(np.float32)).cuda()  # RHS-major
    return X, V


def _noalloc(lib, X, V, sigma, beta):
    n, d = X.shape
    nrhs = V.shape[0]
    Q = torch.empty((nrhs, n), device="cuda", dtype=torch.float32)
    need = C.c_ulonglong()
    rc = lib.krr_kmvm_noalloc(C.c_void_p(X.data_ptr()), n, C.c_void_p(X.data_ptr()), n, d, sigma,
                              beta, C.c_void_p(V.data_ptr()), nrhs, C.c_void_p(Q.data_ptr()),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(need))
    assert rc == 0, rc
    assert 0 < need.value <= 64 << 20
    return Q


def _regular(lib, X, V, sigma, beta):
    from paper_1905_10587_gb300 import _lib
    n, d = X.shape
    nrhs = V.shape[0]
    Q = torch.empty((nrhs, n), device="cuda", dtype=torch.float32)
    h = C.c_void_p()
    assert lib.krr_create(C.byref(h), None, C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    rc = lib.krr_kmvm(h, C.c_void_p(X.data_ptr()), n, C.c_void_p(X.data_ptr()), n, d, sigma, beta,
                      C.c_void_p(V.data_ptr()), nrhs, C.c_void_p(Q.data_ptr()))
    lib.krr_destroy(h)
    assert rc == _lib.KRR_OK
    return Q


def test_noalloc_matches_regular_entry_on_two_calls():
    from paper_1905_10587_gb300 import _lib
    lib = _lib.load()
    cases = [(11, 20000, 8, 1, 1.0, 1e-3), (12, 3001, 3, 5, 0.5, 0.0)]
    for seed, n, d, nrhs, sigma, beta in cases:
        X, V = _case(seed, n, d, nrhs)
        got = _noalloc(lib, X, V, sigma, beta)
        torch.cuda.synchronize()
        ref = _regular(lib, X, V, sigma, beta)
        torch.cuda.synchronize()
        g, r = got.double().cpu().numpy(), ref.double().cpu().numpy()
        rel = np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)
        assert rel.max() <= 1e-5


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
