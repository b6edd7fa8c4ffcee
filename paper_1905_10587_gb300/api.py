"""Thin Python binding over the C ABI (argument marshalling only).

Every computation happens in libkrr's CUDA kernels; this module only checks
shapes, makes tensors contiguous, passes device pointers and the current CUDA
stream, and turns status codes into exceptions.  Multi-column blocks are
exchanged as (n, nrhs) tensors and handed to the library RHS-major.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L


class KRRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{L.STATUS.get(code, code)}: {msg}")
        self.code = code


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _cuda(t: torch.Tensor, dtype: torch.dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return t.contiguous()


def _cols(V: torch.Tensor, dtype: torch.dtype, name: str):
    """(n,) or (n, nrhs) -> RHS-major contiguous (nrhs, n) and a flag for 1-D input."""
    V = _cuda(V, dtype, name)
    if V.dim() == 1:
        return V.reshape(1, -1).contiguous(), True
    if V.dim() != 2:
        raise ValueError(f"{name} must be 1-D or 2-D")
    return V.t().contiguous(), False


def _uncols(Q: torch.Tensor, vec: bool) -> torch.Tensor:
    return Q.reshape(-1) if vec else Q.t()


class KRR:
    """One solver context (workspace, preconditioner state) on the current device and stream."""

    def __init__(self, stream: torch.cuda.Stream | None = None, **opts):
        self.lib = L.load()
        o = L.KrrOpts()
        self.lib.krr_default_opts(C.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.stream = stream or torch.cuda.current_stream()
        h = C.c_void_p()
        rc = self.lib.krr_create(C.byref(h), C.byref(o), C.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise KRRError(rc, "krr_create failed")
        self.h = h
        self._X = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.krr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, allow=(0,)):
        if rc not in allow:
            raise KRRError(rc, self.lib.krr_last_error(self.h).decode())
        return rc

    @property
    def launches(self) -> int:
        return int(self.lib.krr_launch_count(self.h))

    def profile(self, on: bool = True):
        self._check(self.lib.krr_profile_enable(self.h, 1 if on else 0))

    PHASES = ("kmvm", "sketch", "omega", "qrcp", "fgemm", "gram", "chol", "apply", "resid_hp",
              "cgvec", "prep")

    def phase_times(self) -> dict:
        """{phase: (total_ms, count)} of the recorded phases."""
        out = {}
        for ph in self.PHASES:
            ms, cnt = C.c_double(), C.c_longlong()
            self._check(self.lib.krr_profile_read(self.h, ph.encode(), C.byref(ms), C.byref(cnt)))
            out[ph] = (ms.value, cnt.value)
        return out

    # ---------------------------------------------------------------- products
    def kmvm(self, Xr, Xc, V, sigma: float, beta: float = 0.0) -> torch.Tensor:
        """K(Xr, Xc) V + beta V (Section 2.4, Eq. (6))."""
        Xr = _cuda(Xr, torch.float32, "Xr")
        Xc = _cuda(Xc, torch.float32, "Xc")
        Vt, vec = _cols(V, torch.float32, "V")
        Q = torch.empty((Vt.shape[0], Xr.shape[0]), device=Xr.device, dtype=torch.float32)
        self._check(self.lib.krr_kmvm(self.h, _ptr(Xr), Xr.shape[0], _ptr(Xc), Xc.shape[0],
                                      Xr.shape[1], sigma, beta, _ptr(Vt), Vt.shape[0], _ptr(Q)))
        return _uncols(Q, vec)

    def kmvm_dsigma(self, Xr, Xc, v, sigma: float) -> torch.Tensor:
        """(dK(Xr, Xc)/dlog sigma) v for one column v."""
        Xr = _cuda(Xr, torch.float32, "Xr")
        Xc = _cuda(Xc, torch.float32, "Xc")
        v = _cuda(v.reshape(-1), torch.float32, "v")
        Q = torch.empty(Xr.shape[0], device=Xr.device, dtype=torch.float32)
        self._check(self.lib.krr_kmvm_dsigma(self.h, _ptr(Xr), Xr.shape[0], _ptr(Xc), Xc.shape[0],
                                             Xr.shape[1], sigma, _ptr(v), _ptr(Q)))
        return Q

    def residual_hp(self, X, Y, A, sigma: float, beta: float, mode: str = "fp64") -> torch.Tensor:
        """Y - (K + beta I) A in FP64 ("fp64") or float-float ("ff"); A float64, Y float32."""
        X = _cuda(X, torch.float32, "X")
        Yt, vec = _cols(Y, torch.float32, "Y")
        At, _ = _cols(A, torch.float64, "A")
        R = torch.empty_like(At)
        fn = self.lib.krr_residual_ff if mode == "ff" else self.lib.krr_residual_hp
        self._check(fn(self.h, _ptr(X), X.shape[0], X.shape[1], sigma, beta,
                       _ptr(Yt), _ptr(At), Yt.shape[0], _ptr(R)))
        return _uncols(R, vec)

    # ---------------------------------------------------------------- Algorithm 1
    def omega(self, seed: int, l: int, n: int, device=None) -> torch.Tensor:
        """Omega^T (n x l) of Algorithm 1 step 1."""
        Om = torch.empty((n, l), device=device or torch.device("cuda"), dtype=torch.float32)
        self._check(self.lib.krr_omega(self.h, seed, l, n, _ptr(Om)))
        return Om

    def sketch(self, X, sigma: float, l: int, seed: int) -> torch.Tensor:
        """Y = K Omega^T (n x l) of Algorithm 1 step 2."""
        X = _cuda(X, torch.float32, "X")
        Y = torch.empty((X.shape[0], l), device=X.device, dtype=torch.float32)
        self._check(self.lib.krr_sketch(self.h, _ptr(X), X.shape[0], X.shape[1], sigma, l, seed,
                                        _ptr(Y)))
        self._X = None
        return Y

    def sparse_draw(self, seed: int, l: int, r: int, n: int, device=None):
        """Algorithm 2 steps 3-4: row indices R (l x r, int32) and Rademacher signs (l x r)."""
        dev = device or torch.device("cuda")
        R = torch.empty((l, r), device=dev, dtype=torch.int32)
        S = torch.empty((l, r), device=dev, dtype=torch.float32)
        self._check(self.lib.krr_sparse_draw(self.h, seed, l, r, n, _ptr(R), _ptr(S)))
        return R, S

    def sparse_sketch(self, X, sigma: float, l: int, r: int, seed: int) -> torch.Tensor:
        """Y (n x l) of Algorithm 2 steps 5-6: column i = K(X, X_R) v for the i-th draw."""
        X = _cuda(X, torch.float32, "X")
        Y = torch.empty((X.shape[0], l), device=X.device, dtype=torch.float32)
        self._check(self.lib.krr_sparse_sketch(self.h, _ptr(X), X.shape[0], X.shape[1], sigma, l, r,
                                               seed, _ptr(Y)))
        self._X = None
        return Y

    def qrcp(self, Y, k: int):
        """First k pivots of the column-pivoted QR of Y^T and |R_jj| (Y is consumed)."""
        Y = _cuda(Y, torch.float32, "Y").clone()
        piv = torch.empty(k, device=Y.device, dtype=torch.int32)
        rd = torch.empty(k, device=Y.device, dtype=torch.float32)
        self._check(self.lib.krr_qrcp(self.h, _ptr(Y), Y.shape[0], Y.shape[1], k, _ptr(piv), _ptr(rd)))
        return piv, rd

    def strong_rrqr(self, Y, k: int, f: float = 2.0, max_swaps: int = 64):
        """Strong RRQR (Gu-Eisenstat, bound f) of Y^T: (pivots, |R_jj|, swaps, max sqrt(rho))."""
        Y = _cuda(Y, torch.float32, "Y").clone()
        piv = torch.empty(k, device=Y.device, dtype=torch.int32)
        rd = torch.empty(k, device=Y.device, dtype=torch.float32)
        sw, rho = C.c_int(), C.c_double()
        self._check(self.lib.krr_strong_rrqr(self.h, _ptr(Y), Y.shape[0], Y.shape[1], k, f, max_swaps,
                                             _ptr(piv), _ptr(rd), C.byref(sw), C.byref(rho)))
        return piv, rd, sw.value, rho.value

    def anchor_stats(self):
        """(swaps, max sqrt(rho)) of the last build's strong RRQR ((0, 0) for pivoted QR)."""
        sw, rho = C.c_int(), C.c_double()
        self._check(self.lib.krr_anchor_stats(self.h, C.byref(sw), C.byref(rho)))
        return sw.value, rho.value

    def autotune(self, nrhs: int = 1, reps: int = 3):
        """Time the built problem's product for every candidate split (krr_autotune) and keep
        the fastest in the process-wide tuning table; returns (splits, pv_form, ms)."""
        sp, pv, ms = C.c_int(), C.c_int(), C.c_double()
        self._check(self.lib.krr_autotune(self.h, nrhs, reps, C.byref(sp), C.byref(pv), C.byref(ms)))
        return sp.value, pv.value, ms.value

    # ---------------------------------------------------------------- Algorithms 3-5
    def build(self, X, sigma: float, beta: float, k: int, seed: int = 0, anchors=None):
        """Algorithm 5 steps 1-2: anchors (Algorithm 1, or the given ones) and Algorithm 3."""
        X = _cuda(X, torch.float32, "X")
        if anchors is None:
            rc = self.lib.krr_build_precond(self.h, _ptr(X), X.shape[0], X.shape[1], sigma, beta,
                                            k, seed)
        else:
            S = _cuda(anchors, torch.int32, "anchors")
            rc = self.lib.krr_build_precond_anchors(self.h, _ptr(X), X.shape[0], X.shape[1], sigma,
                                                    beta, _ptr(S), S.numel())
        self._check(rc)
        self._X = X   # keeps the points alive: the library reads them during solves
        return self

    def anchors(self) -> torch.Tensor:
        k = C.c_int()
        self._check(self.lib.krr_get_anchors(self.h, None, C.byref(k)))
        S = torch.empty(k.value, device=self._X.device, dtype=torch.int32)
        self._check(self.lib.krr_get_anchors(self.h, _ptr(S), C.byref(k)))
        return S

    def apply_precond(self, R) -> torch.Tensor:
        """(K~ + beta I)^{-1} R (Algorithm 4)."""
        Rt, vec = _cols(R, torch.float32, "R")
        Z = torch.empty_like(Rt)
        self._check(self.lib.krr_precond_apply(self.h, _ptr(Rt), Rt.shape[0], _ptr(Z)))
        return _uncols(Z, vec)

    def solve(self, Y, tol: float = 1e-6, allow_noconv: bool = False):
        """Algorithm 5 step 3: alpha (float64) with ||Y - (K+beta I) alpha|| / ||Y|| <= tol."""
        if self._X is None:
            raise KRRError(L.KRR_E_STATE, "solve before build")
        Yt, vec = _cols(Y, torch.float32, "Y")
        A = torch.empty(Yt.shape, device=Yt.device, dtype=torch.float64)
        info = L.KrrSolveInfo()
        allow = (0, L.KRR_E_NOCONV) if allow_noconv else (0,)
        self._check(self.lib.krr_solve(self.h, _ptr(self._X), _ptr(Yt), Yt.shape[0], tol, _ptr(A),
                                       C.byref(info)), allow)
        out = dict(status=info.status, iters=info.iters, sweeps=info.sweeps, k_eff=info.k_eff,
                   rel_residual=[info.rel_residual[i] for i in range(Yt.shape[0])],
                   build_ms=info.build_ms, solve_ms=info.solve_ms, mvm_count=info.mvm_count,
                   sweep_iters=[info.sweep_iters[i] for i in range(min(8, info.sweeps + 1))],
                   sweep_residual=[info.sweep_residual[i] for i in range(min(8, info.sweeps + 1))],
                   product_form=info.product_form, restarts=info.restarts,
                   recurrence64=info.recurrence64, lanczos_steps=info.lanczos_steps,
                   cond_estimate=info.cond_estimate)
        return _uncols(A, vec), out

    def grad(self, y, Xval, yval, tol: float = 1e-8):
        """Held-out MSE and its gradient w.r.t. (log sigma, log beta, y) for the built problem.

        Returns (loss, dL/dlog sigma, dL/dlog beta, dL/dy as an FP64 tensor)."""
        if self._X is None:
            raise KRRError(L.KRR_E_STATE, "grad before build")
        y = _cuda(y.reshape(-1), torch.float32, "y")
        Xv = _cuda(Xval, torch.float32, "Xval")
        yv = _cuda(yval.reshape(-1), torch.float32, "yval")
        dy = torch.empty(y.shape[0], device=y.device, dtype=torch.float64)
        loss, ds, db = C.c_double(), C.c_double(), C.c_double()
        self._check(self.lib.krr_grad(self.h, _ptr(y), _ptr(Xv), Xv.shape[0], _ptr(yv), tol,
                                      C.byref(loss), C.byref(ds), C.byref(db), _ptr(dy)))
        return loss.value, ds.value, db.value, dy

    def predict(self, Xtest, alpha) -> torch.Tensor:
        """f = K(Xtest, X) alpha (Eq. (1))."""
        Xt = _cuda(Xtest, torch.float32, "Xtest")
        At, vec = _cols(alpha.float() if alpha.dtype != torch.float32 else alpha, torch.float32, "alpha")
        f = torch.empty((At.shape[0], Xt.shape[0]), device=Xt.device, dtype=torch.float32)
        self._check(self.lib.krr_predict(self.h, _ptr(Xt), Xt.shape[0], _ptr(At), At.shape[0], _ptr(f)))
        return _uncols(f, vec)


class ValidationLoss(torch.autograd.Function):
    """Held-out MSE of Gaussian KRR as a differentiable function of (y, log sigma, log beta).

    forward builds the preconditioner for (X, sigma, beta), solves, and runs the adjoint
    solve of krr_grad; backward hands back the stored gradients.  X, Xval, yval, k, seed
    and tol are constants (no gradient)."""

    @staticmethod
    def forward(fctx, y, log_sigma, log_beta, X, Xval, yval, k: int, seed: int = 0, tol: float = 1e-8,
                precision: int = 0):
        sigma = float(torch.exp(log_sigma.detach().double()))
        beta = float(torch.exp(log_beta.detach().double()))
        ctx = KRR(precision=precision)
        ctx.build(X, sigma, beta, k, seed)
        loss, ds, db, dy = ctx.grad(y.detach(), Xval, yval, tol)
        ctx.close()
        fctx.save_for_backward(dy)
        fctx.ds, fctx.db, fctx.ydtype = ds, db, y.dtype
        return torch.tensor(loss, dtype=torch.float64, device=y.device)

    @staticmethod
    def backward(fctx, gout):
        (dy,) = fctx.saved_tensors
        g = gout.to(torch.float64)
        gy = (g * dy).to(fctx.ydtype)
        gs = (g * fctx.ds).reshape(())
        gb = (g * fctx.db).reshape(())
        return gy, gs, gb, None, None, None, None, None, None, None


def validation_loss(y, log_sigma, log_beta, X, Xval, yval, k, seed=0, tol=1e-8, precision=0):
    """Differentiable held-out MSE (see ValidationLoss)."""
    return ValidationLoss.apply(y, log_sigma, log_beta, X, Xval, yval, k, seed, tol, precision)


def peak_probe(kind: int) -> float:
    """Measured issue rate (ops/s) of the whole GPU: 0 FFMA, 1 MUFU ex2, 2 DFMA."""
    lib = L.load()
    v = C.c_double()
    rc = lib.krr_peak_probe(kind, C.byref(v), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise KRRError(rc, "peak probe failed")
    return v.value


def batch_solve(problems, tol: float = 1e-6, seed: int = 0, workers: int = 8, grouped: bool = False,
                **opts):
    """Solve independent problems concurrently (krr_batch_solve), or in lockstep with one
    launch per step over all problems (krr_batch_solve_grouped, grouped=True).

    problems: list of (X (n, d), Y (n, nrhs) or (n,), sigma, beta, k) CUDA tensors/values,
    all with the same number of right-hand sides.  Returns (list of FP64 alpha tensors,
    list of info dicts, list of status codes)."""
    lib = L.load()
    o = L.KrrOpts()
    lib.krr_default_opts(C.byref(o))
    for k, v in opts.items():
        setattr(o, k, v)
    arr = (L.KrrProblem * len(problems))()
    keep, alphas, nrhs = [], [], None
    for i, (X, Y, sigma, beta, k) in enumerate(problems):
        X = _cuda(X, torch.float32, "X")
        Yt, vec = _cols(Y, torch.float32, "Y")
        if nrhs is None:
            nrhs = Yt.shape[0]
        elif nrhs != Yt.shape[0]:
            raise ValueError("all problems need the same number of right-hand sides")
        A = torch.empty(Yt.shape, device=Yt.device, dtype=torch.float64)
        keep += [X, Yt]
        alphas.append((A, vec))
        arr[i] = L.KrrProblem(X.data_ptr(), X.shape[0], X.shape[1], Yt.data_ptr(), sigma, beta, k,
                              A.data_ptr())
    infos = (L.KrrSolveInfo * len(problems))()
    stats = (C.c_int * len(problems))()
    torch.cuda.synchronize()
    fn = lib.krr_batch_solve_grouped if grouped else lib.krr_batch_solve
    rc = fn(arr, len(problems), nrhs, tol, seed, C.byref(o), workers, infos, stats)
    if rc not in (0, L.KRR_E_NOCONV):
        raise KRRError(rc, "batch solve failed")
    out = [_uncols(A, vec) for A, vec in alphas]
    info = [dict(status=f.status, iters=f.iters, sweeps=f.sweeps, k_eff=f.k_eff,
                 rel_residual=[f.rel_residual[j] for j in range(nrhs)], solve_ms=f.solve_ms,
                 build_ms=f.build_ms, mvm_count=f.mvm_count, product_form=f.product_form,
                 restarts=f.restarts)
            for f in infos]
    return out, info, list(stats)


def tc_selftest(variant: int = 0):
    """(mismatches, max_err) of the tcgen05 known-answer test."""
    lib = L.load()
    m, e = C.c_int(), C.c_float()
    rc = lib.krr_tc_selftest(variant, C.byref(m), C.byref(e),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise KRRError(rc, "tensor-core self-test failed to run")
    return m.value, e.value


def solve(X, y, sigma: float, beta: float, k: int, seed: int = 0, tol: float = 1e-6, **opts):
    """One-call solve through the public API.  X, y may live on the host: they are copied
    to the current CUDA device, and alpha comes back on the device of the inputs."""
    host = not X.is_cuda
    dev = torch.device("cuda")
    Xd = X.to(dev, non_blocking=True) if host else X
    yd = y.to(dev, non_blocking=True) if host else y
    ctx = KRR(**opts)
    ctx.build(Xd, sigma, beta, k, seed)
    alpha, info = ctx.solve(yd, tol)
    ctx.close()
    return (alpha.cpu() if host else alpha), info


def tune_save(path: str):
    """Write the process-wide tuning table as JSON (krr_tune_save)."""
    rc = L.load().krr_tune_save(str(path).encode())
    if rc != 0:
        raise KRRError(rc, f"cannot write {path}")


def tune_load(path: str):
    """Add the entries of a JSON tuning file to the table (krr_tune_load)."""
    rc = L.load().krr_tune_load(str(path).encode())
    if rc != 0:
        raise KRRError(rc, f"cannot read {path}")


def tune_get(key: str):
    """(splits, pv_form, ms) of one table entry, or None."""
    sp, pv, ms = C.c_int(), C.c_int(), C.c_double()
    rc = L.load().krr_tune_get(key.encode(), C.byref(sp), C.byref(pv), C.byref(ms))
    return None if rc != 0 else (sp.value, pv.value, ms.value)


def tune_set(key: str, splits: int, pv: int = 0, ms: float = 0.0):
    rc = L.load().krr_tune_set(key.encode(), splits, pv, ms)
    if rc != 0:
        raise KRRError(rc, "bad tuning entry")


def tune_clear():
    L.load().krr_tune_clear()
