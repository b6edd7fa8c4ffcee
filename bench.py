"""Benchmark: preconditioned Gaussian KRR solve on one GB300 (or N independent replicas).

One step = the whole hot path on the resident workload: preconditioner build
(Gaussian sketch, pivoted QR anchors, Nystrom factor, Cholesky; Algorithms 1 and 3)
plus the refined PCG solve to a 1e-6 relative residual (Algorithm 5).  The default
workload is the 10-component Gaussian mixture, n = 100000, d = 8, sigma = 1,
beta = 1e-3, k = 1000 (synthetic, seeded).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "mixture"
METRIC = "KRR solve seconds to 1e-6 rel. residual; kernel-MVM pairs/s vs roofline"
L2_FLUSH_BYTES = 256 << 20


def _workload(n: int | None, rank: int):
    import synth
    kw = {} if n is None else {"n": n}
    return synth.mixture(seed=1000 + rank, **kw)


def _describe(p) -> str:
    return (f"gaussian-mixture n={p.n} d={p.d} sigma={p.sigma:g} beta={p.beta:g} k={p.k} "
            f"l={p.l} nrhs={p.nrhs} tol={p.tol:g}")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int | None):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if self.idx is not None:
            mine = [r for r in rows if r[0] == str(self.idx)]
            rows = mine or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _gpu_index(local_rank: int):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        parts = vis.split(",")
        if local_rank < len(parts) and parts[local_rank].strip().isdigit():
            return int(parts[local_rank])
        return None
    return local_rank


# ------------------------------------------------------------------ CPU oracle baseline
def _grow(fn, first: int, limit: int, budget_s: float):
    """Run fn(m) for m = first, 2 first, ... until one call takes budget_s or m reaches
    limit; return (m, seconds) of the last call."""
    m = first
    while True:
        t0 = time.perf_counter()
        fn(m)
        dt = time.perf_counter() - t0
        if dt >= budget_s or m >= limit:
            return m, dt
        m = min(limit, 2 * m)


def oracle_parts(p, budget_s: float = 3.0) -> dict:
    """Per-part costs of the FP64 oracle (every host core) on the bench workload:
    the kernel product (C helper) per row, the Gaussian sketch (Algorithm 1, l columns)
    per row, pivoted QR of Y^T (dgeqp3) per column on a column sample, the Nystrom
    factor (Algorithm 3) and one preconditioner apply (Algorithm 4) on n / 8 points."""
    from oracle import krr_oracle as O
    import scipy.linalg as sla
    rng = np.random.Generator(np.random.PCG64(7))
    X64 = p.X.astype(np.float64)
    y64 = p.Y[:, 0].astype(np.float64)
    out = {}
    m, dt = _grow(lambda m: O.kmvm_c(X64, y64, p.sigma, p.beta, rows=rng.choice(p.n, m, replace=False)),
                  256, p.n, budget_s)
    out["product_row_s"], out["product_rows"] = dt / m, m
    Om = rng.normal(size=(p.n, p.l))        # the sketch's cost does not depend on Omega's values
    m, dt = _grow(lambda m: O.kmvm_c(X64, Om, p.sigma, 0.0, rows=rng.choice(p.n, m, replace=False)),
                  8, p.n, budget_s)
    out["sketch_row_s"], out["sketch_rows"] = dt / m, m
    del Om
    m, dt = _grow(lambda m: sla.qr(rng.normal(size=(p.l, m)), mode="r", pivoting=True),
                  2048, p.n, budget_s)
    out["qr_col_s"], out["qr_cols"] = dt / m, m
    # the Nystrom factor and one apply cost O(n k^2) and O(n k): timed on n / 8 points
    # with the same k, scaled by 8
    sub = rng.choice(p.n, max(p.k + 1, p.n // 8), replace=False)
    Xs = X64[sub]
    S = rng.choice(len(sub), p.k, replace=False)
    t0 = time.perf_counter()
    M = O.Nystrom(Xs, S, p.sigma, p.beta)
    out["nystrom_s"] = (time.perf_counter() - t0) * p.n / len(sub)
    t0 = time.perf_counter()
    M.apply(y64[sub])
    out["apply_s"] = (time.perf_counter() - t0) * p.n / len(sub)
    out["nystrom_points_timed"] = len(sub)
    del M
    return out


def small_solve_timed() -> dict:
    """A complete oracle solve of the small workload (n = 2000, d = 4, k = 100): Algorithm 1
    anchors, Algorithm 3 preconditioner, PCG (Algorithm 5) with a dense FP64 product."""
    import synth
    from oracle import krr_oracle as O
    a = synth.small()
    t0 = time.perf_counter()
    alpha, its, _, _ = O.solve_krr(a.X, a.Y[:, 0], a.sigma, a.beta, a.k, seed=1, tol=a.tol)
    dt = time.perf_counter() - t0
    res = np.linalg.norm(O.residual(a.X, alpha, a.Y[:, 0], a.sigma, a.beta)) / np.linalg.norm(a.Y)
    return {"workload": "small n=2000 d=4 sigma=0.5 beta=0.01 k=100 tol=1e-6", "seconds": dt,
            "iters": its, "rel_residual": float(res)}


def oracle_estimate(p, parts: dict, products: int, refinements: int) -> float:
    """Seconds of one oracle solve of the bench workload: the build (sketch, pivoted QR,
    Nystrom factor) plus `products` kernel products and preconditioner applies and
    `refinements` true residuals (each one more product)."""
    return (p.n * parts["sketch_row_s"] + p.n * parts["qr_col_s"] + parts["nystrom_s"]
            + products * (p.n * parts["product_row_s"] + parts["apply_s"])
            + refinements * p.n * parts["product_row_s"])


def cpu_baseline(p, products: int, refinements: int, budget_s: float = 3.0) -> dict:
    from oracle import krr_oracle as O
    t0 = time.perf_counter()
    parts = oracle_parts(p, budget_s)
    small = small_solve_timed()
    est = oracle_estimate(p, parts, products, refinements)
    return {"value": est, "unit": "s", "cores": os.cpu_count(), "threads": O.oracle_threads(),
            "kind": "oracle",
            "estimate": True,
            "sample": (f"estimate for one solve of {_describe(p)}: the FP64 oracle's kernel product "
                       f"(C helper, {O.oracle_threads()} threads) timed on {parts['product_rows']} rows, "
                       f"its sketch on {parts['sketch_rows']} rows, dgeqp3 on {parts['qr_cols']} columns "
                       f"of Y^T, the Nystrom factor and one apply on n/8 points; scaled to n rows x "
                       f"({products} products + {refinements} refinement residuals), the counts of "
                       f"this run's GPU solve"),
            "parts": parts, "small_solve_timed": small,
            "elapsed_s": time.perf_counter() - t0}


# products per solve of the bench workload and true residuals, as the GPU path's
# tensor-core form measured them (the reference arm runs without the GPU line)
REF_PRODUCTS, REF_REFINEMENTS = 780, 3


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import krr_oracle as O
    p = _workload(args.n, 0)
    nsteps = args.warmup + args.steps
    per = max(0.3, min(3.0, 100.0 / max(1, nsteps) / 4))
    parts0 = oracle_parts(p, per)        # the one-time build parts, measured once
    vals = []
    for s in range(nsteps):
        # each step re-times the per-iteration parts (product rows, one apply) on a sample
        rng = np.random.Generator(np.random.PCG64(100 + s))
        X64 = p.X.astype(np.float64)
        m, dt = _grow(lambda m: O.kmvm_c(X64, p.Y[:, 0].astype(np.float64), p.sigma, p.beta,
                                         rows=rng.choice(p.n, m, replace=False)), 256, p.n, per)
        parts = dict(parts0, product_row_s=dt / m, product_rows=m)
        if s >= args.warmup:
            vals.append(oracle_estimate(p, parts, REF_PRODUCTS, REF_REFINEMENTS))
    v = float(np.mean(vals))
    small = small_solve_timed()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _describe(p), "l2": "n/a (host)"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": os.cpu_count(),
                             "threads": O.oracle_threads(), "kind": "oracle", "estimate": True,
                             "sample": (f"per step: the FP64 oracle product (C helper) timed on a row "
                                        f"sample, plus the build parts timed once (sketch rows, dgeqp3 "
                                        f"columns, Nystrom factor, one apply); scaled to one solve of "
                                        f"{REF_PRODUCTS} products and {REF_REFINEMENTS} residuals"),
                             "parts": parts0, "small_solve_timed": small},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# DRAM bytes of one product launch (dram__bytes_read.sum + dram__bytes_write.sum from one
# ncu capture of the current kernel on this workload): (form, n, d) -> bytes.  Entries are
# removed whenever the kernel changes and re-taken from a capture of the new one.  The
# V-folded tensor-core product reads both 64-wide BF16 feature sets (2 x 12.8 MB at n = 10^5)
# once from DRAM; the column features' re-reads are L2 hits.
MEASURED_TRAFFIC = {(1, 100000, 8): 25_670_144}


# ------------------------------------------------------------------ roofline of the product
def roofline(p, kms, kcnt, clocks, precision, sms):
    """ALU roofline of the kernel product (the dominant kernel of the solve).

    Per pair (i, j) and right-hand side count r: the FP32 form issues d FFMA for the
    dot product, one FADD for the norms and r FFMA on the FMA pipe plus one ex2 on the
    MUFU; the tensor-core form moves the exponent onto tcgen05 and leaves one ex2 and
    r FFMA (with one right-hand side v folded into the exponent: one ex2 and one FADD).
    Peak pairs/s = min(FMA-pipe rate / FMA ops per pair, MUFU rate), from
    the SM count x 128 FP32 lanes (resp. 32 ex2 per SM per clock on GB300) x the
    largest SM clock seen.
    """
    sm_max = (clocks.get("sm_max_mhz") or 2070.0) * 1e6
    ffma_rate = sms * 128 * sm_max
    mufu_rate = sms * 32 * sm_max
    d, nrhs = p.d, p.nrhs
    fma_per_pair = nrhs if precision == 1 else d + 1 + nrhs
    peak_pairs = min(ffma_rate / fma_per_pair, mufu_rate)
    avg_s = (kms / max(kcnt, 1)) / 1e3
    achieved = (float(p.n) * p.n / avg_s) if kcnt else None
    name = ("k_kmvm_tc<1, 16, true> (tcgen05 BF16x3 exponent GEMM with v folded into the exponent, "
            "ex2 + FADD), (K + beta I) p; the timed phase includes the v partition and the reduction"
            if precision == 1 else "k_kmvm (tiled FP32 kernel product), (K + beta I) p")
    return {"bound": "alu", "achieved": achieved / 1e9 if achieved else None,
            "peak": peak_pairs / 1e9, "unit": "Gpair/s",
            "frac": (achieved / peak_pairs) if achieved else None,
            "traffic": MEASURED_TRAFFIC.get((precision, p.n, p.d)),
            "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
            "kernel": name,
            "peak_basis": (f"derived from unit counts x max clock ({sm_max / 1e6:.0f} MHz): "
                           f"{sms} SMs x 128 FP32 lanes / {fma_per_pair} FMA-pipe ops per pair, "
                           f"{sms} SMs x 32 ex2/clk"),
            "launches": kcnt, "avg_launch_ms": avg_s * 1e3}


# ------------------------------------------------------------------ multi-rank aggregation
def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest of every rank's x (the job ends when its slowest replica ends)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_solve(max_ms: float, steps: int, world: int) -> tuple[float, float]:
    """(ms per step, seconds per solve over the whole job): each of the `world` replicas
    solves its own problem every step, so a step completes `world` solves."""
    ms_per_step = max_ms / steps
    return ms_per_step, ms_per_step / 1e3 / world


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_1905_10587_gb300.build import build
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    build()
    from paper_1905_10587_gb300 import api

    p = _workload(args.n, rank)
    X = torch.from_numpy(p.X).to(dev)
    Y = torch.from_numpy(p.Y).to(dev)
    # work-split tuning (outside the timed region): the table file from an earlier run if
    # there is one, else the product of the built problem timed for every candidate split
    tune = None
    if not args.no_autotune:
        if os.path.exists(args.tune_file):
            try:
                api.tune_load(args.tune_file)
            except api.KRRError:
                pass
        tctx = api.KRR(precision=args.precision)
        tctx.build(X, p.sigma, p.beta, p.k, seed=1)
        width = 64 if args.precision == 1 else p.X.shape[1]
        key = f"form={args.precision} w={width} r=1 lg={int(np.floor(np.log2(p.n)))}"
        got = api.tune_get(key)
        if got is None:
            tctx.autotune(nrhs=1, reps=3)
            got = api.tune_get(key)
        tctx.close()
        tune = {"key": key, "splits": got[0], "pv": got[1], "ms_when_tuned": got[2], "file": args.tune_file}
        if rank == 0:
            try:
                api.tune_save(args.tune_file)
            except api.KRRError:
                pass
    ctx = api.KRR(precision=args.precision, autotune=0 if args.no_autotune else 1)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev, dtype=torch.float32)

    def step():
        ctx.build(X, p.sigma, p.beta, p.k, seed=1)
        return ctx.solve(Y, tol=p.tol)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ctx.profile(True)
    sampler = ClockSampler(_gpu_index(local))
    sampler.start()
    launches0 = ctx.launches
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    total_ms = 0.0
    infos = []
    for _ in range(args.steps):
        flush.fill_(1.0)   # L2 flush between steps (outside the timed events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        alpha, info = step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        infos.append(info)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = ctx.launches - launches0
    clocks = sampler.stop()
    phases = ctx.phase_times()
    ctx.profile(False)

    max_ms = max_over_ranks(total_ms, dist, dev)
    ms_per_step, value = job_seconds_per_solve(max_ms, args.steps, world)

    # ---- dominant kernel: the tiled kernel product of the PCG iterations
    kms, kcnt = phases["kmvm"]
    pairs = float(p.n) * p.n * p.nrhs
    roof = roofline(p, kms, kcnt, clocks, args.precision,
                    torch.cuda.get_device_properties(dev).multi_processor_count)

    out = None
    if rank == 0:
        last = infos[-1]
        out = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
               "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
               "dtype": "f32", "data": "synthetic",
               "config": {"workload": _describe(p), "l2": "flushed between steps (256 MiB write)",
                          "precision": ("tensor-core BF16x3 exponent tiles (tcgen05), FP32 accumulation"
                                        if args.precision == 1 else "FP32 kernel tiles")
                          + "; FP64 CG scalars; float-float residual replacement",
                          "replicas": world, "work_split": tune if tune else "cost model"},
               "roofline": roof, "clocks": clocks, "gpu_launches": launches,
               "mvm_pairs_per_s": pairs * kcnt / (kms / 1e3) if kcnt else None,
               "solve": {"iters": last["iters"], "sweeps": last["sweeps"], "k_eff": last["k_eff"],
                         "mvm_count": last["mvm_count"], "rel_residual": last["rel_residual"][0],
                         "build_ms": last["build_ms"], "solve_ms": last["solve_ms"]},
               "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items() if v[1]}}

    # ---- the other precision form on the same workload and tolerance (reported beside)
    if not args.no_other_form:
        other = 1 - args.precision
        ctx2 = api.KRR(precision=other)
        ctx2.build(X, p.sigma, p.beta, p.k, seed=1)
        ctx2.solve(Y, tol=p.tol)
        torch.cuda.synchronize()
        ctx2.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx2.build(X, p.sigma, p.beta, p.k, seed=1)
        _, inf2 = ctx2.solve(Y, tol=p.tol)
        e1.record(stream)
        e1.synchronize()
        ph2 = ctx2.phase_times()
        ctx2.close()
        if out is not None:
            out["other_form"] = {
                "precision": "FP32 kernel tiles" if other == 0 else "tensor-core tiles",
                "seconds": e0.elapsed_time(e1) / 1e3, "iters": inf2["iters"],
                "rel_residual": inf2["rel_residual"][0],
                "kmvm_avg_ms": ph2["kmvm"][0] / max(ph2["kmvm"][1], 1)}

    # ---- end to end through the public API with host buffers
    if not args.no_e2e:
        Xh = torch.from_numpy(p.X).pin_memory()
        Yh = torch.from_numpy(p.Y[:, 0].copy()).pin_memory()
        e2e_ms = 0.0
        for s in range(1 + args.e2e_steps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            a, _ = api.solve(Xh, Yh, p.sigma, p.beta, p.k, seed=1, tol=p.tol, precision=args.precision)
            e1.record()
            e1.synchronize()
            if s:
                e2e_ms += e0.elapsed_time(e1)
        e2e_max = max_over_ranks(e2e_ms, dist, dev)
        if out is not None:
            out["e2e"] = {"value": job_seconds_per_solve(e2e_max, args.e2e_steps, world)[1], "unit": "s",
                          "h2d_bytes_per_step": int(Xh.numel() * 4 + Yh.numel() * 4),
                          "d2h_bytes_per_step": int(p.n * 8)}

    if out is not None and world == 1 and not args.no_extras:
        sm_hz = (clocks.get("sm_max_mhz") or 2070.0) * 1e6
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        out["batched"] = batched_extra(api, sms, sm_hz)
        out["cube_products"] = cube_extra(api, sms, sm_hz)

    if out is not None:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(p, out["solve"]["mvm_count"], out["solve"]["sweeps"])
        try:
            peaks = {}
            for kind, name in ((0, "ffma_per_s"), (1, "ex2_per_s"), (2, "dfma_per_s")):
                peaks[name] = api.peak_probe(kind)
            out["probe_peaks"] = peaks
        except Exception as e:  # pragma: no cover
            out["probe_peaks"] = {"error": str(e)}
        print(json.dumps(out))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ workloads beside the headline
def _alu_bound(sms: int, sm_hz: float, fma_ops: float) -> float:
    """Pairs/s bound of a kernel product from its FMA-pipe ops and one ex2 per pair."""
    return min(sms * 128 * sm_hz / max(fma_ops, 1e-9), sms * 32 * sm_hz)


def _form_fma_ops(form: int, d: int, nrhs: int, tc_pv: bool = True) -> float:
    """FMA-pipe operations per pair: tensor-core form r FFMA, or with blocks of 8 or 16
    right-hand sides contracted on the tensor cores 2 (the 2^15 scale and the FP16 split's
    mixed FMA), so the ex2 bounds it; FP32 expansion d + 1 + r; exact differences
    2 d + 2 + r (r right-hand sides)."""
    if form == 1:
        return 2 if (tc_pv and nrhs >= 8) else nrhs
    return d + 1 + nrhs if form == 0 else 2 * d + 2 + nrhs


def batched_extra(api, sms: int, sm_hz: float, workers: int = 8) -> dict:
    """The 64-problem batch (n log-uniform in [1e3, 5e4], d in 2..16, 8 RHS) to 1e-6: in lockstep
    with one launch per step over all problems (krr_batch_solve_grouped, tensor-core form),
    and one by one on worker threads (krr_batch_solve) in the tensor-core and FP32 forms.
    `frac` = (the batch's products timed at their ALU bounds) / (batch wall time)."""
    import torch
    import synth
    probs = synth.batched()
    dev = torch.device("cuda")
    args_ = [(torch.from_numpy(q.X).to(dev), torch.from_numpy(q.Y).to(dev), q.sigma, q.beta, max(1, q.k))
             for q in probs]
    out = {"workload": "64 problems, n log-uniform [1e3, 5e4], d in 2..16, X ~ N(0, I), 8 RHS "
                       "sin(w.x), sigma = sqrt(d), beta = 1e-3, k = min(500, n/10), tol 1e-6",
           "workers": workers}
    for prec, name, grouped in ((1, "tensor_core_grouped", True), (1, "tensor_core", False),
                                (0, "fp32", False)):
        api.batch_solve(args_[:4], tol=1e-6, seed=1, workers=workers, precision=prec, grouped=grouped)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, infos, stats = api.batch_solve(args_, tol=1e-6, seed=1, workers=workers, precision=prec,
                                          grouped=grouped)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        tmin = 0.0
        pairs = 0.0
        for q, inf in zip(probs, infos):
            pp = float(q.n) ** 2 * inf["mvm_count"]
            pairs += pp
            form = inf["product_form"]
            tmin += pp / _alu_bound(sms, sm_hz, _form_fma_ops(form, q.d, q.nrhs))
        out[name] = {"seconds": dt, "converged": sum(1 for v in stats if v == 0),
                     "max_rel_residual": max(max(i["rel_residual"]) for i in infos),
                     "iters_total": sum(i["iters"] for i in infos),
                     "escalated": sum(1 for i in infos if i["product_form"] == 2),
                     "product_pairs_per_s": pairs / dt, "frac": tmin / dt,
                     "frac_basis": "sum over problems of (pairs x products) at the product's ALU "
                                   "bound for its final form, over the batch wall time"}
    return out


def cube_extra(api, sms: int, sm_hz: float, reps: int = 3) -> dict:
    """Kernel products of the 10^6-point cube (U[0,10]^3, sigma 0.8, beta 1e-4) for 1 and
    16 right-hand sides in the tensor-core form and the exact-difference form, timed with
    CUDA events (mean of `reps` after one warm-up), against each form's ALU bound."""
    import torch
    import synth
    p = synth.cube3d(nrhs=16)
    X = torch.from_numpy(p.X).cuda()
    Y = torch.from_numpy(p.Y).cuda()
    out = {"workload": f"cube n={p.n} d={p.d} sigma={p.sigma:g} beta={p.beta:g}"}
    for prec, tc_pv in ((1, 1), (2, 1), (1, 0)):
        ctx = api.KRR(precision=prec, tc_pv=tc_pv)
        for nrhs in ((1, 16) if tc_pv else (16,)):
            V = Y[:, :nrhs].contiguous()
            ctx.kmvm(X, X, V, p.sigma, p.beta)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                ctx.kmvm(X, X, V, p.sigma, p.beta)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            rate = float(p.n) ** 2 / (ms / 1e3)
            bound = _alu_bound(sms, sm_hz, _form_fma_ops(prec, p.d, nrhs, bool(tc_pv)))
            key = f"prec{prec}_nrhs{nrhs}" + ("" if tc_pv else "_pv_fma")
            out[key] = {"ms": ms, "pairs_per_s": rate, "frac": rate / bound, "bound_pairs_per_s": bound}
        ctx.close()
    return out


# ------------------------------------------------------------------ batched workload
def run_batched(args):
    """64 independent problems (n log-uniform in [1e3, 5e4], d in 2..16, 8 RHS) solved by the
    batch executor; reported beside the main line, not as the headline."""
    import torch
    from paper_1905_10587_gb300.build import build
    build()
    from paper_1905_10587_gb300 import api
    import synth
    probs = synth.batched()
    args_ = [(torch.from_numpy(p.X).cuda(), torch.from_numpy(p.Y).cuda(), p.sigma, p.beta, max(1, p.k))
             for p in probs]
    api.batch_solve(args_[:4], tol=1e-6, seed=1, workers=args.workers, precision=args.precision,
                    grouped=args.grouped)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    alphas, infos, stats = api.batch_solve(args_, tol=1e-6, seed=1, workers=args.workers,
                                           precision=args.precision, grouped=args.grouped)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    pairs = sum(float(p.n) ** 2 for p in probs)
    print(json.dumps({"metric": "batched KRR solve seconds to 1e-6 rel. residual (64 problems)",
                      "value": dt, "unit": "s", "higher_is_better": False, "n_gpus": 1,
                      "config": {"workload": "64 problems, n log-uniform [1e3, 5e4], d in 2..16, "
                                 "X ~ N(0, I), 8 RHS sin(w.x), sigma = sqrt(d), beta = 1e-3, "
                                 "k = min(500, n/10)", "workers": args.workers,
                                 "precision": args.precision, "grouped": args.grouped},
                      "converged": sum(1 for s in stats if s == 0), "sum_n": sum(p.n for p in probs),
                      "sum_n2_pairs": pairs, "iters_total": sum(i["iters"] for i in infos),
                      "max_rel_residual": max(max(i["rel_residual"]) for i in infos)}))
    return 0


# ------------------------------------------------------------------ gradient workload
def run_gradient(args):
    """Held-out-MSE gradient (krr_grad: solve, adjoint solve, derivative products) on the
    200000 + 20000 point workload, d = 10; checked against central differences of the
    loss in log sigma and log beta.  Reported beside the main line, not as the headline."""
    import torch
    from paper_1905_10587_gb300.build import build
    build()
    from paper_1905_10587_gb300 import api
    import synth
    p = synth.gradient()
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.Y[:, 0].copy()).cuda()
    Xv = torch.from_numpy(p.Xval).cuda()
    yv = torch.from_numpy(p.yval).cuda()
    tol = 1e-6

    def grad_at(log_sigma, log_beta):
        # lambda_max(K) / beta ~ 2.6e7 here: FP64 recurrence vectors from the start
        ctx = api.KRR(precision=args.precision, max_iter=20000, recurrence=1)
        ctx.build(X, float(np.exp(log_sigma)), float(np.exp(log_beta)), p.k, seed=1)
        out = ctx.grad(y, Xv, yv, tol=tol)
        ctx.close()
        return out

    ls0, lb0 = float(np.log(p.sigma)), float(np.log(p.beta))
    grad_at(ls0, lb0)                                  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss, ds, db, dy = grad_at(ls0, lb0)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h = 1e-3
    fd_s = (grad_at(ls0 + h, lb0)[0] - grad_at(ls0 - h, lb0)[0]) / (2 * h)
    fd_b = (grad_at(ls0, lb0 + h)[0] - grad_at(ls0, lb0 - h)[0]) / (2 * h)
    print(json.dumps({"metric": "held-out MSE gradient seconds (build + solve + adjoint solve + "
                                "derivative products)", "value": dt, "unit": "s",
                      "higher_is_better": False, "n_gpus": 1,
                      "config": {"workload": f"n={p.n} train + {p.Xval.shape[0]} held-out, d={p.d}, "
                                             f"X ~ N(0, I), sigma={p.sigma:g}, beta={p.beta:g}, k={p.k}, "
                                             f"solve tol {tol:g}", "precision": args.precision},
                      "loss": loss, "dlogsigma": ds, "dlogbeta": db,
                      "fd_dlogsigma": fd_s, "fd_dlogbeta": fd_b,
                      "rel_diff_dlogsigma": abs(ds - fd_s) / max(abs(fd_s), 1e-300),
                      "rel_diff_dlogbeta": abs(db - fd_b) / max(abs(fd_b), 1e-300),
                      "fd_step": h, "dy_norm": float(dy.norm().item())}))
    return 0


# ------------------------------------------------------------------ 10^6-point cube
def run_cube(args):
    """The 10^6-point cube (U[0,10]^3, sigma 0.8, beta 1e-4, k 2000): preconditioner build and
    kernel-product throughput for 1 and 16 right-hand sides in the tensor-core and
    exact-difference forms.  Its solve to 1e-6 is out of reach in FP32 products (the FP32
    representation of K is off by about 4e-5 in norm against beta = 1e-4), so no solve time
    is claimed; a bounded solve reports the residual reached."""
    import torch
    from paper_1905_10587_gb300.build import build
    build()
    from paper_1905_10587_gb300 import api
    import synth
    p = synth.cube3d(nrhs=16)
    X = torch.from_numpy(p.X).cuda()
    Y = torch.from_numpy(p.Y).cuda()
    out = {"metric": "kernel-product pairs/s and build seconds, 10^6-point cube", "unit": "Tpair/s",
           "n_gpus": 1, "config": {"workload": f"cube n={p.n} d={p.d} sigma={p.sigma:g} beta={p.beta:g} "
                                               f"k={p.k}"}}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for prec in (1, 2):
        ctx = api.KRR(precision=prec)
        for nrhs in (1, 16):
            V = Y[:, :nrhs].contiguous()
            ctx.kmvm(X, X, V, p.sigma, p.beta)
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record()
            ctx.kmvm(X, X, V, p.sigma, p.beta)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            out[f"prec{prec}_nrhs{nrhs}"] = {"ms": ms, "pairs_per_s": float(p.n) ** 2 / (ms / 1e3) / 1e12}
        ctx.close()
    ctx = api.KRR(precision=1, max_iter=args.cube_iters)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.build(X, p.sigma, p.beta, p.k, seed=1)
    torch.cuda.synchronize()
    out["build_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, info = ctx.solve(Y[:, :1].contiguous(), tol=1e-6, allow_noconv=True)
    torch.cuda.synchronize()
    out["bounded_solve"] = {"max_iter": args.cube_iters, "seconds": time.perf_counter() - t0,
                            "iters": info["iters"], "rel_residual": info["rel_residual"][0],
                            "product_form": info["product_form"]}
    ctx.close()
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ Section 5.1 on the GPU
def run_condition(args):
    """Section 5.1's experiment at 10^4 and 10^5 points: cond(K + beta I) (plain CG) and the
    condition number of the system preconditioned with k anchors (k = 100, 500, 1000), each
    from the Lanczos tridiagonal of the solve's own CG coefficients (a lower bound that is
    tight once the extreme Ritz values have converged), with the iterations to 1e-6."""
    import torch
    from paper_1905_10587_gb300.build import build
    build()
    from paper_1905_10587_gb300 import api
    import synth
    sets = [("small recipe (U[0,1]^4, sigma 0.5, beta 1e-2)", synth.small(n=10000)),
            ("mixture recipe (8-D, sigma 1, beta 1e-3)", synth.mixture(n=10000)),
            ("mixture recipe (8-D, sigma 1, beta 1e-3)", synth.mixture(n=100000))]
    rows = []
    for name, p in sets:
        X = torch.from_numpy(p.X).cuda()
        Y = torch.from_numpy(p.Y).cuda()
        for k in (0, 100, 500, 1000):
            # no reliable-update replacement before convergence: the Lanczos estimate uses
            # the whole uninterrupted recurrence
            # anchor_rtol = 0: exactly k anchors unless a Cholesky pivot gives out (k_eff)
            ctx = api.KRR(precision=1, no_precond=1 if k == 0 else 0, max_iter=20000 if k else 3000,
                          refine_max=200, inner_tol=1e-12, anchor_rtol=0.0)
            ctx.build(X, p.sigma, p.beta, max(k, 1), seed=1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = ctx.solve(Y, tol=1e-6, allow_noconv=True)
            torch.cuda.synchronize()
            rows.append({"set": name, "n": p.n, "k": k, "k_eff": info.get("k_eff", 0) if k else 0,
                         "cond_estimate": info["cond_estimate"],
                         "lanczos_steps": info["lanczos_steps"], "iters": info["iters"],
                         "rel_residual": info["rel_residual"][0], "seconds": time.perf_counter() - t0})
            print(json.dumps(rows[-1]), flush=True)
            ctx.close()
    print(json.dumps({"metric": "condition numbers with and without the preconditioner (Section 5.1)",
                      "rows": rows}))
    return 0


def run_product(args):
    """Kernel products alone on the mixture workload (--n points, --nrhs right-hand sides,
    --precision form, P.V form from --tc-pv): --warmup untimed then --steps timed with CUDA
    events; for profiling single kernels on small cases."""
    import torch
    from paper_1905_10587_gb300.build import build
    build()
    from paper_1905_10587_gb300 import api
    p = _workload(args.n, 0)
    X = torch.from_numpy(p.X).cuda()
    rng = np.random.Generator(np.random.PCG64(7))
    V = torch.from_numpy(rng.normal(size=(p.n, args.nrhs)).astype(np.float32)).cuda()
    ctx = api.KRR(precision=args.precision, tc_pv=args.tc_pv)
    for _ in range(args.warmup):
        ctx.kmvm(X, X, V, p.sigma, p.beta)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.kmvm(X, X, V, p.sigma, p.beta)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    print(json.dumps({"metric": "kernel product ms", "value": ms, "unit": "ms", "higher_is_better": False,
                      "n": p.n, "nrhs": args.nrhs, "precision": args.precision, "tc_pv": args.tc_pv,
                      "pairs_per_s": float(p.n) ** 2 / (ms / 1e3)}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None, help="override n (smaller test runs)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-form", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and cube workloads reported beside the headline")
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1],
                    help="kernel product: 0 FP32 tiles, 1 tensor-core tiles (default)")
    ap.add_argument("--workload", default="mixture",
                    choices=["mixture", "batched", "gradient", "cube", "condition", "product"])
    ap.add_argument("--nrhs", type=int, default=16, help="product workload: right-hand sides")
    ap.add_argument("--tc-pv", type=int, default=1, choices=[0, 1, 2],
                    help="product workload: P.V form (opts.tc_pv)")
    ap.add_argument("--cube-iters", type=int, default=300)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--no-autotune", action="store_true",
                    help="split counts from the cost model instead of the tuning table")
    ap.add_argument("--tune-file", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                        ".krr_tune.json"),
                    help="JSON tuning table read before and written after tuning")
    ap.add_argument("--grouped", action="store_true",
                    help="batched workload: lockstep solve with one launch per step over all problems")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "product":
        return run_product(args)
    if args.workload == "gradient":
        return run_gradient(args)
    if args.workload == "cube":
        return run_cube(args)
    if args.workload == "condition":
        return run_condition(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
