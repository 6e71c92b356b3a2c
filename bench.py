#!/usr/bin/env python
"""Benchmark of the Chebyshev-filtered subspace iteration on GB300.

Workload ("paw96"): cubic 40-bohr PAW cell, FFT grid 96^3, G-sphere of 60005 plane waves,
2048 bands, 256 atoms x 8 projectors (N_proj = 2048), seeded synthetic inputs, Chebyshev
degree 4.  One step is one pass of Algorithm 2 through the public API: the filter of
degree 4 on all 2048 bands (cheb_filter) followed by Rayleigh-Ritz in FP64
(rayleigh_ritz); lambda_- of the next step is the largest Ritz value, and the next filter
starts from the projections P^H Y that Rayleigh-Ritz formed for the rotated block (as
Algorithm 2's loop in chebfi_solve does; the first warm-up filter forms its own).

Metric: filter band-H-applications per second = bands x degree / time inside the filter,
for the filter form given by --prec (default: the mixed form).  The FP64 form is timed on
the same workload and reported beside it.  The inputs (2 GB per wavefunction block) are
larger than the 129 MB L2, so no L2 flush is needed between timed steps.

--impl reference times the FP64 oracle (the plain numpy restatement of the method) on the
host cores on a bounded sample of the same workload, with the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Filter band-H-applies/s (mixed vs FP64 form) at <=1e-8 Ha eigenvalue error"
UNIT = "band-H-applies/s"
WORKLOAD = "paw96"
DEGREE = 4


def _traffic(tag: str):
    """DRAM bytes per launch of a kernel at the benchmark workload, from the ncu capture
    recorded in profiles/traffic_paw96.md, or None when the kernel's sources have changed
    since (the record names the files and the SHA-1 of their concatenation) or there is no
    record."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_paw96.md")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if not line.startswith("traffic:"):
            continue
        f = dict(kv.split("=", 1) for kv in line.split()[1:])
        if f.get("tag") != tag:
            continue
        if "files" not in f or "sha1" not in f or "bytes_per_launch" not in f:
            return None
        h = hashlib.sha1()
        for name in f["files"].split(","):
            src = os.path.join(ROOT, name)
            if not os.path.exists(src):
                return None
            h.update(open(src, "rb").read())
        if h.hexdigest() != f["sha1"]:
            return None
        return float(f["bytes_per_launch"])
    return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks sampler
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ multi-rank aggregation
def aggregate(filter_s: float, step_s: float, units_per_rank: float, world: int):
    """Weak scaling over independent replicas: every rank filters its own block; the job's
    time is the slowest rank's (max over ranks) and its throughput counts every rank's units.
    Returns (value, filter_s_max, step_s_max)."""
    import torch
    import torch.distributed as dist
    if world > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([filter_s, step_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        filter_s, step_s = (float(x) for x in t.tolist())
    return world * units_per_rank / filter_s, filter_s, step_s


# ------------------------------------------------------------------ CPU baseline (oracle)
def oracle_setup(cell):
    """The oracle's operator and its one-time filter setup (Section 5.1's G = P^H P and the
    reduced matrix's LU factors), FFTs on every host core; not part of any timing."""
    from oracle import chebyshev as ch
    from oracle.planewave import PWOperator
    op = PWOperator.from_cell(cell)
    op.fft_workers = os.cpu_count()
    return op, ch.filter_setup(op)


def oracle_rate(cell, nbands_sample: int, degree: int, prepared=None):
    """The FP64 oracle's Algorithm-2 filter on a sample of bands: band-applies/s, seconds."""
    import numpy as np
    from oracle import chebyshev as ch
    op, setup = prepared if prepared is not None else oracle_setup(cell)
    Y = np.asfortranarray(cell.Y0[:, :nbands_sample])
    lo, hi = 1.0, float(op.K.max()) + 10.0
    t0 = time.perf_counter()
    ch.filter_reuse(op, Y, degree, lo, hi, setup=setup)
    dt = time.perf_counter() - t0
    return nbands_sample * degree / dt, dt


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from synth import config_cell
    cell = config_cell(WORKLOAD)
    sample = args.ref_bands
    prepared = oracle_setup(cell)
    for _ in range(args.warmup):
        oracle_rate(cell, sample, DEGREE, prepared)
    rates, secs = [], []
    for _ in range(args.steps):
        r, dt = oracle_rate(cell, sample, DEGREE, prepared)
        rates.append(r)
        secs.append(dt)
    value = sample * DEGREE * args.steps / sum(secs)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD + " (96^3 grid, 60005 plane waves, 2048 projectors, PAW, degree 4)",
                   "sample": "%d of 2048 bands per step" % sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d bands x degree %d per step; the oracle's P^H P and reduced-matrix LU "
                                   "formed once before timing; FFTs (scipy) and BLAS on all %d cores"
                                   % (sample, DEGREE, cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ extra measurements
def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # lets ncu restrict a capture to the timed calls
    a.record(st)
    for _ in range(steps):
        fn()
    b_.record(st)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return a.elapsed_time(b_) / steps


def run_extra(args):
    """backward: the filter backward (gY0, gV, gD) at the differentiation workload (48^3 grid,
    8025 plane waves, 32 atoms x 8 projectors, PAW, 128 bands, degree 8), FP64 and FP32 forms;
    unit = band-steps of the adjoint recurrence per second (bands x degree / time).
    refine: S^{-1} by Section 5.1's iterative refinement against the direct Woodbury form on
    the benchmark workload's first 256 bands.
    kpoints: the batched k-point filter (64 k-points of a 48^3 PAW cell, spheres of 3000 to
    12000 plane waves, 128 bands each, FP32, degree 8) against one filter call per k-point,
    and the same batch in the mixed form (projector products on the tensor cores).
    locking: the 48^3 PAW cell (8025 plane waves, 256 bands), 20 sweeps with and without
    locking: FP64 form at degree 10 and residual 1e-9, mixed form at degree 8 (degree 10 trips
    its overflow guard there) and residual 3e-5, above its floor; time, band-applies."""
    import numpy as np
    import torch
    from paper_1406_4350_gb300 import build as b
    from paper_1406_4350_gb300 import F32, F64, MIXED, BOUND_RIGOROUS
    from paper_1406_4350_gb300.chebfi import ChebFI, fortran
    from synth import config_cell
    b.build()
    torch.cuda.set_device(0)
    if args.task == "backward":
        cell = config_cell("paw48", nbands=128)
        deg = 8
        g = ChebFI.from_cell(cell)
        hi = g.upper_bound(BOUND_RIGOROUS)
        Y = fortran(cell.Y0)
        lo = float(g.rayleigh_quotients(Y).max().item())
        rng = np.random.default_rng(8)
        W = fortran(rng.normal(size=cell.Y0.shape) + 1j * rng.normal(size=cell.Y0.shape))
        out = {}
        for name, p in (("f64", F64), ("f32", F32)):
            with Clocks(0) as clk:
                ms = _timed(lambda: g.cheb_filter_backward(Y, W, deg, lo, hi, cell.vloc.shape, cell.D.size, prec=p),
                            args.steps, args.warmup)
                fwd = _timed(lambda: g.cheb_filter(Y.clone(), deg, lo, hi, prec=p), args.steps, args.warmup)
            out[name] = {"value": cell.nbands * deg / (ms / 1e3), "ms_backward": ms, "ms_forward": fwd,
                         "backward_over_forward": ms / fwd, "clocks": clk.summary()}
        line = {"metric": "filter backward band-steps/s (gY0, gV, gD)", "unit": "band-steps/s",
                "value": out["f64"]["value"], "dtype": "f64", "steps": args.steps, "warmup": args.warmup,
                "config": {"workload": "paw48: 48^3 grid, %d plane waves, %d bands, %d projectors, PAW, degree %d, "
                                       "checkpoints every ceil(sqrt(degree))" % (cell.npw, cell.nbands, cell.nproj, deg)},
                "forms": out}
    elif args.task == "locking":
        from paper_1406_4350_gb300 import MIXED
        cell = config_cell("paw48")
        g = ChebFI.from_cell(cell)
        hi = g.upper_bound(BOUND_RIGOROUS)
        k75 = (3 * cell.nbands) // 4
        forms = {}
        # (form, degree, lock tolerance): the tolerance sits above each form's residual floor
        for fname, p, deg, tol in (("f64", F64, 10, 1e-9), ("mixed", MIXED, 8, 3e-5)):
            res = {}
            for name, t in (("full_degree", 0.0), ("locking", tol)):
                Y = fortran(cell.Y0)
                g.solve(Y.clone(), degree=deg, sweeps=1, prec=p, lambda_hi=hi)  # warm-up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ev, rs = g.solve(Y, degree=deg, sweeps=20, prec=p, lambda_hi=hi, lock_tol=t)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                sw, ap = g.solve_stats()
                res[name] = {"s": dt, "sweeps": sw, "band_applies": ap,
                             "max_resid_lowest_75pct": float(rs[:k75].max()), "evals": ev.cpu().numpy()}
            dev = float(np.abs(res["locking"]["evals"][:k75] - res["full_degree"]["evals"][:k75]).max())
            for v in res.values():
                v.pop("evals")
            forms[fname] = {"degree": deg, "lock_tol": tol, "runs": res, "max_eval_diff_lowest_75pct": dev}
        line = {"metric": "locking: band-H-applications and solve time with and without locking", "unit": "s",
                "value": forms["f64"]["runs"]["locking"]["s"], "dtype": "f64",
                "config": {"workload": "paw48: 48^3 grid, %d plane waves, %d bands, PAW, 20 sweeps"
                                       % (cell.npw, cell.nbands)},
                "forms": forms}
    elif args.task == "kpoints":
        from paper_1406_4350_gb300.chebfi import ChebFIBatch
        from synth import kpoint_cells
        cells = kpoint_cells()
        deg = 8
        ctxs = [ChebFI.from_cell(c) for c in cells]
        bt = ChebFIBatch(ctxs, cells[0].nbands)
        Ys = [fortran(c.Y0) for c in cells]
        his = [g_.upper_bound(BOUND_RIGOROUS) for g_ in ctxs]
        los = [float(g_.rayleigh_quotients(Y).max().item()) for g_, Y in zip(ctxs, Ys)]
        shapes, split, tune, split_ms = bt.autotune(F32)
        work = [Y.clone() for Y in Ys]
        l0 = bt.kernel_launches
        with Clocks(0) as clk:
            ms_b = _timed(lambda: bt.cheb_filter(work, deg, los, his, prec=F32), args.steps, args.warmup)
        launches = (bt.kernel_launches - l0) // (args.steps + args.warmup)

        def loop():
            for g_, Y, l, h in zip(ctxs, work, los, his):
                g_.cheb_filter(Y, deg, l, h, prec=F32)
        ms_l = _timed(loop, args.steps, args.warmup)
        units = sum(c.nbands for c in cells) * deg
        # mixed form: the same batch with the projector products as grouped tensor-core GEMMs
        mixed = [Y.clone() for Y in Ys]
        l0 = bt.kernel_launches
        bt.cheb_filter(mixed, deg, los, his, prec=MIXED)
        ms_m = _timed(lambda: bt.cheb_filter(mixed, deg, los, his, prec=MIXED), args.steps, args.warmup)
        launches_m = (bt.kernel_launches - l0) // (args.steps + args.warmup + 1)
        line = {"metric": "batched k-point filter band-H-applies/s", "unit": "band-H-applies/s",
                "value": units / (ms_b / 1e3), "dtype": "f32", "steps": args.steps, "warmup": args.warmup,
                "config": {"workload": "64 k-points of a 48^3 PAW cell (L = 20 bohr, 32 atoms x 8 projectors), "
                                       "spheres %d..%d plane waves, %d bands each, degree %d, one graph replay "
                                       "per step" % (min(c.npw for c in cells), max(c.npw for c in cells),
                                                     cells[0].nbands, deg)},
                "ms_batched": ms_b, "ms_per_kpoint_loop": ms_l, "speedup_over_loop": ms_l / ms_b,
                "gpu_launches_per_call": launches,
                "mixed": {"ms_batched": ms_m, "band_H_applies_per_s": units / (ms_m / 1e3),
                          "gpu_launches_per_call": launches_m}, "autotuned_shapes": shapes, "split_k_PhY": split,
                "autotune_ms": tune.round(4).tolist(), "split_ms": split_ms.round(4).tolist(),
                "clocks": clk.summary()}
    elif args.task == "gemm64":
        # the FP64 complex GEMM engines on one product C = A^H B (m x n, inner k): the modular
        # tensor-core emulation against FP64 FMA on the CUDA cores
        from paper_1406_4350_gb300._lib import GEMM_CUDA_CORES, GEMM_TENSOR
        m, n, k = args.gemm_mnk
        g = ChebFI(0)
        gen = torch.Generator(device="cuda").manual_seed(5)
        A = torch.randn((m, k), dtype=torch.complex128, device="cuda", generator=gen).T
        B = torch.randn((n, k), dtype=torch.complex128, device="cuda", generator=gen).T
        out = {}
        for name, eng in (("tensor", GEMM_TENSOR), ("cuda_cores", GEMM_CUDA_CORES)):
            g.set_fp64_gemm(eng, 14)
            C = torch.zeros((n, m), dtype=torch.complex128, device="cuda").T
            reps = args.steps if eng == GEMM_TENSOR else 1
            ms = _timed(lambda: g.gemm_fp64(A, B, conjA=True, C=C), reps, 1 if eng == GEMM_TENSOR else 0)
            out[name] = {"ms": ms, "tflops_fp64_equivalent": 8.0 * m * n * k / (ms / 1e3) / 1e12, "C": C}
        diff = float((out["tensor"]["C"] - out["cuda_cores"]["C"]).abs().max() / out["cuda_cores"]["C"].abs().max())
        for v in out.values():
            v.pop("C")
        line = {"metric": "FP64 complex GEMM, FP64-equivalent TFLOP/s (modular tensor-core emulation)",
                "unit": "TFLOP/s", "value": out["tensor"]["tflops_fp64_equivalent"], "dtype": "f64",
                "steps": args.steps, "config": {"workload": "C = A^H B, m = %d, n = %d, k = %d, 14 moduli" % (m, n, k)},
                "engines": out, "max_rel_diff": diff}
    elif args.task == "gemm_mixed":
        # the mixed form's tensor-core complex GEMM on the filter's two big shapes at paw96
        # (P^H Z: m = n_proj, n = bands, k = N_pw; P W: m = N_pw, n = bands, k = n_proj), or
        # on --gemm-mnk as a P^H Z-type product
        g = ChebFI(0)
        gen = torch.Generator(device="cuda").manual_seed(6)
        shapes = [("PhY", True, 2048, 2048, 60005), ("PW", False, 60005, 2048, 2048)]
        if args.gemm_mnk_set:
            shapes = [("custom", True, *args.gemm_mnk)]
        out = {}
        for name, conj, m, n, k in shapes:
            A = torch.randn(((m, k) if conj else (k, m)), dtype=torch.complex64, device="cuda", generator=gen).T
            B = torch.randn((n, k), dtype=torch.complex64, device="cuda", generator=gen).T
            C = torch.zeros((n, m), dtype=torch.complex64, device="cuda").T
            ms = _timed(lambda: g.gemm_mixed(A, B, conjA=conj, C=C), args.steps, args.warmup)
            # the GEMM kernel alone (the call also builds the operand planes)
            g.profile(True)
            for _ in range(args.steps):
                g.gemm_mixed(A, B, conjA=conj, C=C)
            torch.cuda.synchronize()
            tot = g.profile_totals()
            g.profile(False)
            kms = tot["gemm_mixed"][0] / tot["gemm_mixed"][1]
            out[name] = {"m": m, "n": n, "k": k, "ms_call": ms, "ms_kernel": kms,
                         "tflops": 8.0 * m * n * k / (kms / 1e3) / 1e12,
                         "tflops_executed_bf16": 3 * 3 * 2.0 * m * n * k / (kms / 1e3) / 1e12,
                         "kernels_ms": {kk: round(v[0] / args.steps, 3) for kk, v in tot.items()}}
            del A, B, C
        first = next(iter(out.values()))
        line = {"metric": "mixed complex GEMM TFLOP/s (complex flops 8mnk)", "unit": "TFLOP/s",
                "value": first["tflops"], "dtype": "bf16x3+f32", "steps": args.steps, "warmup": args.warmup,
                "config": {"workload": "tensor-core complex GEMM, three real products of bf16 pairs"},
                "shapes": out}
    elif args.task == "filter_only":
        # the filter alone (no Rayleigh-Ritz) on a named cell: the command behind the
        # per-kernel counter captures of small cases
        from paper_1406_4350_gb300 import MIXED
        prec = {"mixed": MIXED, "f32": F32, "f64": F64}[args.prec]
        cell = config_cell(args.workload, nbands=args.nbands)
        g = ChebFI.from_cell(cell)
        hi = g.upper_bound(BOUND_RIGOROUS)
        Y = fortran(cell.Y0)
        lo = float(g.rayleigh_quotients(Y).max().item())
        ms = _timed(lambda: g.cheb_filter(Y, DEGREE, lo, hi, prec=prec), args.steps, args.warmup)
        line = {"metric": "filter band-H-applies/s (filter only)", "unit": UNIT,
                "value": Y.shape[1] * DEGREE / (ms / 1e3), "dtype": args.prec, "steps": args.steps,
                "warmup": args.warmup, "ms_per_filter": ms,
                "config": {"workload": "%s: %d^3 grid, %d plane waves, %d bands, %d projectors, degree %d"
                                       % (args.workload, cell.grid[0], cell.npw, Y.shape[1], cell.nproj, DEGREE)}}
    elif args.task == "gate":
        # Accuracy gate at the benchmark workload: Algorithm 2 from the same start in the
        # FP64 form until the residual certificate holds for the lowest 75 % of the bands,
        # then the mixed form for the same sweeps; their Ritz values are compared.
        from paper_1406_4350_gb300 import MIXED
        cell = config_cell(WORKLOAD)
        nb = cell.nbands
        k75 = (3 * nb) // 4
        g = ChebFI.from_cell(cell)
        hi = g.upper_bound(BOUND_RIGOROUS)
        smin = g.overlap_lower_bound()

        def run(prec, sweeps_max, certify):
            Y = fortran(cell.Y0)
            lo = float(g.rayleigh_quotients(Y).max().item())
            hist = []
            ev = rs = None
            # each filter starts from the projections its Rayleigh-Ritz handed over
            pbuf = torch.empty((nb, cell.nproj), dtype=torch.complex128, device="cuda").T
            proj = None
            t0 = time.perf_counter()
            for s_ in range(sweeps_max):
                g.cheb_filter(Y, DEGREE, lo, hi, prec=prec, proj=proj)
                ev, rs = g.rayleigh_ritz(Y, proj=pbuf)
                proj = pbuf
                lo = float(ev.max().item())
                cert = float(rs[:k75].max().item()) / np.sqrt(smin)
                hist.append(cert)
                if certify and cert <= 1e-8:
                    break
            torch.cuda.synchronize()
            return ev.cpu().numpy(), rs.cpu().numpy(), len(hist), hist, time.perf_counter() - t0

        ev64, rs64, n64, h64, t64 = run(F64, args.gate_sweeps, True)
        certified = h64[-1] <= 1e-8
        evmx, rsmx, nmx, hmx, tmx = run(MIXED, n64, False)
        diff = np.abs(evmx[:k75] - ev64[:k75])
        line = {"metric": "config-3 accuracy gate: max |lambda_mixed - lambda_FP64| over the lowest 75% of bands",
                "unit": "Ha", "value": float(diff.max()), "dtype": "f64 / bf16x3+f32",
                "config": {"workload": "paw96: 96^3 grid, %d plane waves, %d bands, %d projectors, PAW, degree %d, "
                                       "Algorithm 2 from the seeded start, lambda_+ rigorous %.4f Ha"
                                       % (cell.npw, nb, cell.nproj, DEGREE, hi)},
                "fp64": {"sweeps": n64, "certified": bool(certified),
                         "certificate_Ha": h64[-1],
                         "certificate": "max over the lowest %d bands of ||H y - theta S y||_2 / sqrt(smin), "
                                        "smin = %.6f a proven lower bound of lambda_min(S): every such Ritz value "
                                        "is within it of an eigenvalue of the pencil" % (k75, smin),
                         "max_residual_lowest_75pct": float(rs64[:k75].max()),
                         "max_residual_all": float(rs64.max()), "lambda_min": float(ev64[0]),
                         "lambda_k75": float(ev64[k75 - 1]), "s": t64, "history": h64},
                "mixed": {"sweeps": nmx, "max_residual_lowest_75pct": float(rsmx[:k75].max()),
                          "max_abs_diff_lowest_75pct_Ha": float(diff.max()),
                          "mean_abs_diff_lowest_75pct_Ha": float(diff.mean()),
                          "max_abs_diff_all_Ha": float(np.abs(evmx - ev64).max()), "s": tmx, "history": hmx},
                "passed": bool(certified and diff.max() <= 1e-8)}
    else:
        cell = config_cell(WORKLOAD, nbands=256)
        g = ChebFI.from_cell(cell)
        X = fortran(cell.Y0)
        res = {}
        ms_direct = _timed(lambda: g.apply_Sinv(X), args.steps, args.warmup)
        its = []
        ms_ref = _timed(lambda: its.append(g.apply_Sinv_refined(X, tol=1e-12)[1]), args.steps, args.warmup)
        a = g.apply_Sinv(X)
        r, _ = g.apply_Sinv_refined(X, tol=1e-12)
        diff = float((a - r).abs().max().item() / X.abs().max().item())
        line = {"metric": "S^-1 application time, refinement vs direct Woodbury", "unit": "ms",
                "value": ms_ref, "dtype": "f64", "steps": args.steps, "warmup": args.warmup,
                "config": {"workload": "paw96: 96^3 grid, %d plane waves, 256 bands, %d projectors, PAW, tol 1e-12"
                                       % (cell.npw, cell.nproj)},
                "ms_direct": ms_direct, "iterations": its[-1], "max_rel_diff": diff}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ native arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "f32", "f64"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed FP64-form filter calls (0: skip)")
    ap.add_argument("--cpu-bands", type=int, default=64, help="bands in the oracle's timed CPU sample")
    ap.add_argument("--ref-bands", type=int, default=64)
    ap.add_argument("--nbands", type=int, default=None, help="override the band count (testing only)")
    ap.add_argument("--workload", default=WORKLOAD, help="synthetic cell (paw96 is the benchmark workload)")
    ap.add_argument("--gemm-mnk", type=int, nargs=3, default=None, help="gemm64 / gemm_mixed: m n k")
    ap.add_argument("--gate-sweeps", type=int, default=120, help="gate: most FP64 sweeps before giving up")
    ap.add_argument("--task", default="filter", choices=["filter", "backward", "refine", "kpoints", "locking", "gate", "filter_only",
                             "gemm64", "gemm_mixed"],
                    help="filter: the benchmark; backward / refine: the differentiation and the "
                         "refinement-Woodbury measurements (their own JSON line)")
    args = ap.parse_args()
    args.gemm_mnk_set = args.gemm_mnk is not None
    if args.gemm_mnk is None:
        args.gemm_mnk = [2048, 2048, 8192]
    if args.impl == "reference":
        return run_reference(args)
    if args.task != "filter":
        return run_extra(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)

    from paper_1406_4350_gb300 import build as b
    from paper_1406_4350_gb300 import F32, F64, MIXED, BOUND_RIGOROUS
    from paper_1406_4350_gb300.chebfi import ChebFI, fortran
    from paper_1406_4350_gb300.parallel import band_range, gather_bands
    from synth import config_cell
    b.build()
    prec = {"mixed": MIXED, "f32": F32, "f64": F64}[args.prec]

    cell = config_cell(args.workload, nbands=args.nbands)
    nb, npw, nq = cell.nbands, cell.npw, cell.nproj
    # one problem split over the ranks by bands (the filter treats bands independently):
    # rank r filters bands [b0, b1); Rayleigh-Ritz gathers the block (the method's exchange
    # step) and every rank keeps its own bands of the rotated block
    b0, b1 = band_range(nb, world, rank)
    g = ChebFI.from_cell(cell, device=local)
    hi = g.upper_bound(BOUND_RIGOROUS)
    Y = fortran(cell.Y0, device="cuda:%d" % local)
    lo = float(g.rayleigh_quotients(Y).max().item())
    if world > 1:
        Y = Y[:, b0:b1].T.contiguous().T

    # measured CUDA-core peaks of this device (the roofline denominators of the SIMT kernels)
    fp64_peak, _ = g.probe_fma_rate(F64)
    fp32_peak, _ = g.probe_fma_rate(F32)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    prof_acc = {"filter": {}, "rr": {}}

    def _acc(phase):
        for k, (ms, cnt, wk) in g.profile_totals().items():
            a = prof_acc[phase].setdefault(k, [0.0, 0, 0.0])
            a[0] += ms
            a[1] += cnt
            a[2] += wk

    # P^H Y of the block that Rayleigh-Ritz has just rotated: that step forms it anyway (for
    # S Y in the residuals), and the next filter starts from it instead of recomputing it,
    # as in chebfi_solve (Algorithm 2's loop); the first warm-up filter computes its own
    proj_full = torch.empty((nb, nq), dtype=torch.complex128, device="cuda:%d" % local).T if nq > 0 else None
    proj = None

    def step(p, timed=None):
        nonlocal lo, Y, proj
        st = torch.cuda.current_stream()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        if timed is not None:
            g.profile(True)
        e0.record(st)
        torch.cuda.nvtx.range_push("filter")
        g.cheb_filter(Y, DEGREE, lo, hi, prec=p, proj=proj)
        torch.cuda.nvtx.range_pop()
        e1.record(st)
        if timed is not None:
            _acc("filter")
            g.profile(True)
        torch.cuda.nvtx.range_push("rr")
        full = gather_bands(Y, nb, world) if world > 1 else Y
        ev, rs = g.rayleigh_ritz(full, proj=proj_full)
        if proj_full is not None:
            proj = proj_full[:, b0:b1]
        if world > 1:
            Y = full[:, b0:b1].clone().T.contiguous().T
        torch.cuda.nvtx.range_pop()
        e2.record(st)
        if timed is not None:
            _acc("rr")
            g.profile(False)
        lo = float(ev.max().item())
        if timed is not None:
            timed.append((e0, e1, e2, ev, rs))

    for _ in range(args.warmup):
        step(prec)
    barrier()
    launches0 = g.kernel_launches
    timed = []
    with Clocks(local) as clk:
        barrier()
        torch.cuda.nvtx.range_push("timed")  # lets ncu restrict a capture to the timed steps
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step(prec, timed)
        barrier()
        wall = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
    launches = g.kernel_launches - launches0
    filt_ms = [a.elapsed_time(b_) for a, b_, c, _, _ in timed]
    rr_ms = [b_.elapsed_time(c) for a, b_, c, _, _ in timed]
    step_ms = [a.elapsed_time(c) for a, b_, c, _, _ in timed]
    ev_last = timed[-1][3].cpu().numpy()
    rs_last = timed[-1][4].cpu().numpy()
    # the job's units: every band of the one problem, degree applications per step
    value, filt_s, step_total = aggregate(sum(filt_ms) / 1e3, sum(step_ms) / 1e3, (b1 - b0) * DEGREE * args.steps,
                                          world)
    value = nb * DEGREE * args.steps / filt_s

    # FP64 form of the same filter, same bands
    fp64 = None
    if args.fp64_steps > 0 and prec != F64:
        # every timed filter starts from the rotated block and its projections, as the
        # mixed form's do (the block is restored between filters, outside the events)
        Yc = Y.clone()
        st = torch.cuda.current_stream()
        g.cheb_filter(Yc, DEGREE, lo, hi, prec=F64, proj=proj)
        barrier()
        g.profile(True)
        evs = []
        for _ in range(args.fp64_steps):
            Yc.copy_(Y)
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            g.cheb_filter(Yc, DEGREE, lo, hi, prec=F64, proj=proj)
            c.record(st)
            evs.append((a, c))
        barrier()
        ms = sum(a.elapsed_time(c) for a, c in evs)
        tot = g.profile_totals()
        g.profile(False)
        fp_s = aggregate(ms / 1e3, 0.0, 0.0, world)[1]  # slowest rank
        fp64 = {"value": nb * DEGREE * args.fp64_steps / fp_s, "unit": UNIT, "ms_per_filter": ms / args.fp64_steps,
                "dtype": "f64 (FFT in double-float pairs on the FP32 units; GEMMs FP64-accurate modular)",
                "kernels_ms": {k: round(v[0] / args.fp64_steps, 3) for k, v in
                               sorted(tot.items(), key=lambda kv: -kv[1][0])[:8]}}
        del Yc

    # end to end through the public API with host buffers: chebfi_cheb_filter_host takes the
    # pinned host block, copies it in, filters it and copies it back every step (band chunks
    # whose copies overlap the neighbouring chunks' filters)
    # (with the rotated block's projections in host memory too, copied in chunk by chunk); the
    # block is restored between calls outside the events, so that every call filters the
    # block its projections belong to; one untimed call first (streams, staging buffers)
    Yh = Y.cpu()
    host = torch.empty((Y.shape[1], npw), dtype=torch.complex128, pin_memory=True).T
    host_p = None
    if proj is not None:
        host_p = torch.empty((proj.shape[1], nq), dtype=torch.complex128, pin_memory=True).T
        host_p.copy_(proj)
    st = torch.cuda.current_stream()
    e2e_ms = 0.0
    for it in range(args.steps + 1):
        host.copy_(Yh)
        barrier()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(st)
        g.cheb_filter_host(host, DEGREE, lo, hi, prec=prec, proj=host_p)
        eb.record(st)
        torch.cuda.synchronize()
        if it > 0:
            e2e_ms += ea.elapsed_time(eb)
    _, e2e_s, _ = aggregate(e2e_ms / 1e3, 0.0, 0.0, world)
    nbytes = npw * (b1 - b0) * 16
    nbytes_p = nq * (b1 - b0) * 16 if host_p is not None else 0
    del Yh

    # rooflines from the library's per-launch CUDA events and each launch's algorithmic work
    # (flops for GEMMs and the Jacobi sweeps, bytes for the FFT passes)
    peaks = _peaks()
    bf16 = peaks.get("bf16_tflops_sustained", 1713.1)
    hbm = peaks.get("hbm_gbs", 6762.3)
    nmod = 14
    # the plane pass's arithmetic: per band and z plane, 96-point line transforms along y on
    # the rows of the active x range (inverse and forward) and along x on every y line
    # (inverse and forward), 5 N log2 N flops each (the usual FFT count), and the real
    # V_loc(r) times complex psi(r) product, 2 flops a point; its launch's recorded work is
    # the column buffer in and out, 2 N ncol per band (elements)
    Ng = int(cell.grid[0])
    xs = (cell.miller[:, 0].astype(np.int64) + Ng // 2) % Ng
    nact = int(xs.max() - xs.min() + 1)
    ncol = len(np.unique(cell.miller[:, 0].astype(np.int64) * 100003 + cell.miller[:, 1]))
    plane_flops_band = Ng * ((2 * nact + 2 * Ng) * 5.0 * Ng * math.log2(Ng) + 2.0 * Ng * Ng)
    plane_elems_band = 2.0 * Ng * ncol

    def roofline(phase, name):
        ms_tot, cnt, work = prof_acc[phase][name]
        avg_s = ms_tot / cnt / 1e3
        out = {"kernel": name, "phase": phase}
        if name.startswith("tc_"):
            # bf16x3: the pipe executes 3 MMAs per algorithmic product
            ach = work / cnt / avg_s / 1e12
            out.update(bound="tensor", unit="TFLOP/s", achieved=ach, peak=bf16, frac=ach / bf16,
                       frac_executed=3 * ach / bf16,
                       peak_source="bf16_tflops_sustained (measured); algorithmic flops, the pipe executes 3x")
        elif name == "k_oz_gemm":
            # FP64 products on the tensor cores: one bf16 GEMM per modulus
            ach = work / cnt / avg_s / 1e12
            out.update(bound="tensor", unit="TFLOP/s", achieved=ach * nmod, peak=bf16, frac=ach * nmod / bf16,
                       fp64_equivalent_tflops=ach, fp64_equivalent_over_fp64_peak=ach / fp64_peak,
                       peak_source="bf16_tflops_sustained (measured); executed = %d moduli x the FP64 flops" % nmod)
        elif name == "k_plane":
            # bound by its FP32 (FP64 in the FP64 phase) arithmetic, not by HBM: the FFT flops
            # per launch over the measured peak of its precision; the HBM fraction beside it
            esz = 16.0 if phase == "rr" or prec == F64 else 8.0
            bands = work / cnt / (plane_elems_band * esz)
            flops = plane_flops_band * bands
            pk = fp64_peak if esz == 16.0 else fp32_peak
            ach = flops / avg_s / 1e12
            out.update(bound="alu", unit="TFLOP/s", achieved=ach, peak=pk, frac=ach / pk,
                       peak_source=("%s FMA rate measured in this run (chebfi_probe_fma_rate); FFT flops "
                                    "5 N log2 N per 96-point line, %d active rows of 96" %
                                    ("FP64" if esz == 16.0 else "FP32", nact)),
                       hbm={"achieved_gbs": work / cnt / avg_s / 1e9, "peak": hbm,
                            "frac": work / cnt / avg_s / 1e9 / hbm},
                       flops_per_launch=flops)
        elif name == "k_jac_sweep":
            ach = work / cnt / avg_s / 1e12
            out.update(bound="alu", unit="TFLOP/s", achieved=ach, peak=fp32_peak, frac=ach / fp32_peak,
                       peak_source="FP32 FMA rate measured in this run (chebfi_probe_fma_rate)")
        elif "gemm" in name:
            ach = work / cnt / avg_s / 1e12
            pk = fp64_peak if prec == F64 else fp32_peak
            out.update(bound="alu", unit="TFLOP/s", achieved=ach, peak=pk, frac=ach / pk,
                       peak_source="FMA rate measured in this run (chebfi_probe_fma_rate)")
        else:
            ach = work / cnt / avg_s / 1e9
            out.update(bound="hbm", unit="GB/s", achieved=ach, peak=hbm, frac=ach / hbm,
                       peak_source="hbm_gbs (measured)")
        out["traffic"] = _traffic(name) if (args.workload == WORKLOAD and args.nbands is None and world == 1) else None
        out.update(avg_launch_ms=avg_s * 1e3, launches_per_step=cnt / args.steps, work_per_launch=work / cnt)
        return out

    def dominant(phase):
        return max((v[0], k) for k, v in prof_acc[phase].items() if v[2] > 0)[1]

    roof = roofline("filter", dominant("filter"))
    # the whole filter against its roofline: sum over its kernels of work / peak, over the time
    ideal = 0.0
    for k, (ms_tot, cnt, work) in prof_acc["filter"].items():
        if work <= 0:
            continue
        r_ = roofline("filter", k)
        if k == "k_plane":  # the larger of its two bounds
            ideal += max(r_["flops_per_launch"] * cnt / (r_["peak"] * 1e12), work / (hbm * 1e9))
            continue
        scale = 1e12 if r_["unit"] == "TFLOP/s" else 1e9
        ideal += work / (r_["peak"] * scale)
    filt_mean_s = statistics.mean(filt_ms) / 1e3
    roof["combined"] = {"frac": ideal / args.steps / filt_mean_s, "ideal_ms": 1e3 * ideal / args.steps,
                        "measured_ms": 1e3 * filt_mean_s,
                        "what": "sum over the filter's kernels of algorithmic work / that kernel's peak, "
                                "over the filter's measured time"}
    roof_rr = roofline("rr", dominant("rr"))

    # eigenvalue state after the timed steps (residual norms in FP64)
    k75 = (3 * nb) // 4
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * step_total / args.steps, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
        "dtype": {"mixed": "bf16x3+f32", "f32": "f32", "f64": "f64"}[args.prec], "data": "synthetic",
        "config": {"workload": "%s: %d^3 grid, %d plane waves, %d bands, %d projectors, PAW=%s, degree 4, one "
                               "filter + FP64 Rayleigh-Ritz per step" % (args.workload, cell.grid[0], npw, nb, nq,
                                                                         cell.Q is not None),
                   "filter_form": args.prec, "l2": "inputs (2 GB per block) larger than L2; no flush",
                   "lambda_hi": "rigorous bound %.4f Ha" % hi,
                   "parallelism": "bands split over %d rank(s), block gathered for Rayleigh-Ritz" % world},
        "phases_ms": {"filter": statistics.mean(filt_ms), "rayleigh_ritz": statistics.mean(rr_ms)},
        "fp64_form": fp64,
        "e2e": {"value": nb * DEGREE * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes + nbytes_p,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "roofline": roof,
        "rr_roofline": roof_rr,
        "measured_peaks": {"fp64_fma_tflops": fp64_peak, "fp32_fma_tflops": fp32_peak, "hbm_gbs": hbm,
                           "bf16_tflops_sustained": bf16},
        "kernels_ms": {ph: {k: round(v[0] / args.steps, 3) for k, v in sorted(prof_acc[ph].items(),
                                                                              key=lambda kv: -kv[1][0])[:12]}
                       for ph in prof_acc},
        "ritz": {"max_residual_lowest_75pct": float(rs_last[:k75].max()), "lambda_min": float(ev_last[0])},
        "clocks": clocks,
        "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and args.cpu_bands > 0:
        prepared = oracle_setup(cell)
        r, dt = oracle_rate(cell, args.cpu_bands, DEGREE, prepared)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "%d of %d bands, degree %d, one filter call (%.1f s); the oracle's "
                                          "P^H P and reduced-matrix LU formed once before timing; FFTs (scipy) "
                                          "and BLAS on all cores" % (args.cpu_bands, nb, DEGREE, dt)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
