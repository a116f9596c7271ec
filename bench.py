"""Benchmark: time-to-1e-9 relative residual of SLD-deflated Jacobi-PCG on the
256x256x128 lognormal-layered point-source workload (8.4M cells, 4x4x4
subdomains x 2 levelsets = 128 deflation vectors), one GB300.

One step = one full solve (steps a4-a8 in one persistent launch: initial
projection, deflated CG iterations, FP64 refinement, back-projection) from a
right-hand side resident in HBM to the solution in HBM, followed by the FP64
true-residual check.  The headline is the FP32-inner / FP64-refined form;
plain FP64 is measured in the same run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With torchrun (N > 1) every rank solves its own replica (the path has no
cross-GPU exchange at this size: "replicas only"); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-9 rel. residual & HBM GB/s: mixed/learned/batched vs plain FP64"
WORKLOAD = "lognormal-layered 256x256x128, point source, 4x4x4 subdomains x 2 levelsets (d=128), tol 1e-9"
# algorithmic bytes per cell: one inner iteration (sweeps A
# and B) and one FP64 refinement step (sweeps O1 and O2).  The TMA sweeps
# stream 16-bit labels.
BYTES_ITER_FP32 = 60   # A: z, p_old, 3 faces, label, p_new  B: p, label, 3 faces, z r/w, xhat r/w
BYTES_ITER_FP64 = 140  # same vectors and faces in FP64 + diag (A, B) and 1/diag (B)
BYTES_OUTER = 152      # O1: x, xhat, b, faces, diag, label, r'  O2: r', label, faces, diag, x r/w, xhat r/w, 1/diag, z, p0, p1
BYTES_ITER_BF16 = 52   # A: z, p_old, 3 BF16 faces, label, p_new  B: p, label, 3 BF16 faces, FP32 1/diag, z r/w, xhat r/w
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) over algorithmic
# bytes of one launch of k_solve_tma<float, float, 8, 3, true, false>, from an
# ncu capture of a 300-iteration launch on this workload; the traffic of a
# full launch is this ratio times its algorithmic bytes.  Must be re-measured
# (or set to None) whenever that kernel changes.
TRAFFIC_RATIO_FP32 = 1.084


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up (NVML initialisation) can hold up the
            # CUDA calls of this process for a large fraction of a second:
            # let it print its first sample before the timed region opens
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 10.0:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    from paper_1510_02148_gb300 import replicas
    return replicas.dist_env()


def cpu_baseline(P, A=None, lab=None, iters_full=None, sample_iters=40, threads=None, single_thread_iters=0):
    """Time the CPU oracle on a bounded sample: `sample_iters` deflated-CG
    iterations (plus its setup), scaled to the full iteration count."""
    import oracle
    oracle.build()
    if threads:
        oracle.set_threads(threads)
    t0 = time.perf_counter()
    if A is None:
        A = oracle.assemble(P.K, P.q, P.bc_type, P.bc_value)
        lab = oracle.labels(P.K, P.S, P.tau, P.L)
    # two runs, 1 and 1 + sample_iters iterations: their difference is the
    # iterations' cost, the rest of the first is the setup (coarse matrix,
    # Cholesky, projection of b), charged once
    t1 = time.perf_counter()
    oracle.dpcg(A, lab, P.d, tol=P.tol, maxiter=1)
    t2 = time.perf_counter()
    r = oracle.dpcg(A, lab, P.d, tol=P.tol, maxiter=1 + sample_iters)
    t3 = time.perf_counter()
    its = max(1, r.iterations - 1)
    per_iter = max(0.0, (t3 - t2) - (t2 - t1)) / its
    setup = max(0.0, (t2 - t1) - per_iter)
    full = iters_full if iters_full else r.iterations
    est_s = (t1 - t0) + setup + per_iter * full
    out = {"value": est_s * 1e3, "unit": "ms", "cores": oracle.max_threads(), "kind": "oracle",
           "sample": f"oracle FP64 DPCG on the full workload: setup {setup:.1f} s, {its} timed iterations "
                     f"({per_iter * 1e3:.0f} ms each), assembly/labels {t1 - t0:.1f} s, "
                     f"scaled to {full} iterations"}
    if single_thread_iters:
        # the same iterations on one core (the oracle's plain loops)
        nt = oracle.max_threads()
        oracle.set_threads(1)
        try:
            t4 = time.perf_counter()
            oracle.dpcg(A, lab, P.d, tol=P.tol, maxiter=1)
            t5 = time.perf_counter()
            oracle.dpcg(A, lab, P.d, tol=P.tol, maxiter=1 + single_thread_iters)
            t6 = time.perf_counter()
        finally:
            oracle.set_threads(nt)
        pi1 = max(0.0, (t6 - t5) - (t5 - t4)) / single_thread_iters
        su1 = max(0.0, (t5 - t4) - pi1)
        out["single_thread"] = {"value": ((t1 - t0) + su1 + pi1 * full) * 1e3, "unit": "ms", "cores": 1,
                                "sample": f"{single_thread_iters} timed iterations ({pi1 * 1e3:.0f} ms each), "
                                          f"setup {su1:.1f} s, scaled to {full} iterations"}
    return out


def bench_c2(sld, torch, reps=1):
    """The 512x512x256 inclusion workload (67M cells, tilted lens/channel
    inclusions at 1e-6 in a K = 1 background, >= 20 % of the volume,
    8x8x8 subdomains x 3 levelsets: d = 1536): BF16 coefficients with an
    FP32 per-cell inverse diagonal (with the refinement's forward-error test,
    and with the residual test alone), FP32 inner, and plain FP64; each with
    the algorithmic GB/s of its persistent kernel against the measured HBM
    peak."""
    from paper_1510_02148_gb300 import workloads as W
    P, frac = W.inclusion_field()
    Kd = torch.from_numpy(P.K.reshape(-1)).cuda()
    t0 = time.perf_counter()
    s = sld.System(Kd, None, P.bc_type, P.bc_value, shape=P.shape)
    s.make_labels(P.S, P.tau, P.L)
    s.build_deflation(P.d)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    x = torch.empty(P.n, dtype=torch.float64, device="cuda")
    peak, peak_kind = _peaks()
    out = {"workload": f"inclusions 512x512x256 ({frac * 100:.1f} % at 1e-6), 8x8x8 subdomains x 3 levelsets "
                       f"(d = {P.d}), tol 1e-9", "n": P.n, "d": P.d, "setup_ms": setup_ms}
    forms = (("bf16", sld.BF16COEF_IR, 0.0, BYTES_ITER_BF16), ("bf16_residual_only", sld.BF16COEF_IR, -1.0, BYTES_ITER_BF16),
             ("fp32_ir", sld.FP32_IR, 0.0, BYTES_ITER_FP32), ("fp64", sld.FP64, 0.0, BYTES_ITER_FP64))
    for name, prec, fwd, bpc in forms:
        s.solve(x=x, precision=prec, fwd_tol=fwd, maxiter=50, raise_on_error=False)  # warm-up (tensor maps, code)
        ms = []
        for _ in range(reps):
            _, i = s.solve(x=x, precision=prec, fwd_tol=fwd)
            ms.append(i.solve_ms)
        kms = statistics.median(ms)
        alg = P.n * (bpc * i.iterations + BYTES_OUTER * i.outer_steps)
        ach = alg / (kms * 1e-3) / 1e9
        out[name] = {"ms": kms, "iterations": i.iterations, "outer_steps": i.outer_steps,
                     "true_relres": i.true_relres, "fwd_err_estimate": i.fwd_err_estimate,
                     "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                  "bytes_per_cell_iter": bpc, "peak_kind": peak_kind}}
    out["speedup_bf16_vs_fp64"] = out["fp64"]["ms"] / out["bf16"]["ms"]
    out["speedup_fp32_vs_fp64"] = out["fp64"]["ms"] / out["fp32_ir"]["ms"]
    s.close()
    return out


def bench_c0(sld, torch, reps=5):
    """The 32^3 layered sandwich (8 z-layers 1 / 1e-6, Dirichlet x-faces,
    2x2x2 subdomains x 2 levelsets: d = 16): L2-resident and barrier-bound,
    reported as time only."""
    from paper_1510_02148_gb300 import workloads as W
    P = W.layered_sandwich()
    s = sld.from_problem(P)
    x = torch.empty(P.n, dtype=torch.float64, device="cuda")
    out = {"workload": "layered sandwich 32^3, 2x2x2 subdomains x 2 levelsets (d = 16), tol 1e-9"}
    for name, prec in (("fp64", sld.FP64), ("fp32_ir", sld.FP32_IR), ("bf16", sld.BF16COEF_IR)):
        s.solve(x=x, precision=prec)
        ms = []
        for _ in range(reps):
            _, i = s.solve(x=x, precision=prec)
            ms.append(i.solve_ms)
        out[name] = {"ms": statistics.median(ms), "iterations": i.iterations, "outer_steps": i.outer_steps,
                     "true_relres": i.true_relres}
    s.close()
    return out


def gmres_bytes(n, m, its, cycles, deflated):
    """Algorithmic bytes of a PDGMRES solve: per Arnoldi step with basis size
    j+1, apply 68 B (raw v, M^-1 v, V_j, w, faces, diag, label), deflation
    52 B (w r/w, faces, diag, label), two dot passes (j+1) 8 + 8 B and two
    orthogonalisation passes (j+1) 8 + 16 B, the second one also reading
    1/diag and writing M^-1 of the next raw vector (+16 B); per cycle the
    residual (apply, deflation, copy with norm and M^-1: 68 + 52 + 32 B);
    plain GMRES drops the deflation pass and the labels."""
    per_step = (184 if deflated else 128)
    per_cycle = (152 if deflated else 96)
    tot = 0
    left = its
    for c in range(cycles):
        k = min(m, left)
        left -= k
        tot += per_cycle + per_step * k + 32 * k * (k + 1) // 2
    return n * tot


def bench_gmres(sld, torch, s, x, P, m=20, tol=1e-6):
    """PDGMRES(m) (the paper's solver: deflated right-Jacobi GMRES, FP64) on
    the bench workload at the paper's tolerance, against plain GMRES(m)
    (capped) and deflated CG to the same tolerance; and RDGMRES(30, 3)
    (harmonic-Ritz deflation) against plain GMRES(30), both capped."""
    out = {"m": m, "tol": tol, "precision": "fp64"}
    for name, defl, cap in (("deflated", True, 20000), ("plain", False, 2000)):
        s.solve_gmres(x=x, m=m, deflate=defl, tol=tol, maxiter=min(cap, 50), raise_on_error=False)  # warm-up
        _, g = s.solve_gmres(x=x, m=m, deflate=defl, tol=tol, maxiter=cap, raise_on_error=False)
        by = gmres_bytes(P.n, m, g.iterations, g.cycles, defl)
        out[name] = {"iterations": g.iterations, "cycles": g.cycles, "ms": g.solve_ms,
                     "converged": g.status == 0, "true_relres": g.true_relres,
                     "ms_per_step": g.solve_ms / max(1, g.iterations),
                     "alg_gbs": by / (g.solve_ms * 1e-3) / 1e9}
    _, c = s.solve(x=x, precision=sld.FP64, tol=tol)
    out["dpcg_fp64_same_tol"] = {"iterations": c.iterations, "ms": c.solve_ms}
    # harmonic-Ritz deflation (RDGMRES(30, 3)) against plain GMRES(30), both capped
    try:
        _, r30 = s.solve_rdgmres(x=x, m=30, d=3, tol=tol, maxiter=4000, raise_on_error=False)
        _, g30 = s.solve_gmres(x=x, m=30, deflate=False, tol=tol, maxiter=4000, raise_on_error=False)
        out["rdgmres_m30_d3"] = {"iterations": r30.iterations, "ms": r30.solve_ms, "converged": r30.status == 0,
                                 "true_relres": r30.true_relres}
        out["gmres_m30_plain"] = {"iterations": g30.iterations, "ms": g30.solve_ms, "converged": g30.status == 0,
                                  "true_relres": g30.true_relres}
    except Exception as ex:  # reported, not fatal to the line
        out["rdgmres_m30_d3"] = {"error": str(ex)}
    return out


def bench_auto_labels(sld, torch, P, x):
    """The same workload deflated with the automatic subdomain-levelset
    labels (face-connected components of each subdomain's levelset classes)
    instead of the plain ones: label construction time, d, the FP32-inner
    and FP64 solves, and PDGMRES(20) to 1e-6."""
    s = sld.System(torch.from_numpy(P.K.reshape(-1)).cuda(), torch.from_numpy(P.q.reshape(-1)).cuda(),
                   P.bc_type, P.bc_value, shape=P.shape)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, d = s.make_labels_cc(P.S, P.tau, P.L)
    torch.cuda.synchronize()
    lab_ms = (time.perf_counter() - t0) * 1e3
    s.build_deflation(d)
    out = {"d": d, "d_plain": P.d, "labels_ms": lab_ms}
    for name, prec in (("fp32_ir", sld.FP32_IR), ("fp64", sld.FP64)):
        s.solve(x=x, precision=prec)
        _, i = s.solve(x=x, precision=prec)
        out[name] = {"ms": i.solve_ms, "iterations": i.iterations, "outer_steps": i.outer_steps,
                     "true_relres": i.true_relres}
    # PDGMRES(20) with these vectors, at the paper's tolerance
    _, g = s.solve_gmres(x=x, m=20, tol=1e-6, maxiter=20000, raise_on_error=False)
    out["pdgmres_m20_tol1e-6"] = {"ms": g.solve_ms, "iterations": g.iterations, "converged": g.status == 0,
                                  "true_relres": g.true_relres}
    s.close()
    return out


def bench_spe10(sld, torch, fp64=False):
    """The paper's SPE10 sweep of plain subdomain deflation (d = 8, 27, 64,
    and d = 1 for reference) on the deflated-CG path, on an SPE10-shaped
    synthetic field (180x220x85): FP32-inner solves with FP64 refinement to
    1e-9, and with fp64 also plain FP64 solves (capped at 30000 iterations:
    on this 7.5-decade field they may stagnate or break down, depending on
    the rounding of E, and take up to a minute of GPU time)."""
    from paper_1510_02148_gb300 import workloads as W
    P = W.spe10_like()
    Kd = torch.from_numpy(P.K.reshape(-1)).cuda()
    qd = torch.from_numpy(P.q.reshape(-1)).cuda()
    s = sld.System(Kd, qd, P.bc_type, P.bc_value, shape=P.shape)
    x = torch.empty(P.n, dtype=torch.float64, device="cuda")
    out = {"workload": f"SPE10-shaped synthetic {P.shape[2]}x{P.shape[1]}x{P.shape[0]} ({P.n} cells)", "runs": []}
    for S in ((1, 1, 1), (2, 2, 2), (3, 3, 3), (4, 4, 4)):
        d = S[0] * S[1] * S[2]
        s.make_labels(S, (), 1)
        s.build_deflation(d)
        row = {"d": d}
        for name, prec in ((("fp64", sld.FP64),) if fp64 else ()) + (("fp32_ir", sld.FP32_IR),):
            s.solve(x=x, precision=prec, maxiter=50, raise_on_error=False)  # warm-up
            _, i = s.solve(x=x, precision=prec, maxiter=30000, raise_on_error=False)
            row[name] = {"ms": i.solve_ms, "iterations": i.iterations, "true_relres": i.true_relres,
                         "converged": i.status == sld.OK}
        out["runs"].append(row)
    s.close()
    return out


def bench_batched(sld, torch, reps=3):
    """64 independent layered cubes (side ~ U{32..160}) in one batched
    persistent launch (FP32 inner, FP64 refinement), against the same
    systems solved one at a time."""
    from paper_1510_02148_gb300 import workloads as W
    probs = W.batch(64, seed=1)
    systems = []
    for P in probs:
        s = sld.System(torch.from_numpy(P.K.reshape(-1)).cuda(), None, P.bc_type, P.bc_value, shape=P.shape)
        s.make_labels(P.S, P.tau, P.L)
        s.build_deflation(P.d)
        systems.append(s)
    xs = [torch.empty(P.n, dtype=torch.float64, device="cuda") for P in probs]
    t0 = time.perf_counter()
    bt = sld.Batch(systems, precision=sld.FP32_IR)
    plan_s = time.perf_counter() - t0
    bt.solve(xs=xs)
    times = []
    infos = None
    for _ in range(reps):
        _, infos = bt.solve(xs=xs)
        times.append(infos[0].solve_ms)
    ms = statistics.median(times)
    seq = 0.0
    for s, x in zip(systems, xs):
        _, i1 = s.solve(x=x, precision=sld.FP32_IR)
        seq += i1.solve_ms
    cells = sum(P.n for P in probs)
    # the batched kernel streams the single solve's arrays (16-bit labels): 60 B per cell-iteration
    alg = sum(P.n * (BYTES_ITER_FP32 * i.iterations + BYTES_OUTER * i.outer_steps) for P, i in zip(probs, infos))
    peak, peak_kind = _peaks()
    gbs = alg / (ms * 1e-3) / 1e9
    out = {"systems": len(probs), "cells": cells, "ms": ms, "solves_per_s": len(probs) / (ms * 1e-3),
           "alg_gbs": gbs,
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                        "traffic": None, "bytes_per_cell_iter": BYTES_ITER_FP32, "peak_kind": peak_kind,
                        "kernel": "k_solve_tma_batch_p<float, float, 8, 3, 1> (one launch, all systems)"},
           "iterations_total": sum(i.iterations for i in infos),
           "max_true_relres": max(i.true_relres for i in infos),
           "one_at_a_time_ms": seq, "speedup_vs_one_at_a_time": seq / ms, "plan": bt.describe(),
           "plan_and_tune_s": plan_s}
    bt.close()
    for s in systems:
        s.close()
    return out


LEARNED_WEIGHTS = os.path.join(ROOT, "paper_1510_02148_gb300", "data", "learned_c4.npz")


def bench_learned(sld, torch, nfields=4):
    """Learned extra deflation vectors on held-out 128^3 lognormal-layered
    fields (contrast 10^c, c ~ U[4, 6], 4x4x2 subdomains x 2 levelsets = 64
    label columns + 8 learned): FP32-inner solves with label deflation alone
    vs label + learned columns, and plain FP64 label deflation; the network
    weights are the committed ones trained by paper_1510_02148_gb300.learned."""
    from paper_1510_02148_gb300 import learned
    if not os.path.exists(LEARNED_WEIGHTS):
        return {"unavailable": "no trained weights committed"}
    params, meta = learned.load_params(LEARNED_WEIGHTS)
    n = int(meta["n"])
    net = sld.Net((n, n, n))
    net.set_params(params.astype(np.float32))
    rows = []
    for seed in range(learned.EVAL_SEED0, learned.EVAL_SEED0 + nfields):
        P = learned.field(seed, n)
        s = learned.build_system(P)
        x = torch.empty(P.n, dtype=torch.float64, device="cuda")
        s.solve(x=x, precision=sld.FP64)
        _, f64 = s.solve(x=x, precision=sld.FP64)
        s.solve(x=x, precision=sld.FP32_IR)
        _, f32 = s.solve(x=x, precision=sld.FP32_IR)
        t0 = time.perf_counter()
        net.infer(s)  # sld_learned_infer: network on the system's K, columns appended to its labels
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        ku = s.deflation_info()[2]
        s.solve(x=x, precision=sld.FP32_IR)
        _, lrn = s.solve(x=x, precision=sld.FP32_IR)
        # the automatic labels (connected components of the levelset classes) instead
        _, dcc = s.make_labels_cc(P.S, P.tau, P.L)
        s.build_deflation(dcc)
        s.solve(x=x, precision=sld.FP32_IR)
        _, cc = s.solve(x=x, precision=sld.FP32_IR)
        rows.append((f64, f32, lrn, setup_ms, ku, cc, dcc))
        s.close()
    net.close()
    med = lambda v: float(statistics.median(v))  # noqa: E731
    return {"workload": f"held-out learned-case fields {n}^3 (seeds {learned.EVAL_SEED0}..), d = 64 + 8 learned",
            "fields": nfields, "trained_on": meta,
            "fp64_plain_ms": med([r[0].solve_ms for r in rows]), "fp64_plain_its": med([r[0].iterations for r in rows]),
            "fp32ir_plain_ms": med([r[1].solve_ms for r in rows]),
            "fp32ir_plain_its": med([r[1].iterations for r in rows]),
            "fp32ir_learned_ms": med([r[2].solve_ms for r in rows]),
            "fp32ir_learned_its": med([r[2].iterations for r in rows]),
            "learned_setup_ms": med([r[3] for r in rows]), "k_used": [r[4] for r in rows],
            "max_true_relres": max(r[2].true_relres for r in rows),
            "speedup_learned_vs_fp64_plain": med([r[0].solve_ms / r[2].solve_ms for r in rows]),
            "speedup_learned_vs_fp32ir_plain": med([r[1].solve_ms / r[2].solve_ms for r in rows]),
            "fp32ir_auto_labels_ms": med([r[5].solve_ms for r in rows]),
            "fp32ir_auto_labels_its": med([r[5].iterations for r in rows]),
            "auto_labels_d": [r[6] for r in rows]}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1510_02148_gb300 import workloads as W
    import oracle
    P = W.lognormal_point_source()
    A = oracle.assemble(P.K, P.q, P.bc_type, P.bc_value)
    lab = oracle.labels(P.K, P.S, P.tau, P.L)
    # the oracle's own full iteration count for this workload, from a full
    # oracle solve recorded by tests/golden/make_ref_iterations.py
    full_iters = int(os.environ.get("SLD_REF_FULL_ITERS", "0")) or None
    if full_iters is None:
        gp = os.path.join(ROOT, "tests", "golden", "ref_iterations.json")
        if os.path.exists(gp):
            with open(gp) as f:
                full_iters = json.load(f).get(P.name, {}).get("iterations")
    vals = []
    cb = None
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(P, A, lab, iters_full=full_iters, sample_iters=8)
        if k >= args.warmup:
            vals.append(cb["value"])
    v = statistics.median(vals)
    full = None
    if args.ref_full_solve:
        # one whole oracle solve, timed, beside the per-step samples: checks
        # the extrapolation and the recorded iteration count
        t0 = time.perf_counter()
        r = oracle.dpcg(A, lab, P.d, tol=P.tol)
        full_ms = (time.perf_counter() - t0) * 1e3
        full = {"ms": full_ms, "iterations": r.iterations, "true_relres": r.true_relres,
                "recorded_iterations": full_iters,
                "iterations_match_record": full_iters is None or r.iterations == full_iters,
                "extrapolated_over_measured": v / full_ms}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "FP64 oracle (CPU)"},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": v,
                             "unit": "ms"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if full is not None:
        line["full_solve_measured"] = full
    print(json.dumps(line), flush=True)
    return 0


def profile_solve(args):
    """One solve of the bench workload (optionally on another grid and with
    an iteration cap), so that a profiler captures exactly one launch of the
    persistent solve kernel."""
    import torch
    from paper_1510_02148_gb300 import _build, sld, workloads as W
    _build.build()
    sld.load()
    shape = tuple(args.shape) if args.shape else (256, 256, 128)
    if args.profile_workload == "inclusions":
        P = W.inclusion_field(*shape, S=(8, 8, 8), a_range=tuple(max(4, int(a * shape[0] / 512)) for a in (16, 96)))[0]
    else:
        P = W.lognormal_point_source(*shape, seed=1)
    q = None if P.q is None else torch.from_numpy(P.q.reshape(-1)).cuda()
    s = sld.System(torch.from_numpy(P.K.reshape(-1)).cuda(), q, P.bc_type, P.bc_value, shape=P.shape)
    s.make_labels(P.S, P.tau, P.L)
    s.build_deflation(P.d)
    x = torch.empty(P.n, dtype=torch.float64, device="cuda")
    prec = {"fp64": sld.FP64, "fp32_ir": sld.FP32_IR, "bf16": sld.BF16COEF_IR}[args.profile_solve]
    kw = {"maxiter": args.maxiter} if args.maxiter > 0 else {}
    _, info = s.solve(x=x, precision=prec, raise_on_error=False, **kw)
    torch.cuda.synchronize()
    s.close()
    print(json.dumps({"profile_solve": args.profile_solve, "shape": shape, "status": info.status,
                      "iterations": info.iterations, "outer_steps": info.outer_steps, "solve_ms": info.solve_ms,
                      "kernel_path": info.kernel_path}), flush=True)
    return 0 if info.status in (sld.OK, sld.ERR_NOT_CONVERGED) else 1


def profile_net(args):
    """The deflation-vector network on a cubic grid (side --shape's nx,
    default 64) with the fixed initial weights of the training driver: one
    forward pass, then --net-steps training steps (forward, subspace loss
    and gradients, Adam) against synthetic targets -- for profiler captures
    of the convolution kernels."""
    import torch
    from paper_1510_02148_gb300 import _build, learned, sld, workloads as W
    _build.build()
    sld.load()
    n = args.shape[0] if args.shape else 64
    P = W.learned_field(0, n=n)
    K = torch.from_numpy(P.K.reshape(-1)).cuda()
    g = torch.Generator(device="cpu").manual_seed(0)
    V = torch.randn((P.n, 8), generator=g, dtype=torch.float32).cuda()
    D = torch.ones(P.n, dtype=torch.float64, device="cuda")
    net = sld.Net((n, n, n))
    net.set_params(learned.init_params(0))
    out = torch.empty((P.n, 8), dtype=torch.float32, device="cuda")
    net.forward(K, out=out)
    losses = []
    for step in range(1, args.net_steps + 1):
        net.forward(K, keep=True)
        losses.append(net.loss_backward(V, D))
        net.adam(1e-3, step)
    torch.cuda.synchronize()
    net.close()
    print(json.dumps({"profile_net": n, "steps": args.net_steps, "losses": losses}), flush=True)
    return 0


def profile_batch(args):
    """One batched launch (no autotune trials: a fixed shape of four CTAs per
    SM) over 16 layered cubes with sides 64..128 -- the batch workload's
    recipe on a narrower side range -- so that a profiler captures exactly
    one launch of the batched solve kernel."""
    import torch
    from paper_1510_02148_gb300 import _build, sld, workloads as W
    _build.build()
    sld.load()
    probs = W.batch(16, side_range=(64, 128), seed=1)
    systems = []
    for P in probs:
        s = sld.System(torch.from_numpy(P.K.reshape(-1)).cuda(), None, P.bc_type, P.bc_value, shape=P.shape)
        s.make_labels(P.S, P.tau, P.L)
        s.build_deflation(P.d)
        systems.append(s)
    xs = [torch.empty(P.n, dtype=torch.float64, device="cuda") for P in probs]
    kw = {"maxiter": args.maxiter} if args.maxiter > 0 else {}
    bt = sld.Batch(systems, precision=sld.FP32_IR, ctas_per_sm=4, **kw)
    _, infos = bt.solve(xs=xs, raise_on_error=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_batch": len(probs), "cells": sum(P.n for P in probs),
                      "iterations": [i.iterations for i in infos], "solve_ms": infos[0].solve_ms}), flush=True)
    bt.close()
    for s in systems:
        s.close()
    return 0 if all(i.status in (sld.OK, sld.ERR_NOT_CONVERGED) for i in infos) else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-gmres", action="store_true")
    ap.add_argument("--no-auto-labels", action="store_true")
    ap.add_argument("--no-spe10", action="store_true")
    ap.add_argument("--spe10-fp64", action="store_true",
                    help="also plain FP64 solves in the SPE10-shaped sweep (about a minute more)")
    ap.add_argument("--no-c2", action="store_true")
    ap.add_argument("--no-c0", action="store_true")
    ap.add_argument("--ref-full-solve", type=int, default=1,
                    help="reference arm: also time one full oracle solve (1) or not (0)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--profile-solve", choices=["fp64", "fp32_ir", "bf16"], default=None,
                    help="set up the workload and run one solve (for profiler captures); no timing line")
    ap.add_argument("--maxiter", type=int, default=0,
                    help="with --profile-solve / --profile-batch: inner iteration cap")
    ap.add_argument("--profile-net", action="store_true",
                    help="run the deflation-vector network (forward, training steps) on a cube (for profiler captures)")
    ap.add_argument("--net-steps", type=int, default=3, help="with --profile-net: training steps")
    ap.add_argument("--profile-batch", action="store_true",
                    help="set up 16 layered cubes and run one batched launch (for profiler captures); no timing line")
    ap.add_argument("--shape", type=int, nargs=3, default=None, help="with --profile-solve: grid nx ny nz")
    ap.add_argument("--profile-workload", choices=["lognormal", "inclusions"], default="lognormal",
                    help="with --profile-solve: the lognormal point-source field or the inclusion field")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_batch:
        return profile_batch(args)
    if args.profile_net:
        return profile_net(args)
    if args.profile_solve:
        return profile_solve(args)

    import torch
    from paper_1510_02148_gb300 import _build, replicas, sld, workloads as W

    world, rank, local = replicas.init(cuda=True)
    torch.cuda.set_device(local)
    _build.build()
    sld.load()
    stream = torch.cuda.current_stream()

    P = W.lognormal_point_source(seed=replicas.replica_seed(rank))
    Kd = torch.from_numpy(P.K.reshape(-1)).cuda()
    qd = torch.from_numpy(P.q.reshape(-1)).cuda()
    t0 = time.perf_counter()
    s = sld.System(Kd, qd, P.bc_type, P.bc_value, stream=stream.cuda_stream, shape=P.shape)
    s.make_labels(P.S, P.tau, P.L)
    s.build_deflation(P.d)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    x = torch.empty(P.n, dtype=torch.float64, device="cuda")

    def barrier():
        replicas.barrier(cuda=True)

    # --- plain FP64 (comparison) ---
    fp64 = []
    for _ in range(1 + args.fp64_steps):
        _, info64 = s.solve(x=x, precision=sld.FP64)
        fp64.append(info64)
    fp64_ms = statistics.median(i.solve_ms for i in fp64[1:])
    # --- mixed precision (headline) ---
    for _ in range(args.warmup):
        s.solve(x=x, precision=sld.FP32_IR)
    infos = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            _, info = s.solve(x=x, precision=sld.FP32_IR)
            infos.append(info)
        ev1.record(stream)
        barrier()
    total_ms = ev0.elapsed_time(ev1)
    ms_step = replicas.max_over_ranks(total_ms / args.steps, cuda=True)
    info = infos[-1]
    kern_ms = statistics.median(i.solve_ms for i in infos)
    n = P.n
    alg_bytes = n * (BYTES_ITER_FP32 * info.iterations + BYTES_OUTER * info.outer_steps)
    hbm_peak, peak_kind = _peaks()
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    alg64 = n * (BYTES_ITER_FP64 * fp64[-1].iterations + BYTES_OUTER * fp64[-1].outer_steps)
    # --- end to end through the public API: host K, q in, host x out ---
    Kh = torch.from_numpy(P.K.reshape(-1)).pin_memory()
    qh = torch.from_numpy(P.q.reshape(-1)).pin_memory()
    xh = torch.empty(P.n, dtype=torch.float64).pin_memory()
    e2e = []
    for k in range(3):
        barrier()
        t = time.perf_counter()
        s2 = sld.System(Kh, qh, P.bc_type, P.bc_value, stream=stream.cuda_stream, shape=P.shape)
        s2.make_labels(P.S, P.tau, P.L)
        s2.build_deflation(P.d)
        s2.solve(x=xh, precision=sld.FP32_IR)
        barrier()
        e2e.append((time.perf_counter() - t) * 1e3)
        s2.close()
    e2e_ms = statistics.median(e2e)

    line = {
        "metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 refinement",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "d": P.d, "precision": "FP32_IR",
                   "l2": "inputs larger than L2 (faces+vectors ~0.9 GB)", "parallelism": "replicas"},
        "iterations": info.iterations, "outer_steps": info.outer_steps, "true_relres": info.true_relres,
        "fp64": {"ms": fp64_ms, "iterations": fp64[-1].iterations, "true_relres": fp64[-1].true_relres,
                 "alg_gbs": alg64 / (fp64_ms * 1e-3) / 1e9},
        "speedup_vs_fp64": fp64_ms / kern_ms,
        "hbm_gbs": achieved,
        "setup_ms": setup_ms,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak,
                     "traffic": (TRAFFIC_RATIO_FP32 * alg_bytes if TRAFFIC_RATIO_FP32 else None),
                     "kernel": "k_solve_tma<float, float, 8, 3, true, false> (persistent, cooperative)", "peak_kind": peak_kind},
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(Kh.numel() * 8 + qh.numel() * 8),
                "d2h_bytes_per_step": int(xh.numel() * 8),
                "what": "sld_build_system(host K, q) + make_labels + build_deflation + sld_solve -> host x"},
        "gpu_launches": 3 * args.steps,
        "clocks": clk.summary(),
    }
    def leg(key, fn, *a):
        # the side legs report an error in their own entry instead of losing the line
        try:
            line[key] = fn(*a)
        except Exception as ex:  # noqa: BLE001
            line[key] = {"error": f"{type(ex).__name__}: {ex}"}

    if not args.no_batched:
        leg("batched", bench_batched, sld, torch)
    if not args.no_learned:
        leg("learned", bench_learned, sld, torch)
    if not args.no_gmres:
        leg("pdgmres", bench_gmres, sld, torch, s, x, P)
    if not args.no_auto_labels:
        leg("auto_labels", bench_auto_labels, sld, torch, P, x)
    if not args.no_spe10:
        leg("spe10_like", bench_spe10, sld, torch, args.spe10_fp64)
    if not args.no_c2:
        leg("c2_inclusions", bench_c2, sld, torch)
    if not args.no_c0:
        leg("c0_sandwich", bench_c0, sld, torch)
    if rank == 0 and not args.no_cpu:
        leg("cpu_baseline", cpu_baseline, P, None, None, fp64[-1].iterations, 30, None, 4)
    s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    replicas.finish()
    return 0


if __name__ == "__main__":
    sys.exit(main())
