#!/usr/bin/env python
"""Time-to-1e-8 of SAIT-preconditioned GMRES and the SAIT-apply HBM bandwidth on one GB300.

Workload (default): 7-point central-difference convection-diffusion on a 128^3
grid (n = 2,097,152, nnz(A) = 14,581,760; convection (1, 0.5, 0.25) scaled to a
cell Peclet number of 0.5), b = A x_true with x_true ~ U[-1, 1] (seeded).  One
step is the whole hot path on the device: ILU(0) factors (GPU, level
scheduled), the SAIT matrices of L and U (m = 3 series terms, row-relative drop
1e-3), and GMRES(50) with z = M_U (M_L r) to a relative residual of 1e-8.

Printed: the benchmark JSON line, last.  `value` is the time to a 1e-8
solution in ms (lower is better); `roofline` is the dominant kernel group of
the step, the SAIT apply (two SELL-32 products), measured live in the timed
steps; `rooflines` adds the A product and the Gram-Schmidt step;
`apply_rooflines` times the apply alone with the factors stored in FP64, FP32
and BF16; `baseline_trisolve` is the same GMRES with the exact
level-scheduled ILU substitutions; `cpu_baseline` is the whole step run by the
FP64 oracle on one host core.  With the extra workloads on (the default), a
`{"bench_detail": ...}` line with their full record comes before the
benchmark line, and `extras` in the benchmark line summarizes it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --case eigen --grid 48               # one extra workload once (profiling)
    python bench.py --summarize-launches launches.csv   # per-kernel table of an ncu launch list
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "time-to-1e-8 residual & SAIT-apply HBM GB/s (% peak) vs level-scheduled trisolve"
APPLY_EVERY = 8  # the timed steps time one SAIT apply in APPLY_EVERY
TOL = 1e-8
RESTART = 50
DROP, TAU = "rowrel", 1e-3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--m", type=int, default=3, help="series terms of SAIT")
    ap.add_argument("--store", default="f64", choices=["f64", "f32", "bf16", "f32x64", "bf16x64"])
    ap.add_argument("--no-extras", action="store_true", help="skip comparator and sweep runs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", choices=["bicgstab", "pcg", "trisolve", "batched", "rhs", "eigen", "adjoint"],
                    help="run one extra workload once at --grid (for profiling) and print its record")
    ap.add_argument("--host-loop", action="store_true",
                    help="with --case: replay the batched solvers' iteration graph from the host instead of "
                         "looping inside a conditional graph node (kernel profilers skip the kernels of graphs "
                         "with conditional nodes)")
    ap.add_argument("--summarize-launches", metavar="CSV",
                    help="print the per-kernel table of an ncu launch list (--metrics gpu__time_duration.sum --csv)")
    return ap.parse_args()


def summarize_launches(path):
    """Per-kernel launches, total time and share of an ncu launch list."""
    import collections
    import csv
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}
    with open(path) as f:
        rows = list(csv.reader(f))
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hdr]
    ki, mi, vi, ui = (h.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hdr + 1:]:
        if len(r) > vi and r[mi] == "gpu__time_duration.sum":
            name = r[ki].split("(")[0].replace("<unnamed>::", "")
            agg[name][0] += 1
            agg[name][1] += float(r[vi].replace(",", "")) * scale[r[ui]]
    tot = sum(v[1] for v in agg.values())
    print(f"launches {sum(v[0] for v in agg.values())}, total {tot / 1e3:.1f} ms (serialised, cold cache)")
    print("| kernel | launches | total ms | share | avg us |\n|---|---|---|---|---|")
    for k, (c, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        if t / tot >= 0.001:
            print(f"| {k} | {c} | {t / 1e3:.2f} | {100 * t / tot:.1f}% | {t / c:.1f} |")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def config_dict(a, A, world=1):
    """The workload, identical for both arms."""
    return {"workload": workload_name(a), "n": A.n, "nnz_A": A.nnz, "m_terms": a.m, "drop": DROP, "tau": TAU,
            "store": a.store, "solver": f"gmres({RESTART})", "tol": TOL,
            "l2": "inputs larger than L2 (A 175 MB, SAIT pair 0.5 GB, GMRES basis 0.86 GB)",
            "parallelism": "replicas" if world > 1 else "single device"}


def workload_name(a):
    return (f"convdiff3d {a.grid}^3 (Pe 0.5): GPU ILU(0) + SAIT(m_terms={a.m}, {DROP} {TAU:g}, "
            f"{a.store}) + GMRES({RESTART}) to {TOL:g}")


# ---- clocks -------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


# ---- the step ----------------------------------------------------------------------
class Problem:
    def __init__(self, grid: int, device):
        import torch
        self.A = synth.convdiff3d(grid)
        xt = synth.uniform(synth.SEED_BASE + 2, self.A.n)
        self.b = self.A.to_scipy() @ xt
        self.host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
                     for k, v in (("rp", self.A.rp), ("ci", self.A.ci), ("va", self.A.va), ("b", self.b))}
        self.dev = {k: v.to(device) for k, v in self.host.items()}
        self.h2d_bytes = sum(v.numel() * v.element_size() for v in self.host.values())
        self.d2h_bytes = self.A.n * 8


def sait_step(sg, ctx, P: Problem, d, m, store, solver="gmres"):
    """One pass of the hot path on device-resident inputs d; returns (x, info, extra)."""
    n = P.A.n
    L, U = sg.sait_ilu0(ctx, n, d["rp"], d["ci"], d["va"])
    ML = sg.sait_build(ctx, L, True, m, DROP, TAU, store=store)
    MU = sg.sait_build(ctx, U, False, m, DROP, TAU, store=store)
    Am = sg.sait_mat_create_csr(ctx, n, d["rp"], d["ci"], d["va"])
    pre = sg.sait_prec_create_sait(ctx, ML, MU)
    if solver == "gmres":
        x, info, st = sg.sait_gmres(ctx, Am, pre, d["b"], restart=RESTART, tol=TOL, maxit=20000)
    else:
        x, info, st = sg.sait_bicgstab(ctx, Am, pre, d["b"], tol=TOL, maxit=20000)
    # the objects are returned so that their teardown falls after the timed region
    return x, info, {"nnz_ML": ML.nnz, "nnz_MU": MU.nnz, "nnz_L": L.nnz, "nnz_U": U.nnz}, \
        (L, U, ML, MU, Am, pre)


def trisolve_step(sg, ctx, P: Problem, d):
    n = P.A.n
    L, U = sg.sait_ilu0(ctx, n, d["rp"], d["ci"], d["va"])
    Am = sg.sait_mat_create_csr(ctx, n, d["rp"], d["ci"], d["va"])
    pre = sg.sait_prec_create_ilu(ctx, L, U)
    x, info, st = sg.sait_gmres(ctx, Am, pre, d["b"], restart=RESTART, tol=TOL, maxit=20000)
    return x, info, sg.sait_prec_levels(pre), (L, U, Am, pre)


def concat_block_diag(mats):
    """Block-diagonal CSR of independent systems (numpy; input assembly only)."""
    n = sum(m.n for m in mats)
    rp = np.zeros(n + 1, dtype=np.int64)
    ci, va, r0, e0 = [], [], 0, 0
    for m in mats:
        rp[r0 + 1:r0 + m.n + 1] = m.rp[1:].astype(np.int64) + e0
        ci.append(m.ci.astype(np.int64) + r0)
        va.append(m.va)
        r0 += m.n
        e0 += m.nnz
    return synth.CSR(n, rp.astype(np.int32), np.concatenate(ci).astype(np.int32), np.concatenate(va))


def batched_workloads(sg, ctx, torch, device, stream):
    """Many independent systems and many right-hand sides (one run each, FP32 and FP64 SAIT)."""
    out = {}
    sides, eps = synth.aniso2d_batch_params(512, synth.SEED_BASE + 4)
    systems = [synth.aniso2d(int(s_), float(e_)) for s_, e_ in zip(sides, eps)]
    A = concat_block_diag(systems)
    ptr = np.concatenate([[0], np.cumsum([m.n for m in systems])]).astype(np.int64)
    b = A.to_scipy() @ synth.uniform(synth.SEED_BASE + 5, A.n)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in
         (("rp", A.rp), ("ci", A.ci), ("va", A.va), ("b", b), ("ptr", ptr))}
    out["tile_autotune"] = sg.sait_batch_autotune(ctx, A.n, d["ptr"]).as_dict()  # setup, before the timed solves

    def solve_batch(store):
        s0, s1, s2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        s0.record(stream)
        L, U = sg.sait_ilu0(ctx, A.n, d["rp"], d["ci"], d["va"])
        ML = sg.sait_build(ctx, L, True, 3, DROP, TAU, store=store)
        MU = sg.sait_build(ctx, U, False, 3, DROP, TAU, store=store)
        s1.record(stream)
        P = sg.sait_prec_create_sait(ctx, ML, MU)
        Am = sg.sait_mat_create_csr(ctx, A.n, d["rp"], d["ci"], d["va"])
        x, info, st, rr, its = sg.sait_bicgstab_batched(ctx, Am, P, d["ptr"], d["b"], tol=TOL, maxit=5000,
                                                        check=False)
        s2.record(stream)
        s2.synchronize()
        row_iters = float((its.cpu().numpy().astype(np.float64) * np.diff(ptr)).sum())
        return info, (s0.elapsed_time(s1), s1.elapsed_time(s2), ML.nnz, MU.nnz, row_iters), (L, U, P, Am, x)

    res = {}
    for store in ("f32", "f32x64", "f64"):
        solve_batch(store)                                   # warm-up (graph capture, pools)
        ms, (info, (b_ms, s_ms, nl, nu, row_iters), keep) = time_region(torch, stream, lambda: solve_batch(store))
        del keep
        it = max(info.graph_replays, 1)
        bytes_it = batched_iter_bytes(A, nl, nu, store, 1, row_iters, it)
        bnd = batched_iter_bound(A, nl, nu, store, 1, row_iters, it)
        res[store] = {"ms": round(ms, 3), "build_ms": round(b_ms, 3), "solve_ms": round(s_ms, 3),
                      "ms_per_iteration": round(s_ms / it, 4), "bytes_per_iteration": bytes_it,
                      "gbs_per_iteration": round(bytes_it / (s_ms / it) / 1e6, 1),
                      "frac_per_iteration": round(bytes_it / (s_ms / it) / 1e6 / peaks()[0], 4),
                      "bound_ms_per_iteration": round(bnd["bound_ms"], 4),
                      "frac_of_bound": round(bnd["bound_ms"] / (s_ms / it), 4), **info.as_dict()}
    out["independent_systems"] = {"nsys": len(systems), "n": A.n, "nnz": A.nnz,
                                  "sides": [int(sides.min()), int(sides.max())], "solver": "bicgstab",
                                  "m_terms": 3, "tol": TOL, **res}
    del d
    torch.cuda.empty_cache()
    # one 128^3 Poisson, 64 right-hand sides
    A = synth.laplace3d(128)
    k = 64
    Xt = synth.uniform(synth.SEED_BASE + 6, (A.n, k))
    B = np.ascontiguousarray(A.to_scipy() @ Xt)
    del Xt
    d = {kk: torch.from_numpy(np.ascontiguousarray(v)).to(device) for kk, v in
         (("rp", A.rp), ("ci", A.ci), ("va", A.va), ("B", B))}
    del B

    def solve_multi(store):
        s0, s1, s2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        s0.record(stream)
        L, U = sg.sait_ilu0(ctx, A.n, d["rp"], d["ci"], d["va"])
        ML = sg.sait_build(ctx, L, True, 3, DROP, TAU, store=store)
        MU = sg.sait_build(ctx, U, False, 3, DROP, TAU, store=store)
        s1.record(stream)
        P = sg.sait_prec_create_sait(ctx, ML, MU)
        Am = sg.sait_mat_create_csr(ctx, A.n, d["rp"], d["ci"], d["va"])
        X, info, st, rr, its = sg.sait_bicgstab_multi(ctx, Am, P, d["B"], tol=TOL, maxit=5000, check=False)
        s2.record(stream)
        s2.synchronize()
        row_iters = float(its.cpu().numpy().astype(np.float64).sum()) * A.n
        return info, (s0.elapsed_time(s1), s1.elapsed_time(s2), ML.nnz, MU.nnz, row_iters), (L, U, P, Am, X)

    res = {}
    for store in ("f32", "f32x64", "f64"):
        solve_multi(store)
        ms, (info, (b_ms, s_ms, nl, nu, row_iters), keep) = time_region(torch, stream, lambda: solve_multi(store))
        del keep
        it = max(info.graph_replays, 1)
        bytes_it = batched_iter_bytes(A, nl, nu, store, k, row_iters, it)
        bnd = batched_iter_bound(A, nl, nu, store, k, row_iters, it)
        res[store] = {"ms": round(ms, 3), "build_ms": round(b_ms, 3), "solve_ms": round(s_ms, 3),
                      "ms_per_iteration": round(s_ms / it, 4), "bytes_per_iteration": bytes_it,
                      "gbs_per_iteration": round(bytes_it / (s_ms / it) / 1e6, 1),
                      "frac_per_iteration": round(bytes_it / (s_ms / it) / 1e6 / peaks()[0], 4),
                      "bound_ms_per_iteration": round(bnd["bound_ms"], 4),
                      "frac_of_bound": round(bnd["bound_ms"] / (s_ms / it), 4), **info.as_dict()}
    out["many_rhs"] = {"n": A.n, "k": k, "solver": "bicgstab", "m_terms": 3, "tol": TOL, **res}
    del d
    torch.cuda.empty_cache()
    return out


def eigen_workload(sg, ctx, torch, device, stream, factors="ilut"):
    """16 smallest eigenpairs of 96^3 log-normal diffusion by SAIT-preconditioned LOBPCG."""
    A = synth.varcoef3d(96, 1.0, synth.SEED_BASE + 3)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in
         (("rp", A.rp), ("ci", A.ci), ("va", A.va))}
    X0 = torch.from_numpy(synth.uniform(synth.SEED_BASE + 10, (A.n, 16))).to(device)

    def solve(store):
        if factors == "ilut":
            L, U = sg.sait_ilut(ctx, A.n, d["rp"], d["ci"], d["va"], 1e-4, 10)
        else:
            L, U = sg.sait_ilu0(ctx, A.n, d["rp"], d["ci"], d["va"])
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, DROP, TAU, store=store),
                                     sg.sait_build(ctx, U, False, 3, DROP, TAU, store=store))
        Am = sg.sait_mat_create_csr(ctx, A.n, d["rp"], d["ci"], d["va"])
        lam, X, info, st = sg.sait_lobpcg(ctx, Am, P, X0.clone(), tol=TOL, maxit=1000, check=False)
        return lam, info, st, (L, U, P, Am, X)

    out = {"n": A.n, "k": 16, "factors": factors, "m_terms": 3, "tol": TOL}
    ref = None
    for store in ("f64", "f32", "bf16"):
        solve(store)
        ms, (lam, info, st, keep) = time_region(torch, stream, lambda: solve(store))
        del keep
        lam = lam.cpu().numpy()
        if ref is None:
            ref = lam
        out[store] = {"ms": round(ms, 3), "iters": info.iters, "max_resid": info.rel_resid, "status": st,
                      "max_rel_eig_diff_vs_f64": float(np.abs(lam - ref).max() / np.abs(ref).max()),
                      "lambda_min": float(lam[0]), "lambda_max": float(lam[-1])}
    out["vs_oracle"] = eigen_vs_oracle(sg, ctx, torch, device)
    return out


def eigen_vs_oracle(sg, ctx, torch, device):
    """The same eigenproblem at the size of the stored FP64 oracle run
    (tests/golden/eigen_varcoef<G>.json, written by make_eigen_fixture.py): the
    largest relative eigenvalue error of each storage against the oracle."""
    here = os.path.join(ROOT, "tests", "golden")
    fixtures = sorted(f for f in os.listdir(here) if f.startswith("eigen_varcoef") and f.endswith(".json"))
    if not fixtures:
        return None
    with open(os.path.join(here, fixtures[-1])) as f:
        fx = json.load(f)
    A = synth.varcoef3d(fx["grid"], 1.0, synth.SEED_BASE + 3)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in
         (("rp", A.rp), ("ci", A.ci), ("va", A.va))}
    X0 = torch.from_numpy(synth.uniform(synth.SEED_BASE + 10, (A.n, fx["k"]))).to(device)
    ref8 = np.array(fx["tol_1e-8"]["lambda"])
    ref11 = np.array(fx["tol_1e-11"]["lambda"])
    out = {"grid": fx["grid"], "n": A.n, "oracle_iters_1e-8": fx["tol_1e-8"]["iters"]}
    for store in ("f64", "f32", "bf16"):
        L, U = sg.sait_ilut(ctx, A.n, d["rp"], d["ci"], d["va"], 1e-4, 10)
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, DROP, TAU, store=store),
                                     sg.sait_build(ctx, U, False, 3, DROP, TAU, store=store))
        Am = sg.sait_mat_create_csr(ctx, A.n, d["rp"], d["ci"], d["va"])
        lam, X, info, st = sg.sait_lobpcg(ctx, Am, P, X0.clone(), tol=TOL, maxit=1000, check=False)
        lam = lam.cpu().numpy()
        out[store] = {"iters": info.iters, "status": st,
                      "max_rel_eig_err_vs_oracle": float(np.abs(lam - ref8).max() / np.abs(ref8).max()),
                      "max_rel_eig_err_vs_oracle_tight": float(np.abs(lam - ref11).max() / np.abs(ref11).max())}
    return out


def paper_replica_workload(sg, ctx, torch, device, stream):
    """Section 4's experiment on the GPU: 100^3 Laplacian, level-0 and level-1 ILU,
    PCG to 1e-10 with SAIT_Thr(tau, 10), SAIT_Pat(p, 10), the exact substitution
    and k Jacobi sweeps."""
    A = synth.laplace3d(100)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in
         (("rp", A.rp), ("ci", A.ci), ("va", A.va))}
    b = torch.from_numpy(synth.uniform(synth.SEED_BASE, A.n, 0.0, 1.0)).to(device)
    Am = sg.sait_mat_create_csr(ctx, A.n, d["rp"], d["ci"], d["va"])
    tol, m = 1e-10, 10

    def pcg(P):
        sg.sait_pcg(ctx, Am, P, b, tol=tol, maxit=2000, check=False)    # warm-up
        ms, (_, info, st) = time_region(torch, stream,
                                        lambda: sg.sait_pcg(ctx, Am, P, b, tol=tol, maxit=2000, check=False))
        return {"iters": info.iters, "pcg_ms": round(ms, 3), "rel_resid": info.rel_resid, "status": st}

    out = {"n": A.n, "tol": tol, "m": m, "maxit": 2000}
    for level in (0, 1):
        ms_f, (L, U) = time_region(torch, stream, lambda: sg.sait_iluk(ctx, A.n, d["rp"], d["ci"], d["va"], level))
        lev = {"ilu_ms": round(ms_f, 3), "nnz_L": L.nnz, "exact_ilu": pcg(sg.sait_prec_create_ilu(ctx, L, U)),
               "rows": []}
        for name, drop, tau, p in [("SAIT_Thr(0.05,10)", "abs", 0.05, 0), ("SAIT_Thr(0.02,10)", "abs", 0.02, 0),
                                   ("SAIT_Thr(0.01,10)", "abs", 0.01, 0), ("SAIT_Pat(1,10)", "pattern", 0.0, 1),
                                   ("SAIT_Pat(2,10)", "pattern", 0.0, 2), ("SAIT_Pat(3,10)", "pattern", 0.0, 3)]:
            terms = m + 1 + p
            sg.sait_build(ctx, L, True, terms, drop, tau, p)       # warm-up
            ms_b, (ML, MU) = time_region(torch, stream, lambda: (sg.sait_build(ctx, L, True, terms, drop, tau, p),
                                                                 sg.sait_build(ctx, U, False, terms, drop, tau, p)))
            row = {"name": name, "ratio": round(MU.nnz / U.nnz, 2), "build_ms": round(ms_b, 3)}
            row.update(pcg(sg.sait_prec_create_sait(ctx, ML, MU)))
            row["total_ms"] = round(row["build_ms"] + row["pcg_ms"], 3)
            lev["rows"].append(row)
        lev["jacobi"] = [{"sweeps": k, **pcg(sg.sait_prec_create_jacobi(ctx, L, U, k))} for k in (1, 2, 3, 4, 10)]
        out[f"level{level}"] = lev
    return out


def autotune_workload(sg, ctx, torch, device, stream, P: "Problem", m, store):
    """Product autotuning on the benchmark matrices: every candidate kernel's time and the choice."""
    d = P.dev
    L, U = sg.sait_ilu0(ctx, P.A.n, d["rp"], d["ci"], d["va"])
    ML = sg.sait_build(ctx, L, True, m, DROP, TAU, store=store)
    MU = sg.sait_build(ctx, U, False, m, DROP, TAU, store=store)
    Am = sg.sait_mat_create_csr(ctx, P.A.n, d["rp"], d["ci"], d["va"])
    return {"A": sg.sait_mat_autotune(ctx, Am).as_dict(), "M_L": sg.sait_mat_autotune(ctx, ML).as_dict(),
            "M_U": sg.sait_mat_autotune(ctx, MU).as_dict()}


PARAM_CANDIDATES = [
    {"m_terms": 2, "drop": "rowrel", "tau": 1e-3}, {"m_terms": 3, "drop": "rowrel", "tau": 1e-3},
    {"m_terms": 4, "drop": "rowrel", "tau": 1e-3}, {"m_terms": 3, "drop": "rowrel", "tau": 3e-3},
    {"m_terms": 4, "drop": "rowrel", "tau": 1e-2}, {"m_terms": 4, "drop": "hybrid", "tau": 1e-2, "p": 1},
    {"m_terms": 3, "drop": "pattern", "p": 1},
]


def optimal_params_workload(sg, ctx, P: "Problem", store):
    """The optimal parameters of Section 3 on the benchmark problem: each
    candidate's SAIT build + GMRES(50) solve timed by sait_tune_params."""
    n = P.A.n
    d = P.dev
    L, U = sg.sait_ilu0(ctx, n, d["rp"], d["ci"], d["va"])
    Am = sg.sait_mat_create_csr(ctx, n, d["rp"], d["ci"], d["va"])
    _, rep = sg.sait_tune_params(ctx, Am, L, U, d["b"], PARAM_CANDIDATES, solver="gmres", restart=RESTART,
                                 tol=TOL, maxit=20000, store=store, count_build=True)
    out = rep.as_dict(PARAM_CANDIDATES)
    out["chosen_param"] = PARAM_CANDIDATES[rep.chosen] if rep.chosen >= 0 else None
    out["measure"] = "build_ms + solve_ms (one solve per preconditioner), ILU(0) excluded"
    return out


def adjoint_workload(sg, ctx, torch, device, stream):
    """Forward + backward of the differentiable solve on 64^3 log-normal diffusion."""
    from paper_2106_12836_gb300.autograd import SolveOptions, sait_solve
    A = synth.varcoef3d(64, 1.0, synth.SEED_BASE + 7)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in
         (("rp", A.rp), ("ci", A.ci), ("va", A.va))}
    b = torch.from_numpy(synth.uniform(synth.SEED_BASE + 8, A.n)).to(device)
    xt = torch.from_numpy(synth.uniform(synth.SEED_BASE + 9, A.n)).to(device)
    opts = SolveOptions(restart=50, tol=TOL, store="f32")

    def run():
        vals = d["va"].clone().requires_grad_(True)
        bb = b.clone().requires_grad_(True)
        x = sait_solve(vals, bb, d["rp"], d["ci"], ctx, opts)
        loss = 0.5 * ((x - xt) ** 2).sum()
        loss.backward()
        return vals.grad

    run()
    ms, _ = time_region(torch, stream, run)
    return {"n": A.n, "ms_forward_backward": round(ms, 3), "store": "f32", "restart": 50, "tol": TOL}


def apply_precisions(sg, ctx, torch, device, stream, P: "Problem", m, flush_l2, peak, reps=20):
    """The SAIT apply z = M_U (M_L r) of the benchmark factors stored in FP64, FP32
    and BF16: each apply timed alone with CUDA events on the context stream, L2
    flushed before each, against its algorithmic bytes."""
    d = P.dev
    L, U = sg.sait_ilu0(ctx, P.A.n, d["rp"], d["ci"], d["va"])
    r = torch.from_numpy(synth.uniform(synth.SEED_BASE + 11, P.A.n)).to(device)
    z = torch.empty_like(r)
    out = {}
    for store in ("f64", "f32", "bf16"):
        ML = sg.sait_build(ctx, L, True, m, DROP, TAU, store=store)
        MU = sg.sait_build(ctx, U, False, m, DROP, TAU, store=store)
        for _ in range(3):
            sg.sait_apply(ctx, ML, MU, r, z)
        ms = []
        for _ in range(reps):
            flush_l2()
            t, _ = time_region(torch, stream, lambda: sg.sait_apply(ctx, ML, MU, r, z))
            ms.append(t)
        t = statistics.median(ms)
        b = apply_bytes(P.A.n, ML.nnz, MU.nnz, store)
        out[store] = {"ms": round(t, 4), "algorithmic_bytes": b, "achieved": round(b / t / 1e6, 1),
                      "peak": peak, "unit": "GB/s", "frac": round(b / t / 1e6 / peak, 4)}
        del ML, MU
    return out


def batched_iter_bytes(A, nnz_ml, nnz_mu, store, k, row_iters=None, replays=1):
    """Algorithmic bytes of one batched BiCGSTAB iteration over all systems (k
    right-hand sides; k = 1 for the independent systems): two SAIT applies and
    two products with A, each matrix read once for all k columns, and the 22
    FP64 vector passes of the recurrences (dots, p, s, x and r updates).  The
    products run over every row in every iteration; the vector passes skip the
    systems (columns) that have converged, so with row_iters = the sum over
    systems of iterations x rows (n x the sum of the columns' iterations) they
    are counted for the rows still iterating, averaged over the replays."""
    n = A.n
    sv = {"f64": 8, "f32": 4, "bf16": 2, "f32x64": 4, "bf16x64": 2}[store]
    vec = 32 if store in ("f64", "f32x64", "bf16x64") else 24        # r in, w out + in, z out, per column
    apply_b = (nnz_ml + nnz_mu) * (sv + 4) + 2 * 4 * (n + 1) + vec * n * k
    spmv_b = A.nnz * 12 + 4 * (n + 1) + 16 * n * k
    vec_rows = n * k if row_iters is None else row_iters / replays
    return int(2 * apply_b + 2 * spmv_b + 22 * 8 * vec_rows)


# FP64 fused multiply-adds per SM per clock on GB300 (152 SMs, 2070 MHz maximum
# clock: 1.26 TFLOP/s, the nominal FP64 rate); the 64^3 x 64 block product with
# A ran 115.9 M FMAs in 203.7 us at 92.3% FP64-pipe busy (ncu), 1.96 per SM clock.
FP64_FMA_PER_SM_CLK = 2
SM_COUNT, SM_MAX_MHZ = 152, 2070


def fp64_fma_rate():
    """FP64 multiply-adds per second at the maximum SM clock."""
    return FP64_FMA_PER_SM_CLK * SM_COUNT * SM_MAX_MHZ * 1e6


def batched_iter_bound(A, nnz_ml, nnz_mu, store, k, row_iters=None, replays=1):
    """Lower bound (ms) on one batched BiCGSTAB iteration: each part of the
    iteration takes at least the longer of its algorithmic bytes at the
    measured copy bandwidth and its FP64 multiply-adds at the FP64 rate.  With
    k columns every matrix entry feeds k FP64 multiply-adds, so for k = 64 the
    products of A (and, in the FP64-arithmetic storage modes, the two SAIT
    products) are bound by the FP64 pipe, not by HBM.  The FP32 storage mode
    multiplies in FP32, whose rate is 64 times the FP64 one.  The vector passes
    do 12 FP64 multiply-adds per iterating row and column (6 dot terms, 6 in the
    updates) against 176 bytes."""
    n = A.n
    bw = peaks()[0] * 1e6       # bytes per ms
    fma = fp64_fma_rate() / 1e3  # per ms
    sv = {"f64": 8, "f32": 4, "bf16": 2, "f32x64": 4, "bf16x64": 2}[store]
    vec = 32 if store in ("f64", "f32x64", "bf16x64") else 24
    apply_b = (nnz_ml + nnz_mu) * (sv + 4) + 2 * 4 * (n + 1) + vec * n * k
    apply_f = (nnz_ml + nnz_mu) * k if store in ("f64", "f32x64", "bf16x64") else 0
    spmv_b = A.nnz * 12 + 4 * (n + 1) + 16 * n * k
    spmv_f = A.nnz * k
    vec_rows = n * k if row_iters is None else row_iters / replays
    parts = [(apply_b, apply_f)] * 2 + [(spmv_b, spmv_f)] * 2 + [(22 * 8 * vec_rows, 12 * vec_rows)]
    return {"bound_ms": sum(max(b / bw, f / fma) for b, f in parts),
            "fp64_fma": int(sum(f for _, f in parts)),
            "fp64_bound_parts": sum(1 for b, f in parts if f / fma > b / bw)}


def apply_bytes(n, nnz_l, nnz_u, store):
    sv = {"f64": 8, "f32": 4, "bf16": 2, "f32x64": 4, "bf16x64": 2}[store]
    vec = 32 * n if store in ("f64", "f32x64", "bf16x64") else 24 * n   # r in, w out+in, z out
    return (nnz_l + nnz_u) * (sv + 4) + 2 * 4 * (n + 1) + vec


# DRAM bytes (read + write) per launch from ncu captures, scaled to the benchmark size
# where the capture ran on a smaller grid: the two SELL-32 FP64 products of one SAIT
# apply on the 96^3 factors (8,709,408 entries each) moved 115,658,752 B (M_L) and
# 115,724,544 B (M_U); scaled by entries to the two 128^3 factors (20,726,144 each).
TRAFFIC = {"128:3:f64": {"apply": round((115658752 + 115724544) * 20726144 / 8709408)}}


def ortho_bytes(n, iters, restart):
    """Algorithmic bytes of the DCGS2 Gram-Schmidt work of `iters` Arnoldi steps."""
    total, left = 0, iters
    while left > 0:
        steps = min(left, restart)
        for j in range(steps):
            # DCGS2 step j over the j final basis vectors kept as (hi FP32, m16) pairs:
            #   dual dot sweep  read hi (4 B per vector), fl32(u) and w (FP64)
            #   update sweep    read hi + m16 (6 B per vector), read u and w (FP64), write
            #                   w1' (FP64), v_j's hi and m16 and fl32(w1')
            total += 10 * j * n + (4 + 8 + 16 + 8 + 6 + 4) * n
        left -= steps
    return total


def spmv_a_bytes(A):
    return A.nnz * 12 + 4 * (A.n + 1) + 16 * A.n


def time_region(torch, ctx_stream, fn):
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(ctx_stream)
    out = fn()
    e.record(ctx_stream)
    e.synchronize()
    return s.elapsed_time(e), out


# ---- CPU baseline: the oracle, the whole solve ------------------------------------
def oracle_problem(grid):
    """The benchmark's matrix and right-hand side (same seed as the GPU arm)."""
    A = synth.convdiff3d(grid)
    xt = synth.uniform(synth.SEED_BASE + 2, A.n)
    return A, A.to_scipy() @ xt


def oracle_solve(A, b, m, maxit=20000):
    """One full step on the host: oracle ILU(0) + SAIT build of L and U + GMRES(50)
    to the tolerance, one thread.  Returns (ms, sample description, steps, relres)."""
    import oracle
    t0 = time.perf_counter()
    L, U = oracle.ilu0(A)
    ML = oracle.sait(L, m, DROP, TAU)
    MU = oracle.sait(U, m, DROP, TAU)
    t1 = time.perf_counter()
    _, it, rr, st = oracle.gmres(A, b, "sait", ML, MU, restart=RESTART, tol=TOL, maxit=maxit)
    t2 = time.perf_counter()
    sample = (f"oracle, 1 thread, the whole step measured (nothing scaled): ILU(0) + SAIT build of L and U "
              f"({t1 - t0:.2f} s) and GMRES({RESTART}) to {TOL:g}, {it} Arnoldi steps ({t2 - t1:.2f} s, "
              f"status {st}, relres {rr:.2e})")
    return (t2 - t0) * 1e3, sample, it, rr


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A, b = oracle_problem(a.grid)
    # warm-up (untimed): page the oracle and the problem in with a bounded step,
    # the factors and one GMRES cycle
    for _ in range(a.warmup):
        oracle_solve(A, b, a.m, maxit=RESTART)
    vals, last = [], ""
    for _ in range(a.steps):
        v, sample, _, _ = oracle_solve(A, b, a.m)
        vals.append(v)
        last = sample
    v = statistics.mean(vals)
    print(json.dumps({
        "metric": METRIC, "impl": "reference", "value": round(v, 1), "unit": "ms", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(a, A),
        "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": 1, "kind": "oracle", "sample": last,
                         "step_ms": [round(x, 1) for x in vals]},
        "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def max_over_ranks(dist, value: float, device) -> float:
    """The slowest replica's time: every rank solves its own system (weak scaling)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


# ---- our arm -----------------------------------------------------------------------
def run_ours(a):
    import torch
    import paper_2106_12836_gb300 as sg
    from paper_2106_12836_gb300 import build as sgb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    sgb.build()
    peak, peak_kind = peaks()

    P = Problem(a.grid, device)
    n = P.A.n
    ctx = sg.Context()
    stream = ctx.stream
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=device)

    def flush_l2():
        flush.fill_(1)

    # The timed steps record CUDA events around every APPLY_EVERY-th SAIT apply only
    # (the dominant kernel, whose roofline they give): events between kernels cost
    # launch overlap.  The other groups' times come from as many further steps with
    # every call of every group timed.  The timers are on during the warm-up too, so
    # their CUDA events already exist when the timed steps start.
    sg.sait_ctx_set_timing(ctx, True)
    sg.sait_ctx_set_timing_groups(ctx, ["apply"], APPLY_EVERY)
    for _ in range(max(a.warmup, 0)):
        res = sait_step(sg, ctx, P, P.dev, a.m, a.store)
        del res
    torch.cuda.synchronize()
    sg.sait_ctx_stats(ctx, reset=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(1.0)  # let the sampler start up before the timed steps (its start-up competes for the host)
    times, infos, extra = [], [], {}
    for _ in range(a.steps):
        flush_l2()
        ms, (x, info, extra, keep) = time_region(torch, stream,
                                                 lambda: sait_step(sg, ctx, P, P.dev, a.m, a.store))
        del keep
        times.append(ms)
        infos.append(info.as_dict())
    torch.cuda.synchronize()
    clk = clocks.stop()
    stats = sg.sait_ctx_stats(ctx, reset=True).as_dict()
    # the same steps again with every group timed: the breakdown and the other rooflines
    sg.sait_ctx_set_timing_groups(ctx, None, 1)
    times_all = []
    for _ in range(a.steps):
        flush_l2()
        ms, (_, _, _, keep) = time_region(torch, stream, lambda: sait_step(sg, ctx, P, P.dev, a.m, a.store))
        del keep
        times_all.append(ms)
    torch.cuda.synchronize()
    stats_all = sg.sait_ctx_stats(ctx, reset=True).as_dict()
    sg.sait_ctx_set_timing(ctx, False)
    ms_step = statistics.mean(times)
    if dist:
        ms_step = max_over_ranks(dist, ms_step, device)
        dist.barrier()
    torch.cuda.synchronize()

    # true residual of the last solution, checked in FP64 on the host
    xr = x.cpu().numpy()
    relres = float(np.linalg.norm(P.b - P.A.to_scipy() @ xr) / np.linalg.norm(P.b))

    # ---- end to end through the C ABI from host (pinned) buffers
    def e2e():
        d = {k: v.to(device, non_blocking=True) for k, v in P.host.items()}
        xx, _, _, keep = sait_step(sg, ctx, P, d, a.m, a.store)
        return xx.to("cpu", non_blocking=True), keep, d

    # one untimed pass first: the device copies of the inputs come from torch's
    # caching allocator, whose first request for them maps new memory
    flush_l2()
    _ = time_region(torch, stream, e2e)
    del _
    e2e_times = []
    for _ in range(min(a.steps, 3)):
        flush_l2()
        ms, _ = time_region(torch, stream, e2e)
        e2e_times.append(ms)

    # ---- rooflines from the live timers of the timed steps
    iters = infos[-1]["iters"]
    groups = {g: stats_all[g]["ms"] for g in ("apply", "spmv", "ortho", "build", "ilu")}
    ab = apply_bytes(n, extra["nnz_ML"], extra["nnz_MU"], a.store)
    apply_ms = stats["apply"]["ms"] / max(stats["apply"]["calls"], 1)
    ob = ortho_bytes(n, iters, RESTART) * a.steps
    ortho_ms = stats_all["ortho"]["ms"]
    sb = spmv_a_bytes(P.A)
    spmv_ms = stats_all["spmv"]["ms"] / max(stats_all["spmv"]["calls"], 1)
    rl = {
        "apply": {"kernel": "k_spmv_sell x2 (M_L then M_U, SELL-32), one SAIT apply", "bound": "hbm",
                  "achieved": ab / apply_ms / 1e6, "bytes": ab, "ms": apply_ms,
                  "calls": stats["apply"]["calls"]},
        "ortho": {"kernel": "GMRES DCGS2 step (k_dcgs_dot with its scalar step, k_dcgs_update with the rotation)",
                  "bound": "hbm", "achieved": ob / max(ortho_ms, 1e-9) / 1e6,
                  "bytes": ob / max(stats_all["ortho"]["calls"], 1),
                  "ms": ortho_ms / max(stats_all["ortho"]["calls"], 1), "calls": stats_all["ortho"]["calls"]},
        "spmv": {"kernel": "k_spmv_sell (A, FP64)", "bound": "hbm", "achieved": sb / spmv_ms / 1e6,
                 "bytes": sb, "ms": spmv_ms, "calls": stats_all["spmv"]["calls"]},
    }
    for r in rl.values():
        r.update(peak=peak, unit="GB/s", frac=r["achieved"] / peak, peak_kind=peak_kind)
    # The dominant kernel is k_spmv_sell (the largest share of the ncu launch list; it
    # serves the SAIT apply and the A product), reported through the SAIT apply.
    dom = "apply"
    traffic = {"apply": None, "ortho": None, "spmv": None}
    traffic.update(TRAFFIC.get(f"{a.grid}:{a.m}:{a.store}", {}))

    def roof(g, full=True):
        r = rl[g]
        o = {"bound": r["bound"], "achieved": round(r["achieved"], 1), "peak": peak, "unit": "GB/s",
             "frac": round(r["frac"], 4), "traffic": traffic.get(g), "algorithmic_bytes_per_launch": int(r["bytes"]),
             "avg_ms": round(r["ms"], 4), "launches_timed": r["calls"]}
        if full:
            o.update(kernel=r["kernel"], peak_source=f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)")
        return o

    out = {
        "metric": METRIC, "value": round(ms_step, 3), "unit": "ms", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(a, P.A, world),
        "l2_flush": "a 512 MB write before every timed step",
        "clocks": clk,
        "e2e": {"value": round(statistics.mean(e2e_times), 3), "unit": "ms",
                "h2d_bytes_per_step": P.h2d_bytes, "d2h_bytes_per_step": P.d2h_bytes},
        "gpu_launches": stats["launches"],
        "roofline": roof(dom),
        # per group: achieved GB/s, fraction of peak, average ms per launch
        "rooflines": {g: {"achieved": round(rl[g]["achieved"], 1), "frac": round(rl[g]["frac"], 4),
                          "avg_ms": round(rl[g]["ms"], 4)} for g in rl},
        "solve": {"iters": iters, "cycles": infos[-1]["cycles"], "rel_resid_host_check": float(f"{relres:.4e}"),
                  "step_ms_min_max": [round(min(times), 3), round(max(times), 3)], **extra},
        "breakdown_ms_per_step": {g: round(v / a.steps, 3) for g, v in groups.items()},
        "group_timing": {"timed_steps": f"CUDA events around every {APPLY_EVERY}th SAIT apply only (roofline)",
                         "breakdown_and_other_rooflines": f"{a.steps} further steps with every group timed, "
                                                          f"{statistics.mean(times_all):.3f} ms per step"},
    }

    detail = {}
    if not a.no_extras:
        # exact level-scheduled ILU substitution in the same GMRES (comparator)
        flush_l2()
        sg.sait_ctx_set_timing(ctx, True)
        sg.sait_ctx_stats(ctx, reset=True)
        ms_t, (xt_, info_t, levels, keep) = time_region(torch, stream, lambda: trisolve_step(sg, ctx, P, P.dev))
        del keep
        st_t = sg.sait_ctx_stats(ctx, reset=True).as_dict()
        baseline = {
            "ms": round(ms_t, 3), "iters": info_t.iters, "rel_resid": float(f"{info_t.rel_resid:.3e}"),
            "levels": list(levels),
            "avg_trisolve_pair_ms": round(st_t["trisolve"]["ms"] / max(st_t["trisolve"]["calls"], 1), 4),
            "speedup_of_sait": round(ms_t / ms_step, 3)}
        sg.sait_ctx_set_timing(ctx, False)
        # the apply with the factors stored in FP64 / FP32 / BF16
        apr = apply_precisions(sg, ctx, torch, device, stream, P, a.m, flush_l2, peak)
        detail["apply_rooflines"] = apr
        # the whole step with reduced-precision SAIT storage (one run each)
        ss = {}
        for store in ("f32", "bf16"):
            sait_step(sg, ctx, P, P.dev, a.m, store)
            flush_l2()
            ms_s, (xs, info_s, _, keep) = time_region(torch, stream,
                                                      lambda: sait_step(sg, ctx, P, P.dev, a.m, store))
            del keep
            rr = float(np.linalg.norm(P.b - P.A.to_scipy() @ xs.cpu().numpy()) / np.linalg.norm(P.b))
            ss[store] = {"ms": round(ms_s, 3), "iters": info_s.iters, "rel_resid_host_check": rr}
        store_sweep = ss
        # BiCGSTAB with the same SAIT preconditioner
        flush_l2()
        ms_b, (_, info_b, _, keep) = time_region(
            torch, stream, lambda: sait_step(sg, ctx, P, P.dev, a.m, a.store, "bicgstab"))
        del keep
        detail["bicgstab"] = {"ms": round(ms_b, 3), "iters": info_b.iters, "rel_resid": info_b.rel_resid}
        # m sweep (one run each)
        sweep = []
        sg.sait_ctx_set_timing(ctx, True)
        for m in (2, 3, 4, 6):
            flush_l2()
            sg.sait_ctx_stats(ctx, reset=True)
            ms_m, (_, info_m, ex_m, keep) = time_region(torch, stream,
                                                        lambda: sait_step(sg, ctx, P, P.dev, m, a.store))
            del keep
            st_m = sg.sait_ctx_stats(ctx, reset=True).as_dict()
            sweep.append({"m_terms": m, "ms": round(ms_m, 3), "iters": info_m.iters,
                          "nnz_ML": ex_m["nnz_ML"], "nnz_MU": ex_m["nnz_MU"],
                          "build_ms": round(st_m["build"]["ms"], 3),
                          "apply_ms": round(st_m["apply"]["ms"] / max(st_m["apply"]["calls"], 1), 4)})
        detail["m_sweep"] = sweep
        sg.sait_ctx_set_timing(ctx, False)
        detail["batched"] = batched_workloads(sg, ctx, torch, device, stream)
        detail["adjoint"] = adjoint_workload(sg, ctx, torch, device, stream)
        detail["eigen"] = eigen_workload(sg, ctx, torch, device, stream)
        detail["paper_replica"] = paper_replica_workload(sg, ctx, torch, device, stream)
        detail["autotune"] = autotune_workload(sg, ctx, torch, device, stream, P, a.m, a.store)
        detail["optimal_params"] = optimal_params_workload(sg, ctx, P, a.store)
        out["extras"] = summarize_extras(detail)
        # the apply with FP64 / FP32 / BF16 factors: [ms, fraction of peak]
        out["apply_rooflines"] = {k: [v["ms"], v["frac"]] for k, v in apr.items()}
        out["store_sweep"] = store_sweep
        out["baseline_trisolve"] = baseline

    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        A_h, b_h = oracle_problem(a.grid)
        v, sample, it_o, _ = oracle_solve(A_h, b_h, a.m)
        out["cpu_baseline"] = {"value": round(v, 1), "unit": "ms", "cores": 1, "kind": "oracle",
                               "sample": sample, "oracle_steps": it_o}
    if rank == 0:
        if detail:
            # the full record of the extra workloads first; the benchmark line is the last line
            print(json.dumps({"bench_detail": detail}), flush=True)
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def summarize_extras(d):
    """A few numbers per extra workload, short enough to stay in the benchmark line."""
    s = {}
    if "bicgstab" in d:
        s["bicgstab"] = {k: d["bicgstab"][k] for k in ("ms", "iters")}
    if "m_sweep" in d:
        s["m_sweep_ms"] = {str(r["m_terms"]): round(r["ms"], 1) for r in d["m_sweep"]}
    if "batched" in d:
        b = d["batched"]
        for key, name in (("independent_systems", "batched_512"), ("many_rhs", "rhs_64")):
            # per storage: [build ms, solve ms, max iterations, GB/s per iteration, fraction of
            # the HBM peak, fraction of the HBM + FP64 bound]
            s[name] = {st: [round(b[key][st]["build_ms"], 1), round(b[key][st]["solve_ms"], 1),
                            b[key][st]["max_iters"], round(b[key][st]["gbs_per_iteration"]),
                            b[key][st]["frac_per_iteration"], b[key][st]["frac_of_bound"]]
                       for st in ("f64", "f32", "f32x64") if st in b[key]}
    if "adjoint" in d:
        s["adjoint_ms"] = d["adjoint"]["ms_forward_backward"]
    if "eigen" in d:
        e = d["eigen"]
        # per storage at 96^3: [ms, iterations, eigenvalue difference to the FP64 run]
        s["eigen96"] = {k: [round(e[k]["ms"]), e[k]["iters"], float(f"{e[k]['max_rel_eig_diff_vs_f64']:.1e}")]
                        for k in ("f64", "f32", "bf16") if k in e}
        vo = e.get("vs_oracle")
        if vo:
            s[f"eig_err_vs_oracle_{vo['grid']}"] = {k: float(f"{vo[k]['max_rel_eig_err_vs_oracle']:.1e}")
                                                   for k in ("f64", "f32", "bf16") if k in vo}
    if "paper_replica" in d:
        p = d["paper_replica"]
        short = {"SAIT_Thr(0.05,10)": "T.05", "SAIT_Thr(0.02,10)": "T.02", "SAIT_Thr(0.01,10)": "T.01",
                 "SAIT_Pat(1,10)": "P1", "SAIT_Pat(2,10)": "P2", "SAIT_Pat(3,10)": "P3"}
        # per row: [nnz ratio, PCG iterations]; exact: the substitution's iterations
        s["paper_replica"] = {f"L{lv}": {"exact": p[f"level{lv}"]["exact_ilu"]["iters"],
                                         **{short[r["name"]]: [r["ratio"], r["iters"]]
                                            for r in p[f"level{lv}"]["rows"]}} for lv in (0, 1)}
    if "optimal_params" in d:
        s["optimal_params_chosen"] = d["optimal_params"].get("chosen_param")
    return s


def run_case(a):
    """One extra workload, once, at a size chosen for profiling (--grid): the
    same code paths as the benchmark's extras."""
    import torch
    import paper_2106_12836_gb300 as sg
    from paper_2106_12836_gb300 import build as sgb
    sgb.build()
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    ctx = sg.Context()
    stream = ctx.stream
    if a.host_loop:
        sg.sait_ctx_set_device_loop(ctx, False)
    g = a.grid
    if a.case in ("bicgstab", "trisolve"):
        P = Problem(g, device)
        if a.case == "bicgstab":
            _, info, _, keep = sait_step(sg, ctx, P, P.dev, a.m, a.store, "bicgstab")
        else:
            _, info, _, keep = trisolve_step(sg, ctx, P, P.dev)
        out = {"case": a.case, "n": P.A.n, "iters": info.iters, "rel_resid": info.rel_resid}
        del keep
    elif a.case == "pcg":
        A = synth.laplace3d(g)
        d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in
             (("rp", A.rp), ("ci", A.ci), ("va", A.va))}
        b = torch.from_numpy(synth.uniform(synth.SEED_BASE, A.n, 0.0, 1.0)).to(device)
        Am = sg.sait_mat_create_csr(ctx, A.n, d["rp"], d["ci"], d["va"])
        L, U = sg.sait_ilu0(ctx, A.n, d["rp"], d["ci"], d["va"])
        P1 = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 11, "abs", 0.05),
                                      sg.sait_build(ctx, U, False, 11, "abs", 0.05))
        _, i1, _ = sg.sait_pcg(ctx, Am, P1, b, tol=1e-10)
        _, i2, _ = sg.sait_pcg(ctx, Am, sg.sait_prec_create_jacobi(ctx, L, U, 2), b, tol=1e-10)
        out = {"case": a.case, "n": A.n, "sait_iters": i1.iters, "jacobi2_iters": i2.iters}
    elif a.case == "batched":
        sides, eps = synth.aniso2d_batch_params(64, synth.SEED_BASE + 4, smax=min(256, max(16, g)))
        systems = [synth.aniso2d(int(s_), float(e_)) for s_, e_ in zip(sides, eps)]
        A = concat_block_diag(systems)
        ptr = np.concatenate([[0], np.cumsum([m.n for m in systems])]).astype(np.int64)
        b = A.to_scipy() @ synth.uniform(synth.SEED_BASE + 5, A.n)
        d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in
             (("rp", A.rp), ("ci", A.ci), ("va", A.va), ("b", b), ("ptr", ptr))}
        L, U = sg.sait_ilu0(ctx, A.n, d["rp"], d["ci"], d["va"])
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, DROP, TAU, store="f32"),
                                     sg.sait_build(ctx, U, False, 3, DROP, TAU, store="f32"))
        Am = sg.sait_mat_create_csr(ctx, A.n, d["rp"], d["ci"], d["va"])
        _, info, st, _, _ = sg.sait_bicgstab_batched(ctx, Am, P, d["ptr"], d["b"], tol=TOL, maxit=5000, check=False)
        out = {"case": a.case, "n": A.n, **info.as_dict()}
    elif a.case == "rhs":
        A = synth.laplace3d(g)
        k = 64
        B = np.ascontiguousarray(A.to_scipy() @ synth.uniform(synth.SEED_BASE + 6, (A.n, k)))
        d = {kk: torch.from_numpy(np.ascontiguousarray(v)).to(device) for kk, v in
             (("rp", A.rp), ("ci", A.ci), ("va", A.va), ("B", B))}
        L, U = sg.sait_ilu0(ctx, A.n, d["rp"], d["ci"], d["va"])
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, DROP, TAU, store="f32"),
                                     sg.sait_build(ctx, U, False, 3, DROP, TAU, store="f32"))
        Am = sg.sait_mat_create_csr(ctx, A.n, d["rp"], d["ci"], d["va"])
        _, info, st, _, _ = sg.sait_bicgstab_multi(ctx, Am, P, d["B"], tol=TOL, maxit=5000, check=False)
        out = {"case": a.case, "n": A.n, "k": k, **info.as_dict()}
    elif a.case == "eigen":
        A = synth.varcoef3d(g, 1.0, synth.SEED_BASE + 3)
        d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in
             (("rp", A.rp), ("ci", A.ci), ("va", A.va))}
        X0 = torch.from_numpy(synth.uniform(synth.SEED_BASE + 10, (A.n, 16))).to(device)
        L, U = sg.sait_ilut(ctx, A.n, d["rp"], d["ci"], d["va"], 1e-4, 10)
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, DROP, TAU, store=a.store),
                                     sg.sait_build(ctx, U, False, 3, DROP, TAU, store=a.store))
        Am = sg.sait_mat_create_csr(ctx, A.n, d["rp"], d["ci"], d["va"])
        lam, X, info, st = sg.sait_lobpcg(ctx, Am, P, X0, tol=TOL, maxit=1000, check=False)
        out = {"case": a.case, "n": A.n, "iters": info.iters, "lambda_min": float(lam[0])}
    else:
        out = {"case": a.case, **adjoint_workload(sg, ctx, torch, device, stream)}
    torch.cuda.synchronize()
    print(json.dumps(out), flush=True)
    ctx.close()


def main():
    a = parse()
    if a.summarize_launches:
        summarize_launches(a.summarize_launches)
        return
    if a.case:
        run_case(a)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
