#!/usr/bin/env python3
"""Benchmark: s-step GMRES with randomized block orthogonalization on one GB300.

Workload (default, one "step"): s-step GMRES(m=60, s=5) on the 7-point 3D Poisson
matrix of a 100^3 grid (n = 1e6, FP64 CSR, Dirichlet), Jacobi right
preconditioner, monomial matrix-powers basis, b = A*1, x0 = 0, solved to a 1e-10
true relative residual -- once with one-stage randomized BCGS2 and once with the
two-stage scheme (s_hat = 20).  `value` is the mean time to solution per solve.
The working set (CSR 88 MB + basis 490 MB + vectors) exceeds the 129 MB L2, so no
L2 flush is needed between steps.

Also reported (the block orthogonalization alone, V = 2^24 x 61 glued blocks,
two-stage s_hat = 30 and one-stage, FP64 and mixed precision): orthogonalized
columns/s, algorithmic HBM GB/s and ||I - Q^T Q||_2, under "orth".

At one GPU it also runs the stress workload's two-stage solves (3D convection-diffusion
256^3, s=10, s_hat=50, m=100, float64 and mixed precision, learned SPAI with Jacobi
fallback) under "stress"; --stress adds the one-stage and Jacobi-only runs, --no-stress
skips it.

`--impl reference` times the CPU oracle (numpy/scipy) on a bounded sample of the
same workload and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "orth cols/s & HBM GB/s at ‖I−QᵀQ‖≤1e-13; s-step GMRES time to 1e-10"
WORKLOAD = "s-step GMRES(m=60, s=5) one-stage + two-stage (s_hat=20), 3D Poisson 7-pt 100^3 (n=1e6), Jacobi, b=A*1, tol 1e-10"
N_GRID, M, S, S_HAT, TOL = 100, 60, 5, 20, 1e-10
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.07e9   # SMs x FP64 FMA/clk/SM x 2 flop x max SM clock


def max_over_ranks(value: float, dist=None, device="cuda") -> float:
    """The largest `value` over all ranks of the process group (the slowest rank
    decides a timing); `value` itself without a process group."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    p = {}
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    return {"hbm_gbs": float(p.get("hbm_gbs", 6800.0)),
            "hbm_src": "measured" if "hbm_gbs" in p else "fallback"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"rbo_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(", ") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import synth
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2503_16717_gb300 as rbo

    A = synth.poisson3d_csr(N_GRID)
    b_host = synth.ones_rhs(A)
    args.n_rows = A.n
    Ad = rbo.DeviceCSR.from_host(A)
    bd = torch.from_numpy(b_host).cuda()
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    launches = {"n": 0}
    last = {}

    def solve(s_hat):
        x.zero_()
        _, info = rbo.sstep_gmres(Ad, bd, x, s=S, s_hat=s_hat, m=M, tol=TOL)
        if info["status"] != 0:
            raise RuntimeError(f"sstep_gmres failed: {info}")
        launches["n"] += info["kernel_launches"] + 1
        return info

    def step():
        last["one"] = solve(0)
        last["two"] = solve(S_HAT)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    # unprofiled timing (the reported value)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches["n"] = 0
    with Clocks(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            step()
        ev1.record()
        barrier()
    ms = ev0.elapsed_time(ev1)
    gpu_launches = launches["n"]
    ms = max_over_ranks(ms, dist, "cuda")
    ms_per_step = ms / args.steps
    sec_per_solve = ms_per_step / 2.0 / 1e3

    # the same solves in float32-pair arithmetic (RBO_PREC_DF64)
    df64 = None
    if not args.no_df64:
        def solve_df(s_hat):
            x.zero_()
            _, info = rbo.sstep_gmres(Ad, bd, x, s=S, s_hat=s_hat, m=M, tol=TOL,
                                      precision=rbo.PREC_DF64)
            if info["status"] != 0:
                raise RuntimeError(f"sstep_gmres df64 failed: {info}")
            return info
        solve_df(0)
        solve_df(S_HAT)
        barrier()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record()
        for _ in range(args.steps):
            i1 = solve_df(0)
            i2 = solve_df(S_HAT)
        d1.record()
        barrier()
        dms = d0.elapsed_time(d1) / args.steps
        df64 = {"s_per_solve": dms / 2.0 / 1e3, "ms_per_step": dms,
                "one_stage": {"iterations": i1["iterations"], "relres": i1["relres"]},
                "two_stage": {"iterations": i2["iterations"], "relres": i2["relres"]}}

    # the same solves with the wide Gram passes on the tensor cores (RBO_PREC_OZAKI:
    # exact digit products, float64 tolerances)
    ozaki = None
    if not args.no_ozaki:
        def solve_oz(s_hat):
            x.zero_()
            _, info = rbo.sstep_gmres(Ad, bd, x, s=S, s_hat=s_hat, m=M, tol=TOL,
                                      precision=rbo.PREC_OZAKI)
            if info["status"] != 0:
                raise RuntimeError(f"sstep_gmres ozaki failed: {info}")
            return info
        solve_oz(0)
        solve_oz(S_HAT)
        barrier()
        z0, z1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        z0.record()
        for _ in range(args.steps):
            o1 = solve_oz(0)
            o2 = solve_oz(S_HAT)
        z1.record()
        barrier()
        zms = z0.elapsed_time(z1) / args.steps
        ozaki = {"s_per_solve": zms / 2.0 / 1e3, "ms_per_step": zms,
                 "one_stage": {"iterations": o1["iterations"], "relres": o1["relres"]},
                 "two_stage": {"iterations": o2["iterations"], "relres": o2["relres"]}}

    # the two-stage solve with BCGS-PIP preprocessing (the paper's deterministic
    # two-stage comparator), same problem
    def solve_pip():
        x.zero_()
        return rbo.sstep_gmres(Ad, bd, x, s=S, s_hat=S_HAT, m=M, tol=TOL,
                               preproc=rbo.PREPROC_PIP)[1]
    solve_pip()
    barrier()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    ipip = solve_pip()
    p1.record()
    barrier()
    pip = {"s_per_solve": p0.elapsed_time(p1) / 1e3, "status": ipip["status"],
           "iterations": ipip["iterations"], "restarts": ipip["restarts"], "relres": ipip["relres"],
           "breakdown_stage": ipip["breakdown_stage_name"]}

    # per-kernel times with CUDA events around each library launch (same steps again)
    if args.no_prof:
        prof, roofline, ms_prof = None, None, None
    else:
        prof, roofline, ms_prof = profile_steps(rbo, torch, step, barrier, args)
        if df64 is not None:
            def step_df():
                solve_df(0)
                solve_df(S_HAT)
            prof_df, _, _ = profile_steps(rbo, torch, step_df, barrier, args)
            df64["rowpass_ms_per_step"] = prof_df["rowpass"]["ms"] / args.steps
            df64["rowpass_by_role"] = {k: {"ms": v["ms"], "tflops": v["tflops"]}
                                       for k, v in prof_df["rowpass_by_role"].items()}

    # end-to-end through the public API with host buffers
    e2e = None if args.no_e2e else run_e2e(rbo, torch, A, b_host, args)

    orth = run_orth(rbo, torch, args) if (rank == 0 and not args.no_orth) else None
    learned_res = run_learned(rbo, torch, args) if (rank == 0 and not args.no_learned) else None
    stress_res = None
    if rank == 0 and (args.stress or (world == 1 and not args.no_stress)):
        stress_res = run_stress(rbo, torch, args, core_only=not args.stress)
    bases_res = run_stress_bases(rbo, torch, args) if (rank == 0 and args.stress_bases) else None
    sweep_res = run_s_sweep(rbo, torch, Ad, bd, args) if (rank == 0 and args.s_sweep) else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(A, b_host, last["one"]["iterations"])

    if rank == 0:
        one, two = last["one"], last["two"]
        line = {
            "metric": METRIC, "value": sec_per_solve, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": A.n, "nnz": A.nnz, "m": M, "s": S, "s_hat": S_HAT,
                       "tol": TOL, "l2": "working set > L2 (no flush)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "solves": {
                "one_stage": {"iterations": one["iterations"], "restarts": one["restarts"],
                              "relres": one["relres"], "kernel_launches": one["kernel_launches"]},
                "two_stage": {"iterations": two["iterations"], "restarts": two["restarts"],
                              "relres": two["relres"], "kernel_launches": two["kernel_launches"]},
            },
            "df64": df64,
            "ozaki": ozaki,
            "two_stage_pip": pip,
            "ms_per_step_profiled": ms_prof,
            "kernels": prof,
            "roofline": roofline,
            "e2e": e2e,
            "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
            "orth": orth,
            "learned": learned_res,
            "stress": stress_res,
            "stress_bases": bases_res,
            "s_sweep": sweep_res,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def measured_traffic(passes, n, launches):
    """DRAM bytes per row-pass launch of the step, from the committed one-kernel captures
    of the two row-pass instances (profiles/rowpass_traffic.json): the Gram instance's
    DRAM/algorithmic ratio applied to the roles without a sketch, and for the update +
    sketch roles their algorithmic bytes plus the measured schedule-record bytes per row.
    None when a row-pass source has changed since the counters were taken."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        with open(os.path.join(here, "profiles", "rowpass_traffic.json")) as f:
            rec = json.load(f)
        sha = {}
        for src in ("rowpass.cu", "rowpass_sk.cu"):
            with open(os.path.join(here, "paper_2503_16717_gb300", "csrc", src), "rb") as f:
                sha[src] = hashlib.sha256(f.read()).hexdigest()
    except (OSError, ValueError):
        return None
    if rec.get("sources_sha256") != sha or not launches:
        return None
    ratio = rec["instances"]["gram"]["ratio"]
    per_row = rec["instances"]["update_sketch"]["schedule_record_bytes_per_row"]
    total = 0.0
    for name, r in passes.items():
        if "update_sketch" in name:
            total += r["bytes"] + per_row * n * r["launches"]
        else:
            total += ratio * r["bytes"]
    return total / launches


def profile_steps(rbo, torch, step, barrier, args):
    rbo.profile_reset()
    rbo.profile_enable(True)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    barrier()
    ms_prof = e0.elapsed_time(e1) / args.steps
    prof = {k: rbo.profile_read(v) for k, v in
            (("rowpass", rbo.PROF_ROWPASS), ("spmv", rbo.PROF_SPMV), ("vector", rbo.PROF_VECTOR))}
    names = {1: "P1_gram", 2: "P2_update_sketch", 3: "P3_trsm_gram", 4: "P4_trsm_gram2",
             5: "P5_reorth_update_gram", 6: "P6_trsm", 7: "T1_gram", 8: "T2_update_sketch",
             9: "T3_forward_subst_gram", 10: "T4_trsm_gram2", 11: "T5_reorth_update_gram",
             12: "T6_trsm", 13: "normalise", 14: "T2p_pip_gram", 0: "other"}
    passes = {}
    for tag, nm in names.items():
        r = rbo.profile_read(8 + tag)
        if r["launches"]:
            r["share_of_rowpass"] = r["ms"] / max(prof["rowpass"]["ms"], 1e-9)
            r["tflops"] = r["flops"] / (r["ms"] / 1e3) / 1e12 if r["ms"] > 0 else 0.0
            r["gbs"] = r["bytes"] / (r["ms"] / 1e3) / 1e9 if r["ms"] > 0 else 0.0
            passes[nm] = r
    prof["rowpass_by_role"] = passes
    rbo.profile_enable(False)
    rp = prof["rowpass"]
    avg_ms = rp["ms"] / max(rp["launches"], 1)
    achieved_flops = rp["flops"] / (rp["ms"] / 1e3) if rp["ms"] > 0 else 0.0
    roofline = {"bound": "alu", "kernel": "rowpass_kernel<0> (fused float64 row pass, all roles)",
                "achieved": achieved_flops / 1e12, "peak": FP64_PEAK_DERIVED / 1e12,
                "unit": "TFLOP/s", "frac": achieved_flops / FP64_PEAK_DERIVED,
                "peak_src": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (FP64 1.25 TFLOP/s nominal)",
                "traffic": measured_traffic(passes, args.n_rows, rp["launches"]),
                "traffic_src": "estimated from one-kernel captures (profiles/rowpass_traffic.json)",
                "launches": rp["launches"], "avg_launch_us": avg_ms * 1e3,
                "hbm_gbs_algorithmic": rp["bytes"] / (rp["ms"] / 1e3) / 1e9 if rp["ms"] > 0 else 0.0,
                "share_of_step": rp["ms"] / args.steps / ms_prof if ms_prof > 0 else None}

    return prof, roofline, ms_prof



def run_e2e(rbo, torch, A, b_host, args):
    """Same solve through the public API, with the matrix and b copied from pinned host
    memory and x read back, every step (one-stage + two-stage solve per step)."""
    import numpy as np
    rp = torch.from_numpy(A.rowptr).pin_memory()
    cl = torch.from_numpy(A.col).pin_memory()
    vl = torch.from_numpy(A.val).pin_memory()
    bh = torch.from_numpy(b_host).pin_memory()
    xh = torch.empty(A.n, dtype=torch.float64).pin_memory()
    h2d = (rp.numel() * 4 + cl.numel() * 4 + vl.numel() * 8 + bh.numel() * 8) * 2
    d2h = xh.numel() * 8 * 2

    def one():
        for s_hat in (0, S_HAT):
            Ad = rbo.DeviceCSR.__new__(rbo.DeviceCSR)
            Ad.n, Ad.nnz = A.n, A.nnz
            Ad.rowptr = rp.cuda(non_blocking=True)
            Ad.col = cl.cuda(non_blocking=True)
            Ad.val = vl.cuda(non_blocking=True)
            bd = bh.cuda(non_blocking=True)
            x, info = rbo.sstep_gmres(Ad, bd, s=S, s_hat=s_hat, m=M, tol=TOL)
            xh.copy_(x, non_blocking=True)
            torch.cuda.synchronize()
            if info["status"] != 0:
                raise RuntimeError(info)

    one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = (time.perf_counter() - t0) / args.steps
    return {"value": dt / 2.0, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


ORTH_TOL = 1e-13   # the metric counts columns/s and GB/s only at ||I - Q^T Q||_2 <= 1e-13
PREC_NAMES = ("fp64", "mixed", "df64", "ozaki")


def _orth_bytes(scheme, c, s, s_hat, n):
    """Algorithmic bytes of one orthogonalization: col-passes of the scheme (every
    n-row column read or written once per pass), times 8n."""
    k = s
    if scheme == "one":
        passes = 2 + sum(4 * p + 11 * k for p in range(1, c, k))
    elif scheme == "two_pip":
        # per panel: C1 Gram (P+k), update (P+2k), PIP reduction (p'+k), forward
        # substitution (p'+2k); big-panel end as RandBCGS2
        passes = 2
        for P in range(1, c, s_hat):
            for j in range(s_hat // s):
                pp = j * k
                passes += (P + k) + (P + 2 * k) + (pp + k) + (pp + 2 * k)
            passes += (P + 2 * s_hat) + (P + 2 * s_hat) + 2 * s_hat
    else:
        passes = 2
        for P in range(1, c, s_hat):
            for j in range(s_hat // s):
                pp = j * k
                passes += (P + k) + (P + 2 * k) + (pp + 2 * k)
            passes += (P + 2 * s_hat) + (P + 2 * s_hat) + 2 * s_hat
    return passes * 8.0 * n


def _orth_call(rbo, sk, Wm, scheme, s, s_hat, prec):
    if scheme == "two":
        return rbo.block_orth_two_stage(sk, Wm, s, s_hat, v0=True, precision=prec, raise_on_error=False)
    if scheme == "two_pip":
        return rbo.block_orth_two_stage(None, Wm, s, s_hat, v0=True, precision=prec,
                                        raise_on_error=False, preproc=rbo.PREPROC_PIP)
    return rbo.block_orth_one_stage(sk, Wm, s, v0=True, precision=prec, raise_on_error=False)


def _orth_err_gpu(rbo, Wm, c):
    import numpy as np
    G = rbo.gram(Wm, Wm)
    return float(np.max(np.abs(np.linalg.eigvalsh(np.eye(c) - 0.5 * (G + G.T)))))


def _rel_fro(torch, A, B):
    """||A - B||_F / ||B||_F on the device, one column at a time (no n x c temporary)."""
    num = den = 0.0
    for j in range(B.shape[1]):
        num += float(torch.sum((A[:, j] - B[:, j]) ** 2))
        den += float(torch.sum(B[:, j] ** 2))
    return (num / den) ** 0.5 if den > 0 else num ** 0.5


def _orth_vs_oracle(rbo, torch, V0, c, s, s_hat, nrows=20000):
    """Every scheme and precision on the first `nrows` rows of the workload's V
    against the CPU oracle (the same sketch): relative R and Q errors."""
    import numpy as np
    from oracle import metrics, orth
    from oracle.sketch import Sketch as OSketch
    Vh = V0[:, :nrows].t().contiguous().cpu().numpy()      # nrows x c
    osk = OSketch(nrows, 4 * c, 8, 42)
    refs = {"one": orth.block_orth_one_stage(Vh, s, osk, v0=True),
            "two": orth.block_orth_two_stage(Vh, s, s_hat, osk, v0=True)}
    sk = rbo.sketch_create(nrows, 4 * c, 8, 42)
    out = []
    for scheme in ("one", "two"):
        ref = refs[scheme]
        for prec in (rbo.PREC_FP64, rbo.PREC_MIXED, rbo.PREC_DF64, rbo.PREC_OZAKI):
            Wd = rbo.colmajor(nrows, c)
            Wd.copy_(torch.from_numpy(Vh))
            o = _orth_call(rbo, sk, Wd, scheme, s, s_hat, prec)
            row = {"scheme": scheme, "precision": PREC_NAMES[prec], "rows": nrows,
                   "status": o.info["status"]}
            if o.info["status"] == 0:
                Q = Wd.cpu().numpy()
                row["r_err_vs_oracle"] = metrics.rel_diff(o.R, ref.R)
                row["q_err_vs_oracle"] = metrics.rel_diff(Q, ref.Q)
                row["orth_err"] = metrics.orth_error(Q)
                row["backward_err"] = metrics.backward_error(Vh, Q, o.R)
            out.append(row)
    return out


def _orth_oracle_timing(torch, V0, c, s, s_hat, nrows=1 << 20):
    """The CPU oracle's block orthogonalization of the workload, timed on its first
    `nrows` rows (one-stage and two-stage, the same sketch parameters) and scaled
    linearly to the full row count: every step of both schemes is a pass over the rows
    or a small factorisation, so the time grows in proportion to n.  A labelled
    estimate, on the host cores."""
    from oracle import orth
    from oracle.sketch import Sketch as OSketch
    n = V0.shape[1]
    nrows = min(nrows, n)
    Vh = V0[:, :nrows].t().contiguous().cpu().numpy()      # nrows x c
    osk = OSketch(nrows, 4 * c, 8, 42)
    t = {}
    for scheme in ("one", "two"):
        t0 = time.perf_counter()
        if scheme == "one":
            orth.block_orth_one_stage(Vh, s, osk, v0=True)
        else:
            orth.block_orth_two_stage(Vh, s, s_hat, osk, v0=True)
        t[scheme] = time.perf_counter() - t0
    scale = n / nrows
    return {"kind": "oracle", "estimate": True, "rows_sampled": nrows, "rows": n,
            "cores": _cpu_threads(),
            "sample_s": t, "est_s": {k: v * scale for k, v in t.items()},
            "est_cols_per_s": {k: c / (v * scale) for k, v in t.items()}}


def run_orth(rbo, torch, args):
    """Block orthogonalization alone on V = 2^24 x 61 (v0 + 12 glued blocks of 5).

    Per (kappa, scheme, precision): time, ||I - Q^T Q||_2 and, only for calls that
    return status 0 at ||I - Q^T Q||_2 <= 1e-13 (the metric's condition), columns/s and
    algorithmic GB/s; a failed call keeps its status and error and reports no
    throughput.  Mixed and float32-pair results carry their relative R and Q errors
    against the float64 result on the same input, and at kappa = 1e4 every precision is
    also compared with the CPU oracle on the first 20000 rows."""
    import numpy as np
    import synth
    n, nb, s, s_hat = 1 << 24, 12, 5, 30
    c = nb * s + 1
    out = []
    kappas = [1e8] if args.quick_orth else [1e4, 1e8, 1e12, 1e14]
    sk = rbo.sketch_create(n, 4 * c, 8, 42)
    V0 = synth.glued_blocks_torch(n, nb, s, kappas[0], seed=1, v0=True, device="cuda")
    W = torch.empty_like(V0)
    Q64 = torch.empty_like(V0)
    vs_oracle = None
    oracle_time = None
    for kappa in kappas:
        if kappa != kappas[0]:
            del V0
            torch.cuda.empty_cache()
            V0 = synth.glued_blocks_torch(n, nb, s, kappa, seed=1, v0=True, device="cuda")
        if kappa == 1e4 and not args.no_cpu:
            vs_oracle = _orth_vs_oracle(rbo, torch, V0, c, s, s_hat)
            oracle_time = _orth_oracle_timing(torch, V0, c, s, s_hat)
        for scheme in ("two", "one", "two_pip"):
            R64 = None
            for prec in ((rbo.PREC_FP64,) if scheme == "two_pip" else
                         (rbo.PREC_FP64, rbo.PREC_MIXED, rbo.PREC_DF64, rbo.PREC_OZAKI)):
                Wm = W.t()  # n x c column-major view
                times = []
                info = None
                for rep in range(3):
                    W.copy_(V0)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    o = _orth_call(rbo, sk, Wm, scheme, s, s_hat, prec)
                    e1.record()
                    torch.cuda.synchronize()
                    if rep > 0:
                        times.append(e0.elapsed_time(e1))
                    info = o.info
                ms = min(times)
                status = info["status"]
                oe = _orth_err_gpu(rbo, Wm, c) if status == 0 else None
                valid = status == 0 and oe is not None and oe <= ORTH_TOL
                gb = _orth_bytes(scheme, c, s, s_hat, n) / 1e9
                row = {"kappa": kappa, "scheme": scheme, "precision": PREC_NAMES[prec],
                       "status": status, "ms": ms, "orth_err": oe, "valid": valid,
                       "cols_per_s": c / (ms / 1e3) if valid else None,
                       "hbm_gbs_algorithmic": gb / (ms / 1e3) if valid else None,
                       "launches": info["kernel_launches"], "fallbacks": info.get("fallbacks", 0)}
                if status != 0:
                    row["breakdown_stage"] = info.get("breakdown_stage_name")
                if prec == rbo.PREC_FP64 and status == 0:
                    Q64.copy_(W)
                    R64 = o.R.copy()
                elif prec != rbo.PREC_FP64 and R64 is not None and status == 0:
                    nr = np.linalg.norm(R64)
                    row["r_err_vs_fp64"] = float(np.linalg.norm(o.R - R64) / nr)
                    row["q_err_vs_fp64"] = _rel_fro(torch, W.t(), Q64.t())
                out.append(row)
    # sketch types (Section 5.2): the same orthogonalizations (kappa of the last
    # sweep entry) with the Gaussian, Count and Count-Gauss maps
    kinds = [("sparse_sign", dict(d=4 * c, zeta=8)),
             ("count", dict(d=4 * c, zeta=1)),
             ("gaussian", dict(d=2 * s_hat, kind=rbo.SKETCH_GAUSSIAN)),
             ("count_gauss", dict(d=2 * s_hat, kind=rbo.SKETCH_COUNT_GAUSS, d_inner=4 * c))]
    types = []
    for name, kw in kinds:
        skt = rbo.sketch_create(n, kw.pop("d"), seed=42, **kw)
        for scheme in ("one", "two"):
            Wm = W.t()
            times = []
            for rep_ in range(3):
                W.copy_(V0)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                o = _orth_call(rbo, skt, Wm, scheme, s, s_hat, rbo.PREC_FP64)
                e1.record()
                torch.cuda.synchronize()
                if rep_ > 0:
                    times.append(e0.elapsed_time(e1))
            ms = min(times)
            oe = _orth_err_gpu(rbo, Wm, c) if o.info["status"] == 0 else None
            valid = o.info["status"] == 0 and oe is not None and oe <= ORTH_TOL
            gb = _orth_bytes(scheme, c, s, s_hat, n) / 1e9
            types.append({"sketch": name, "d": skt.d, "scheme": scheme, "kappa": kappas[-1],
                          "status": o.info["status"], "ms": ms, "orth_err": oe, "valid": valid,
                          "cols_per_s": c / (ms / 1e3) if valid else None,
                          "hbm_gbs_algorithmic": gb / (ms / 1e3) if valid else None})
    del V0, W, Q64
    torch.cuda.empty_cache()
    return {"n": n, "cols": c, "s": s, "s_hat": s_hat, "d": 4 * c, "results": out,
            "sketch_types": types, "vs_oracle_20000_rows": vs_oracle,
            "cpu_oracle_kappa_1e4": oracle_time}


def run_learned(rbo, torch, args):
    """Learned SPAI preconditioner on the convection-diffusion family (config 3): train
    on 256 generated instances at 512^2 with residuals from Jacobi s-step GMRES,
    evaluate s-step GMRES(m=60, s=5, s_hat=30) to 1e-10 against Jacobi on unseen
    instances at 2048^2 (n = 4.19M): the first 4 of the 32 by default, all 32 with
    --learned-full; --learned-quick: 32 training instances at 128^2 and 2 evaluation
    instances at 512^2."""
    import numpy as np
    import synth
    from paper_2503_16717_gb300 import learned
    if args.learned_quick:
        n_train, N_train, n_eval, N_eval = 32, 128, 2, 512
    else:
        n_train, N_train, N_eval = 256, 512, 2048
        n_eval = 32 if args.learned_full else 4
    t0 = time.perf_counter()
    train_set = learned.make_instances(synth.convdiff2d_csr, range(3000, 3000 + n_train), N_train)
    t_gen = time.perf_counter() - t0
    net = rbo.GNN(seed=2)
    hist = learned.train(net, train_set, epochs=8, lr=3e-3, lr_decay=0.8)
    jac = rbo.GNN(seed=0)
    # kernel timing: one training step and one inference
    A0 = train_set[0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        net.loss_grad(A0.A, A0.R)
    e1.record()
    torch.cuda.synchronize()
    grad_ms = e0.elapsed_time(e1) / 5
    del train_set
    rows = []
    infer_ms = None
    for sd in range(4000, 4000 + n_eval):
        Ah, meta = synth.convdiff2d_csr(N_eval, sd)
        A = rbo.DeviceCSR.from_host(Ah)
        b = torch.from_numpy(synth.ones_rhs(Ah)).cuda()
        if infer_ms is None:
            net.infer(A)
            torch.cuda.synchronize()
            e0.record()
            net.infer(A)
            e1.record()
            torch.cuda.synchronize()
            infer_ms = e0.elapsed_time(e1)
            nnz_eval, n_eval_nodes = A.nnz, A.n
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        x, info, used = learned.solve(net, A, b, jacobi=jac, s=5, s_hat=30, m=60, tol=1e-10)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        _, ij = rbo.sstep_gmres(A, b, s=5, s_hat=30, m=60, tol=1e-10)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        rows.append({"seed": sd, "peclet": meta["peclet"], "learned_used": bool(used),
                     "iters_learned": info["iterations"], "iters_jacobi": ij["iterations"],
                     "relres_learned": info["relres"], "relres_jacobi": ij["relres"],
                     "s_learned": t2 - t1, "s_jacobi": t3 - t2,
                     "loss_learned": info["learned_loss"], "loss_jacobi": info["jacobi_loss"]})
        del A, b, x
    il = float(np.mean([r["iters_learned"] for r in rows]))
    ij_ = float(np.mean([r["iters_jacobi"] for r in rows]))
    bytes_infer = gnn_infer_bytes(n_eval_nodes, nnz_eval)
    return {"train": {"instances": n_train, "grid": N_train, "epochs": 8,
                      "epoch_loss": hist["epoch_loss"], "train_s": hist["seconds"],
                      "generate_s": t_gen, "loss_grad_ms": grad_ms},
            "eval": {"instances": n_eval, "grid": N_eval, "mean_iters_learned": il,
                     "mean_iters_jacobi": ij_, "iteration_ratio": il / ij_,
                     "mean_s_learned": float(np.mean([r["s_learned"] for r in rows])),
                     "mean_s_jacobi": float(np.mean([r["s_jacobi"] for r in rows])),
                     "rows": rows},
            "infer_ms": infer_ms, "infer_edges": nnz_eval,
            "infer_gbs_algorithmic": bytes_infer / (infer_ms / 1e3) / 1e9 if infer_ms else None}


def gnn_infer_bytes(n: int, nnz: int) -> int:
    """Algorithmic bytes of one inference of the learned-SPAI network (float32
    activations of width 32 = 128 bytes per row).  Per edge: graph build 56 (column,
    value, transpose position, features written), 3 message layers 3 x (4 column + 128
    h_j gathered + 128 m written) + the edge states e_1 written, read, e_2 written, read
    (512) + 12 features + 4 decoder term written, 3 node updates reading m (3 x 128),
    decoder 28 (row, column, term, two node terms, M written) -> 1776.  Per node: graph
    and features 16, encoder 8 + 128, 3 node updates reading h (384) and writing h_1,
    h_2 (256), decoder terms 8 written, diagonal inverse 8 read, row pointers 16 -> 824."""
    return 1776 * nnz + 824 * n


def run_gnn_kernels(rbo, torch, grid: int = 2048):
    """Kernel times of the learned-SPAI network alone (--gnn-only): one inference on an
    unseen grid^2 convection-diffusion instance (2048^2 by default: n = 4.19M, 21M
    edges; --gnn-grid sets the grid) and one loss and
    gradient on a 512^2 training instance with 8 residual columns, each timed with CUDA
    events over 5 calls after a warm-up call.  Weights: the initial ones plus seeded
    N(0, 0.05^2) noise (the cost does not depend on their values)."""
    import numpy as np
    import synth
    net = rbo.GNN(seed=2)
    rng = np.random.default_rng(1)
    th = net.get_params()
    net.set_params((th + rng.standard_normal(th.shape) * 0.05).astype(np.float32))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    Ah, _ = synth.convdiff2d_csr(grid, 4000)
    A = rbo.DeviceCSR.from_host(Ah)
    infer_ms = timed(lambda: net.infer(A))
    Bh, _ = synth.convdiff2d_csr(512, 3000)
    B = rbo.DeviceCSR.from_host(Bh)
    R = rbo.colmajor(Bh.n, 8)
    R.copy_(torch.from_numpy(np.random.default_rng(2).standard_normal((Bh.n, 8))))
    grad_ms = timed(lambda: net.loss_grad(B, R))
    return {"infer_ms": infer_ms, "infer_n": int(A.n), "infer_edges": int(A.nnz),
            "infer_gbs_algorithmic": gnn_infer_bytes(A.n, A.nnz) / (infer_ms / 1e3) / 1e9,
            "loss_grad_ms": grad_ms, "loss_grad_n": int(B.n), "loss_grad_edges": int(B.nnz),
            "residual_columns": 8}


def run_s_sweep(rbo, torch, Ad, bd, args):
    """Time to solution of the benchmark problem against the block size s (Sec. 8:
    sketching keeps larger s stable): one-stage and two-stage (s_hat = the smallest
    multiple of s that is >= 20 and divides m), monomial, Newton and Chebyshev basis."""
    out = []
    x = torch.zeros(Ad.n, dtype=torch.float64, device="cuda")
    for s_ in (5, 10, 15, 20, 30):
        sh = next(v for v in range(s_, M + 1, s_) if v >= 20 and M % v == 0)
        for s_hat in ((0, sh) if sh > s_ else (0,)):
            for basis in (rbo.BASIS_MONOMIAL, rbo.BASIS_NEWTON, rbo.BASIS_CHEBYSHEV):
                def go():
                    x.zero_()
                    return rbo.sstep_gmres(Ad, bd, x, s=s_, s_hat=s_hat, m=M, tol=TOL,
                                           basis=basis)[1]
                go()
                torch.cuda.synchronize()
                t = time.perf_counter()
                info = go()
                torch.cuda.synchronize()
                out.append({"s": s_, "s_hat": s_hat or s_, "scheme": "two" if s_hat > s_ else "one",
                            "basis": {rbo.BASIS_MONOMIAL: "monomial", rbo.BASIS_NEWTON: "newton",
                                      rbo.BASIS_CHEBYSHEV: "chebyshev"}[basis],
                            "status": info["status"], "iterations": info["iterations"],
                            "restarts": info["restarts"], "relres": info["relres"],
                            "s_per_solve": time.perf_counter() - t})
    return out


def run_stress(rbo, torch, args, core_only=False):
    """Nonsymmetric 3D convection-diffusion, 7-point upwind, anisotropy (1, 1, 1e-3),
    Peclet 100 (seed 7), N^3 cells; s-step GMRES(m=100, s=10) to 1e-10:
    one-stage with CholQR2 (the deterministic baseline) and with RandCholQR, then two-stage
    RandBCGS2 (s_hat=50) in float64 and mixed precision with Jacobi and with the
    learned SPAI (trained on smaller instances of the family; Jacobi fallback).
    core_only (the default run at one GPU): only the two-stage float64 and mixed solves
    with the learned SPAI and its Jacobi fallback, the runs the stress workload names."""
    import numpy as np
    import synth
    from paper_2503_16717_gb300 import learned
    N = args.stress_n
    t0 = time.perf_counter()
    Ah, meta = synth.convdiff3d_csr(N, seed=7)
    A = rbo.DeviceCSR.from_host(Ah)
    b = torch.from_numpy(synth.ones_rhs(Ah)).cuda()
    t_gen = time.perf_counter() - t0
    del Ah
    out = {"N": N, "n": A.n, "nnz": A.nnz, "s": 10, "s_hat": 50, "m": 100, "tol": 1e-10,
           "wind": meta["w"], "generate_s": t_gen, "max_restarts": args.stress_restarts}

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t

    def row(info, sec, **kw):
        d = {"status": info["status"], "converged": info["converged"],
             "iterations": info["iterations"], "restarts": info["restarts"],
             "relres": info["relres"], "fallbacks": info["fallbacks"], "s": sec}
        if info["status"] != 0:
            d["breakdown"] = {k: info.get(k) for k in ("breakdown_block", "breakdown_column",
                                                       "breakdown_stage_name")}
        d.update(kw)
        return d

    out["core_only"] = core_only
    if not core_only:
        # the deterministic baseline: one-stage with CholQR2 on the monomial panels
        (_, info), sec = timed(lambda: rbo.sstep_gmres(A, b, s=10, m=100, tol=1e-10,
                                                       max_restarts=args.stress_restarts,
                                                       intra=rbo.INTRA_CHOLQR2))
        out["cholqr2_one_stage"] = row(info, sec)
        # the randomized one-stage scheme on the same panels
        (_, info), sec = timed(lambda: rbo.sstep_gmres(A, b, s=10, m=100, tol=1e-10,
                                                       max_restarts=args.stress_restarts))
        out["randcholqr_one_stage"] = row(info, sec)
    # the learned SPAI, trained on the same family at 48^3
    t0 = time.perf_counter()
    train_set = learned.make_instances(lambda n_, sd: synth.convdiff3d_csr(n_, sd), range(100, 116), 48,
                                       s=10, m=100)
    net = rbo.GNN(seed=2)
    hist = learned.train(net, train_set, epochs=8, lr=3e-3, lr_decay=0.8)
    out["train"] = {"instances": 16, "grid": 48, "epoch_loss": hist["epoch_loss"],
                    "s": time.perf_counter() - t0}
    del train_set
    jac = rbo.GNN(seed=0)
    runs = []
    for prec, pn in ((rbo.PREC_FP64, "fp64"), (rbo.PREC_MIXED, "mixed")):
        if not core_only:
            (_, info), sec = timed(lambda: rbo.sstep_gmres(A, b, s=10, s_hat=50, m=100,
                                                           tol=1e-10, precision=prec,
                                                           max_restarts=args.stress_restarts))
            runs.append(row(info, sec, precision=pn, precond="jacobi"))
        (res, sec) = timed(lambda: learned.solve(net, A, b, jacobi=jac, s=10, s_hat=50, m=100,
                                                 tol=1e-10, precision=prec,
                                                 max_restarts=args.stress_restarts))
        _, info, used = res
        runs.append(row(info, sec, precision=pn, precond="learned" if used else "jacobi (fallback)",
                        loss_learned=info["learned_loss"], loss_jacobi=info["jacobi_loss"]))
    out["runs"] = runs
    del A, b
    torch.cuda.empty_cache()
    return out


def run_stress_bases(rbo, torch, args):
    """The stress problem (3D convection-diffusion, anisotropy (1, 1, 1e-3), Peclet 100,
    seed 7, N^3 cells) solved by one-stage RandCholQR s-step GMRES(m=100) to 1e-10 with
    the monomial, Newton and Chebyshev bases at s = 10, 20 and 25 (Section 4 names the
    Newton and Chebyshev bases as the stabler matrix-powers bases)."""
    import synth
    N = args.stress_n
    t0 = time.perf_counter()
    Ah, meta = synth.convdiff3d_csr(N, seed=7)
    A = rbo.DeviceCSR.from_host(Ah)
    b = torch.from_numpy(synth.ones_rhs(Ah)).cuda()
    out = {"N": N, "n": A.n, "nnz": A.nnz, "m": 100, "tol": 1e-10,
           "generate_s": time.perf_counter() - t0, "runs": []}
    del Ah
    names = {rbo.BASIS_MONOMIAL: "monomial", rbo.BASIS_NEWTON: "newton",
             rbo.BASIS_CHEBYSHEV: "chebyshev"}
    for s_ in (10, 20, 25):
        for basis in (rbo.BASIS_MONOMIAL, rbo.BASIS_NEWTON, rbo.BASIS_CHEBYSHEV):
            torch.cuda.synchronize()
            t = time.perf_counter()
            _, info = rbo.sstep_gmres(A, b, s=s_, m=100, tol=1e-10, basis=basis,
                                      max_restarts=args.stress_restarts)
            torch.cuda.synchronize()
            out["runs"].append({"s": s_, "basis": names[basis], "status": info["status"],
                                "converged": info["converged"], "iterations": info["iterations"],
                                "restarts": info["restarts"], "relres": info["relres"],
                                "s_per_solve": time.perf_counter() - t})
    del A, b
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------------------------------
def oracle_solve_estimate(A, b, scheme: str, cycles: int, iterations: int):
    """Seconds of one full oracle solve of the workload, from a bounded sample: the
    setup (scaling, sketch, first residual; a call with no restart cycle) plus the
    per-iteration time of `cycles` restart cycles, scaled to `iterations`.
    Returns (estimate, sampled iterations, sampled seconds)."""
    from oracle import krylov
    kw = dict(s=S, m=M, tol=TOL) if scheme == "one" else dict(s=S, m=M, s_hat=S_HAT, scheme="two",
                                                              tol=TOL)
    t0 = time.perf_counter()
    krylov.sstep_gmres(A, b, max_restarts=0, **kw)
    t1 = time.perf_counter()
    res = krylov.sstep_gmres(A, b, max_restarts=cycles, **kw)
    t2 = time.perf_counter()
    setup, its = t1 - t0, max(res.iterations, 1)
    per_it = max((t2 - t1) - setup, 0.0) / its
    return setup + per_it * iterations, its, t2 - t0


def cpu_baseline(A, b, gpu_iterations, budget_cycles=2):
    """The oracle's one-stage s-step GMRES on the same problem: setup plus
    `budget_cycles` restart cycles, scaled by iterations to the GPU solve's count."""
    est, its, dt = oracle_solve_estimate(A, b, "one", budget_cycles, gpu_iterations)
    return {"value": est, "unit": "s", "cores": _cpu_threads(), "kind": "oracle",
            "sample": f"setup + {its} iterations ({budget_cycles} restart cycles) of the one-stage "
                      f"solve in {dt:.1f} s, scaled to {gpu_iterations} iterations"}


def _cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count()


def _golden_iterations():
    """Converged iteration counts of the workload from the oracle's own full solves
    (tests/golden/gmres_poisson100.json, written by the oracle-only script beside it)."""
    path = os.path.join(ROOT, "tests", "golden", "gmres_poisson100.json")
    with open(path) as f:
        g = json.load(f)
    return {"one": int(g["one_stage"]["iterations"]), "two": int(g["two_stage"]["iterations"])}, g


def run_reference(args):
    """The CPU oracle on the workload, as it stands, on the host cores.  A full oracle
    solve takes minutes, so each step is a bounded sample: one restart cycle of the
    one-stage and one of the two-stage solve (60 iterations each).  `value` is the
    per-solve time these samples extrapolate to: the setup (Jacobi scaling, sketch,
    first residual; timed once, in the first warm-up step) plus the sampled
    per-iteration time times the iteration count at which the oracle's own full solves
    of this workload converge (read from the committed golden file).  `ms_per_step` is
    the measured wall time of one sampled step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    from oracle import krylov
    A = synth.poisson3d_csr(N_GRID)
    b = synth.ones_rhs(A)
    its_full, gold = _golden_iterations()
    kw = {"one": dict(s=S, m=M, tol=TOL),
          "two": dict(s=S, m=M, s_hat=S_HAT, scheme="two", tol=TOL)}
    setup = {}
    for sch in ("one", "two"):
        t0 = time.perf_counter()
        krylov.sstep_gmres(A, b, max_restarts=0, **kw[sch])
        setup[sch] = time.perf_counter() - t0
    per_it = {"one": [], "two": []}
    step_s = []
    for it in range(max(args.warmup, 0) + args.steps):
        t_step = time.perf_counter()
        for sch in ("one", "two"):
            t0 = time.perf_counter()
            r = krylov.sstep_gmres(A, b, max_restarts=1, **kw[sch])
            dt = time.perf_counter() - t0
            if it >= args.warmup:
                per_it[sch].append(max(dt - setup[sch], 0.0) / max(r.iterations, 1))
        if it >= args.warmup:
            step_s.append(time.perf_counter() - t_step)
    est = {sch: setup[sch] + statistics.mean(per_it[sch]) * its_full[sch] for sch in ("one", "two")}
    v = (est["one"] + est["two"]) / 2.0
    ms_step = statistics.mean(step_s) * 1e3
    sample = (f"per step: one restart cycle ({M} iterations) of the one-stage and of the two-stage "
              f"solve; setup timed once; per-iteration time scaled to the oracle's converged "
              f"iteration counts ({its_full['one']} one-stage, {its_full['two']} two-stage, "
              f"tests/golden/gmres_poisson100.json)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "estimate": True,
            "config": {"workload": WORKLOAD, "n": A.n},
            "estimate_per_solve_s": est, "setup_s": setup,
            "cpu_baseline": {"value": v, "unit": "s", "kind": "oracle", "cores": _cpu_threads(),
                             "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-orth", action="store_true")
    ap.add_argument("--quick-orth", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-prof", action="store_true")
    ap.add_argument("--no-df64", action="store_true")
    ap.add_argument("--no-ozaki", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--learned-full", action="store_true")
    ap.add_argument("--learned-quick", action="store_true")
    ap.add_argument("--stress", action="store_true",
                    help="the full 3D convection-diffusion stress study (s=10, s_hat=50, m=100): "
                         "also the one-stage CholQR2 and RandCholQR runs and the Jacobi-only "
                         "two-stage runs; without it a run on one GPU does the two-stage float64 "
                         "and mixed solves with the learned SPAI")
    ap.add_argument("--no-stress", action="store_true",
                    help="skip the stress solves of the default run")
    ap.add_argument("--stress-n", type=int, default=256, help="grid points per side of the stress case")
    ap.add_argument("--stress-restarts", type=int, default=100)
    ap.add_argument("--stress-bases", action="store_true",
                    help="also solve the stress problem with the monomial, Newton and Chebyshev "
                         "bases at s = 10, 20, 25")
    ap.add_argument("--s-sweep", action="store_true",
                    help="also time the workload's solves for s in 5, 10, 15, 20, 30")
    ap.add_argument("--gnn-only", action="store_true",
                    help="only time the learned-SPAI network's inference (2048^2) and loss and "
                         "gradient (512^2), print them as one JSON object and exit")
    ap.add_argument("--gnn-grid", type=int, default=2048,
                    help="grid points per side of the --gnn-only inference instance")
    args = ap.parse_args()
    if args.gnn_only:
        import torch
        import paper_2503_16717_gb300 as rbo
        print(json.dumps({"gnn_kernels": run_gnn_kernels(rbo, torch, args.gnn_grid)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
