"""Benchmark: one structure-preserving spectral division (sign + split) of a
definite pseudosymmetric Casida matrix of order n on one GB300.

A step is one call of pssd_split on an H already resident in HBM: bounds,
Cholesky congruence, the two-step Zolotarev sign with its stopping test, the
invariant-subspace bases and the projected blocks A11, A22 and Q.

Default workload: n = 16384 (k = 8192), d1, d2 log-uniform in [1e-2, 1e2]
(kappa <= 1e4), synthetic, seeded.  Each H is 2.1 GB, larger than the 129 MB
L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 16384] [--impl ours|reference]

Under torchrun each rank runs its own replica (the path is not sharded), the
time is the max over ranks and value = whole-job seconds per solve.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "n=16384 split: s/solve & TFLOP/s, mixed vs plain FP64 at ‖S²−I‖≤1e-12·n"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t, device="cpu"):
    """The job's time: the largest of the ranks' times (needs an initialised
    process group; NCCL on the GPU machine, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        fd, self.path = tempfile.mkstemp(prefix="pssd_clocks_", suffix=".csv")
        os.close(fd)
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1])); mx.append(float(v[2]))
            except ValueError:
                continue
            for nm, val in zip(names, v[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


ORACLE_SIZES = (256, 384, 512)


def _oracle_solve(n_s, seed=0):
    """One oracle sign (Alg. 8, scalar-loop pivoted elimination of Eq. ZoloIt2,
    the r shifted systems in r threads) + split (Alg. 7) of an order-n_s input
    of the workload's distribution; returns (seconds, threads used)."""
    import casida_inputs as G
    import oracle as O
    H, _, _ = G.casida(n_s // 2, ("loguniform", 1e-2, 1e2), seed=seed)
    t0 = time.perf_counter()
    S, info = O.sign_alg(H)
    O.split_alg(H, None, S)
    return time.perf_counter() - t0, max(info["r"])


def cpu_baseline_sample(n_target=16384):
    """The oracle on a bounded sample of the same workload (about 12 s of host
    work): one solve at each of n = 256, 384, 512, a least-squares fit of
    t = c n^3 through them, and the fit evaluated at n_target (extrapolated;
    the oracle's dense steps are O(n^3))."""
    ts, thr = [], 1
    for n_s in ORACLE_SIZES:
        t, r = _oracle_solve(n_s)
        ts.append(t); thr = max(thr, r)
    x = [float(n) ** 3 for n in ORACLE_SIZES]
    c = sum(a * b for a, b in zip(x, ts)) / sum(a * a for a in x)
    # log-log slope of the measurements, to show how close to n^3 they are
    lx = [math.log(n) for n in ORACLE_SIZES]; ly = [math.log(t) for t in ts]
    mx, my = sum(lx) / 3, sum(ly) / 3
    slope = sum((a - mx) * (b - my) for a, b in zip(lx, ly)) / sum((a - mx) ** 2 for a in lx)
    return {"value": c * n_target ** 3, "unit": "s/solve", "cores": thr, "kind": "oracle",
            "sample": "oracle sign (Alg. 8: scalar-loop pivoted elimination of Eq. ZoloIt2, r shifted systems in "
                      "r threads) + split (Alg. 7) of one Casida input of the workload's distribution at each of "
                      "n = %s: %s s; t = c n^3 fitted (measured log-log slope %.2f) and evaluated at n = %d "
                      "(extrapolated); cores = threads the shifted solves used (max r); numpy matmuls use the "
                      "host BLAS" % (", ".join(map(str, ORACLE_SIZES)), ", ".join("%.2f" % t for t in ts),
                                     slope, n_target),
            "measured_s": dict(zip(map(str, ORACLE_SIZES), ts)), "loglog_slope": slope}


def run_reference(args):
    """The oracle as it stands on the host cores: each step is one bounded
    sample of the workload (one oracle sign + split at n = 384, about 3 s),
    reported in the metric's unit by n^3 scaling to n = 16384 (extrapolated);
    ms_per_step is the measured time of a step."""
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    n_s = 384
    for i in range(args.warmup):
        _oracle_solve(n_s, seed=i)
    ts, thr = [], 1
    for i in range(args.steps):
        t, r = _oracle_solve(n_s, seed=100 + i)
        ts.append(t); thr = max(thr, r)
    tm = statistics.median(ts)
    v = tm * (args.n / n_s) ** 3
    cb = {"value": v, "unit": "s/solve", "cores": thr, "kind": "oracle",
          "sample": "each step: oracle sign (Alg. 8) + split (Alg. 7) of one n=%d Casida input of the workload's "
                    "distribution (median %.2f s), scaled by (%d/%d)^3 to s/solve at n=%d (extrapolated)"
                    % (n_s, tm, args.n, n_s, args.n)}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/solve", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tm * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "casida_n%d_log1e-2_1e2 split" % args.n, "n": args.n,
                       "sample_n": n_s, "note": "value extrapolated by n^3 from the sample; ms_per_step measured"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "s/solve", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gemm_probe(args):
    """One n x n x n contraction C = A B through a single engine of the library
    (the engines' test hooks), W warm-ups and K timed launches, CUDA events."""
    import torch

    import paper_2203_08900_gb300 as P
    from paper_2203_08900_gb300 import build as B
    B.build()
    n = args.n
    g = torch.Generator(device="cuda"); g.manual_seed(5)
    f64 = args.gemm_probe in ("dfma", "df", "oz")
    dt = torch.float64 if f64 else torch.float32
    A = torch.randn(n, n, device="cuda", dtype=dt, generator=g)
    Bm = torch.randn(n, n, device="cuda", dtype=dt, generator=g)
    h = P.Handle()

    def run():
        if f64:
            return P.test_gemm_f64(A, Bm, engine={"dfma": 0, "df": 1, "oz": 2}[args.gemm_probe], handle=h)
        return P.test_gemm_f32(A, Bm, use_tc=args.gemm_probe == "tc", handle=h)

    for _ in range(args.warmup):
        C = run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        C = run()
    e1.record(); torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    ref = (A.double() @ Bm.double())
    err = float((C.double() - ref).abs().max() / (A.double().abs() @ Bm.double().abs()).max())
    print(json.dumps({"metric": "gemm probe", "engine": args.gemm_probe, "n": n, "s_per_gemm": t,
                      "tflops": 2.0 * n ** 3 / t / 1e12, "max_rel_err": err,
                      "note": "includes the engine's operand preparation passes"}))
    return 0


def _seconds_by_k(ks, infos):
    """Sum of the instances' own call times (each on its worker thread), by block order k."""
    bins = [(16, 64), (64, 256), (256, 1025)]
    out = {}
    for lo, hi in bins:
        sel = [i for i, k in enumerate(ks) if lo <= k < hi]
        out["k%d-%d" % (lo, hi - 1)] = {"instances": len(sel), "seconds": sum(infos[i]["seconds"] for i in sel)}
    return out


def run_batch(args):
    """Batched workload: one step = pssd_eig_batched over `count` instances."""
    import torch

    import casida_inputs as G
    import paper_2203_08900_gb300 as P
    from paper_2203_08900_gb300 import build as B
    B.build()
    ws, rank, local = dist_env()
    if ws > 1:   # independent batches per rank (weak scaling), no data-path collective
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    ks = G.batch_sizes(args.batch_count, 16, 1024, seed=0)
    Hs = []
    for i, k in enumerate(ks):
        H, _, _ = G.casida_torch(int(k), ("uniform", 0.5, 50.0), seed=10000 + rank * args.batch_count + i,
                                 device=dev)
        Hs.append(H.contiguous())
    torch.cuda.synchronize()
    prec = {"fp64": P.PSSD_FP64, "mixed": P.PSSD_MIXED, "fp64e": P.PSSD_FP64_EMULATED}[args.precision]
    stream = torch.cuda.current_stream()
    h = P.Handle(stream)
    for _ in range(args.warmup):
        P.eig_batched(Hs, handle=h, precision=prec)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    h.profile_reset()
    l0 = h.launch_count()
    ph0 = P.launch_count_phases()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        Ds, Vs, infos = P.eig_batched(Hs, handle=h, precision=prec)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ck = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    if ws > 1:
        t = max_over_ranks(t, dev)
    # accuracy over the batch (untimed): max relative eigen-residual
    res = 0.0
    with torch.no_grad():
        for H, D, V in zip(Hs, Ds, Vs):
            res = max(res, float(torch.linalg.norm(H @ V - V * D) / torch.linalg.norm(H)))
    n3 = float(sum((2.0 * k) ** 3 for k in ks))
    line = {"metric": "batched diagonalisation: instances/s", "value": ws * args.batch_count * args.steps / t,
            "unit": "instances/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "batch of %d Casida matrices, k log-uniform [16,1024], d ~ U[0.5,50]"
                       % args.batch_count, "sum_n3": n3, "precision": args.precision},
            "max_rel_residual": res, "gpu_launches": h.launch_count() - l0,
            "launches_by_phase": {k: v - ph0[k] for k, v in P.launch_count_phases().items()},
            "host_seconds_by_k": _seconds_by_k(ks, infos), "clocks": ck}
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "fp64e"],
                    help="fp64: native FP64; mixed: FP32 Zolotarev + FP64-accurate refinement; "
                         "fp64e: the FP64 algorithm with every contraction FP64-accurate on the BF16 tensor cores")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP64-emulated and plain-FP64 solves on the same input")
    ap.add_argument("--workload", default="split", choices=["split", "batch"],
                    help="split: one n x n sign + split per step (headline); batch: full diagonalisation of "
                         "512 Casida matrices with k log-uniform in [16, 1024], d ~ U[0.5, 50]")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--numpy-inputs", action="store_true",
                    help="draw H with the numpy generator at any n (keeps torch's GPU linear algebra, which "
                         "some profiler setups cannot load, out of the run)")
    ap.add_argument("--gemm-probe", default=None, choices=["dfma", "df", "oz", "tc", "f32"],
                    help="time one n x n x n contraction on one engine (no solve)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.gemm_probe:
        return run_gemm_probe(args)

    import numpy as np
    import torch

    import casida_inputs as G
    import paper_2203_08900_gb300 as P

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2203_08900_gb300 import build as B
    B.build()
    peaks = measured_peaks()
    n = args.n
    k = n // 2
    dist_d = ("loguniform", 1e-2, 1e2)
    if n <= 4096 or args.numpy_inputs:   # numpy generator (also keeps torch's GPU linear algebra out of profiler runs)
        Hn, d1, d2 = G.casida(k, dist_d, seed=1234 + rank)
        H = torch.from_numpy(Hn).to(dev)
    else:
        H, d1, d2 = G.casida_torch(k, dist_d, seed=1234 + rank, device=dev)
    H = H.contiguous()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    h = P.Handle(stream)
    p = n // 2

    PREC = {"fp64": P.PSSD_FP64, "mixed": P.PSSD_MIXED, "fp64e": P.PSSD_FP64_EMULATED}
    prec = PREC[args.precision]

    def step(pr=prec):
        return P.split(H, handle=h, precision=pr)

    infos = []
    for _ in range(args.warmup):
        Q, A11, A22, pp, info = step()
        infos.append(info)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    h.profile(True); h.profile_reset()
    l0 = h.launch_count()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")     # ncu --nvtx --nvtx-include "timed/" lists these launches only
    e0.record(stream)
    for _ in range(args.steps):
        Q, A11, A22, pp, info = step()
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if ws > 1:
        dist.barrier()
    ck = clocks.stop()
    h.profile(False)
    launches = h.launch_count() - l0
    t = e0.elapsed_time(e1) / 1e3
    if ws > 1:
        t = max_over_ranks(t, dev)
    kinds = {P.KIND_NAMES[i]: h.profile_read(i) for i in range(len(P.KIND_NAMES))}
    last = infos[-1]
    rs = [x for x in last["r_used"][:last["passes"]]]
    # algorithmic FLOPs: the library's exact structural count of every contraction it launched
    fl = sum(kinds[kk]["flops"] for kk in ("dgemm", "sgemm", "dfgemm", "tcgemm", "ozgemm", "chol_leaf")) / args.steps
    solves = args.steps * ws
    s_per_solve = t / solves
    table = kernel_table(kinds, t, args.steps, peaks)
    dom = max(["dgemm", "sgemm", "dfgemm", "tcgemm", "ozgemm"], key=lambda kk: kinds[kk]["ms"])
    roof = dict(table[dom])
    roof.update({"kernel": KERNEL_NAMES[dom], "traffic": roof.pop("traffic_per_launch", None),
                 "traffic_note": "bytes per launch: ncu DRAM bytes per flop of a 4096^3 launch x this step's "
                                 "flops per launch; about 3.5x the algorithmic slice and C bytes (L2 re-reads)"})
    acc = split_accuracy(P, torch, H, Q, p, dev)
    # the metric's condition on S itself: S = L^{-T} sign(K) L^T from pssd_sign in the same
    # precision mode, ||S^2 - I||_F and ||SH - HS||_F / ||H||_F computed by the library (untimed)
    S_chk, info_s = P.sign(H, handle=h, precision=prec, flags=P.FLAG_RESIDUALS)
    del S_chk
    acc.update({"s2_resid_sign": info_s["s2_resid"], "s2_bound": 1e-12 * n,
                "s2_ok": bool(info_s["s2_resid"] <= 1e-12 * n), "comm_rel_sign": info_s["comm_resid"],
                "split_backerr_K": last["split_backerr"], "comm_rel_split_lib": last["comm_resid"]})
    line = {
        "metric": METRIC, "value": s_per_solve, "unit": "s/solve", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f32+f64", "fp64e": "f64 (emulated on bf16 tensor cores)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": "casida_n%d_log1e-2_1e2 split (sign+split), %s path" % (n, args.precision), "n": n,
                   "k": k, "precision": args.precision, "l2": "inputs larger than L2 (2.1 GB per H), no flush",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "tflops": fl * solves / t / 1e12, "algorithmic_flops_per_solve": fl,
        "r_per_pass": rs, "restarts": last["restarts"], "alpha": last["alpha"], "beta": last["beta"],
        "accuracy": acc,
        "roofline": roof,
        "kernels": table,
        "gpu_launches": launches,
        "clocks": ck,
    }
    line["mixed_info"] = {"fp32_steps": last.get("fp32_steps"), "ns_steps": last.get("ns_steps"),
                          "ns_resid_K_basis": last.get("ns_resid")} if args.precision == "mixed" else None
    if not args.no_e2e and rank == 0:
        # end to end through the public API with HOST buffers: H2D of H, the solve, D2H of Q, A11, A22
        Hh = H.cpu().pin_memory()
        Qh = torch.empty((n, n), dtype=torch.float64).pin_memory()
        A11h = torch.empty((p, p), dtype=torch.float64).pin_memory()
        A22h = torch.empty((n - p, n - p), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True); f1 = torch.cuda.Event(enable_timing=True)
        fa = torch.cuda.Event(enable_timing=True); fb = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        Hd = Hh.to(dev, non_blocking=True)
        fa.record(stream)
        Q2, B11, B22, _, _ = P.split(Hd, handle=h, precision=prec)
        fb.record(stream)
        Qh.copy_(Q2, non_blocking=True); A11h.copy_(B11, non_blocking=True); A22h.copy_(B22, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        te = f0.elapsed_time(f1) / 1e3
        hb, db = 8 * n * n, 8 * (n * n + p * p + (n - p) ** 2)
        line["e2e"] = {"value": te, "unit": "s/solve", "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db,
                       "h2d_GBps": hb / (f0.elapsed_time(fa) / 1e3) / 1e9,
                       "d2h_GBps": db / (fb.elapsed_time(f1) / 1e3) / 1e9,
                       "note": "pinned host buffers; copy rates from events around the copies"}
        del Q2, B11, B22, Hd
    if rank == 0 and ws == 1 and not args.no_compare:   # the comparison arms: single-process runs only
        # the other precision modes on the same input, same handle (workspace already grown)
        for name in ("fp64e", "fp64"):
            if name == args.precision:
                continue
            reps = 1 if name == "fp64" else max(1, min(3, args.steps))
            if name == "fp64e":
                step(PREC[name])          # one warm-up (the slice engine's extra workspace)
            torch.cuda.synchronize()
            h.profile(True); h.profile_reset()
            g0 = torch.cuda.Event(enable_timing=True); g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(reps):
                Qf, A11f, A22f, _, infof = step(PREC[name])
            g1.record(stream)
            torch.cuda.synchronize()
            h.profile(False)
            tf = g0.elapsed_time(g1) / 1e3 / reps
            kf = {P.KIND_NAMES[i]: h.profile_read(i) for i in range(len(P.KIND_NAMES))}
            tab = kernel_table(kf, tf * reps, reps, peaks)
            domf = max(["dgemm", "dfgemm", "ozgemm"], key=lambda kk: kf[kk]["ms"])
            with torch.no_grad():
                dA = float(torch.linalg.norm(torch.linalg.eigvalsh(A11f) - torch.linalg.eigvalsh(A11))
                           / torch.linalg.norm(torch.linalg.eigvalsh(A11f)))
            accf = split_accuracy(P, torch, H, Qf, p, dev)
            accf.update({"split_backerr_K": infof["split_backerr"], "comm_rel_split_lib": infof["comm_resid"]})
            line["plain_fp64" if name == "fp64" else "fp64_emulated"] = {
                "s_per_solve": tf, "speedup_vs_this_path": tf / s_per_solve,
                "timed_solves": reps, "accuracy": accf,
                "A11_spectrum_rel_diff_vs_headline_path": dA,
                "dominant_kernel": dict(tab[domf], kernel=KERNEL_NAMES[domf]),
                "kernels": tab, "r_per_pass": infof["r_used"][:infof["passes"]],
                "note": "same input and handle" + ("; timed after the FP64-emulated solves (workspace allocated)"
                                                   if name == "fp64" else "; 1 warm-up")}
            del Qf, A11f, A22f
        if "plain_fp64" in line and "fp64_emulated" in line:
            line["fp64_emulated"]["speedup_vs_plain_fp64"] = (line["plain_fp64"]["s_per_solve"]
                                                              / line["fp64_emulated"]["s_per_solve"])
        # the structure-aware split of the same H from its blocks A, B (k x k polar factor of
        # C = L_P^T L_R), FP64-emulated and plain FP64
        Ab = H[:k, :k].contiguous(); Bb = H[:k, k:].contiguous()
        for name in ("fp64e", "fp64"):
            reps = max(1, min(3, args.steps)) if name == "fp64e" else 1
            if name == "fp64e":
                P.casida_split(Ab, Bb, handle=h, precision=PREC[name])  # warm-up (FP64 reuses its workspace)
            torch.cuda.synchronize()
            h.profile(True); h.profile_reset()
            g0 = torch.cuda.Event(enable_timing=True); g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(reps):
                Qc, A11c, A22c, _, infoc = P.casida_split(Ab, Bb, handle=h, precision=PREC[name])
            g1.record(stream)
            torch.cuda.synchronize()
            h.profile(False)
            tc = g0.elapsed_time(g1) / 1e3 / reps
            kc = {P.KIND_NAMES[i]: h.profile_read(i) for i in range(len(P.KIND_NAMES))}
            tab = kernel_table(kc, tc * reps, reps, peaks)
            accc = split_accuracy(P, torch, H, Qc, p, dev)
            accc.update({"split_backerr_K": infoc["split_backerr"], "comm_rel_split_lib": infoc["comm_resid"]})
            entry = {"s_per_solve": tc, "timed_solves": reps, "accuracy": accc,
                     "r_per_pass": infoc["r_used"][:infoc["passes"]], "kernels": tab,
                     "note": "pssd_casida_split on the blocks A, B of the same H; k x k work"
                             + ("; 1 warm-up" if name == "fp64e" else "; timed after the FP64-emulated solves")}
            if "plain_fp64" in line:
                entry["speedup_vs_plain_fp64_nxn"] = line["plain_fp64"]["s_per_solve"] / tc
            line["structure_aware_" + ("fp64e" if name == "fp64e" else "fp64")] = entry
            del Qc, A11c, A22c
        # full diagonalisation of the same H (structure-aware, FP64-emulated): one warm-up, one
        # timed solve; ||HV - VD||_F / ||H||_F and the Sigma-orthogonality checked by cuBLAS, untimed
        P.casida_eig(Ab, Bb, handle=h, precision=P.PSSD_FP64_EMULATED)
        torch.cuda.synchronize()
        h.profile(True); h.profile_reset()
        g0 = torch.cuda.Event(enable_timing=True); g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        De, Ve, infoe = P.casida_eig(Ab, Bb, handle=h, precision=P.PSSD_FP64_EMULATED)
        g1.record(stream)
        torch.cuda.synchronize()
        h.profile(False)
        te_eig = g0.elapsed_time(g1) / 1e3
        ke = {P.KIND_NAMES[i]: h.profile_read(i) for i in range(len(P.KIND_NAMES))}
        with torch.no_grad():
            R = torch.addmm(Ve * De[None, :], H, Ve, beta=-1.0)
            res = float(torch.linalg.norm(R) / torch.linalg.norm(H))
            del R
            gen = torch.Generator(device=dev); gen.manual_seed(11)
            Xp = torch.randn(n, 16, dtype=torch.float64, device=dev, generator=gen)
            Jv = torch.cat([torch.ones(k, dtype=torch.float64, device=dev), -torch.ones(k, dtype=torch.float64, device=dev)])
            vsv = float(torch.linalg.norm(Ve.T @ (Jv[:, None] * (Ve @ Xp)) - torch.sign(De)[:, None] * Xp)
                        / torch.linalg.norm(Xp))
        line["structure_aware_eig_fp64e"] = {
            "s_per_solve": te_eig, "timed_solves": 1, "levels": infoe["levels"],
            "residual_HV_VD_rel": res, "residual_bound": 1e-11,
            "vsigma_orth_probe": vsv, "vsigma_bound": 1e-12 * n,
            "kernels": kernel_table(ke, te_eig, 1, peaks),
            "note": "pssd_casida_eig on the blocks A, B of the same H (1 warm-up); checks untimed"}
        del De, Ve
        del Ab, Bb
        # the paper's Tab. ItRuntime on this GPU: Example 2 (n = 5000, A = Sigma Q D Q^T, Sigma random
        # +-1, Q = orth(rand(n)), D equally spaced in [1, kappa]), one split per method and kappa,
        # FP64-emulated; iterations, seconds and the split backward error ||Q+^T Sigma A Q-|| / ||A||
        ne = 5000
        ge = torch.Generator(device=dev); ge.manual_seed(0)
        Qe, _ = torch.linalg.qr(torch.rand(ne, ne, dtype=torch.float64, device=dev, generator=ge))
        sge = torch.where(torch.rand(ne, dtype=torch.float64, device=dev, generator=ge) < 0.5, 1.0, -1.0)
        sig_e = sge.to(torch.int8).cpu().numpy()
        table_m = {}
        for kap in (1e2, 1e8, 1e12):
            De = torch.linspace(1.0, kap, ne, dtype=torch.float64, device=dev)
            Me = (Qe * De[None, :]) @ Qe.T
            Ae = (sge[:, None] * (0.5 * (Me + Me.T))).contiguous()
            del Me
            for mname, mcode in (("zolo_pd", P.METHOD_ZOLO), ("sigma_dwh", P.METHOD_DWH), ("newton", P.METHOD_NEWTON)):
                try:
                    P.split(Ae, sigma=sig_e, handle=h, precision=P.PSSD_FP64_EMULATED, method=mcode)
                    torch.cuda.synchronize()
                    g0 = torch.cuda.Event(enable_timing=True); g1 = torch.cuda.Event(enable_timing=True)
                    g0.record(stream)
                    _, _, _, _, ie = P.split(Ae, sigma=sig_e, handle=h, precision=P.PSSD_FP64_EMULATED, method=mcode)
                    g1.record(stream)
                    torch.cuda.synchronize()
                    _, _, _, _, ir = P.split(Ae, sigma=sig_e, handle=h, precision=P.PSSD_FP64_EMULATED, method=mcode,
                                             flags=P.FLAG_RESIDUALS)
                    table_m["%s_kappa%.0e" % (mname, kap)] = {
                        "iterations": ie["iterations"], "seconds": g0.elapsed_time(g1) / 1e3,
                        "split_backerr": ir["split_backerr"], "r_per_pass": ie["r_used"][:ie["passes"]]
                        if mcode == P.METHOD_ZOLO else None}
                except P.PssdError as err:
                    table_m["%s_kappa%.0e" % (mname, kap)] = {"status": err.status}
            del Ae, De
        line["methods_example2_n5000"] = {"precision": "fp64e", "results": table_m,
                                          "note": "Sec. 6 Example 2 recipe on the GPU; the paper's Tab. ItRuntime "
                                                  "ran MATLAB on a laptop CPU (context, not a target)"}
        del Qe
        # gradient workload: the step-reversal adjoint of <G, S> + sum of positive eigenvalues at n = 2048
        # (d ~ U[1,10], G symmetric N(0,1)), FP64: one warm-up, one timed backward (its forward included)
        ka = 1024
        Ha, _, _ = G.casida_torch(ka, ("uniform", 1.0, 10.0), seed=2048, device=dev)
        ga = torch.Generator(device=dev); ga.manual_seed(3)
        Ga = torch.randn(2 * ka, 2 * ka, dtype=torch.float64, device=dev, generator=ga)
        Ga = 0.5 * (Ga + Ga.T)
        P.sign_vjp_rev(Ha, Ga, pos_weight=1.0, handle=h)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True); g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        Hbar = P.sign_vjp_rev(Ha, Ga, pos_weight=1.0, handle=h)
        g1.record(stream)
        torch.cuda.synchronize()
        line["adjoint_n2048"] = {"s_per_gradient": g0.elapsed_time(g1) / 1e3, "precision": "fp64",
                                 "gradient_fro_norm": float(torch.linalg.norm(Hbar)),
                                 "note": "pssd_sign_vjp_rev: forward Zolotarev sign with its record + reversed steps, "
                                         "congruence and Cholesky; loss <G,S> + sum of positive eigenvalues"}
        del Ha, Ga, Hbar
        # batch workload: 512 Casida matrices, k log-uniform in [16, 1024], d ~ U[0.5, 50], mixed precision,
        # pssd_eig_batched: one warm-up, one timed call; max relative residual checked untimed
        ks = G.batch_sizes(512, 16, 1024, seed=0)
        Hs = [G.casida_torch(int(kk), ("uniform", 0.5, 50.0), seed=10000 + i, device=dev)[0].contiguous()
              for i, kk in enumerate(ks)]
        torch.cuda.synchronize()
        P.eig_batched(Hs, handle=h, precision=P.PSSD_MIXED)
        torch.cuda.synchronize()
        lb0 = h.launch_count()
        ph0 = P.launch_count_phases()
        g0 = torch.cuda.Event(enable_timing=True); g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        Ds, Vs, binfo = P.eig_batched(Hs, handle=h, precision=P.PSSD_MIXED)
        g1.record(stream)
        torch.cuda.synchronize()
        tb = g0.elapsed_time(g1) / 1e3
        with torch.no_grad():
            resb = max(float(torch.linalg.norm(Hx @ Vx - Vx * Dx) / torch.linalg.norm(Hx))
                       for Hx, Dx, Vx in zip(Hs, Ds, Vs))
        line["batch_512_casida"] = {"s_per_step": tb, "instances_per_s": len(Hs) / tb, "instances": len(Hs),
                                 "precision": "mixed", "max_rel_residual": resb,
                                 "gpu_launches": h.launch_count() - lb0,
                                 "launches_by_phase": {k: v - ph0[k] for k, v in P.launch_count_phases().items()},
                                 "host_seconds_by_k": _seconds_by_k(ks, binfo),
                                 "note": "pssd_eig_batched (host work queue over 16 worker streams)"}
        del Hs, Ds, Vs
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(n)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


KERNEL_NAMES = {"dgemm": "gemm_kernel<GM_F64> (FP64 DFMA, 64x64x16 tiles)",
                "sgemm": "gemm_kernel<GM_F32> (FP32 FFMA)",
                "dfgemm": "gemm_kernel<GM_DF> (FP64 emulated with float pairs on the FP32 pipe)",
                "tcgemm": "tc_gemm_kernel (tcgen05 kind::tf32, 3xTF32)",
                "ozgemm": "oz_gemm_kernel (tcgen05 kind::f16 BF16, 36 integer-slice products)"}


def measured_peaks():
    """HBM copy bandwidth and BF16 dense throughput measured on this machine type
    (MEASURED_PEAKS.json beside this file).  Fails loudly when absent: every
    roofline fraction is taken against these measured numbers."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    with open(path) as f:
        d = json.load(f)
    return {"hbm_gbs": float(d["hbm_gbs"]), "bf16": float(d["bf16_tflops"]),
            "bf16_sustained": float(d["bf16_tflops_sustained"])}


def kernel_table(kinds, t_total_s, steps, peaks):
    """Per kind of kernel: time per step, share of the step, launches, and the
    achieved rate against its roof.  Contractions: algorithmic FLOPs in the
    pipe's own operations (3 TF32 products per 3xTF32 product, 36 BF16 slice
    products per slice product) over the kernel's event-timed duration, against
    the SUSTAINED measured BF16 peak (x 1.1/2.25, the nominal TF32/BF16 ratio,
    for TF32) since these kernels run inside a seconds-long step, or against the
    derived FP64 / FP32 ALU roofs.  Memory-bound passes: algorithmic bytes over
    duration against the measured HBM copy bandwidth."""
    fp64_roof = 152 * 2 * 2 * 2.07e9 / 1e12        # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
    fp32_roof = 152 * 128 * 2 * 2.07e9 / 1e12      # 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz
    tensor = {"tcgemm": (3.0, peaks["bf16_sustained"] * 1.1 / 2.25,
                         "of measured: sustained BF16 x 1.1/2.25 (TF32 nominal ratio); 3 TF32 products counted"),
              "ozgemm": (36.0, peaks["bf16_sustained"],
                         "of measured: sustained BF16; 36 BF16 slice products counted (FP64-equivalent = /36)")}
    alu = {"dgemm": (fp64_roof, "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz"),
           "sgemm": (fp32_roof, "derived: 152 SM x 128 FFMA/clk x 2 flop x 2.07 GHz"),
           "dfgemm": (fp32_roof / 13.0, "derived: FP32 issue rate / 13 instructions per multiply-add x 2 flop"),
           "chol_leaf": (fp64_roof, "derived FP64 roof; the leaf is latency-bound (sequential columns)")}
    # DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per product of the pipe's own
    # operations, from one ncu capture of each tensor-core kernel on a 4096^3 product:
    # oz_gemm_kernel 2.346 GB for 36 x 2 x 4096^3 BF16 slice flops, tc_gemm_kernel 0.763 GB for
    # 3 x 2 x 4096^3 TF32 flops.  A launch's traffic is taken in proportion to its flops (the tile
    # shape fixes the bytes moved per flop).
    traffic_per_flop = {"ozgemm": 2.346e9 / (36 * 2 * 4096.0 ** 3), "tcgemm": 0.763e9 / (3 * 2 * 4096.0 ** 3)}
    out = {}
    for name, v in kinds.items():
        if v["launches"] == 0:
            continue
        ms = v["ms"]
        row = {"ms_per_step": ms / steps, "share_of_step": ms / 1e3 / t_total_s if t_total_s > 0 else None,
               "launches_per_step": v["launches"] / steps}
        if name in tensor:
            f, pk, note = tensor[name]
            a = v["flops"] * f / (ms / 1e3) / 1e12
            row.update({"bound": "tensor", "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                        "peak_note": note,
                        "traffic_per_launch": traffic_per_flop[name] * v["flops"] * f / v["launches"],
                        "algorithmic_flops_per_launch": v["flops"] * f / v["launches"]})
        elif name in alu:
            pk, note = alu[name]
            a = v["flops"] / (ms / 1e3) / 1e12
            row.update({"bound": "alu", "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                        "peak_note": note})
        elif v.get("bytes", 0) > 0:
            a = v["bytes"] / (ms / 1e3) / 1e9
            row.update({"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": a / peaks["hbm_gbs"], "bytes_per_step": v["bytes"] / steps,
                        "peak_note": "of measured HBM copy bandwidth; algorithmic bytes of the passes that count them"})
        out[name] = row
    return out


def split_accuracy(P, torch, H, Q, p, dev):
    """Accuracy of a split, measured outside the timed region: S = Q Q^T Sigma,
    randomized estimates of ||S^2 - I||_F and ||SH - HS||_F / ||H||_F, and the
    (Sigma, Sigma_hat)-orthogonality defect of Q."""
    n = H.shape[0]
    with torch.no_grad():
        J = torch.cat([torch.ones(p, device=dev, dtype=torch.float64),
                       -torch.ones(n - p, device=dev, dtype=torch.float64)])
        g = torch.Generator(device=dev); g.manual_seed(7)
        X = torch.randn(n, 16, device=dev, dtype=torch.float64, generator=g)
        Sx = lambda Y: Q @ (Q.T @ (J[:, None] * Y))
        R = Sx(Sx(X)) - X
        s2 = float(torch.linalg.norm(R) / 4.0)                     # E||(S^2-I)x||^2 = ||S^2-I||_F^2
        C = Sx(H @ X) - H @ Sx(X)
        comm = float(torch.linalg.norm(C) / 4.0 / torch.linalg.norm(H))
        QJQ = float(torch.linalg.norm(Q.T @ (J[:, None] * Q) - torch.diag(J)) / torch.linalg.norm(Q) ** 2)
    return {"s2_resid_est_from_Q": s2, "comm_rel_est_from_Q": comm, "qjq_rel_defect": QJQ}


if __name__ == "__main__":
    sys.exit(main())
