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
import os
import statistics
import subprocess
import sys
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
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_%d.csv" % os.getpid())
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
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
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def cpu_baseline_sample(seconds_target=20.0):
    """The oracle (Alg. 8 + Alg. 7 in scalar-loop FP64 C) on a bounded sample
    of the same workload: the same generator at n = 512 (k = 256), timed on the
    host cores, scaled to n = 16384 by n^3."""
    import casida_inputs as G
    import oracle as O
    n_s = 512
    H, _, _ = G.casida(n_s // 2, ("loguniform", 1e-2, 1e2), seed=0)
    t0 = time.perf_counter()
    S, info = O.sign_alg(H)
    O.split_alg(H, None, S)
    t = time.perf_counter() - t0
    scale = (16384 / n_s) ** 3
    return {"value": t * scale, "unit": "s/solve", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle sign (Alg. 8, scalar-loop pivoted elimination) + split (Alg. 7) of one n=%d "
                      "Casida input of the same distribution: %.2f s measured, scaled by (16384/%d)^3 = %d "
                      "to s/solve at n=16384 (extrapolated)" % (n_s, t, n_s, int(scale)),
            "measured_s": t, "measured_n": n_s}


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    vals = []
    for _ in range(args.warmup):
        cpu_baseline_sample()
    for _ in range(args.steps):
        vals.append(cpu_baseline_sample())
    v = statistics.median([x["value"] for x in vals])
    cb = dict(vals[-1]); cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/solve", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "casida_n16384_log1e-2_1e2 split (oracle sample n=512, n^3-scaled)"},
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
            "max_rel_residual": res, "gpu_launches": h.launch_count() - l0, "clocks": ck}
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
                         "fp64e: the FP64 algorithm with FP64 emulated on the FP32 pipe")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP64 comparison solve")
    ap.add_argument("--workload", default="split", choices=["split", "batch"],
                    help="split: one n x n sign + split per step (headline); batch: full diagonalisation of "
                         "512 Casida matrices with k log-uniform in [16, 1024], d ~ U[0.5, 50]")
    ap.add_argument("--batch-count", type=int, default=512)
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
    n = args.n
    k = n // 2
    dist_d = ("loguniform", 1e-2, 1e2)
    if n <= 4096:   # numpy generator (also keeps torch's GPU linear algebra out of profiler runs)
        Hn, d1, d2 = G.casida(k, dist_d, seed=1234 + rank)
        H = torch.from_numpy(Hn).to(dev)
    else:
        H, d1, d2 = G.casida_torch(k, dist_d, seed=1234 + rank, device=dev)
    H = H.contiguous()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    h = P.Handle(stream)
    p = n // 2

    prec = {"fp64": P.PSSD_FP64, "mixed": P.PSSD_MIXED, "fp64e": P.PSSD_FP64_EMULATED}[args.precision]

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
    e0.record(stream)
    for _ in range(args.steps):
        Q, A11, A22, pp, info = step()
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ck = clocks.stop()
    h.profile(False)
    launches = h.launch_count() - l0
    t = e0.elapsed_time(e1) / 1e3
    if ws > 1:
        t = max_over_ranks(t, dev)
    kinds = {P.KIND_NAMES[i]: h.profile_read(i) for i in range(len(P.KIND_NAMES))}
    # dominant kernel of this precision mode
    dom = max(["dgemm", "sgemm", "dfgemm", "tcgemm", "ozgemm"], key=lambda kk: kinds[kk]["ms"])
    gemm = kinds[dom]
    last = infos[-1]
    rs = [x for x in last["r_used"][:last["passes"]]]
    # algorithmic FLOPs: the library's exact structural count of every contraction it launched
    fl = sum(kinds[kk]["flops"] for kk in ("dgemm", "sgemm", "dfgemm", "tcgemm", "ozgemm", "chol_leaf")) / args.steps
    solves = args.steps * ws
    s_per_solve = t / solves
    # accuracy of the split, measured outside the timed region: S = Q Q^T Sigma,
    # randomized estimates of ||S^2 - I||_F and ||S H - H S||_F / ||H||_F
    with torch.no_grad():
        J = torch.cat([torch.ones(p, device=dev, dtype=torch.float64), -torch.ones(n - p, device=dev, dtype=torch.float64)])
        g = torch.Generator(device=dev); g.manual_seed(7)
        X = torch.randn(n, 16, device=dev, dtype=torch.float64, generator=g)
        Sx = lambda Y: Q @ (Q.T @ (J[:, None] * Y))
        R = Sx(Sx(X)) - X
        s2 = float(torch.linalg.norm(R) / 4.0)                     # E||(S^2-I)x||^2 = ||S^2-I||_F^2
        C = Sx(H @ X) - H @ Sx(X)
        comm = float(torch.linalg.norm(C) / 4.0 / torch.linalg.norm(H))
        QJQ = float(torch.linalg.norm(Q.T @ (J[:, None] * Q) - torch.diag(J)) / torch.linalg.norm(Q) ** 2)
    # the metric's condition on S itself: S = L^{-T} sign(K) L^T from pssd_sign in the same
    # precision mode, ||S^2 - I||_F computed by the library (untimed)
    S_chk, info_s = P.sign(H, handle=h, precision=prec, flags=P.FLAG_RESIDUALS)
    s2_sign = info_s["s2_resid"]
    del S_chk
    peak_fp64 = 152 * 2 * 2 * 2.07e9 / 1e12        # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
    peak_fp32 = 152 * 128 * 2 * 2.07e9 / 1e12      # 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz
    achieved = (gemm["flops"] / gemm["launches"]) / (gemm["ms"] / gemm["launches"] / 1e3) / 1e12 if gemm["launches"] else None
    # the FP64-emulating kernel spends 13 FP32 instructions per multiply-add (see the design notes):
    # its ALU roof is the FP32 issue rate / 6.5 in FP64-equivalent FLOP/s
    bf16_meas = 1901.5    # measured cuBLAS BF16 dense TFLOP/s on this machine's GB300 (burst)
    try:
        bf16_meas = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        pass
    # tensor-core kernels are reported in the tensor pipe's own operations:
    #   tcgemm: 3 TF32 products per FP32 product; TF32 peak = BF16 peak x (1.1 / 2.25) nominal ratio
    #   ozgemm: 36 BF16 slice products per FP64 product; peak = measured BF16
    tensor_factor = {"tcgemm": 3.0, "ozgemm": 36.0}.get(dom, 1.0)
    if achieved is not None:
        achieved *= tensor_factor
    peak_dom = {"dgemm": peak_fp64, "sgemm": peak_fp32, "dfgemm": peak_fp32 / 13.0,
                "tcgemm": bf16_meas * 1.1 / 2.25, "ozgemm": bf16_meas}[dom]
    line = {
        "metric": METRIC, "value": s_per_solve, "unit": "s/solve", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32+f64", "fp64e": "f64 (emulated on f32)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": "casida_n%d_log1e-2_1e2 split (sign+split), %s path" % (n, args.precision), "n": n,
                   "k": k, "precision": args.precision, "l2": "inputs larger than L2 (2.1 GB per H), no flush",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "tflops": fl * solves / t / 1e12, "algorithmic_flops_per_solve": fl,
        "r_per_pass": rs, "restarts": last["restarts"], "alpha": last["alpha"], "beta": last["beta"],
        "accuracy": {"s2_resid_sign": s2_sign, "s2_bound": 1e-12 * n, "s2_ok": bool(s2_sign <= 1e-12 * n),
                     "s2_resid_est_from_Q": s2, "comm_rel_est_from_Q": comm, "qjq_rel_defect": QJQ,
                     "split_backerr_K": last["split_backerr"]},
        "roofline": {"kernel": {"dgemm": "gemm_kernel<GM_F64> (FP64 DFMA, 64x64x16 tiles)",
                                "sgemm": "gemm_kernel<GM_F32> (FP32 FFMA)",
                                "dfgemm": "gemm_kernel<GM_DF> (FP64 emulated on the FP32 pipe)",
                                "tcgemm": "tc_gemm_kernel (tcgen05 kind::tf32, 3xTF32)",
                                "ozgemm": "oz_gemm_kernel (tcgen05 kind::f16 BF16, 36 integer-slice products)"}[dom],
                     "bound": "tensor" if dom in ("tcgemm", "ozgemm") else "alu",
                     "achieved": achieved, "peak": peak_dom, "unit": "TFLOP/s",
                     "frac": (achieved / peak_dom) if achieved else None, "traffic": None,
                     "peak_note": {"dgemm": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz (cuBLAS DGEMM measured 1.09)",
                                   "sgemm": "derived: 152 SM x 128 FFMA/clk x 2 flop x 2.07 GHz",
                                   "dfgemm": "derived: FP32 issue rate (152 SM x 128/clk x 2.07 GHz) / 13 instructions per multiply-add x 2 flop",
                                   "tcgemm": "of measured: BF16 burst x 1.1/2.25 (TF32 nominal ratio); achieved counts the 3 TF32 products",
                                   "ozgemm": "of measured: BF16 burst; achieved counts the 36 BF16 slice products (FP64-equivalent = achieved/36)"}[dom],
                     "share_of_step": gemm["ms"] / 1e3 / t if t > 0 else None},
        "kernels": kinds,
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
        f0.record(stream)
        Hd = Hh.to(dev, non_blocking=True)
        Q2, B11, B22, _, _ = P.split(Hd, handle=h, precision=prec)
        Qh.copy_(Q2, non_blocking=True); A11h.copy_(B11, non_blocking=True); A22h.copy_(B22, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        te = f0.elapsed_time(f1) / 1e3
        line["e2e"] = {"value": te, "unit": "s/solve", "h2d_bytes_per_step": 8 * n * n,
                       "d2h_bytes_per_step": 8 * (n * n + p * p + (n - p) ** 2)}
    if rank == 0 and not args.no_compare and args.precision != "fp64":
        # plain FP64 on the same input: one untimed warm-up (allocations), one timed solve
        step(P.PSSD_FP64)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True); g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        Qf, A11f, A22f, _, infof = step(P.PSSD_FP64)
        g1.record(stream)
        torch.cuda.synchronize()
        tf = g0.elapsed_time(g1) / 1e3
        with torch.no_grad():
            dA = float(torch.linalg.norm(torch.linalg.eigvalsh(A11f) - torch.linalg.eigvalsh(A11))
                       / torch.linalg.norm(torch.linalg.eigvalsh(A11f)))
        line["plain_fp64"] = {"s_per_solve": tf, "speedup_of_this_path": tf / s_per_solve,
                              "split_backerr": infof["split_backerr"],
                              "A11_spectrum_rel_diff_vs_this_path": dA,
                              "note": "same input, 1 warm-up + 1 timed solve"}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
