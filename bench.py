#!/usr/bin/env python
"""Benchmark of the RSM hot path on one GB300 (or N replicas under torchrun).

One step = one full decomposition of the paper-scale synthetic workload
(m = 131072, n = 1024, r = 8, rho = 0.7, sigma = 1e-3, l = 9, 20000 submatrices):
mask packing, column sampling, row selection + Gram, minor vectors, M, the
eigensolve of M, the per-row solves for U and the error e, all in librsm.so.

Headline form: Y in FP32, FP32 Gram and normal equations, FP64 minor vectors,
M, eigensolve and r x r solves; its V is checked against the plain FP64 form
(itself parity-tested against the FP64 oracle) at <= 1e-6 subspace angle.
The plain FP64 form is timed beside it.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead (bounded samples of the same workload, single core).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decomps/s & submatrices/s at ≤1e-6 subspace angle vs FP64 oracle; p50/p99 lat"
WORKLOAD = "paper_131072x1024"
STAGES = ["setup", "pack_mask", "sample_cols", "select_gram", "minor_scatter", "eig_M", "solve_U", "residual", "total"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--fp64-steps", type=int, default=0, help="timed steps of the FP64 form (default max(3, steps/4))")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)  # internal: CPU worker
    return ap.parse_args()


# ----------------------------------------------------------------- oracle (CPU) legs

def oracle_sample(trial_sample: int, row_sample: int, seed: int = 0) -> dict:
    """Time the FP64 oracle on a bounded sample of the workload and extrapolate to one decomposition.

    Sample: ``trial_sample`` of the I submatrices (row scan, SVD, accumulation),
    the full eigensolve of M, and U plus the residual on ``row_sample`` of the m rows.
    """
    import oracle
    from oracle import rsm as orsm
    from workloads import config_problem

    p = config_problem(WORKLOAD)
    cols = orsm.sample_columns(p.n, p.l, trial_sample, p.seed)
    t0 = time.perf_counter()
    Zs = []
    for t in range(trial_sample):
        R = orsm.select_rows(p.W, cols[t])
        if R.size < p.l:
            Zs.append(None)
            continue
        Zs.append(orsm.minor_vectors(np.asarray(p.Y[np.ix_(R, cols[t])]), p.l - p.r))
    M = orsm.accumulate_M(p.n, cols, Zs)
    t_trials = time.perf_counter() - t0
    t0 = time.perf_counter()
    V, _ = orsm.eig_smallest(M, p.r)
    t_eig = time.perf_counter() - t0
    t0 = time.perf_counter()
    U, _ = orsm.solve_U(p.Y[:row_sample], p.W[:row_sample], V)
    orsm.residual(p.Y[:row_sample], p.W[:row_sample], U, V)
    t_rows = time.perf_counter() - t0
    est = t_trials * p.trials / trial_sample + t_eig + t_rows * p.m / row_sample
    return dict(decomps_per_s=1.0 / est, submatrices_per_s=trial_sample / t_trials, est_s_per_decomp=est,
                t_trials=t_trials, t_eig=t_eig, t_rows=t_rows,
                sample=f"{trial_sample} of {p.trials} submatrices + full eigensolve of M + U and e on "
                       f"{row_sample} of {p.m} rows, extrapolated to one decomposition")


def run_oracle_worker(trial_sample: int, row_sample: int) -> dict:
    """Run oracle_sample in a single-threaded child process (BLAS pinned to one thread)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample",
                          f"{trial_sample},{row_sample}"], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, out_path: str):
        self.out_path = out_path
        self.proc = None

    def start(self):
        try:
            self.f = open(self.out_path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # nvidia-smi takes a moment to emit its first sample
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.out_path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) == 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        idx = sorted({r[0] for r in rows})
        want = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        gpu = want if want in idx else idx[0]
        rows = [r for r in rows if r[0] == gpu]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- helpers

def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def traffic_record(summary: str):
    """DRAM bytes per launch of the dominant kernel from its committed ncu summary.

    The summary (a text file under profiles/) carries ``source``,
    ``source_sha256``, ``launches_per_step`` and ``dram_bytes_per_launch`` lines;
    the record is used only while the kernel source still has that hash.
    """
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for line in f:
            parts = line.strip().split(":", 1)
            if len(parts) == 2 and parts[0] in ("source", "source_sha256", "launches_per_step", "dram_bytes_per_launch"):
                rec[parts[0]] = parts[1].strip()
    if len(rec) < 4:
        return None
    with open(os.path.join(ROOT, rec["source"]), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != rec["source_sha256"]:
            return None
    return {"launches_per_step": int(rec["launches_per_step"]), "dram_bytes_per_launch": int(rec["dram_bytes_per_launch"])}


def dist_setup(n_gpus: int):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier_sync(ws, device=None):
    """Drain the device, then (N > 1) a barrier over all ranks, then drain again."""
    import torch
    cuda = device is None or getattr(device, "type", "cuda") == "cuda"
    if cuda:
        torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    if cuda:
        torch.cuda.synchronize()


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """The largest x over all ranks (the slowest rank's time decides)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device if device is not None else "cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws: int, steps: int, max_ms: float) -> float:
    """Whole-job decompositions per second: every rank ran `steps` decompositions in at most max_ms."""
    return ws * steps / (max_ms / 1e3)


def subspace_sin(A, B) -> float:
    """sin of the largest principal angle between the column spans of A and B (orthonormal columns).

    A and B are small (n x r); the angle is evaluated on the host."""
    a = A.detach().cpu().numpy()
    b = B.detach().cpu().numpy()
    return float(np.linalg.norm(b - a @ (a.T @ b), ord=2))


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q / 100.0
    f, c = math.floor(k), math.ceil(k)
    return xs[f] + (xs[c] - xs[f]) * (k - f)


# ----------------------------------------------------------------- GPU arm

def bench_mine(args):
    import torch

    import paper_1411_0814_gb300 as rsm
    from workloads import config_problem

    ws, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    # a stream of our own (not the legacy default stream, which would serialise
    # with the copy stream of the end-to-end measurement)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    p = config_problem(WORKLOAD)
    Y64 = torch.from_numpy(np.ascontiguousarray(p.Y.T)).to(dev).t()  # column-major m x n
    Y32 = Y64.to(torch.float32)
    W = torch.from_numpy(np.ascontiguousarray(p.W.T)).to(dev).t()
    torch.cuda.synchronize()
    h = rsm.RSM(dev.index, stream=stream)
    common = dict(trials=p.trials, l=p.l, seed=p.seed, variant=p.variant)
    mixed = rsm.Problem(Y32, W, p.r, gram="f32", solve="f32", **common)
    fp64 = rsm.Problem(Y64, W, p.r, gram="f64", solve="f64", **common)

    def timed(prob, steps, warmup):
        for _ in range(warmup):
            h.decompose(prob)
        barrier_sync(ws)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        results = []
        evs[0].record(stream)
        for k in range(steps):
            results.append(h.decompose(prob))
            evs[k + 1].record(stream)
        barrier_sync(ws)
        per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
        return evs[0].elapsed_time(evs[-1]), per, results

    # headline: mixed form, inputs resident in HBM
    import tempfile
    clocks = ClockSampler(os.path.join(tempfile.gettempdir(), f"rsm_clocks_rank{rank}_{os.getpid()}.csv"))
    for _ in range(args.warmup):
        h.decompose(mixed)
    clocks.start()
    total_ms, per, res = timed(mixed, args.steps, 0)
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms, ws)
    last = res[-1]
    assert last.status == 0, f"mixed form status {last.status}"

    # plain FP64 form on the same GPU
    k64 = args.fp64_steps or max(3, args.steps // 4)
    total64, per64, res64 = timed(fp64, k64, 1)
    assert res64[-1].status == 0
    angle = math.asin(min(1.0, subspace_sin(fp64.V, mixed.V)))

    # end to end through the public API: host (pinned) -> device, decompose, device -> host.
    # Every step copies its own inputs in and its results out inside the timed
    # region; the copies of step k + 1's inputs run on a copy stream while step k
    # computes (two device buffer sets).
    e2e = None
    if not args.no_e2e:
        hY = torch.empty((p.n, p.m), dtype=torch.float32, pin_memory=True)
        hY.copy_(Y32.t())
        hW = torch.empty((p.n, p.m), dtype=torch.uint8, pin_memory=True)
        hW.copy_(W.t())
        hU = torch.empty((p.r, p.m), dtype=torch.float64, pin_memory=True)
        hV = torch.empty((p.r, p.n), dtype=torch.float64, pin_memory=True)
        sets = []
        for _ in range(2):
            dY = torch.empty((p.n, p.m), dtype=torch.float32, device=dev)
            dW = torch.empty((p.n, p.m), dtype=torch.uint8, device=dev)
            sets.append((dY, dW, rsm.Problem(dY.t(), dW.t(), p.r, gram="f32", solve="f32", **common)))
        cs = torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]

        def e2e_run(steps):
            with torch.cuda.stream(cs):
                sets[0][0].copy_(hY, non_blocking=True)
                sets[0][1].copy_(hW, non_blocking=True)
                ev_in[0].record(cs)
            for k in range(steps):
                dY, dW, prob_k = sets[k % 2]
                stream.wait_event(ev_in[k % 2])
                if k + 1 < steps:  # the next step's inputs, while this one computes
                    nY, nW, _ = sets[(k + 1) % 2]
                    with torch.cuda.stream(cs):
                        nY.copy_(hY, non_blocking=True)
                        nW.copy_(hW, non_blocking=True)
                        ev_in[(k + 1) % 2].record(cs)
                h.decompose(prob_k)
                with torch.cuda.stream(cs):
                    cs.wait_stream(stream)
                    hU.copy_(prob_k.U.t(), non_blocking=True)
                    hV.copy_(prob_k.V.t(), non_blocking=True)
            stream.wait_stream(cs)

        e2e_run(max(1, args.warmup))
        barrier_sync(ws)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        e2e_run(args.steps)
        s1.record(stream)
        barrier_sync(ws)
        e2e_ms = max_over_ranks(s0.elapsed_time(s1), ws)
        h2d = hY.numel() * 4 + hW.numel()
        d2h = hU.numel() * 8 + hV.numel() * 8
        e2e = {"value": replica_throughput(ws, args.steps, e2e_ms), "unit": "decomps/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms / args.steps,
               "note": "pinned host Y (FP32) and W copied in, U and V copied out, every step; step k+1's "
                       "inputs copy on a second stream while step k computes"}

    # roofline of the dominant kernel: fused row selection + Gram (HBM-bound)
    stage = {k: statistics.median([r_.stage_ms[k] for r_ in res]) for k in STAGES}
    stage64 = {k: statistics.median([r_.stage_ms[k] for r_ in res64]) for k in STAGES}
    dominant = max((k for k in STAGES if k not in ("total", "setup")), key=lambda k: stage[k])
    nwords = (p.m + 31) // 32
    P_l = p.l * (p.l + 1) // 2
    alg_bytes = (p.trials * (p.l * nwords * 4 + P_l * 8 + p.l * 4 + 4) + last.rows_selected * p.l * 4)
    sg_ms = stage["select_gram"]
    peaks = measured_peaks()
    achieved = alg_bytes / (sg_ms * 1e-3) / 1e9
    trec = traffic_record("k_gram_slab_paper_131072x1024.md")
    launches = trec["launches_per_step"] if trec else 16  # row slabs of 32 MiB of FP32 Y
    traffic = trec["dram_bytes_per_launch"] if trec else None
    roofline = {"kernel": "k_gram_slab<2,9> (row-slab selection + FP32 Gram)", "bound": "hbm",
                "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": int(alg_bytes / launches), "launches_per_step": launches,
                "launch_ms": round(sg_ms / launches, 4), "peak_source": peaks["source"] + " (copy bandwidth)",
                "note": "traffic (DRAM bytes per launch, ncu) is ~10x below the algorithmic bytes: the slab "
                        "schedule serves repeated reads from L2; the kernel is bound by L2 sector reads"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            o = run_oracle_worker(2000, 16384)
            cpu = {"value": o["decomps_per_s"], "unit": "decomps/s", "cores": 1, "kind": "oracle",
                   "sample": o["sample"], "submatrices_per_s": o["submatrices_per_s"],
                   "est_s_per_decomp": o["est_s_per_decomp"]}
        except Exception as ex:  # report, do not hide
            cpu = {"value": None, "unit": "decomps/s", "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}

    launches_per_step = last.kernel_launches
    out = {
        "metric": METRIC,
        "value": replica_throughput(ws, args.steps, total_ms),
        "unit": "decomps/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "fp32+fp64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": p.m, "n": p.n, "r": p.r, "rho": p.rho, "sigma": p.sigma, "l": p.l,
                   "trials": p.trials, "form": "Y, Gram and normal equations FP32; minor vectors, M, eigensolve "
                                                 "and r x r solves FP64",
                   "l2": "inputs larger than L2 (Y fp32 537 MB, W 134 MB)", "parallelism": f"replicas x{ws}"},
        "submatrices_per_s": ws * args.steps * last.accepted_trials / (total_ms / 1e3),
        "submatrices_per_s_gram_stage": last.accepted_trials / (stage["select_gram"] * 1e-3),
        "latency_ms": {"p50": pct(per, 50), "p99": pct(per, 99)},
        "angle_vs_fp64_form": angle,
        "eig_factor_bits": last.eig_factor_bits,
        "eig_iterations": last.eig_iterations,
        "fp64_form": {"value": replica_throughput(ws, k64, max_over_ranks(total64, ws)), "unit": "decomps/s", "ms_per_step": total64 / k64,
                      "latency_ms": {"p50": pct(per64, 50), "p99": pct(per64, 99)}, "stage_ms": stage64},
        "stage_ms": stage,
        "dominant_stage": dominant,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    h.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------- reference arm (the oracle)

def bench_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from workloads import config_problem

    p = config_problem(WORKLOAD)
    trial_sample, row_sample = 300, 2048
    per_decomp = []
    t_start = time.perf_counter()
    for k in range(args.warmup + args.steps):
        o = run_oracle_worker(trial_sample, row_sample)
        if k >= args.warmup:
            per_decomp.append(o["est_s_per_decomp"])
    est = statistics.mean(per_decomp)
    value = 1.0 / est
    sample = (f"each step: {trial_sample} of {p.trials} submatrices + full eigensolve of M + U and e on "
              f"{row_sample} of {p.m} rows, extrapolated to one decomposition")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "decomps/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": est * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "m": p.m, "n": p.n, "r": p.r, "rho": p.rho, "sigma": p.sigma, "l": p.l,
                      "trials": p.trials, "form": "FP64 CPU oracle (numpy), one core"},
           "cpu_baseline": {"value": value, "unit": "decomps/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "decomps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": time.perf_counter() - t_start}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.oracle_sample:
        ts, rs = (int(x) for x in args.oracle_sample.split(","))
        print(json.dumps(oracle_sample(ts, rs)))
        return
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_mine(args)


if __name__ == "__main__":
    main()
