#!/usr/bin/env python
"""Benchmark of the RSM hot path on one GB300 (or N replicas under torchrun).

One step = one full decomposition of the paper-scale synthetic workload
(m = 131072, n = 1024, r = 8, rho = 0.7, sigma = 1e-3, l = 9, 20000 submatrices):
mask packing, column sampling, row selection + Gram, minor vectors, M, the
eigensolve of M, the per-row solves for U and the error e, all in librsm.so.

Headline form: Y in FP32, FP32 Gram and FP32 accumulation of the normal
equations (tensor cores); FP64 minor vectors, M, eigensolve (FP32-pair
iteration ended by an FP64 refinement pass) and r x r solves.  Its V-hat is
compared with the FP64 oracle's V-hat for this workload (stored by
tests/golden/make_oracle_goldens.py, which calls only the oracle): the
subspace angle must be <= 1e-6.  The plain FP64 form is timed beside it and
held to 1e-10.

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
WORKLOADS = ["paper_131072x1024", "noiseless_2048x128", "trajectory_4096x144", "batched256", "serving", "fig1_sweep"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--workload", choices=WORKLOADS, default=WORKLOAD,
                    help="paper_131072x1024 (default, the headline); the others are measured on demand")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serving: length of the arrival stream")
    ap.add_argument("--batched-gram", choices=["f32", "f32x2"], default="f32",
                    help="batched256 / serving: the per-trial Gram form of the mixed batched form")
    ap.add_argument("--fp64-steps", type=int, default=0, help="timed steps of the FP64 form (default max(3, steps/4))")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="paper workload: keep the default Gram schedule instead of rsm_autotune's choice")
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


# ----------------------------------------------------------------- the oracle on all host cores
# The oracle's functions, unchanged, driven over P processes: the draws are
# split into P contiguous chunks (row scan + SVD per draw in the workers), M is
# accumulated in the parent in ascending draw order (the oracle's order), its
# eigensolve runs in the parent, and U and the residual are split by rows.
# Each worker builds the workload itself once (not timed).
_POOL_PROBLEM = None


def _pool_init(workload):
    import os as _os
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        _os.environ[k] = "1"
    global _POOL_PROBLEM
    from workloads import config_problem
    _POOL_PROBLEM = config_problem(workload)


def _pool_trials(args):
    from oracle import rsm as orsm
    cols, = args
    p = _POOL_PROBLEM
    out = []
    for c in cols:
        R = orsm.select_rows(p.W, c)
        out.append(None if R.size < p.l else orsm.minor_vectors(np.asarray(p.Y[np.ix_(R, c)]), p.l - p.r))
    return out


def _pool_rows(args):
    from oracle import rsm as orsm
    i0, i1, V = args
    p = _POOL_PROBLEM
    U, _ = orsm.solve_U(p.Y[i0:i1], p.W[i0:i1], V)
    w = p.W[i0:i1].astype(np.float64)
    d = (np.asarray(p.Y[i0:i1], dtype=np.float64) - U @ V.T) * w
    return float(np.sum(d * d)), float(np.sum(w))


class OraclePool:
    """One whole decomposition by the oracle on `procs` host processes."""

    def __init__(self, workload: str, procs: int):
        import multiprocessing as mp
        from workloads import config_problem
        self.p = config_problem(workload)
        self.procs = procs
        # one BLAS thread per worker: the children read these when they start
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        os.environ.update({k: "1" for k in saved})
        try:
            self.pool = mp.get_context("spawn").Pool(procs, initializer=_pool_init, initargs=(workload,))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.pool.map(_pool_rows, [(0, 1, np.zeros((self.p.n, self.p.r)))] * procs)  # wait for the workers

    def decompose(self) -> dict:
        from oracle import rsm as orsm
        p = self.p
        t0 = time.perf_counter()
        cols = orsm.sample_columns(p.n, p.l, p.trials, p.seed)
        chunks = np.array_split(np.arange(p.trials), self.procs * 4)
        Zs = [z for part in self.pool.map(_pool_trials, [(cols[c],) for c in chunks]) for z in part]
        M = orsm.accumulate_M(p.n, cols, Zs)
        V, evals = orsm.eig_smallest(M, p.r)
        bounds = np.linspace(0, p.m, self.procs * 4 + 1).astype(int)
        parts = self.pool.map(_pool_rows, [(bounds[k], bounds[k + 1], V) for k in range(len(bounds) - 1)])
        e = float(np.sqrt(sum(a for a, _ in parts) / sum(b for _, b in parts)))
        return {"seconds": time.perf_counter() - t0, "V": V, "e": e, "accepted": sum(z is not None for z in Zs)}

    def close(self):
        self.pool.terminate()
        self.pool.join()


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


def oracle_golden(p):
    """The FP64 oracle's V-hat of this workload (tests/golden), or None if absent or for another workload."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{WORKLOAD}.npz")
    if not os.path.exists(path):
        return None
    g = np.load(path)
    if (int(g["m"]), int(g["n"]), int(g["r"]), int(g["trials"]), int(g["seed"])) != (p.m, p.n, p.r, p.trials, p.seed):
        return None
    return {k: g[k] for k in g.files}


def gather_probe(dev, stream, per_line: int) -> float:
    """Loads per second from random 128-byte lines of a 32 MiB L2-resident buffer (rsm_probe_gather), per_line
    distinct sectors of each line (1: the L1 line rate, 4: the L2 sector rate), best of 5."""
    import torch

    import paper_1411_0814_gb300 as rsm
    lib = rsm.lib()
    buf = torch.rand(1 << 23, device=dev)
    blocks, per = 152 * 16, 256
    out = torch.empty(blocks * 256, device=dev)
    best = None
    for k in range(7):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = lib.rsm_probe_gather(buf.data_ptr(), buf.numel(), blocks, per, per_line, out.data_ptr(),
                                  stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if st != 0:
            return None
        if k >= 2:
            rate = blocks * 256 * per / (e0.elapsed_time(e1) * 1e-3)
            best = rate if best is None else max(best, rate)
    return best


def gpu_numa_cpus(dev):
    """(NUMA node of the GPU's PCI function, the CPUs of that node this process may use), or (None, None)."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev)
        bus = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bus}/numa_node") as f:
            node = int(f.read().strip())
        if node < 0:
            return None, None
        with open(f"/sys/devices/system/node/node{node}/cpulist") as f:
            cpus = set()
            for part in f.read().strip().split(","):
                a, _, b = part.partition("-")
                cpus.update(range(int(a), int(b or a) + 1))
        cpus &= os.sched_getaffinity(0)
        return node, (cpus or None)
    except Exception:
        return None, None


def pinned_near(dev, shape, dtype, fill=None):
    """A pinned host tensor whose pages are first touched from the CPUs of the GPU's NUMA node
    (the process's CPU affinity is narrowed for the allocation and the fill, then restored)."""
    import torch
    node, cpus = gpu_numa_cpus(dev)
    old = os.sched_getaffinity(0)
    try:
        if cpus:
            os.sched_setaffinity(0, cpus)
        t = torch.empty(shape, dtype=dtype, pin_memory=True)
        if fill is not None:
            t.copy_(fill)
        else:
            t.zero_()
    finally:
        if cpus:
            os.sched_setaffinity(0, old)
    return t, node


def h2d_rate(src, dst, stream, reps=3) -> float:
    """GB/s of one pinned host -> device copy of src into dst on `stream` (best of reps)."""
    import torch
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            dst.copy_(src, non_blocking=True)
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return src.numel() * src.element_size() / (best * 1e-3) / 1e9


def subspace_angle_np(a, b) -> float:
    qa, _ = np.linalg.qr(a)
    qb, _ = np.linalg.qr(b)
    return float(math.asin(min(1.0, np.linalg.norm(qb - qa @ (qa.T @ qb), ord=2))))


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

    # the Gram-stage choice a user would make once per problem shape (before any timing);
    # the FP64 form and the end-to-end problems share the handle and so the choice
    tune = None if args.no_autotune else h.autotune(mixed, reps=2)
    if tune is not None:
        h.autotune(fp64, reps=1)

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
    gold = oracle_golden(p)
    angle_oracle = angle_oracle64 = None
    if gold is not None:
        angle_oracle = subspace_angle_np(mixed.V.detach().cpu().numpy(), gold["V"])
        angle_oracle64 = subspace_angle_np(fp64.V.detach().cpu().numpy(), gold["V"])

    # end to end through the public API: host (pinned) -> device, decompose, device -> host.
    # Every step copies its own inputs in and its results out inside the timed
    # region; the copies of step k + 1's inputs run on a copy stream while step k
    # computes (two device buffer sets).
    e2e = None
    if not args.no_e2e:
        hY, numa = pinned_near(dev, (p.n, p.m), torch.float32, Y32.t())
        hW, _ = pinned_near(dev, (p.n, p.m), torch.uint8, W.t())
        hU, _ = pinned_near(dev, (p.r, p.m), torch.float64)
        hV, _ = pinned_near(dev, (p.r, p.n), torch.float64)
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
        h2d_gbs = h2d_rate(hY, sets[0][0], cs)
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
               "h2d_gbs": round(h2d_gbs, 1), "h2d_ms_per_step": round(h2d / (h2d_gbs * 1e9) * 1e3, 3),
               "host_numa_node": numa,
               "note": "pinned host Y (FP32) and W copied in, U and V copied out, every step; step k+1's "
                       "inputs copy on a second stream while step k computes; h2d_gbs is one pinned copy "
                       "of Y alone, so a step cannot be shorter than h2d_ms_per_step; the pinned buffers are "
                       "first touched from the CPUs of the GPU's NUMA node (host_numa_node)"}

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
    # one launch per row slab: 32 MiB of FP32 Y by default, or the autotuner's slab size
    slab_mib = tune["slab_mib"] if tune is not None and tune["schedule"] == "slab" else 32
    slab_rows = max(1024, ((slab_mib << 20) // (p.n * 4)) // 32 * 32)
    launches = -(-p.m // slab_rows)
    # DRAM bytes per launch from the committed ncu summary (taken at its own slab size; the slab
    # launches read Y once between them, so the bytes per launch scale with the rows per launch)
    trec = traffic_record("k_gram_slab_paper_131072x1024.md")
    traffic = (int(trec["dram_bytes_per_launch"] * trec["launches_per_step"] / launches) if trec else None)
    # the L2 sector ceiling (rsm_probe_gather, measured here) against the slab Gram's sectors: per
    # trial and column, the 8-row sectors that hold a selected row (rows selected with probability
    # q = p_t / m: a fraction 1 - (1 - q)^8 of the m / 8 sectors), plus the mask words (8 per sector)
    gather = gather_probe(dev, stream, 4)
    q = last.rows_selected / (p.trials * p.m)
    mask_sectors = p.trials * p.l * ((p.m + 31) // 32) / 8
    gathers = p.trials * p.l * (p.m / 8.0) * (1.0 - (1.0 - q) ** 8) + mask_sectors
    gather_rate = gathers / (sg_ms * 1e-3)
    # the L1 line ceiling: a warp load of 32 sorted selected rows touches one 128-byte line per
    # lane, except where a row lies in the same 32-row line as the previous lane's row (gap g < 32
    # with probability (32 - g) / 32 for a gap of g rows, P(g) = q (1 - q)^(g - 1)); the mask
    # reads are one line per warp load of 32 words
    line_rate = gather_probe(dev, stream, 1)
    share = sum((32 - g) / 32.0 * q * (1.0 - q) ** (g - 1) for g in range(1, 32))
    lines = last.rows_selected * p.l * (1.0 - share) + p.trials * p.l * ((p.m + 31) // 32) / 32
    lines_rate = lines / (sg_ms * 1e-3)
    roofline = {"kernel": "k_gram_slab<2,9,0> (row-slab selection + FP32 Gram)", "bound": "hbm",
                "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": int(alg_bytes / launches), "launches_per_step": launches,
                "launch_ms": round(sg_ms / launches, 4), "peak_source": peaks["source"] + " (copy bandwidth)",
                "l1_line_ceiling": {"achieved_lines_per_s": lines_rate, "peak_lines_per_s": line_rate,
                                    "frac": lines_rate / line_rate if line_rate else None, "lines_per_step": lines,
                                    "peak_source": "rsm_probe_gather per_line = 1, measured in this run (every "
                                                   "4-byte load on its own random 128-byte line of a 32 MiB "
                                                   "L2-resident buffer)"},
                "l2_sector_ceiling": {"achieved_sectors_per_s": gather_rate, "peak_sectors_per_s": gather,
                                      "frac": gather_rate / gather if gather else None,
                                      "sectors_per_step": gathers,
                                      "peak_source": "rsm_probe_gather per_line = 4, measured in this run "
                                                     "(four 32-byte sectors of each random 128-byte line)"},
                "note": "traffic (DRAM bytes per launch, ncu) is ~10x below the algorithmic bytes: the slab "
                        "schedule serves repeated reads from L2.  Rows are chosen by data, so a gathered "
                        "element costs a 128-byte line lookup in L1 and a 32-byte sector from L2; the line "
                        "lookups bound the kernel (l1_line_ceiling)"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:  # every host core: one whole decomposition, timed
            procs = len(os.sched_getaffinity(0))
            pool = OraclePool(WORKLOAD, procs)
            try:
                o = pool.decompose()
            finally:
                pool.close()
            one = run_oracle_worker(2000, 16384)
            cpu = {"value": 1.0 / o["seconds"], "unit": "decomps/s", "cores": procs, "nproc": os.cpu_count(),
                   "kind": "oracle", "sample": "one whole decomposition (all 20000 draws, all rows), draws and rows "
                                               f"split over {procs} processes, M reduced in draw order",
                   "seconds": o["seconds"],
                   "angle_gpu_vs_this": subspace_angle_np(mixed.V.detach().cpu().numpy(), o["V"]),
                   "single_core": {"value": one["decomps_per_s"], "unit": "decomps/s", "cores": 1,
                                   "sample": one["sample"], "submatrices_per_s": one["submatrices_per_s"]}}
        except Exception as ex:  # report, do not hide
            cpu = {"value": None, "unit": "decomps/s", "cores": None, "kind": "oracle", "sample": f"failed: {ex}"}

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
                   "trials": p.trials,
                   "form": "Y FP32; per-trial Gram FP32; normal equations N_i, b_i accumulated in FP32 (tensor "
                           "cores, TF32 head + tail); minor vectors FP64 (FP32 Jacobi + FP64 Newton); M FP64 "
                           "(fixed-point sums); eigensolve of M FP32-pair block iteration + FP64 refinement "
                           "(FP64 residual reported); r x r Cholesky solves FP64",
                   "l2": "inputs larger than L2 (Y fp32 537 MB, W 134 MB)", "parallelism": f"replicas x{ws}",
                   "gram_schedule": tune if tune is not None else "default (32 MiB row slabs)"},
        "submatrices_per_s": ws * args.steps * last.accepted_trials / (total_ms / 1e3),
        "submatrices_per_s_gram_stage": last.accepted_trials / (stage["select_gram"] * 1e-3),
        "latency_ms": {"p50": pct(per, 50), "p99": pct(per, 99)},
        "angle_vs_oracle": angle_oracle,
        "angle_vs_oracle_tol": 1e-6,
        "angle_vs_fp64_form": angle,
        "eig_factor_bits": last.eig_factor_bits,
        "eig_iterations": last.eig_iterations,
        "fp64_form": {"value": replica_throughput(ws, k64, max_over_ranks(total64, ws)), "unit": "decomps/s", "ms_per_step": total64 / k64,
                      "angle_vs_oracle": angle_oracle64, "angle_vs_oracle_tol": 1e-10,
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


# ----------------------------------------------------------------- the other workloads (on demand)

def _device_problem(p, dtype, dev):
    import torch
    Y = torch.from_numpy(np.ascontiguousarray(p.Y.T)).to(dev, dtype=dtype).t()
    W = torch.from_numpy(np.ascontiguousarray(p.W.T)).to(dev).t()
    return Y, W


def _line(args, name, value, unit, ms_per_step, dtype, config, **extra):
    out = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": dtype, "data": "synthetic", "config": dict(workload=name, **config)}
    out.update(extra)
    print(json.dumps(out), flush=True)


def _timed_calls(fn, steps, stream):
    import torch
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    out = []
    torch.cuda.synchronize()
    evs[0].record(stream)
    for k in range(steps):
        out.append(fn())
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    return evs[0].elapsed_time(evs[-1]), per, out


def bench_single(args):
    """The small single-problem workloads (FP64 form, latency bound): the noiseless
    2048 x 128 problem and the 4096 x 144 trajectory stand-in.  The oracle runs
    one whole decomposition on one host core (these sizes take seconds)."""
    import torch

    import oracle
    import paper_1411_0814_gb300 as rsm
    from workloads import config_problem

    name = args.workload
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    p = config_problem(name)
    Y, W = _device_problem(p, torch.float64, dev)
    h = rsm.RSM(0, stream=stream)
    common = dict(trials=p.trials, l=p.l, seed=p.seed, variant=p.variant, gram="f64", solve="f64")
    prob = rsm.Problem(Y, W, p.r, **common)
    for _ in range(max(3, args.warmup)):
        h.decompose(prob)
    import tempfile
    clocks = ClockSampler(os.path.join(tempfile.gettempdir(), f"rsm_clocks_{os.getpid()}.csv"))
    clocks.start()
    total, per, res = _timed_calls(lambda: h.decompose(prob), args.steps, stream)
    clk = clocks.stop()
    last = res[-1]
    stage = {k: statistics.median([r_.stage_ms[k] for r_ in res]) for k in STAGES}
    # end to end: host Y, W copied in, U, V copied out, every step
    hY = torch.from_numpy(np.ascontiguousarray(p.Y.T)).pin_memory()
    hW = torch.from_numpy(np.ascontiguousarray(p.W.T)).pin_memory()
    hU = torch.empty((p.r, p.m), dtype=torch.float64, pin_memory=True)
    hV = torch.empty((p.r, p.n), dtype=torch.float64, pin_memory=True)
    dY = torch.empty((p.n, p.m), dtype=torch.float64, device=dev)
    dW = torch.empty((p.n, p.m), dtype=torch.uint8, device=dev)
    eprob = rsm.Problem(dY.t(), dW.t(), p.r, **common)

    def e2e_step():
        dY.copy_(hY, non_blocking=True)
        dW.copy_(hW, non_blocking=True)
        r_ = h.decompose(eprob)
        hU.copy_(eprob.U.t(), non_blocking=True)
        hV.copy_(eprob.V.t(), non_blocking=True)
        return r_
    for _ in range(3):
        e2e_step()
    e2e_ms, _, _ = _timed_calls(e2e_step, args.steps, stream)
    # the oracle: one whole decomposition, one core
    t0 = time.perf_counter()
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, variant=p.variant)
    t_oracle = time.perf_counter() - t0
    angle = oracle.subspace_angle(prob.V.cpu().numpy(), o.V)
    _line(args, name, 1e3 * args.steps / total, "decomps/s", total / args.steps, "f64",
          dict(m=p.m, n=p.n, r=p.r, l=p.l, trials=p.trials, variant=p.variant, form="FP64 throughout",
               l2="inputs smaller than L2; consecutive decompositions of the same resident problem"),
          latency_ms={"p50": pct(per, 50), "p99": pct(per, 99)}, stage_ms=stage,
          submatrices_per_s=args.steps * last.accepted_trials / (total * 1e-3),
          status=last.status, accepted_trials=last.accepted_trials, angle_vs_oracle=angle, angle_vs_oracle_tol=1e-10,
          accepted_trials_oracle=o.accepted_trials, e=last.e, e_oracle=o.e,
          e2e={"value": 1e3 * args.steps / e2e_ms, "unit": "decomps/s", "ms_per_step": e2e_ms / args.steps,
               "h2d_bytes_per_step": int(hY.numel() * 8 + hW.numel()), "d2h_bytes_per_step": int((hU.numel() + hV.numel()) * 8)},
          cpu_baseline={"value": 1.0 / t_oracle, "unit": "decomps/s", "cores": 1, "nproc": os.cpu_count(),
                        "kind": "oracle", "sample": "one whole decomposition"},
          gpu_launches=int(last.kernel_launches * args.steps), clocks=clk)
    h.close()


def bench_batched(args):
    """The batched uneven workload: 256 independent problems (m log-uniform in
    [4096, 65536], n in 64..512, r in 2..16, rho in [0.5, 0.9]) in one
    rsm_decompose_batch call (FP32 Y, the given Gram form, FP64 minor vectors, M,
    eigensolve and solves), against the plain per-problem FP64 form (each
    problem alone, FP64 Y, Gram and solves) on the same GPU."""
    import torch

    import oracle
    import paper_1411_0814_gb300 as rsm
    from workloads import batched_problem, batched_problem_specs

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    specs = batched_problem_specs(256)
    t0 = time.perf_counter()
    dev64, dev32, meta = [], [], []
    for i, sp in enumerate(specs):
        p = batched_problem(sp)
        Y64, W = _device_problem(p, torch.float64, dev)
        dev64.append((Y64, W))
        dev32.append(Y64.to(torch.float32))
        meta.append((p.r, p.l, p.trials, p.seed, p.m, p.n))
        del p
    t_gen = time.perf_counter() - t0
    h = rsm.RSM(0, stream=stream)
    mixed = [rsm.Problem(dev32[i], dev64[i][1], r, trials=t, l=l, seed=sd, problem_id=i, gram=args.batched_gram,
                         solve="f32") for i, (r, l, t, sd, m, n) in enumerate(meta)]
    plain = [rsm.Problem(dev64[i][0], dev64[i][1], r, trials=t, l=l, seed=sd, problem_id=i, gram="f64", solve="f64")
             for i, (r, l, t, sd, m, n) in enumerate(meta)]
    for _ in range(max(1, args.warmup)):
        resm = h.decompose_batch(mixed)
    import tempfile
    clocks = ClockSampler(os.path.join(tempfile.gettempdir(), f"rsm_clocks_{os.getpid()}.csv"))
    clocks.start()
    total, per, outs = _timed_calls(lambda: h.decompose_batch(mixed), args.steps, stream)
    clk = clocks.stop()
    resm = outs[-1]
    # plain per-problem FP64 form: each problem alone, one pass over all 256 (after one warm-up pass)
    for pr in plain[:8]:
        h.decompose(pr)
    t64, per64, res64 = _timed_calls(lambda: [h.decompose(pr) for pr in plain], 1, stream)
    alone_ms = []
    for pr in plain[:32]:  # per-problem latencies of the FP64 form
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        h.decompose(pr)
        s1.record(stream)
        torch.cuda.synchronize()
        alone_ms.append(s0.elapsed_time(s1))
    # accuracy on the problems whose oracle result is stored (tests/golden)
    angles, angles64 = {}, {}
    for i in (47, 80, 181, 201, 215):
        path = os.path.join(ROOT, "tests", "golden", f"oracle_batched_{i:03d}.npz")
        if os.path.exists(path):
            g = np.load(path)
            angles[i] = subspace_angle_np(mixed[i].V.cpu().numpy(), g["V"])
            angles64[i] = subspace_angle_np(plain[i].V.cpu().numpy(), g["V"])
    statuses = [r_.status for r_ in resm]
    n_ok = sum(1 for s_ in statuses if s_ in (0, 4))
    stage = {k: float(resm[0].stage_ms[k]) for k in STAGES}
    _line(args, "batched256", 256e3 * args.steps / total, "decomps/s", total / args.steps, "fp32+fp64",
          dict(problems=256, m_range=[4096, 65536], n_range=[64, 512], r_range=[2, 16], rho_range=[0.5, 0.9],
               trials="20 n per problem", form=f"one rsm_decompose_batch call: Y FP32, Gram {args.batched_gram}, "
                                                 "normal equations accumulated in FP32 (tensor cores) + one FP32 "
                                                 "refinement step; minor vectors, M, eigensolve and r x r solves FP64",
               l2="inputs larger than L2 (Y fp32 6.6 GB)"),
          latency_ms={"p50": pct(per, 50), "p99": pct(per, 99), "what": "whole batch of 256"},
          determined=n_ok, underdetermined=statuses.count(3),
          submatrices_per_s=sum(r_.accepted_trials for r_ in resm) * args.steps / (total * 1e-3),
          stage_ms=stage, angle_vs_oracle=angles, angle_vs_oracle_tol=1e-6,
          fp64_per_problem={"value": 256e3 / t64, "unit": "decomps/s", "ms_per_pass": t64,
                            "latency_ms_alone": {"p50": pct(alone_ms, 50), "p99": pct(alone_ms, 99),
                                                 "what": "first 32 problems, each alone"},
                            "angle_vs_oracle": angles64, "angle_vs_oracle_tol": 1e-10},
          speedup_vs_fp64_per_problem=(256e3 * args.steps / total) / (256e3 / t64),
          gpu_launches=int(resm[0].kernel_launches * args.steps), setup_s=t_gen, clocks=clk)
    h.close()


def bench_serving(args):
    """The serving stream: Poisson arrivals at 200 requests/s for --serve-seconds,
    each a problem of the batched uneven distribution (a pool of 32 resident
    problems) or, with probability 5%, the large request (m = 262144, n = 2048,
    r = 16, rho = 0.8).  FP32 inputs resident on the device; requests go through
    rsm_submit and are polled; latency = completion - arrival on the host clock.
    The same request list is then run through the plain per-problem FP64 form
    (each request alone, synchronously) for its throughput and latencies."""
    import torch

    import paper_1411_0814_gb300 as rsm
    from workloads import batched_problem, batched_problem_specs, config_problem, serving_arrivals

    dev = torch.device("cuda", 0)
    specs = batched_problem_specs(256)[:32]
    pool = []
    for i, sp in enumerate(specs):
        p = batched_problem(sp)
        Y64, W = _device_problem(p, torch.float64, dev)
        pool.append(dict(Y32=Y64.to(torch.float32), Y64=Y64, W=W, r=p.r, l=p.l, trials=p.trials, seed=p.seed, pid=i))
        del p
    pl = config_problem("serving_large_262144x2048")
    Y64, W = _device_problem(pl, torch.float64, dev)
    large = dict(Y32=Y64.to(torch.float32), Y64=None, W=W, r=pl.r, l=pl.l, trials=pl.trials, seed=pl.seed, pid=1000)
    del Y64, pl
    torch.cuda.synchronize()
    times, kinds = serving_arrivals(200.0, args.serve_seconds, 0.05, pool_small=32)

    def make(k, form):
        q = large if k < 0 else pool[k]
        if form == "mixed":
            return rsm.Problem(q["Y32"], q["W"], q["r"], trials=q["trials"], l=q["l"], seed=q["seed"],
                               problem_id=q["pid"], gram=args.batched_gram, solve="f32")
        return rsm.Problem(q["Y64"], q["W"], q["r"], trials=q["trials"], l=q["l"], seed=q["seed"],
                           problem_id=q["pid"], gram="f64", solve="f64")

    # each kind alone first (synchronous, the same form): stage times of the large request and of a small one
    ha = rsm.RSM(0)
    alone = {}
    for k in (-1, 0):
        for _ in range(2):
            r_ = ha.decompose(make(k, "mixed"))
        alone["large" if k < 0 else "small_0"] = {"ms": r_.stage_ms["total"], "stage_ms": r_.stage_ms,
                                                  "status": r_.status}
    ha.close()
    h = rsm.RSM(0, max_slots=4)
    for k in (-1, 0, 1):  # warm the slots' workspaces with both request kinds
        t = h.submit(make(k, "mixed"))
        h.wait(t, timeout_ns=120 * 10 ** 9)
        h.release(t)
    import tempfile
    clocks = ClockSampler(os.path.join(tempfile.gettempdir(), f"rsm_clocks_{os.getpid()}.csv"))
    clocks.start()
    pending = {}
    lat, lat_small, lat_large, queue_ms, run_ms = [], [], [], [], []
    statuses = []
    max_pending = 0
    start = time.perf_counter()
    i = 0
    n = len(times)
    while i < n or pending:
        now = time.perf_counter() - start
        if i < n and now >= times[i]:
            prob = make(int(kinds[i]), "mixed")
            t = h.submit(prob)
            pending[t] = (times[i], int(kinds[i]), prob)
            i += 1
            max_pending = max(max_pending, len(pending))
            continue
        done = []
        for t, (t_arr, kind, prob) in pending.items():
            res = h.poll(t)
            if res is not None:
                tl = (time.perf_counter() - start - t_arr) * 1e3
                lat.append(tl)
                (lat_large if kind < 0 else lat_small).append(tl)
                queue_ms.append(res.queue_ms)
                run_ms.append(res.run_ms)
                statuses.append(res.status)
                done.append(t)
        for t in done:
            h.release(t)
            del pending[t]
        if not done:
            wait = (times[i] - (time.perf_counter() - start)) if i < n else 2e-4
            time.sleep(min(max(wait, 0.0), 2e-4))
    wall = time.perf_counter() - start
    clk = clocks.stop()
    h.close()
    # the plain per-problem FP64 form over the same kinds of requests (each alone,
    # synchronous); the large request's FP64 form needs its FP64 Y, built here
    hs = rsm.RSM(0)
    small_kinds = [int(k) for k in kinds if k >= 0][:200]
    s_lat = []
    for k in small_kinds[:8]:
        hs.decompose(make(k, "fp64"))
    for k in small_kinds:
        t0 = time.perf_counter()
        hs.decompose(make(k, "fp64"))
        s_lat.append((time.perf_counter() - t0) * 1e3)
    pl = config_problem("serving_large_262144x2048")
    large["Y64"], _ = _device_problem(pl, torch.float64, dev)
    del pl
    l_lat = []
    for _ in range(3):
        t0 = time.perf_counter()
        hs.decompose(make(-1, "fp64"))
        l_lat.append((time.perf_counter() - t0) * 1e3)
    hs.close()
    frac_large = float(np.mean(kinds < 0))
    mean64 = (1 - frac_large) * statistics.mean(s_lat) + frac_large * statistics.mean(l_lat)
    mix64 = s_lat + l_lat * max(1, round(frac_large * len(s_lat) / max(1, len(l_lat))))
    _line(args, "serving", len(lat) / wall, "decomps/s", wall * 1e3 / max(1, len(lat)), "fp32+fp64",
          dict(rate_hz=200, seconds=args.serve_seconds, large_frac=0.05, pool_small=32,
               large=dict(m=262144, n=2048, r=16, rho=0.8, l=17, trials=40960), max_slots=4,
               form=f"rsm_submit / rsm_poll, continuous batching; Y FP32, Gram {args.batched_gram}, FP32 normal "
                    "equations, FP64 minor vectors, M, eigensolve, r x r solves"),
          requests=len(lat), arrivals=n, wall_s=wall,
          latency_ms={"p50": pct(lat, 50), "p99": pct(lat, 99), "small_p50": pct(lat_small, 50),
                      "small_p99": pct(lat_small, 99), "large_p50": pct(lat_large, 50), "large_p99": pct(lat_large, 99)},
          queue_ms={"mean": statistics.mean(queue_ms), "p99": pct(queue_ms, 99)},
          run_ms={"mean": statistics.mean(run_ms), "p99": pct(run_ms, 99)}, max_in_flight=max_pending, alone=alone,
          statuses={str(s_): statuses.count(s_) for s_ in sorted(set(statuses))},
          fp64_per_problem={"value": 1e3 / mean64, "unit": "decomps/s", "what": "each request alone, synchronous, "
                            "same request mix (200 small + 3 large)",
                            "latency_ms": {"p50": pct(mix64, 50), "p99": pct(mix64, 99),
                                           "small_p50": pct(s_lat, 50), "large_mean": statistics.mean(l_lat)}},
          clocks=clk)


# Table 1 of the paper (Section V-A): m, n, rho, sigma, printed time t (s) and error e (Matlab, FP64,
# one core of an i5-3470; context only)
TABLE1 = [(65536, 1024, 0.2, 0.2, 52.4, 0.1987), (98304, 1024, 0.2, 0.2, 64.3, 0.1986),
          (131072, 1024, 0.2, 0.2, 79.1, 0.1985), (131072, 768, 0.2, 0.2, 59.1, 0.1981),
          (131072, 512, 0.2, 0.2, 53.0, 0.1971), (131072, 1024, 0.5, 0.1, 84.2, 0.0997),
          (131072, 1024, 0.4, 0.1, 75.7, 0.0996), (131072, 1024, 0.3, 0.1, 59.1, 0.0995),
          (131072, 1024, 0.3, 0.3, 59.5, 0.2985), (131072, 1024, 0.3, 0.5, 60.4, 0.4976)]


def bench_fig1(args):
    """The scaling sweep of Figure 1 on the shapes of Table 1 (r = 3, M1 with
    l = 4, I = 20 n submatrices): time per decomposition against m and n on the
    GPU (FP64 form, as the paper's Matlab) and for the oracle on one host core
    (a bounded sample extrapolated), with the error e beside the paper's."""
    import torch

    import paper_1411_0814_gb300 as rsm
    from workloads import lowrank_problem

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    h = rsm.RSM(0, stream=stream)
    rows = []
    for (m, n, rho, sigma, t_paper, e_paper) in TABLE1:
        p = lowrank_problem(m, n, 3, rho, sigma, l=4, trials=20 * n, seed=0)
        Y, W = _device_problem(p, torch.float64, dev)
        prob = rsm.Problem(Y, W, 3, trials=p.trials, l=4, seed=0, gram="f64", solve="f64")
        for _ in range(2):
            h.decompose(prob)
        total, per, res = _timed_calls(lambda: h.decompose(prob), max(3, args.steps // 10), stream)
        k = len(per)
        t_gpu = total / k
        o = oracle_sample_problem(p, trial_sample=200, row_sample=2048)
        rows.append(dict(m=m, n=n, rho=rho, sigma=sigma, gpu_ms=t_gpu, gpu_decomps_per_s=1e3 / t_gpu,
                         e_gpu=res[-1].e, status=res[-1].status, accepted=res[-1].accepted_trials,
                         oracle_s_est=o["est_s_per_decomp"], oracle_sample=o["sample"],
                         paper_t_s=t_paper, paper_e=e_paper))
        print(json.dumps(rows[-1]), flush=True)
        del Y, W, prob, p
        torch.cuda.empty_cache()
    _line(args, "fig1_sweep", statistics.mean(r_["gpu_decomps_per_s"] for r_ in rows), "decomps/s",
          statistics.mean(r_["gpu_ms"] for r_ in rows), "f64",
          dict(shapes="Table 1 (Section V-A)", r=3, l=4, trials="20 n", form="FP64 throughout"), sweep=rows,
          note="paper times are Matlab FP64 on one core of an i5-3470 (context only)")
    h.close()


def oracle_sample_problem(p, trial_sample: int, row_sample: int) -> dict:
    """oracle_sample for a given problem, in this process (BLAS threads as configured)."""
    import oracle
    from oracle import rsm as orsm
    cols = orsm.sample_columns(p.n, p.l, trial_sample, p.seed)
    t0 = time.perf_counter()
    Zs = []
    for t in range(trial_sample):
        R = orsm.select_rows(p.W, cols[t])
        Zs.append(None if R.size < p.l else orsm.minor_vectors(np.asarray(p.Y[np.ix_(R, cols[t])]), p.l - p.r))
    M = orsm.accumulate_M(p.n, cols, Zs)
    t_trials = time.perf_counter() - t0
    t0 = time.perf_counter()
    V, _ = orsm.eig_smallest(M, p.r)
    t_eig = time.perf_counter() - t0
    t0 = time.perf_counter()
    U, _ = orsm.solve_U(p.Y[:row_sample], p.W[:row_sample], V)
    oracle.residual(p.Y[:row_sample], p.W[:row_sample], U, V)
    t_rows = time.perf_counter() - t0
    est = t_trials * p.trials / trial_sample + t_eig + t_rows * p.m / row_sample
    return dict(est_s_per_decomp=est, sample=f"{trial_sample} of {p.trials} submatrices + full eigensolve of M + "
                                               f"U and e on {row_sample} of {p.m} rows, extrapolated")


# ----------------------------------------------------------------- reference arm (the oracle)

def bench_reference(args):
    """The FP64 oracle as it stands, on every host core: each step is one whole
    decomposition of the workload (draws and rows split over processes, M
    reduced in draw order), about 3-5 s each on 16 cores."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    procs = len(os.sched_getaffinity(0))
    t_start = time.perf_counter()
    pool = OraclePool(WORKLOAD, procs)
    p = pool.p
    steps, warmup = args.steps, args.warmup
    secs = []
    try:
        for k in range(warmup + steps):
            o = pool.decompose()
            if k >= warmup:
                secs.append(o["seconds"])
    finally:
        pool.close()
    total = sum(secs)
    value = len(secs) / total
    sample = (f"whole decompositions (all {p.trials} draws, all {p.m} rows) on {procs} processes; "
              f"{len(secs)} timed after {warmup} untimed")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "decomps/s", "n_gpus": ws,
           "steps": len(secs), "warmup": warmup, "ms_per_step": total * 1e3 / len(secs), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "m": p.m, "n": p.n, "r": p.r, "rho": p.rho, "sigma": p.sigma, "l": p.l,
                      "trials": p.trials, "form": f"FP64 CPU oracle (numpy), {procs} host processes"},
           "cpu_baseline": {"value": value, "unit": "decomps/s", "cores": procs, "nproc": os.cpu_count(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "decomps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "e": o["e"],
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
    elif args.workload == WORKLOAD:
        bench_mine(args)
    else:
        {"noiseless_2048x128": bench_single, "trajectory_4096x144": bench_single, "batched256": bench_batched,
         "serving": bench_serving, "fig1_sweep": bench_fig1}[args.workload](args)


if __name__ == "__main__":
    main()
