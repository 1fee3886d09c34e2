"""Write the oracle's results on full-size workloads to tests/golden/oracle_<case>.npz.

The GPU parity tests compare the CUDA path at full size against these files,
because the FP64 oracle takes minutes per decomposition at these sizes.  This
script calls only ``oracle`` (and the input generators of ``workloads``); no
value in the files comes from the CUDA path.

Each file holds, for one workload: the sampler and size parameters (so a test
can check that the fixture matches the workload it builds), the oracle's
status and accepted-trial count, V-hat (n x r), the smallest eigenvalues of M,
the largest eigenvalue and the trace of M, the error e of eq. (ep), and U-hat on a seeded sample of rows (``row_idx``,
``U_rows``) for basis-free checks of U V^T on those rows.

Usage: python tests/golden/make_oracle_goldens.py [case ...]   (default: all)
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

# the batched uneven workload at its true sizes: a subset that spans its range
# (the largest r and n, m above 30000, one problem with too few rows per trial)
BATCHED_SUBSET = (47, 80, 140, 181, 201, 215)
ROW_SAMPLE = 512


def _cases():
    c = {"paper_131072x1024": ("config", "paper_131072x1024"),
         "serving_large_262144x2048": ("config", "serving_large_262144x2048")}
    for i in BATCHED_SUBSET:
        c[f"batched_{i:03d}"] = ("batched", i)
    return c


def _problem(kind, key):
    sys.path.insert(0, ROOT)
    from workloads import batched_problem, batched_problem_specs, config_problem
    if kind == "config":
        return config_problem(key), 0
    spec = batched_problem_specs(256)[key]
    return batched_problem(spec), key  # problem id = index in the batch


def run_case(name: str) -> str:
    sys.path.insert(0, ROOT)
    import oracle
    kind, key = _cases()[name]
    t0 = time.time()
    p, pid = _problem(kind, key)
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, problem_id=pid, variant=p.variant)
    out = dict(m=p.m, n=p.n, r=p.r, l=p.l, trials=p.trials, seed=p.seed, problem_id=pid, rho=p.rho, sigma=p.sigma,
               status=o.status, accepted_trials=o.accepted_trials, V=o.V, evals=o.evals[:min(p.n, p.r + 8)],
               lambda_max=float(o.evals[-1]), trace_M=float(np.trace(o.M)), e=o.e)
    if o.U is not None:
        rng = np.random.default_rng(20241)
        idx = np.sort(rng.choice(p.m, min(ROW_SAMPLE, p.m), replace=False))
        out.update(row_idx=idx, U_rows=o.U[idx])
    np.savez_compressed(os.path.join(HERE, f"oracle_{name}.npz"), **out)
    return f"{name}: status {o.status}, accepted {o.accepted_trials}, e {o.e:.6e}, {time.time() - t0:.0f} s"


def main(argv):
    names = argv or list(_cases())
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    with mp.get_context("spawn").Pool(min(len(names), os.cpu_count() or 1)) as pool:
        for line in pool.imap_unordered(run_case, names):
            print(line, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
