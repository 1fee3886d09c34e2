"""Run decompositions of one named synthetic workload, for profilers.

    python -m paper_1411_0814_gb300.profile_case --workload paper_131072x1024 --form mixed --repeat 2

Builds the workload on the host (seeded), copies Y and W to the device once,
and runs `repeat` decompositions back to back through the C ABI, then prints
one line with the status and the stage times of the last one.  Forms: "mixed"
(Y, Gram and normal equations in FP32; minor vectors, M, eigensolve and r x r
solves in FP64), "f32x2" (FP64 Y, Gram in FP32 pairs), "fp64" (everything FP64).
"""
import argparse
import json

import numpy as np
import torch

from . import rsm


def main():
    from workloads import CONFIGS, config_problem

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="paper_131072x1024", choices=sorted(CONFIGS))
    ap.add_argument("--form", default="mixed", choices=["mixed", "f32x2", "fp64"])
    ap.add_argument("--repeat", type=int, default=2)
    a = ap.parse_args()
    p = config_problem(a.workload)
    dtype = torch.float32 if a.form == "mixed" else torch.float64
    Y = torch.from_numpy(np.ascontiguousarray(p.Y.T)).to("cuda", dtype=dtype).t()
    W = torch.from_numpy(np.ascontiguousarray(p.W.T)).to("cuda").t()
    gram, solve = {"mixed": ("f32", "f32"), "f32x2": ("f32x2", "f64"), "fp64": ("f64", "f64")}[a.form]
    prob = rsm.Problem(Y, W, p.r, trials=p.trials, l=p.l, seed=p.seed, variant=p.variant, gram=gram, solve=solve)
    with rsm.RSM(0) as h:
        for _ in range(a.repeat):
            res = h.decompose(prob)
    print(json.dumps({"workload": a.workload, "form": a.form, "status": res.status,
                      "accepted_trials": res.accepted_trials, "stage_ms": res.stage_ms}))


if __name__ == "__main__":
    main()
