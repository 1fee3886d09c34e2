"""Seeded generators for the RSM workloads.

Paper workload (Section V-A, eq. construct.Y): the ground truth is a product of
two standard-normal factors, the noise is sigma times a standard-normal matrix,
and an entry is known when a standard uniform draw falls below rho.  The mask
test is taken as ``u < rho`` on [0, 1), the half-open form of the paper's
``rand(m, n) <= rho`` on (0, 1); the two differ only on a set of measure zero.

Storage: every matrix is column-major m x n (a Fortran-ordered numpy array), the
layout the CUDA path reads; ``W`` is uint8 with values 0/1.

Nothing here samples columns, selects rows or solves anything: the module only
draws inputs, so the oracle and the CUDA path can share it.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """One low-rank-with-missing-entries instance (Section II notation)."""

    Y: np.ndarray  # m x n, Fortran order, float64 or float32
    W: np.ndarray  # m x n, Fortran order, uint8 (1 = known, eq. problem)
    r: int  # target rank
    l: int  # columns per submatrix (M1), usually r + 1
    trials: int  # number of submatrix draws (I in Section IV-A step 1)
    seed: int  # key of the column sampler
    variant: str = "random"  # "random" (M1) or "adjacent" (contiguous columns)
    sigma: float = 0.0  # noise level used to build Y
    rho: float = 1.0  # Bernoulli density used to build W
    U_bar: Optional[np.ndarray] = None  # ground-truth left factor (m x r)
    V_bar: Optional[np.ndarray] = None  # ground-truth right factor (n x r)
    name: str = ""

    @property
    def m(self) -> int:
        return self.Y.shape[0]

    @property
    def n(self) -> int:
        return self.Y.shape[1]


def _streams(seed: int, k: int):
    return [np.random.Generator(np.random.PCG64(s)) for s in np.random.SeedSequence(seed).spawn(k)]


def lowrank_problem(m: int, n: int, r: int, rho: float, sigma: float, *, l: Optional[int] = None,
                    trials: Optional[int] = None, seed: int = 0, dtype=np.float64,
                    variant: str = "random", chunk_cols: int = 64, name: str = "") -> Problem:
    """Eq. (construct.Y): Y = randn(m,r) randn(r,n) + sigma randn(m,n), W = rand(m,n) < rho.

    Columns are generated in chunks so that the peak host memory stays near the
    size of Y itself.
    """
    g_fac, g_noise, g_mask = _streams(seed, 3)
    U = g_fac.standard_normal((m, r))
    V = g_fac.standard_normal((n, r))  # Y_bar = U V^T, so V^T is randn(r, n)
    Yt = np.empty((n, m), dtype=dtype)  # row j of Yt is column j of Y
    Wt = np.empty((n, m), dtype=np.uint8)
    for j0 in range(0, n, chunk_cols):
        j1 = min(n, j0 + chunk_cols)
        blk = V[j0:j1] @ U.T
        if sigma != 0.0:
            blk += sigma * g_noise.standard_normal((j1 - j0, m))
        Yt[j0:j1] = blk
        Wt[j0:j1] = g_mask.random((j1 - j0, m)) < rho
    l = r + 1 if l is None else l
    trials = 20 * n if trials is None else trials
    return Problem(Y=Yt.T, W=Wt.T, r=r, l=l, trials=trials, seed=seed, variant=variant,
                   sigma=sigma, rho=rho, U_bar=U, V_bar=V, name=name)


def trajectory_problem(m: int = 4096, views: int = 72, rank: int = 4, sigma: float = 0.5,
                       min_views: int = 4, max_views: int = 20, l: int = 5,
                       trials: Optional[int] = None, seed: int = 0, name: str = "") -> Problem:
    """Structured-mask stand-in for the paper's turntable sequences (Section V-B).

    Points are [X Y Z 1] with X, Y, Z uniform; a random projection of rank 4
    maps them to 2 coordinates per view; every column is then rescaled
    affinely to [0, 500] (the constant column keeps the rank at 4); Gaussian
    noise of the given sigma is added.  Each point is visible over one
    contiguous window of whole views: length uniform in [min_views, max_views],
    start uniform over the positions that keep the window inside the sequence.
    """
    g_pts, g_proj, g_noise, g_win = _streams(seed, 4)
    n = 2 * views
    P = np.concatenate([g_pts.random((m, rank - 1)), np.ones((m, 1))], axis=1)
    Vp = g_proj.standard_normal((n, rank))
    Ybar = P @ Vp.T
    lo, hi = Ybar.min(axis=0), Ybar.max(axis=0)
    scale = 500.0 / (hi - lo)
    Ybar = (Ybar - lo) * scale
    # the affine map keeps the rank: column j becomes P (scale_j Vp_j) - lo_j scale_j * 1
    Vbar = Vp * scale[:, None]
    Vbar[:, rank - 1] -= lo * scale
    Y = Ybar + sigma * g_noise.standard_normal((m, n))
    length = g_win.integers(min_views, max_views + 1, size=m)
    start = np.floor(g_win.random(m) * (views - length + 1)).astype(np.int64)
    view_idx = np.arange(views)[None, :]
    vis = (view_idx >= start[:, None]) & (view_idx < (start + length)[:, None])
    W = np.repeat(vis, 2, axis=1).astype(np.uint8)
    trials = 20 * n if trials is None else trials
    return Problem(Y=np.asfortranarray(Y), W=np.asfortranarray(W), r=rank, l=l, trials=trials,
                   seed=seed, variant="adjacent", sigma=sigma, rho=float(W.mean()),
                   U_bar=P, V_bar=Vbar, name=name)


def batched_problem_specs(count: int = 256, seed: int = 0, m_range=(4096, 65536), n_range=(64, 512),
                          r_range=(2, 16), rho_range=(0.5, 0.9), sigma: float = 1e-4):
    """Size distribution of the batched uneven workload: one dict per problem."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed).spawn(1)[0]))
    out = []
    for i in range(count):
        m = int(round(math.exp(g.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        n = int(g.integers(n_range[0], n_range[1] + 1))
        r = int(g.integers(r_range[0], r_range[1] + 1))
        rho = float(g.uniform(rho_range[0], rho_range[1]))
        out.append(dict(m=m, n=n, r=r, rho=rho, sigma=sigma, l=r + 1, trials=20 * n, seed=i))
    return out


def serving_arrivals(rate_hz: float = 200.0, duration_s: float = 60.0, large_frac: float = 0.05,
                     pool_small: int = 32, seed: int = 0):
    """Poisson arrival times and request kinds for the serving stream.

    Returns (times_s, kinds) where kind >= 0 indexes a small problem of the
    batched distribution and kind == -1 marks a large request.
    """
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed + 7919).spawn(1)[0]))
    gaps = g.exponential(1.0 / rate_hz, size=int(rate_hz * duration_s * 2) + 16)
    times = np.cumsum(gaps)
    times = times[times < duration_s]
    large = g.random(times.size) < large_frac
    kinds = np.where(large, -1, g.integers(0, pool_small, size=times.size))
    return times, kinds


LARGE_SERVING = dict(m=262144, n=2048, r=16, rho=0.8, sigma=1e-4, l=17, trials=20 * 2048)


def batched_problem(spec: dict, dtype=np.float64) -> Problem:
    """One problem of the batched uneven workload from its spec (batched_problem_specs)."""
    return lowrank_problem(spec["m"], spec["n"], spec["r"], spec["rho"], spec["sigma"], l=spec["l"],
                           trials=spec["trials"], seed=spec["seed"], dtype=dtype)

CONFIGS = {
    "noiseless_2048x128": dict(m=2048, n=128, r=4, rho=0.8, sigma=0.0, l=5, trials=2000, seed=0),
    "paper_131072x1024": dict(m=131072, n=1024, r=8, rho=0.7, sigma=1e-3, l=9, trials=20000, seed=0),
    "trajectory_4096x144": dict(kind="trajectory", m=4096, views=72, rank=4, sigma=0.5, l=5, trials=2880, seed=0),
    "serving_large_262144x2048": dict(LARGE_SERVING, seed=0),
}


def config_problem(name: str, dtype=np.float64, **over) -> Problem:
    """Build one of the named single-problem workloads (optionally overriding fields)."""
    spec = dict(CONFIGS[name])
    spec.update(over)
    if spec.pop("kind", None) == "trajectory":
        return trajectory_problem(name=name, **spec)
    return lowrank_problem(spec.pop("m"), spec.pop("n"), spec.pop("r"), spec.pop("rho"), spec.pop("sigma"),
                           dtype=dtype, name=name, **spec)
