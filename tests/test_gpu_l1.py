"""The L1 forms of V-hat and U-hat on the device against the oracle's IRLS
(Section IV-A, eq. solve.barV_L1_norm and eq. solve.barU with the L1 norm;
oracle/robust.py): the same number of reweighting steps from the L2 solution,
the same delta_V and delta_U.

* Two grossly corrupted columns: the device's L1 V-hat must match the oracle's
  and, like it, recover the ground truth on the other columns while the L2
  form does not.  The reweighted M_w is less well conditioned than M (the
  smaller delta_V, the more so: its Davis-Kahan floor is ~2e-9 at 1e-4, ~1e-7
  at 1e-6), so the floor of the oracle's last M_w is asserted below 1e-8 and
  the FP64 form held to 10 times it, the FP32 form to 1e-6 plus that.
* U-hat: in the FP64 form U V^T on the known entries within 1e-8 relative of
  the oracle's L1 rows.  In the FP32 form (FP32 sums of the reweighted normal
  equations) the rows themselves are not a stable target: least-absolute-
  deviation solutions move a lot when a residual near delta changes its weight
  by orders of magnitude, so the form is held to the objective the rows
  minimise, sum |y - u . v| over the known entries: within 1e-5 relative of the
  oracle's, the FP32 forms' tolerance on U V^T (1e-6 in the FP64 form).
* Noiseless data: exact recovery.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import robust
from tests.gpu_helpers import known_relative_diff, to_device
from workloads import lowrank_problem

pytestmark = pytest.mark.gpu

import paper_1411_0814_gb300 as rsm  # noqa: E402

ITERS, DV, DU = 8, 1e-4, 1e-3


def _corrupted():
    p = lowrank_problem(2048, 64, 3, 0.8, 1e-3, trials=1280, seed=7)
    p.Y = np.asfortranarray(p.Y.copy())
    p.Y[:, [5, 40]] += 5 * np.random.default_rng(1).standard_normal((p.m, 2))
    return p, np.setdiff1d(np.arange(p.n), [5, 40])


def _oracle_l1(p):
    o = oracle.decompose(p.Y, p.W, p.r, p.l, p.trials, p.seed, solve_u=False)
    V1, ev, _ = robust.eig_smallest_l1(p.n, o.cols, o.Z, p.r, ITERS, DV, o.V)
    U1 = robust.solve_U_l1(p.Y, p.W, V1, ITERS, DU)
    return o, V1, ev, U1


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_l1_forms_match_oracle_on_corrupted_columns(form):
    p, good = _corrupted()
    o, V1, ev, U1 = _oracle_l1(p)
    floor = 100 * 2.0 ** -52 * ev[-1] / (ev[p.r] - ev[p.r - 1])
    assert floor <= 1e-8, floor
    dtype = torch.float64 if form == "fp64" else torch.float32
    Y, W = to_device(p, dtype)
    prec = "f64" if form == "fp64" else "f32"
    with rsm.RSM(0) as h:
        l1 = h.decompose(rsm.Problem(Y, W, p.r, trials=p.trials, seed=p.seed, gram=prec, solve=prec, norm="l1",
                                     irls_iters=ITERS, irls_delta_v=DV, irls_delta_u=DU))
        l2 = h.decompose(rsm.Problem(Y, W, p.r, trials=p.trials, seed=p.seed, gram=prec, solve=prec))
    Vg, Ug = l1.V.cpu().numpy(), l1.U.cpu().numpy()
    ang = oracle.subspace_angle(Vg, V1)
    truth1 = oracle.subspace_angle(Vg[good], p.V_bar[good])
    truth2 = oracle.subspace_angle(l2.V.cpu().numpy()[good], p.V_bar[good])
    Yref = p.Y if form == "fp64" else np.asarray(p.Y, dtype=np.float32).astype(np.float64)
    rel = known_relative_diff(Ug, Vg, U1, V1, p.W, Yref)
    print(f"{form}: angle to oracle L1 {ang:.2e}, to truth L1 {truth1:.2e} L2 {truth2:.2e}, rows {rel:.2e}, "
          f"e {l1.e:.6e}")
    assert l1.status == 0
    assert ang <= 10 * floor + (0.0 if form == "fp64" else 1e-6)
    assert truth1 < 1e-3 and truth2 > 0.05
    f_g = robust.l1_objective_U(Yref, p.W, Ug, Vg)
    f_o = robust.l1_objective_U(Yref, p.W, U1, V1)
    print(f"{form}: L1 objective device {f_g:.9e} oracle {f_o:.9e}")
    if form == "fp64":
        assert rel <= 1e-8
    # FP32 form: least absolute deviations move with the FP32 rounding of the data, so the
    # objective is held to the FP32 forms' tolerance on U V^T (1e-5 relative)
    assert abs(f_g - f_o) <= (1e-6 if form == "fp64" else 1e-5) * f_o


def test_l1_forms_noiseless_exact():
    p = lowrank_problem(2048, 64, 3, 0.8, 0.0, trials=1280, seed=3)
    Y, W = to_device(p)
    with rsm.RSM(0) as h:
        res = h.decompose(rsm.Problem(Y, W, p.r, trials=p.trials, seed=p.seed, norm="l1", irls_iters=4))
    assert res.status == 0
    assert oracle.subspace_angle(res.V.cpu().numpy(), p.V_bar) <= 1e-10
    w = p.W != 0
    fit = res.U.cpu().numpy() @ res.V.cpu().numpy().T
    assert np.max(np.abs((fit - p.Y)[w])) <= 1e-9 * np.max(np.abs(p.Y))
