"""Shared helpers of the GPU tests: move a workload to the device, run the
library, and compare against the oracle."""
import numpy as np
import torch

import oracle


def to_device(prob, dtype=torch.float64):
    """Column-major device copies of Y and W of a workloads.Problem."""
    Y = torch.from_numpy(np.ascontiguousarray(prob.Y.T)).to("cuda", dtype=dtype).t()  # (m, n), stride (1, m)
    W = torch.from_numpy(np.ascontiguousarray(prob.W.T)).to("cuda").t()
    return Y, W


def projector_distance(A, B):
    """|| A A^T - B B^T ||_F for matrices with orthonormal columns."""
    return float(np.linalg.norm(A @ A.T - B @ B.T))


def minor_bound(Asub, nm, eps):
    """Rounding bound of the Gram-based minor subspace of Asub (p x l) relative to its SVD.

    The Gram's entries carry absolute errors of order sqrt(p) eps sigma_1^2; the
    minor subspace moves by that over the eigen-gap sigma_{l-nm}^2 - sigma_{l-nm+1}^2.
    """
    s = np.linalg.svd(Asub, compute_uv=False)
    p, l = Asub.shape
    gap = s[l - nm - 1] ** 2 - s[l - nm] ** 2
    return 16.0 * np.sqrt(p) * eps * s[0] ** 2 / max(gap, 1e-300) + 1e-13


def known_relative_diff(U1, V1, U2, V2, W, Y):
    """|| W o (U1 V1^T - U2 V2^T) ||_F / || W o Y ||_F, chunked over rows."""
    num = 0.0
    den = 0.0
    m = W.shape[0]
    for i0 in range(0, m, 8192):
        i1 = min(m, i0 + 8192)
        w = W[i0:i1].astype(np.float64)
        d = (U1[i0:i1] @ V1.T - U2[i0:i1] @ V2.T) * w
        num += float(np.sum(d * d))
        den += float(np.sum((np.asarray(Y[i0:i1], dtype=np.float64) * w) ** 2))
    return float(np.sqrt(num / den))


def check_near_degenerate(res, o, p, floor_max=1e-6):
    """Parity for a problem whose M is near-degenerate at the rank gap.

    When the Davis-Kahan floor f = 100 u lambda_max / (lambda_{r+1} - lambda_r)
    of FP64 eigenvectors is far above 1e-10, no FP64 solver defines V-hat to
    1e-10, so the test asserts instead, against the oracle:
      * f itself is at most floor_max (the problem is not arbitrarily degenerate);
      * status, accepted trials bit for bit, and M to 1e-12 relative;
      * V-hat is an invariant subspace of the oracle's M to FP64 working accuracy
        (backward error ||M_o V_g - V_g (V_g^T M_o V_g)|| <= 1e-12 lambda_max)
        with orthonormal columns;
      * the subspace angle to the oracle's V-hat is at most 10 f, and U V^T on the
        known entries agrees to 10 f relative.
    """
    import numpy as np
    import oracle
    ev = o.evals
    f = 100 * 2.0 ** -52 * max(abs(ev[-1]), 1.0) / max(ev[p.r] - ev[p.r - 1], 1e-300)
    assert f <= floor_max, f
    assert res.status == o.status and res.accepted_trials == o.accepted_trials
    if res.M is not None:
        Mg = res.M.detach().cpu().numpy()
        assert np.linalg.norm(Mg - o.M) <= 1e-12 * np.linalg.norm(o.M)
    Vg = res.V.detach().cpu().numpy()
    assert np.allclose(Vg.T @ Vg, np.eye(p.r), atol=1e-12)
    MV = o.M @ Vg
    back = np.linalg.norm(MV - Vg @ (Vg.T @ MV), ord=2)
    ang = oracle.subspace_angle(Vg, o.V)
    rel = known_relative_diff(res.U.detach().cpu().numpy(), Vg, o.U, o.V, p.W, p.Y)
    print(f"near-degenerate M: floor {f:.2e} backward {back / ev[-1]:.2e} angle {ang:.2e} recon {rel:.2e}")
    assert back <= 1e-12 * ev[-1]
    assert ang <= 10 * f
    assert rel <= 10 * f
