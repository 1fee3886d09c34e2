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
