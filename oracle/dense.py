"""Eq. 4 for a fully connected leftover block (the SK workload): plain sum over
all 2^|R| leftover states per sample, FP64.  Test infrastructure only.

  log Z_R(s) = -beta E_1(s) + ln sum_r exp(-beta E_2(s, r)),
  -beta E_2(s, r) = beta [ sum_{i<j in R} J_ij r_i r_j + sum_{i in R, k in W} J_ik r_i s_k ].
"""
import numpy as np
import torch

from .ising import DT, all_configs, w_energy_term


def coupling_matrix(n, ei, ej, J) -> torch.Tensor:
    """Symmetric n x n matrix with the bond couplings, zero diagonal."""
    J = torch.as_tensor(J, dtype=DT) if not torch.is_tensor(J) else J
    M = torch.zeros(n, n, dtype=DT)
    M = M.index_put((torch.as_tensor(np.asarray(ei), dtype=torch.int64),
                     torch.as_tensor(np.asarray(ej), dtype=torch.int64)), J, accumulate=True)
    return M + M.T


def log_zr_dense(n, ei, ej, J, beta, W, sW: torch.Tensor, chunk: int = 64, field=None) -> torch.Tensor:
    """Plain 2^|R| sum for each row of sW [B, |W|] (|R| <= 20).  `field`
    ([B] or a scalar): a uniform field on R, added to every R spin's field."""
    W = np.asarray(W, np.int64)
    R = np.setdiff1d(np.arange(n), W)
    M = coupling_matrix(n, ei, ej, J)
    Wt, Rt = torch.as_tensor(W), torch.as_tensor(R)
    J_RR = M[Rt][:, Rt]
    J_RW = M[Rt][:, Wt]
    rc = all_configs(len(R))  # [S, |R|]
    e_rr = 0.5 * ((rc @ J_RR) * rc).sum(1)  # sum_{i<j} J_ij r_i r_j
    sW = sW.to(DT)
    out = []
    for start in range(0, sW.shape[0], chunk):
        h = sW[start:start + chunk] @ J_RW.T  # [b, |R|] fields from W
        if field is not None:
            h = h + (field[start:start + chunk][:, None] if torch.is_tensor(field) and field.dim() > 0 else field)
        expo = beta * (e_rr[None, :] + h @ rc.T)  # [b, S]
        out.append(torch.logsumexp(expo, dim=1))
    return w_energy_term(ei, ej, J, beta, W, sW) + torch.cat(out)
