"""Helpers shared by the GPU parity tests: run the CUDA path through the
C-ABI binding, run the FP64 oracle on the same inputs, compare."""
from __future__ import annotations

import numpy as np

from oracle import rqlp_oracle as orc

# Tolerances, FP32 or BF16x3 path vs the FP64 oracle: leading-k |L_ii|
# relative 1e-4 (the target; both arithmetic forms meet it without widening),
# ||Q^T Q - I||_F <= 1e-5 (CholeskyQR2 in FP32 leaves ~1e-6), relative residual
# within 1e-3 (relative) of the oracle's or within RES_FLOOR of it when the
# residual is at the pass arithmetic's rounding level. Entries of the leading
# k columns of Q, P and of L's leading block differ by <= elem_atol (default
# 2e-4): an entry error of qf(X) is about kappa(X(:, 1:k)) times the unit
# roundoff of the passes (6e-8 in FP32, ~2^-16 with two BF16 parts), and
# kappa <= ~1e2 on the leading blocks of these workloads.
TOL_LII = 1e-4
TOL_ORTH = 1e-5
TOL_RES = 1e-3


def run_gpu(A, Om, k, p, q, precision=0, small_fp64=False, parts=0, literal=False, fused=False):
    import torch

    from paper_2110_01011_gb300 import rqlp
    dA = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda()
    dO = torch.from_numpy(np.ascontiguousarray(Om, dtype=np.float32)).cuda()
    Q, L, P, info, diag = rqlp.factor(dA, k, p, q, dO, precision=precision, small_fp64=small_fp64, parts=parts,
                                      literal=literal, fused=fused)
    torch.cuda.synchronize()
    return (Q.double().cpu().numpy(), L.double().cpu().numpy(), P.double().cpu().numpy(),
            info.cpu().numpy(), diag.cpu().numpy())


def relres(A, Q, L, P):
    A = np.asarray(A, dtype=np.float64)
    return np.linalg.norm(A - (Q @ L) @ P.T) / np.linalg.norm(A)


# Absolute floor for the relative residual when the oracle's is at rounding
# level (rank(A) <= d): a few units of the pass arithmetic's roundoff
# (FP32 6e-8; BF16x3 keeps ~16 bits per operand, ~1.5e-5).
RES_FLOOR = {0: 1e-6, 1: 2e-5}


def compare(A, Om, k, p, q, gpu, elem_atol=2e-4, precision=0, literal=False):
    """Compare GPU factors with the oracle; returns a dict of measured errors
    and asserts the tolerances. literal: the oracle runs step 5 as
    Algorithm 1 prints it."""
    Qg, Lg, Pg, info, diag = gpu
    A64 = np.asarray(A, dtype=np.float64)
    chain = orc.rand_qlp_literal if literal else orc.rand_qlp
    ref = chain(A64, np.asarray(Om, dtype=np.float64), q)
    d = k + p
    assert info[0] == 0, f"info={info}"
    err = {}
    err["orthQ"] = np.linalg.norm(Qg.T @ Qg - np.eye(d))
    err["orthP"] = np.linalg.norm(Pg.T @ Pg - np.eye(d))
    err["Lii_rel"] = np.max(np.abs(np.diag(Lg)[:k] - np.diag(ref.L)[:k]) / np.abs(np.diag(ref.L)[:k]))
    rg, ro = relres(A64, Qg, Lg, Pg), relres(A64, ref.Q, ref.L, ref.P)
    err["res_gpu"], err["res_oracle"] = rg, ro
    err["res_rel"] = abs(rg - ro) / ro if ro > 0 else abs(rg)
    err["Q_lead"] = np.max(np.abs(Qg[:, :k] - ref.Q[:, :k]))
    err["P_lead"] = np.max(np.abs(Pg[:, :k] - ref.P[:, :k]))
    err["L_lead"] = np.max(np.abs(Lg[:k, :k] - ref.L[:k, :k])) / np.abs(ref.L).max()
    err["L_upper_zero"] = float(np.abs(np.triu(Lg, 1)).max()) if d > 1 else 0.0
    nA2 = np.linalg.norm(A64) ** 2
    nL2 = float((Lg * Lg).sum())
    err["diag_A2_rel"] = abs(diag[0] - nA2) / nA2
    # d_diag = [||A||^2, ||L||^2, ||A||^2 - ||L||^2, shifted Choleskys]
    err["diag_L2_rel"] = abs(diag[1] - nL2) / nL2
    err["diag_res2"] = abs(diag[2] - (diag[0] - diag[1])) / nA2
    assert err["L_upper_zero"] == 0.0
    assert (np.diag(Lg) > 0).all()
    assert err["orthQ"] <= TOL_ORTH, err
    assert err["orthP"] <= TOL_ORTH, err
    assert err["Lii_rel"] <= TOL_LII, err
    assert err["res_rel"] <= TOL_RES or abs(rg - ro) <= RES_FLOOR[precision], err
    assert err["Q_lead"] <= elem_atol and err["P_lead"] <= elem_atol, err
    assert err["L_lead"] <= elem_atol, err
    assert err["diag_A2_rel"] <= 1e-6, err
    assert err["diag_L2_rel"] <= 1e-6 and err["diag_res2"] <= 1e-12, err
    assert diag[3] == np.round(diag[3]) and diag[3] >= 0, err
    return err
