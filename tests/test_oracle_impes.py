"""Pins of the oracle's true-IMPES reduction (§5.3: D_ss = diag(A_ss^T e), D_ps = diag(A_ps^T e), column-sum
lumping of the saturation derivatives).

Each TPFA face flux depends on the upstream saturation only, and enters the rows of its two cells with
opposite signs (conservation), so every flux term cancels in a column sum: the column sums of A_ss and A_ps
are the accumulation derivatives alone.  True-IMPES on the full Jacobian therefore gives the S_pp that
quasi-IMPES gives on the same Jacobian generated without the flux saturation derivatives (whose A_ss and
A_ps are diagonal, while A_sp and A_pp, and so the flow row scaling, are unchanged)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("cfg,kw", [(0, dict(nx=6, ny=5, nz=4)), (1, dict(nx=12, ny=10, nz=6)),
                                    (2, dict(nx=10, ny=20, nz=12))])
def test_true_impes_lumps_the_flux_saturation_derivatives(cfg, kw):
    full = oracle.System(oracle.default_params(cfg, **kw))
    nosat = oracle.System(oracle.default_params(cfg, flags=oracle.OR_ALL & ~oracle.OR_FLUX_SAT, **kw))
    assert full.alpha_f == nosat.alpha_f
    # the saturation derivatives do couple neighbours in the full Jacobian
    rp, ci, v = full.blocks["ff"]
    off = np.repeat(np.arange(len(rp) - 1), np.diff(rp)) != ci
    assert np.abs(v.reshape(-1, 4)[off, 0]).max() > 0
    sp_true = oracle.Prec(full, oracle.default_prec_params(cpr_reduction=oracle.CPR_TRUE_IMPES)).spp()[2]
    sp_q_nosat = oracle.Prec(nosat, oracle.default_prec_params(cpr_reduction=oracle.CPR_QUASI_IMPES)).spp()[2]
    sp_q_full = oracle.Prec(full, oracle.default_prec_params(cpr_reduction=oracle.CPR_QUASI_IMPES)).spp()[2]
    scale = np.abs(sp_true).max()
    assert np.abs(sp_true - sp_q_nosat).max() <= 1e-12 * scale
    assert np.abs(sp_true - sp_q_full).max() > 1e-6 * scale  # the two reductions differ on the full Jacobian


def test_true_and_quasi_impes_agree_without_face_coupling():
    flags = oracle.OR_ALL & ~oracle.OR_FLUX & ~oracle.OR_FLUX_SAT
    s = oracle.System(oracle.default_params(0, nx=5, ny=4, nz=3, flags=flags))
    a = oracle.Prec(s, oracle.default_prec_params(cpr_reduction=oracle.CPR_TRUE_IMPES))
    b = oracle.Prec(s, oracle.default_prec_params(cpr_reduction=oracle.CPR_QUASI_IMPES))
    assert np.array_equal(a.spp()[2], b.spp()[2])
    v = np.random.default_rng(1).standard_normal(s.n)
    assert np.array_equal(a.apply(v), b.apply(v))


def test_true_impes_fgmres_converges():
    s = oracle.System(oracle.default_params(1, nx=12, ny=10, nz=6))
    x, st = oracle.Prec(s, oracle.default_prec_params(cpr_reduction=oracle.CPR_TRUE_IMPES)).fgmres(tol=1e-8)
    assert st.converged and np.linalg.norm(s.rhs - s.spmv(x)) <= 1e-8 * np.linalg.norm(s.rhs)
