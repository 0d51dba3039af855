"""Pins of the oracle's row-sum-lumped fixed-stress diagonal (the §5.1 remark on the algebraic fixed
stress: D_sp = -diag(A_su A_uu^{-1} A_up e), D_pp = -diag(A_pu A_uu^{-1} A_up e)).

Probing with the constant pressure vector: with the exact A_uu^{-1}, the lumped S_ff reproduces the
exact Schur complement S = A_ff - A_fu A_uu^{-1} A_uf (Eq. (LU) of §5.1) on that vector, row by row:
(A_ff + D) e_p = S e_p, with e_p = 1 on every pressure unknown and 0 on every saturation.  The Schur
complement is formed densely by a library solve on a tiny grid."""
import numpy as np
import pytest

import oracle


def dense_blocks(s):
    A = s.dense()
    nu = s.n_u
    return A[:nu, :nu], A[:nu, nu:], A[nu:, :nu], A[nu:, nu:]


@pytest.mark.parametrize("cfg,kw", [(0, dict(nx=4, ny=3, nz=3)), (1, dict(nx=5, ny=4, nz=3))])
def test_exact_rsl_reproduces_the_schur_complement_on_constant_pressure(cfg, kw):
    s = oracle.System(oracle.default_params(cfg, **kw))
    P = oracle.Prec(s, oracle.default_prec_params(fs_mode=oracle.FS_RSL_EXACT))
    D = P.fs_diag().reshape(-1, 2)
    Auu, Auf, Afu, Aff = dense_blocks(s)
    S = Aff - Afu @ np.linalg.solve(Auu, Auf)
    ep = np.zeros(2 * s.n_cells)
    ep[1::2] = 1.0
    lhs = (Aff @ ep).reshape(-1, 2) + D
    rhs = (S @ ep).reshape(-1, 2)
    assert np.allclose(lhs, rhs, rtol=1e-9, atol=1e-12 * np.abs(rhs).max())
    # the lumped diagonal is not the generator's K_dr-based one (the two approximations differ)
    assert not np.allclose(D.ravel(), s.d_fs, rtol=1e-3)


def test_rsl_with_the_mechanics_vcycle_converges():
    s = oracle.System(oracle.default_params(1, nx=12, ny=10, nz=6))
    P = oracle.Prec(s, oracle.default_prec_params(fs_mode=oracle.FS_RSL))
    D = P.fs_diag().reshape(-1, 2)
    assert np.all(np.isfinite(D))
    x, st = P.fgmres(tol=1e-8)
    assert st.converged and np.linalg.norm(s.rhs - s.spmv(x)) <= 1e-8 * np.linalg.norm(s.rhs)
