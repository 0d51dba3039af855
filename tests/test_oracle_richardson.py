"""Pins of the oracle's sequential fixed-stress strategy (§5.4 remark: the two-stage preconditioner inside a
Richardson iteration x <- x + M^{-1}(b - A x)).  Its error propagator is E = I - M^{-1} A:
  * M = A^{-1}: E = 0, one pass solves the system;
  * M the exact block-triangular factor of §5.1 (exact A_uu and exact Schur complement): M^{-1} A is unit
    upper block-triangular, E is strictly upper block-triangular, E^2 = 0, two passes solve the system;
  * with the inexact two-stage preconditioner the iteration still converges, in more passes than FGMRES."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def sys0():
    return oracle.System(oracle.default_params(0, nx=4, ny=3, nz=3))


def test_exact_inverse_one_pass(sys0):
    P = oracle.Prec(sys0, oracle.default_prec_params(full_exact=1))
    x, st = P.richardson(tol=1e-10)
    assert st.converged and st.iters == 1


def test_exact_block_factor_two_passes(sys0):
    pp = oracle.default_prec_params(mech_mode=oracle.MECH_EXACT, flow_mode=oracle.FLOW_EXACT_SCHUR)
    P = oracle.Prec(sys0, pp)
    x, st = P.richardson(tol=1e-10, max_iters=2)
    assert st.converged and st.iters == 2
    # one pass is not enough: the coupling block of E is not zero
    _, st1 = P.richardson(tol=1e-10, max_iters=1)
    assert not st1.converged and st1.true_relres > 1e-6
    xe = sys0.dense_solve(sys0.rhs)
    assert np.linalg.norm(x - xe) <= 1e-8 * np.linalg.norm(xe)


def test_two_stage_richardson_converges_slower_than_fgmres():
    s = oracle.System(oracle.default_params(1, nx=12, ny=10, nz=6))
    P = oracle.Prec(s)
    x, st = P.richardson(tol=1e-8, max_iters=2000)
    _, sf = P.fgmres(tol=1e-8)
    assert st.converged and np.linalg.norm(s.rhs - s.spmv(x)) <= 1e-8 * np.linalg.norm(s.rhs)
    assert st.iters > sf.iters
