"""Pins of the oracle's rigid-body-mode smoothed aggregation (MECH_AMG_RBM: AMG on the full A_uu with the six
rigid-body modes as near-nullspace, the usual alternative to the separate-displacement-component
approximation of §5.2):

  * the oracle's modes annihilate the pure-Neumann elasticity block (so they are rigid-body modes, with the
    right rotation signs);
  * per aggregate the tentative prolongator has orthonormal columns and reproduces the modes, P_tent B_c = B
    on the aggregated nodes (the six modes lie in the range of P_tent);
  * on a pure-Neumann block, where A B = 0, the smoothed prolongator reproduces the modes too, P B_c = B, and
    every Galerkin operator annihilates its level's coarse modes, A_c B_c = 0;
  * with the coarsest level at the finest (coarse_max above the node count) the V-cycle is the exact solve;
  * the V-cycle contracts the error on the Dirichlet-constrained block, and FGMRES with it converges."""
import numpy as np
import pytest

import oracle
from oracle import OR_ALL, OR_DIRICHLET, OR_GRAVITY
from tests.test_oracle_generator import _uu_dense


def rbm_prec(s, **kw):
    return oracle.Prec(s, oracle.default_prec_params(mech_mode=oracle.MECH_AMG_RBM, **kw))


def neumann(cfg=1, **kw):
    return oracle.System(oracle.default_params(cfg, flags=OR_ALL & ~(OR_GRAVITY | OR_DIRICHLET), **kw))


def bsr_dense(rp, ci, v, ncols):
    n, br, bc = len(rp) - 1, v.shape[1], v.shape[2]
    D = np.zeros((n * br, ncols * bc))
    for i in range(n):
        for q in range(rp[i], rp[i + 1]):
            D[i * br:(i + 1) * br, ci[q] * bc:(ci[q] + 1) * bc] = v[q]
    return D


def test_modes_annihilate_the_pure_neumann_block():
    s = neumann(0)
    B = oracle.rigid_body_modes(s.nx, s.ny, s.nz)
    A = _uu_dense(s)
    assert np.abs(A @ B).max() <= 1e-11 * np.abs(A).sum(1).max() * np.abs(B).max()
    assert np.linalg.matrix_rank(B) == 6


@pytest.mark.parametrize("cfg,kw", [(0, dict(nx=6, ny=5, nz=4)), (1, dict(nx=10, ny=8, nz=6))])
def test_tentative_prolongator_reproduces_the_modes(cfg, kw):
    s = oracle.System(oracle.default_params(cfg, **kw))
    P = rbm_prec(s, coarse_max_u=20)
    assert P.rbm_nlevels() >= 2
    for l in range(P.rbm_nlevels() - 1):
        sh, shc = P.rbm_shape(l), P.rbm_shape(l + 1)
        agg, B, Pt, _ = P.rbm_data(l)
        _, Bc, _, _ = P.rbm_data(l + 1)
        b = sh["b"]
        assert shc["n"] == sh["nagg"] and shc["b"] == 6
        on = np.repeat(agg >= 0, b)
        for a in range(sh["nagg"]):
            rows = np.repeat(agg == a, b)
            Q = Pt[rows]
            G = Q.T @ Q
            keep = np.abs(np.diag(G)) > 0.5
            assert keep.sum() >= 3
            assert np.abs(G - np.diag(keep.astype(float))).max() <= 1e-12
            assert np.abs(Q @ Bc[6 * a:6 * a + 6] - B[rows]).max() <= 1e-12 * max(1.0, np.abs(B[rows]).max())
        assert np.all(Pt[~on] == 0.0)


@pytest.mark.parametrize("cfg,kw", [(0, dict(nx=6, ny=5, nz=4)), (1, dict(nx=9, ny=8, nz=6))])
def test_smoothed_prolongator_and_galerkin_keep_the_modes(cfg, kw):
    s = neumann(cfg, **kw)
    P = rbm_prec(s, coarse_max_u=4)
    nl = P.rbm_nlevels()
    assert nl >= 3, [P.rbm_shape(l) for l in range(nl)]
    for l in range(nl - 1):
        sh = P.rbm_shape(l)
        agg, B, _, _ = P.rbm_data(l)
        _, Bc, _, _ = P.rbm_data(l + 1)
        rp, ci, v = P.rbm_prolongator(l)
        Pd = bsr_dense(rp, ci, v, sh["nagg"])
        Bn = np.abs(B).max()
        assert np.abs(Pd @ Bc - B).max() <= 1e-9 * Bn, l
        rp, ci, v = P.rbm_level(l)
        A = bsr_dense(rp, ci, v, len(rp) - 1)
        rp, ci, v = P.rbm_level(l + 1)
        Ac = bsr_dense(rp, ci, v, len(rp) - 1)
        # scale of the Galerkin products' terms (A_c itself is all rounding where one aggregate is left)
        scale = (np.abs(Pd).T @ np.abs(A) @ np.abs(Pd)).max()
        assert np.abs(Ac - Ac.T).max() <= 1e-13 * scale
        assert np.abs(Ac @ Bc).max() <= 1e-11 * scale * np.abs(Bc).sum(1).max(), l


def test_single_level_vcycle_is_the_exact_solve():
    s = oracle.System(oracle.default_params(0, nx=4, ny=3, nz=3))
    P = rbm_prec(s, coarse_max_u=10 ** 6)
    assert P.rbm_nlevels() == 1
    A = _uu_dense(s)
    b = np.random.default_rng(2).standard_normal(3 * s.n_nodes)
    x = P.rbm_vcycle(b)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)


def test_vcycle_contracts_and_fgmres_converges():
    s = oracle.System(oracle.default_params(1, nx=12, ny=10, nz=6))
    P = rbm_prec(s, coarse_max_u=30)
    assert P.rbm_nlevels() >= 3
    A = _uu_dense(s)
    rng = np.random.default_rng(3)
    xs = rng.standard_normal(3 * s.n_nodes)
    b = A @ xs
    # stationary iteration x <- x + M (b - A x): the error shrinks by a factor per V-cycle
    x = np.zeros_like(b)
    e0 = np.linalg.norm(xs)
    for _ in range(8):
        x = x + P.rbm_vcycle(b - A @ x)
    assert np.linalg.norm(x - xs) <= 0.2 * e0
    _, st = P.fgmres(tol=1e-8)
    assert st.converged and st.true_relres <= 1e-8


def test_prolongator_smoothing_lowers_the_energy():
    # P = (I - omega D^{-1} A) P_tent with 0 < omega lambda_max(D^{-1} A) < 2 is an A-norm contraction on
    # every column: each coarse basis function has no more energy than its tentative one, and strictly
    # less for most of them
    # (without gravity the elasticity block is symmetric; the Dirichlet base makes it definite)
    s = oracle.System(oracle.default_params(1, nx=9, ny=8, nz=6, flags=OR_ALL & ~OR_GRAVITY))
    P = rbm_prec(s, coarse_max_u=20)
    sh = P.rbm_shape(0)
    agg, B, Pt, lam = P.rbm_data(0)
    rp, ci, v = P.rbm_prolongator(0)
    Pd = bsr_dense(rp, ci, v, sh["nagg"])
    rp, ci, v = P.rbm_level(0)
    A = bsr_dense(rp, ci, v, len(rp) - 1)
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    b = sh["b"]
    Ptd = np.zeros((Pt.shape[0], 6 * sh["nagg"]))
    for i in np.nonzero(agg >= 0)[0]:
        Ptd[i * b:(i + 1) * b, 6 * agg[i]:6 * agg[i] + 6] = Pt[i * b:(i + 1) * b]
    e_t = np.einsum("ik,ij,jk->k", Ptd, A, Ptd)
    e_s = np.einsum("ik,ij,jk->k", Pd, A, Pd)
    live = e_t > 0
    assert np.all(e_s[live] <= e_t[live] * (1 + 1e-12))
    assert np.mean(e_s[live] < 0.9 * e_t[live]) > 0.5
