"""Pins of the oracle's block Gauss-Seidel local stage (§5.3 option 1: sweeps of block Gauss-Seidel on the
interleaved S_ff^(FS), 2x2 cell blocks), taken with the cells in red-black order.

  * k sweeps from zero equal the stationary iteration x <- x + (D + L)^{-1} (w - S x) of the red-black
    permuted matrix, with D + L its block lower triangle, formed densely with numpy;
  * with no face coupling (no TPFA terms) S_ff^(FS) is block diagonal and one sweep is the exact local
    solve, so Algorithm 1 with this local stage equals Algorithm 1 with an exact local stage."""
import numpy as np
import pytest

import oracle


def dense_sff(s):
    """S_ff^(FS) = A_ff + blockdiag([[0, D_sp], [0, D_pp]]) (§5.1), interleaved (s, p) per cell, dense."""
    rp, ci, v = s.blocks["ff"]
    nc = s.n_cells
    S = np.zeros((2 * nc, 2 * nc))
    v = v.reshape(-1, 2, 2)
    for i in range(nc):
        for q in range(rp[i], rp[i + 1]):
            S[2 * i:2 * i + 2, 2 * ci[q]:2 * ci[q] + 2] += v[q]
        S[2 * i, 2 * i + 1] += s.d_fs[2 * i]
        S[2 * i + 1, 2 * i + 1] += s.d_fs[2 * i + 1]
    return S


def red_black_order(nx, ny, nz):
    cells = np.arange(nx * ny * nz)
    i, j, k = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    colour = (i + j + k) % 2
    return np.concatenate([cells[colour == 0], cells[colour == 1]])


@pytest.mark.parametrize("sweeps", [1, 2, 3])
@pytest.mark.parametrize("cfg,kw", [(0, dict(nx=5, ny=4, nz=3)), (1, dict(nx=6, ny=5, nz=4))])
def test_gs_sweeps_equal_the_stationary_iteration(cfg, kw, sweeps):
    s = oracle.System(oracle.default_params(cfg, **kw))
    P = oracle.Prec(s, oracle.default_prec_params(local_mode=oracle.LOCAL_GS, local_sweeps=sweeps))
    S = dense_sff(s)
    order = red_black_order(s.nx, s.ny, s.nz)
    perm = np.stack([2 * order, 2 * order + 1], axis=1).ravel()  # dof permutation, cell blocks kept whole
    Sp = S[np.ix_(perm, perm)]
    DL = np.zeros_like(Sp)
    for bi in range(len(order)):
        DL[2 * bi:2 * bi + 2, :2 * bi + 2] = Sp[2 * bi:2 * bi + 2, :2 * bi + 2]
    w = np.random.default_rng(5).standard_normal(2 * s.n_cells)
    wp = w[perm]
    x = np.zeros_like(wp)
    for _ in range(sweeps):
        x = x + np.linalg.solve(DL, wp - Sp @ x)
    expect = np.empty_like(x)
    expect[perm] = x
    got = P.gs_apply(w, sweeps)
    assert np.linalg.norm(got - expect) <= 1e-12 * np.linalg.norm(expect)


def test_gs_is_exact_without_face_coupling():
    flags = oracle.OR_ALL & ~oracle.OR_FLUX & ~oracle.OR_FLUX_SAT
    s = oracle.System(oracle.default_params(0, nx=4, ny=3, nz=3, flags=flags))
    v = np.random.default_rng(2).standard_normal(s.n)
    z_gs = oracle.Prec(s, oracle.default_prec_params(local_mode=oracle.LOCAL_GS, local_sweeps=1)).apply(v)
    z_ex = oracle.Prec(s, oracle.default_prec_params(local_mode=oracle.LOCAL_EXACT)).apply(v)
    assert np.linalg.norm(z_gs - z_ex) <= 1e-12 * np.linalg.norm(z_ex)


def test_gs_local_stage_fgmres_reaches_tolerance():
    s = oracle.System(oracle.default_params(1, nx=12, ny=10, nz=6))
    P = oracle.Prec(s, oracle.default_prec_params(local_mode=oracle.LOCAL_GS))
    x, st = P.fgmres(tol=1e-8)
    r = s.rhs - s.spmv(x)
    assert st.converged and np.linalg.norm(r) <= 1e-8 * np.linalg.norm(s.rhs)
