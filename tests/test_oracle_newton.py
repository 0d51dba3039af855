"""Pins of the oracle's Newton driver for one time step (§4 and its remarks on inexact Newton), with the
two-stage preconditioned FGMRES as the inner solver:

  * the Jacobian at a state away from the base one is the derivative of the residual there: central
    differences of the (independently pinned) residual reproduce Jacobian columns at base + dx;
  * the converged iterate satisfies the discrete equations: the residual, evaluated afresh, is below the
    nonlinear tolerance;
  * with tight inner solves the convergence is superlinear (from the second step each reduction factor is
    smaller than the previous);
  * the fixed Krylov tolerance of the paper's runs and Eisenstat-Walker forcing reach the same state, the
    latter with fewer Krylov iterations;
  * the forcing term follows the paper's formula and safeguard on hand-worked values."""
import numpy as np
import pytest

import oracle


def _scaled_rows(s, r):
    rs = r.copy()
    rs[:s.n_u] /= s.alpha_u
    rs[s.n_u:] /= s.alpha_f
    rs[:s.n_u][s.dirichlet.astype(bool)] = 0.0
    return rs


def test_jacobian_at_an_offset_state_is_the_residual_derivative():
    gp = oracle.default_params(0, nx=4, ny=3, nz=3)
    s0 = oracle.System(gp)
    rng = np.random.default_rng(1)
    dx = np.zeros(s0.n)
    dx[:s0.n_u] = 1e-3 * rng.standard_normal(s0.n_u)
    dx[:s0.n_u][s0.dirichlet.astype(bool)] = 0.0
    dx[s0.n_u::2] = 0.02 * rng.standard_normal(s0.n_cells)
    dx[s0.n_u + 1::2] = 2e5 * rng.standard_normal(s0.n_cells)
    s = oracle.System(gp, dx)
    J = s.dense()  # scaled rows, pressure columns in MPa, Dirichlet rows as identity
    free = np.concatenate([~s0.dirichlet.astype(bool), np.ones(s0.n_f, bool)])
    for col in list(range(0, s0.n_u, 37)) + list(range(s0.n_u, s0.n, 29)):
        if not free[col]:
            continue
        pcol = col >= s0.n_u and (col - s0.n_u) % 2 == 1
        h = 1.0 if pcol else (1e-6 if col < s0.n_u else 1e-6)
        e = np.zeros(s0.n)
        e[col] = h
        d = (oracle.residual(gp, dx + e) - oracle.residual(gp, dx - e)) / (2 * h)
        if pcol:
            d = d * 1e6  # pressure column in MPa
        fd = _scaled_rows(s, d)[free]
        jc = J[free, col]
        # the Jacobian evaluates the porosity in the mechanics blocks at the element-mean strain, the residual
        # at each Gauss point: with a 1e-3 displacement field they differ by that strain's spread
        assert np.linalg.norm(fd - jc) <= 1e-3 * max(np.linalg.norm(jc), 1e-12), col


@pytest.mark.parametrize("cfg,kw", [(0, {}), (1, dict(nx=12, ny=10, nz=6))])
def test_newton_converges_to_a_root(cfg, kw):
    gp = oracle.default_params(cfg, **kw)
    s0 = oracle.System(gp)
    x, st = oracle.newton(gp, np_=oracle.default_newton_params(forcing=oracle.FORCING_FIXED, eta_fixed=1e-11,
                                                                  rtol=1e-10))
    assert st["converged"] and st["newton_iters"] <= 6
    r0 = np.linalg.norm(_scaled_rows(s0, oracle.residual(gp, np.zeros(s0.n))))
    r = np.linalg.norm(_scaled_rows(s0, oracle.residual(gp, x)))
    assert r <= 1e-10 * r0
    assert abs(r - st["rnorm"][-1]) <= 1e-9 * r0
    # superlinear once the iterate is close: from the second step on each reduction factor is smaller than
    # the one before
    f = [st["rnorm"][k + 1] / st["rnorm"][k] for k in range(st["newton_iters"])]
    assert all(f[k + 1] < f[k] for k in range(1, len(f) - 1)), f
    assert f[-1] < 1e-3


def test_fixed_tolerance_and_eisenstat_walker_reach_the_same_state():
    gp = oracle.default_params(1, nx=12, ny=10, nz=6)
    xf, sf = oracle.newton(gp, np_=oracle.default_newton_params(forcing=oracle.FORCING_FIXED, rtol=1e-8))
    xe, se = oracle.newton(gp, np_=oracle.default_newton_params(forcing=oracle.FORCING_EW, rtol=1e-8))
    assert sf["converged"] and se["converged"]
    nu = 3 * (gp.nx + 1) * (gp.ny + 1) * (gp.nz + 1)
    for part in (slice(0, nu), slice(nu, None, 2), slice(nu + 1, None, 2)):
        assert np.linalg.norm(xe[part] - xf[part]) <= 1e-5 * np.linalg.norm(xf[part])
    assert se["linear_iters"] < sf["linear_iters"]
    assert se["eta"][0] == pytest.approx(0.1)


def test_forcing_term_hand_worked_values():
    np_ = oracle.default_newton_params(rtol=1e-8)  # gamma 0.9, omega 2, eta0 0.1, eta_max 0.1
    assert oracle.ew_eta(np_, 0, 5.0, 5.0, 0.1, 10.0) == pytest.approx(0.1)
    # gamma (r_k / r_{k-1})^omega = 0.9 * 0.01 = 0.009; safeguard 0.9 * 0.1^2 = 0.009 is not above 0.1
    assert oracle.ew_eta(np_, 1, 1.0, 10.0, 0.1, 10.0) == pytest.approx(0.009)
    # the safeguard: gamma eta_prev^omega = 0.9 * 0.5^2 = 0.225 > 0.1 lifts eta to 0.225, then the cap 0.1
    big = oracle.default_newton_params(ew_eta_max=1.0, rtol=1e-8)
    assert oracle.ew_eta(big, 1, 1.0, 10.0, 0.5, 10.0) == pytest.approx(0.225)
    assert oracle.ew_eta(np_, 1, 1.0, 10.0, 0.5, 10.0) == pytest.approx(0.1)
    # the floor: no tighter than half the nonlinear tolerance relative to the current residual
    assert oracle.ew_eta(np_, 3, 1e-7, 1e-2, 1e-4, 10.0) == pytest.approx(0.5 * 1e-8 * 10.0 / 1e-7)
    fixed = oracle.default_newton_params(forcing=oracle.FORCING_FIXED, eta_fixed=1e-6, rtol=1e-8)
    assert oracle.ew_eta(fixed, 2, 1.0, 2.0, 0.1, 10.0) == 1e-6


def test_default_tolerances_are_the_papers():
    # Table 1: Newton tolerance 1e-5, Krylov tolerance 1e-6; the forcing parameters of the §4 remark
    np_ = oracle.default_newton_params()
    assert np_.rtol == 1e-5 and np_.eta_fixed == 1e-6
    assert (np_.ew_gamma, np_.ew_omega, np_.ew_eta0) == (0.9, 2.0, 0.1)


def test_library_forcing_term_equals_the_oracles():
    # the library's host-side forcing rule (ps_newton_eta) against the oracle's on a spread of inputs
    import itertools
    import paper_1812_05540_gb300 as ps
    for forcing in (oracle.FORCING_FIXED, oracle.FORCING_EW):
        o = oracle.default_newton_params(forcing=forcing)
        p = ps.ps_newton_params_default(forcing=forcing)
        for k, rk, rkm1, eta_prev, r0 in itertools.product((0, 1, 4), (1e-7, 0.3, 2.0), (1e-3, 1.0, 5.0),
                                                             (1e-4, 0.1, 0.6), (10.0,)):
            assert ps.ps_newton_eta(p, k, rk, rkm1, eta_prev, r0) == oracle.ew_eta(o, k, rk, rkm1, eta_prev, r0)


def test_well_jacobian_is_the_residual_derivative():
    # the Peaceman well terms (§3 well model) of the Jacobian at an offset state are the derivatives of the
    # residual's well sources: central differences on the well cells' columns; a planted sign or density
    # mistake in either side fails it
    gp = oracle.default_params(0, nx=4, ny=3, nz=3, flags=oracle.OR_ALL | oracle.OR_WELLS)
    s0 = oracle.System(gp)
    rng = np.random.default_rng(5)
    dx = np.zeros(s0.n)
    dx[s0.n_u::2] = 0.02 * rng.standard_normal(s0.n_cells)
    dx[s0.n_u + 1::2] = 2e5 * rng.standard_normal(s0.n_cells)
    s = oracle.System(gp, dx)
    J = s.dense()
    nx, ny, nz = gp.nx, gp.ny, gp.nz
    wells = [i + nx * (j + ny * k) for k in range(nz) for (i, j) in ((0, 0), (nx - 1, ny - 1))]
    for c in wells:
        for comp, h in ((0, 1e-6), (1, 1.0)):
            col = s0.n_u + 2 * c + comp
            e = np.zeros(s0.n)
            e[col] = h
            d = (oracle.residual(gp, dx + e) - oracle.residual(gp, dx - e)) / (2 * h)
            if comp == 1:
                d = d * 1e6
            fd = _scaled_rows(s, d)[s0.n_u:]
            jc = J[s0.n_u:, col]
            assert np.linalg.norm(fd - jc) <= 1e-5 * max(np.linalg.norm(jc), 1e-12), (c, comp)


def test_wells_inject_water_and_produce_both_phases():
    # at the base state the injector column gains wetting-phase mass only and the producer column loses mass of
    # both phases (the 5 MPa bottom-hole offsets of Table 1 set the signs): the residual's well sources
    gp = oracle.default_params(0, nx=4, ny=3, nz=3)
    gw = oracle.default_params(0, nx=4, ny=3, nz=3, flags=oracle.OR_ALL | oracle.OR_WELLS)
    s0 = oracle.System(gp)
    x = np.zeros(s0.n)
    dr = oracle.residual(gw, x) - oracle.residual(gp, x)
    nx, ny, nz = gp.nx, gp.ny, gp.nz
    nu = s0.n_u
    inj = [i for i in range(s0.n_cells) if i % nx == 0 and (i // nx) % ny == 0]
    prod = [i for i in range(s0.n_cells) if i % nx == nx - 1 and (i // nx) % ny == ny - 1]
    other = [c for c in range(s0.n_cells) if c not in inj and c not in prod]
    assert np.all(dr[:nu] == 0.0)
    assert all(dr[nu + 2 * c] < 0 and dr[nu + 2 * c + 1] == 0.0 for c in inj)  # -dt q^I_w < 0
    assert all(dr[nu + 2 * c] > 0 and dr[nu + 2 * c + 1] > 0 for c in prod)  # +dt q^P_l > 0
    assert all(dr[nu + 2 * c] == 0.0 and dr[nu + 2 * c + 1] == 0.0 for c in other)


def test_wells_need_cells_wider_than_the_wellbore():
    # Eq. (well_index) needs Peaceman's radius 0.28 sqrt(2) h / 2 above the well radius 0.1524 m: both the
    # oracle and the library refuse wells on cells of 0.5 m (the library before touching the device)
    import ctypes
    import paper_1812_05540_gb300 as ps
    gp = oracle.default_params(0, nx=4, ny=3, nz=3, h=0.5, flags=oracle.OR_ALL | oracle.OR_WELLS)
    with pytest.raises(ValueError):
        oracle.residual(gp, np.zeros(3 * 5 * 4 * 4 + 2 * 36))
    with pytest.raises(RuntimeError):
        oracle.System(gp)
    g = ps.ps_gen_default(0)
    g.nx, g.ny, g.nz, g.h = 4, 3, 3, 0.5
    g.flags = ps.PS_GEN_ALL | ps.PS_GEN_WELLS
    out = ctypes.POINTER(ps.ps_system)()
    assert ps.lib().ps_generate(ctypes.byref(g), None, ctypes.byref(out)) == ps.PS_ERR_INVALID
    assert not out
