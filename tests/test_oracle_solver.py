"""Pins of the oracle's preconditioner and Krylov solver (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import OR_ACCUM, OR_ALL, OR_FLUX, OR_FLUX_SAT, OR_COUPLING, OR_GRAVITY, OR_SCALE, OR_DIRICHLET


@pytest.fixture(scope="module")
def sys0():
    return oracle.System(oracle.default_params(0))


def test_dense_lu_matches_library(sys0):
    x = sys0.dense_solve(sys0.rhs)
    xr = np.linalg.solve(sys0.dense(), sys0.rhs)
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)


@pytest.mark.parametrize("pp", [dict(), dict(coarse_max_u=16, coarse_max_p=16), dict(smoother=0)])
def test_fgmres_matches_dense_lu(sys0, pp):
    # brute force: FGMRES to 1e-12 agrees with the direct solution within cond * 1e-12
    xd = sys0.dense_solve(sys0.rhs)
    P = oracle.Prec(sys0, oracle.default_prec_params(**pp))
    x, st = P.fgmres(tol=1e-12)
    assert st.converged and st.true_relres <= 1e-12
    cond = np.linalg.cond(sys0.dense())
    assert np.linalg.norm(x - xd) <= 10 * cond * 1e-12 * np.linalg.norm(xd)
    x8, st8 = P.fgmres(tol=1e-8)
    assert st8.converged and st8.true_relres <= 1e-8 and st8.iters <= st.iters


def test_exact_inverse_one_iteration(sys0):
    # M = A^{-1}: one Krylov step
    P = oracle.Prec(sys0, oracle.default_prec_params(full_exact=1))
    x, st = P.fgmres(tol=1e-10)
    assert st.iters == 1 and st.true_relres <= 1e-10


def test_exact_block_factor_two_iterations(sys0):
    # §5.1: M^{-1} = L^{-1} gives L^{-1}A = U, unit upper triangular with (U - I)^2 = 0,
    # so GMRES needs at most two iterations.
    P = oracle.Prec(sys0, oracle.default_prec_params(mech_mode=oracle.MECH_EXACT,
                                                     flow_mode=oracle.FLOW_EXACT_SCHUR))
    x, st = P.fgmres(tol=1e-10)
    assert st.iters <= 2 and st.true_relres <= 1e-10


def test_exact_local_stage_makes_cpr_exact(sys0):
    # Eq. (mult_prec_op) of §5.3: with M_L = (S_ff^FS)^{-1}, M_ff^{-1} = S^{-1} regardless of M_G,
    # so Algorithm 1 steps 2-8 equal a direct S_ff^(FS) solve after step 2.
    rng = np.random.default_rng(1)
    v = rng.standard_normal(sys0.n)
    Pa = oracle.Prec(sys0, oracle.default_prec_params(local_mode=oracle.LOCAL_EXACT, coarse_max_p=16))
    Pb = oracle.Prec(sys0, oracle.default_prec_params(flow_mode=oracle.FLOW_EXACT_FS))
    za, zb = Pa.apply(v), Pb.apply(v)
    assert np.linalg.norm(za - zb) <= 1e-10 * np.linalg.norm(zb)
    # and step 1 is the same mechanics V-cycle in both
    assert np.array_equal(za[:sys0.n_u], zb[:sys0.n_u])


def _sff_dense(s):
    rp, ci, v = s.blocks["ff"]
    v = v.reshape(-1, 2, 2).copy()
    for c in range(s.n_cells):
        q = rp[c] + list(ci[rp[c]:rp[c + 1]]).index(c)
        v[q, 0, 1] += s.d_fs[2 * c]
        v[q, 1, 1] += s.d_fs[2 * c + 1]
    S = np.zeros((s.n_f, s.n_f))
    for i in range(s.n_cells):
        for q in range(rp[i], rp[i + 1]):
            S[2 * i:2 * i + 2, 2 * ci[q]:2 * ci[q] + 2] = v[q]
    return S


def test_fixed_stress_and_qimpes_reduction():
    # §5.1 S_ff^(FS) adds D_sp, D_pp = V b^2/K_dr (s rho_w, (1-s) rho_nw) to the accumulation diagonal;
    # §5.3 quasi-IMPES S_pp equals the exact second Schur complement when A_ss and A_ps are diagonal.
    gp = oracle.default_params(0, flags=OR_ALL & ~OR_FLUX_SAT)
    s = oracle.System(gp)
    f = s.fields
    Kdr = f["E"] / (3 * (1 - 2 * f["nu"]))
    dp = f["p"] - gp.p_ref
    V = gp.h ** 3
    Dsp = V * gp.biot ** 2 / Kdr * f["sw"] * gp.rho_w0 * (1 + gp.c_w * dp) * 1e6 / s.alpha_f
    Dpp = V * gp.biot ** 2 / Kdr * (1 - f["sw"]) * gp.rho_nw0 * (1 + gp.c_nw * dp) * 1e6 / s.alpha_f
    assert np.allclose(s.d_fs[0::2], Dsp, rtol=1e-13) and np.allclose(s.d_fs[1::2], Dpp, rtol=1e-13)
    S = _sff_dense(s)
    Ass, Asp, Aps, App = S[0::2, 0::2], S[0::2, 1::2], S[1::2, 0::2], S[1::2, 1::2]
    assert np.count_nonzero(Ass - np.diag(np.diag(Ass))) == 0
    assert np.count_nonzero(Aps - np.diag(np.diag(Aps))) == 0
    exact = App - Aps @ np.linalg.solve(Ass, Asp)
    P = oracle.Prec(s)
    rp, ci, v = P.spp()
    Spp = sp.csr_matrix((v, ci, rp), shape=(s.n_cells, s.n_cells)).toarray()
    assert np.abs(Spp - exact).max() <= 1e-12 * np.abs(exact).max()


def test_ilu0_exact_on_cell_chain():
    # a 1-D chain of cells has a block tridiagonal S_ff: ILU(0) is its exact LU
    s = oracle.System(oracle.default_params(0, nx=9, ny=1, nz=1))
    P = oracle.Prec(s)
    S = _sff_dense(s)
    w = np.random.default_rng(2).standard_normal(s.n_f)
    assert np.linalg.norm(P.ilu_apply(w) - np.linalg.solve(S, w)) <= 1e-10 * np.linalg.norm(np.linalg.solve(S, w))


def test_block_ilu0_equals_pointwise_ilu0():
    # §5.3 option 2 is pointwise ILU(0) on the interleaved system; with full 2x2 cell blocks the
    # pattern is closed under the block structure and block ILU(0) gives the same factors.
    s = oracle.System(oracle.default_params(0, nx=3, ny=3, nz=2))
    S = _sff_dense(s)
    n = S.shape[0]
    pat = S != 0
    for c in range(s.n_cells):
        pat[2 * c:2 * c + 2, 2 * c:2 * c + 2] = True
    A = S.copy()
    for i in range(1, n):  # textbook IKJ ILU(0), pointwise
        for k in range(i):
            if not pat[i, k]:
                continue
            A[i, k] /= A[k, k]
            for j in range(k + 1, n):
                if pat[i, j]:
                    A[i, j] -= A[i, k] * A[k, j]
    L = np.tril(A, -1) + np.eye(n)
    U = np.triu(A)
    w = np.random.default_rng(3).standard_normal(n)
    ref = np.linalg.solve(U, np.linalg.solve(L, w))
    P = oracle.Prec(s)
    assert np.linalg.norm(P.ilu_apply(w) - ref) <= 1e-12 * np.linalg.norm(ref)


def test_amg_direct_when_small(sys0):
    P = oracle.Prec(sys0, oracle.default_prec_params(coarse_max_u=10**6, coarse_max_p=10**6))
    assert P.nlevels(0) == 1 and P.nlevels(1) == 1
    rp, ci, v = P.level(1, 0)
    A = sp.csr_matrix((v[:, 0], ci, rp))
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    assert np.linalg.norm(A @ P.vcycle(1, 0, b) - b) <= 1e-12 * np.linalg.norm(b)


def _strength_graph(rp, ci, v, theta):
    n = len(rp) - 1
    A = sp.csr_matrix((np.abs(v).sum(1), ci, rp), shape=(n, n))
    d = A.diagonal()
    At = A.T.tocsr()
    M = A.maximum(At).tocoo()
    keep = (M.row != M.col) & (M.data >= theta * np.sqrt(d[M.row] * d[M.col])) & (M.data > 0)
    G = sp.csr_matrix((np.ones(keep.sum()), (M.row[keep], M.col[keep])), shape=(n, n))
    return G


@pytest.mark.parametrize("which", [0, 1])
def test_aggregation_and_galerkin_hierarchy(which):
    # amg(.) of §5.2/§5.3 as smoothed aggregation: aggregates cover every coupled row, roots form a
    # distance-2 maximal independent set of the strength graph, P = (I - w D^{-1} A) P_tent with
    # w = (4/3)/lambda_Gershgorin, and A_c = P^T A P (Galerkin).
    s = oracle.System(oracle.default_params(1, nx=16, ny=16, nz=8))
    pp = oracle.default_prec_params(coarse_max_u=40, coarse_max_p=40)
    P = oracle.Prec(s, pp)
    nl = P.nlevels(which)
    assert nl >= 3
    theta = pp.theta_u if which == 0 else pp.theta_p
    for l in range(nl - 1):
        rp, ci, v = P.level(which, l)
        n, nc = len(rp) - 1, v.shape[1]
        agg, na = P.aggregates(which, l)
        G = _strength_graph(rp, ci, v, theta * 0.5 ** l)
        # exactly the rows with a strong connection are aggregated (isolated rows are left
        # to the smoother)
        coupled = np.diff(G.indptr) > 0
        assert np.all((agg >= 0) == coupled) and agg.max() == na - 1
        G1 = (G + sp.eye(n)).tocsr()
        G2 = (G1 @ G1).tocsr()
        roots = P.roots(which, l)
        assert roots.sum() == na
        # aggregate ids follow the root order
        assert np.array_equal(agg[roots], np.arange(na))
        # distance-2 independence of the roots
        RR = G2[roots][:, roots]
        assert (RR - sp.diags(RR.diagonal())).nnz == 0
        # maximality: every coupled node lies within distance 2 of a root
        assert np.all((G2 @ roots.astype(float))[coupled] > 0)
        # every strong neighbour of a root joins the root's aggregate
        for r in np.where(roots)[0]:
            nb = G.indices[G.indptr[r]:G.indptr[r + 1]]
            assert np.all(agg[nb] == agg[r])
        # smoothed prolongator and Galerkin product, per component
        prp, pci, pv = P.prolongator(which, l)
        crp, cci, cv = P.level(which, l + 1)
        for c in range(nc):
            A = sp.csr_matrix((v[:, c], ci, rp), shape=(n, n))
            Pm = sp.csr_matrix((pv[:, c], pci, prp), shape=(n, na))
            T = sp.csr_matrix((np.ones(coupled.sum()), (np.where(coupled)[0], agg[coupled])), shape=(n, na))
            d = A.diagonal()
            lam = (abs(A).sum(1).A1 / np.abs(d)).max()
            Pref = T - (4 / 3) / lam * sp.diags(1 / d) @ A @ T
            assert abs(Pm - Pref).max() <= 1e-13 * abs(Pref).max()
            Ac = sp.csr_matrix((cv[:, c], cci, crp), shape=(na, na))
            Aref = Pm.T @ A @ Pm
            assert abs(Ac - Aref).max() <= 1e-12 * abs(Aref).max()


def test_vcycle_contracts():
    # V-cycle used as a stationary iteration reduces the error in the energy norm
    s = oracle.System(oracle.default_params(1, nx=16, ny=16, nz=8))
    P = oracle.Prec(s, oracle.default_prec_params(coarse_max_u=40, coarse_max_p=40))
    for which, comp in ((0, 0), (0, 2), (1, 0)):
        rp, ci, v = P.level(which, 0)
        A = sp.csr_matrix((v[:, comp], ci, rp))
        e = np.random.default_rng(5).standard_normal(A.shape[0])
        if which == 0:
            e[s.dirichlet[comp::3].astype(bool)] = 0
        for _ in range(6):
            e2 = e + P.vcycle(which, comp, -(A @ e))
            ratio = np.sqrt((e2 @ (A @ e2)) / (e @ (A @ e)))
            e = e2
        assert ratio < 0.8


def test_fgmres_diagonal_distinct_eigenvalues():
    # GMRES terminates in k steps on a diagonal operator with k distinct eigenvalues
    for k in (1, 3, 7):
        vals = np.repeat(np.linspace(1.0, 5.0, k), 40)
        b = np.random.default_rng(k).standard_normal(len(vals))
        x, st = oracle.fgmres_diag(vals, b, tol=1e-12)
        assert st.iters == k and np.allclose(x, b / vals, rtol=1e-10)


def test_fgmres_restart_converges_to_same_solution(sys0):
    P = oracle.Prec(sys0)
    x1, st1 = P.fgmres(tol=1e-10)
    x2, st2 = P.fgmres(tol=1e-10, restart=7)
    assert st2.converged and st2.restarts > 0
    assert np.linalg.norm(x1 - x2) <= 1e-6 * np.linalg.norm(x1)


def test_terzaghi_consolidation():
    # Generator <-> physics: 1-D consolidation under a top load with a drained top (textbook
    # closed form), built from the same element and TPFA routines as the Jacobian.
    E, nu, b, kap, mu, phi0, sig, nz, h = 1e9, 0.25, 0.8, 1e-13, 1e-3, 0.2, 1e6, 20, 1.0
    H = nz * h
    Kdr = E / (3 * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    Kv = Kdr + 4 * G / 3
    S = (b - phi0) * (1 - b) / Kdr
    cv = (kap / mu) / (S + b * b / Kv)
    p0 = b * sig / (Kv * S + b * b)
    T = H * H / cv
    dt = T / 1000
    t, p, p0n, cvn, nr = oracle.terzaghi(nz=nz, h=h, E=E, nu=nu, biot=b, kappa=kap, mu=mu, phi0=phi0,
                                         rho0=1000.0, sigma0=sig, dt=dt, nsteps=300)
    assert p0n == pytest.approx(p0, rel=1e-10)
    assert cvn == pytest.approx(cv, rel=1e-12)
    # linear problem: one Newton step is exact up to round-off (an inconsistent Jacobian gives O(1e-1))
    assert nr <= 1e-5
    zc = (np.arange(nz) + 0.5) * h
    zd = H - zc  # depth below the drained top
    m = np.arange(200)[:, None]
    for ti, pi in zip(t, p):
        if ti < 0.05 * T:
            continue
        ser = (4 * p0 / np.pi) * np.sum(np.sin((2 * m + 1) * np.pi * zd / (2 * H)) / (2 * m + 1)
                                        * np.exp(-(2 * m + 1) ** 2 * np.pi ** 2 * cv * ti / (4 * H * H)), axis=0)
        assert np.abs(pi - ser).max() <= 0.02 * p0, (ti / T, np.abs(pi - ser).max() / p0)


def _periodic_laplacian(n, eps):
    # circulant tridiag(-1, 2 + eps, -1): diag(A) = 2 + eps and l1 row sums 4 + eps in every row,
    # Fourier modes cos(2 pi k i / n) are eigenvectors with eigenvalue 2 + eps - 2 cos(2 pi k / n)
    rp = np.arange(0, 3 * n + 1, 3, dtype=np.int64)
    ci, v = [], []
    for i in range(n):
        row = sorted([((i - 1) % n, -1.0), (i, 2.0 + eps), ((i + 1) % n, -1.0)])
        ci += [c for c, _ in row]
        v += [a for _, a in row]
    return rp, np.array(ci, dtype=np.int32), np.array(v)


@pytest.mark.parametrize("degree", [1, 2, 3, 4])
@pytest.mark.parametrize("ratio", [20.0, 7.0])
def test_chebyshev_smoother_error_polynomial(degree, ratio):
    # Chebyshev smoothing on D^{-1}A over [lmax/ratio, lmax], lmax = the Gershgorin bound (Adams et al.
    # 2003): the error of each eigenvector of D^{-1}A is multiplied by the scaled Chebyshev polynomial
    # p_m(t) = T_m((theta - t)/delta) / T_m(theta/delta), from x = 0 and from a nonzero start
    n, eps = 64, 0.5
    rp, ci, v = _periodic_laplacian(n, eps)
    lmax = (4.0 + eps) / (2.0 + eps)
    lmin = lmax / ratio
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)

    def p(t):
        return np.polynomial.chebyshev.chebval((theta - t) / delta, [0] * degree + [1]) / \
            np.polynomial.chebyshev.chebval(theta / delta, [0] * degree + [1])

    i = np.arange(n)
    A = np.zeros((n, n))
    for r in range(n):
        A[r, ci[rp[r]:rp[r + 1]]] = v[rp[r]:rp[r + 1]]
    for k in (1, 5, 16, 31):
        vk = np.cos(2 * np.pi * k * i / n)
        mu = (2.0 + eps - 2.0 * np.cos(2 * np.pi * k / n)) / (2.0 + eps)
        x = oracle.smoother_apply(rp, ci, v, A @ vk, 1, degree, ratio)
        assert np.allclose(x, (1.0 - p(mu)) * vk, rtol=0, atol=1e-12)
        # nonzero start x0 = 0.5 v_j: error v_k - 0.5 v_j
        j = 3
        vj = np.cos(2 * np.pi * j * i / n)
        muj = (2.0 + eps - 2.0 * np.cos(2 * np.pi * j / n)) / (2.0 + eps)
        x = oracle.smoother_apply(rp, ci, v, A @ vk, 1, degree, ratio, x0=0.5 * vj)
        expect = vk - (p(mu) * vk - 0.5 * p(muj) * vj)
        assert np.allclose(x, expect, rtol=0, atol=1e-12)


@pytest.mark.parametrize("sweeps", [1, 2, 5])
def test_l1_jacobi_smoother_error_factor(sweeps):
    # l1-Jacobi (Baker et al. 2011): e <- (I - D_l1^{-1} A) e with D_l1 = diag(sum_j |a_ij|); on the
    # circulant operator D_l1 = (4 + eps) I, so each Fourier mode is damped by (1 - lambda/(4+eps))^s
    n, eps = 48, 0.25
    rp, ci, v = _periodic_laplacian(n, eps)
    i = np.arange(n)
    A = np.zeros((n, n))
    for r in range(n):
        A[r, ci[rp[r]:rp[r + 1]]] = v[rp[r]:rp[r + 1]]
    for k in (0, 2, 12, 24):
        vk = np.cos(2 * np.pi * k * i / n)
        lam = 2.0 + eps - 2.0 * np.cos(2 * np.pi * k / n)
        g = (1.0 - lam / (4.0 + eps)) ** sweeps
        x = oracle.smoother_apply(rp, ci, v, A @ vk, 0, sweeps)
        assert np.allclose(x, (1.0 - g) * vk, rtol=0, atol=1e-12)


def test_reuse_keeps_the_mechanics_hierarchy_and_takes_the_new_flow_stage():
    # flow-setup reuse (§5.4): M_uu built from one Jacobian, everything else from the next Newton step's
    kw = dict(nx=8, ny=7, nz=5)
    s1 = oracle.System(oracle.default_params(1, **kw))
    s2 = oracle.System(oracle.default_params(1, dp_amp=2e6, **kw))
    assert not np.array_equal(s1.blocks["uu"][2], s2.blocks["uu"][2])
    assert not np.array_equal(s1.blocks["ff"][2], s2.blocks["ff"][2])
    P1, P2 = oracle.Prec(s1), oracle.Prec(s2)
    R = oracle.Prec(s2, mech_system=s1)
    b = np.random.default_rng(0).standard_normal(s1.n_nodes)
    for c in range(3):
        assert np.array_equal(R.vcycle(0, c, b), P1.vcycle(0, c, b))
    assert np.array_equal(R.spp()[2], P2.spp()[2])
    assert np.array_equal(R.vcycle(1, 0, b[:s2.n_cells]), P2.vcycle(1, 0, b[:s2.n_cells]))
    x, st = R.fgmres(tol=1e-8)
    assert st.converged and np.linalg.norm(s2.rhs - s2.spmv(x)) <= 1e-8 * np.linalg.norm(s2.rhs)
