"""Pins of the oracle's Jacobian generator against what the paper and the
mathematics fix (no GPU).  Each test names the passage it checks."""
import os

import numpy as np
import pytest

import oracle
from oracle import (OR_ACCUM, OR_ALL, OR_COUPLING, OR_DIRICHLET, OR_FLUX, OR_FLUX_SAT, OR_GRAVITY,
                    OR_SCALE)

MD = 9.869233e-16


def homogeneous(**kw):
    return oracle.default_params(0, field_kind=oracle.FIELDS_HOMOGENEOUS, **kw)


def test_splitmix64_published_vector():
    # Vigna's splitmix64 seeded with 0: first three outputs
    L = oracle.lib()
    golden = 0x9E3779B97F4A7C15
    outs = [L.or_splitmix64((k * golden) & (2**64 - 1)) for k in range(3)]
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


@pytest.mark.parametrize("row", _golden_rows("table2_staircase_dofs.txt"))
def test_dof_counts_match_table2(row):
    # §6.1 Table 2: 88,307 and 680,419 DoF on the staircase meshes (all nodes x3 + 2 per cell)
    nx, ny, nz, dof = (int(t) for t in row)
    gp = homogeneous(nx=nx, ny=ny, nz=nz, flags=OR_ACCUM)
    s = oracle.System(gp)
    assert s.n == dof
    assert s.n_u == 3 * (nx + 1) * (ny + 1) * (nz + 1) and s.n_f == 2 * nx * ny * nz


def test_generator_constants_match_table1():
    # §6 Table 1: reference densities and residual saturations used by every configuration
    gp = oracle.default_params(0)
    for name, value, _unit in _golden_rows("table1_parameters.txt"):
        assert getattr(gp, name) == float(value), name


def test_reference_integrals_closed_forms():
    # Q1 on a cube of edge h: int N_a = h^3/8, int dN_a/dx_d = +-h^2/4,
    # int (dN_a/dx)^2 = h/9, partition of unity kills sums over b.
    h = 3.0
    G, IN, IdN, INdN = oracle.ref_integrals(h)
    assert np.allclose(IN, h**3 / 8, rtol=1e-14)
    for a in range(8):
        for d in range(3):
            sign = 1.0 if (a >> d) & 1 else -1.0
            assert IdN[a, d] == pytest.approx(sign * h * h / 4, rel=1e-14)
            assert G[a, a, d, d] == pytest.approx(h / 9, rel=1e-13)
    assert np.abs(G.sum(axis=1)).max() < 1e-12 * h
    assert np.abs(INdN.sum(axis=1)).max() < 1e-12 * h * h
    assert np.allclose(G, G.transpose(1, 0, 3, 2), atol=1e-14 * h)
    # int N_a dN_b/dx_e + int N_b dN_a/dx_e = int d(N_a N_b)/dx_e = boundary flux of N_a N_b
    S = INdN + INdN.transpose(1, 0, 2)
    for a in range(8):
        for b in range(8):
            for e in range(3):
                if (a >> e) & 1 != (b >> e) & 1:
                    continue
                # both on the same face along e: +-(face integral of product) = +-h^2 * m
                same = [(a >> d) & 1 == (b >> d) & 1 for d in range(3) if d != e]
                m = np.prod([1 / 3 if sm else 1 / 6 for sm in same])
                sign = 1.0 if (a >> e) & 1 else -1.0
                assert S[a, b, e] == pytest.approx(sign * h * h * m, rel=1e-12)


def _uu_dense(s):
    rp, ci, v = s.blocks["uu"]
    v = v.reshape(-1, 3, 3)
    A = np.zeros((s.n_u, s.n_u))
    for i in range(s.n_nodes):
        for q in range(rp[i], rp[i + 1]):
            A[3 * i:3 * i + 3, 3 * ci[q]:3 * ci[q] + 3] = v[q]
    return A


def _node_xyz(s):
    nx, ny, nz, h = s.nx, s.ny, s.nz, s.h
    idx = np.arange(s.n_nodes)
    return np.stack([(idx % (nx + 1)) * h, (idx // (nx + 1)) % (ny + 1) * h, idx // ((nx + 1) * (ny + 1)) * h], 1)


def test_rigid_body_modes_in_pure_neumann_nullspace():
    # §5.2 elasticity block without Dirichlet and gravity: six rigid-body modes are in its null space
    gp = oracle.default_params(0, flags=OR_ALL & ~(OR_GRAVITY | OR_DIRICHLET))
    s = oracle.System(gp)
    A = _uu_dense(s)
    X = _node_xyz(s)
    modes = []
    for d in range(3):
        m = np.zeros((s.n_nodes, 3)); m[:, d] = 1; modes.append(m)
    for (a, b) in ((0, 1), (1, 2), (2, 0)):
        m = np.zeros((s.n_nodes, 3)); m[:, a] = -X[:, b]; m[:, b] = X[:, a]; modes.append(m)
    An = np.abs(A).sum(1).max()
    for m in modes:
        r = A @ m.ravel()
        assert np.abs(r).max() <= 1e-12 * An * np.abs(m).max()
    # and the gravity-free block is symmetric
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()


def test_patch_test_affine_displacement():
    # homogeneous Q1 elasticity reproduces constant stress: interior nodal forces vanish
    gp = homogeneous(nx=4, ny=3, nz=3, flags=OR_ALL & ~(OR_GRAVITY | OR_DIRICHLET))
    s = oracle.System(gp)
    A = _uu_dense(s)
    X = _node_xyz(s)
    Gm = np.array([[1e-3, 2e-4, -3e-4], [5e-4, -2e-3, 1e-4], [0.0, 7e-4, 1.5e-3]])
    u = X @ Gm.T + np.array([0.1, -0.2, 0.3])
    f = (A @ u.ravel()).reshape(-1, 3)
    nx, ny, nz = s.nx, s.ny, s.nz
    idx = np.arange(s.n_nodes)
    i, j, k = idx % (nx + 1), (idx // (nx + 1)) % (ny + 1), idx // ((nx + 1) * (ny + 1))
    interior = (i > 0) & (i < nx) & (j > 0) & (j < ny) & (k > 0) & (k < nz)
    assert interior.sum() > 0
    assert np.abs(f[interior]).max() <= 1e-12 * np.abs(f).max()


def test_tpfa_zero_row_sums_and_transmissibility():
    # App. A / Eq. (8): with incompressible fluids and no gravity the pressure part of the
    # face Jacobian has zero row sums; for uniform kappa, Upsilon = kappa |f| / h.
    gp = homogeneous(nx=5, ny=4, nz=3, flags=OR_FLUX | OR_FLUX_SAT, c_w=0.0, c_nw=0.0, c_r=0.0, dp_amp=2e6)
    s = oracle.System(gp)
    rp, ci, v = s.blocks["ff"]
    v = v.reshape(-1, 2, 2)
    for i in range(s.n_cells):
        blk = v[rp[i]:rp[i + 1]]
        assert abs(blk[:, 0, 1].sum()) <= 1e-12 * np.abs(blk[:, 0, 1]).max()
        assert abs(blk[:, 1, 1].sum()) <= 1e-12 * np.abs(blk[:, 1, 1]).max()
    # off-diagonal oil pressure entry of cell 0 -> its x neighbour: -dt rho lam Upsilon
    h, kap = gp.h, gp.kappa0
    sh = (gp.sw0 - gp.s_wr) / (1 - gp.s_wr - gp.s_nwr)
    lam_nw = (1 - sh) ** 2 / gp.mu_nw
    q = rp[0] + list(ci[rp[0]:rp[1]]).index(1)
    assert v[q, 1, 1] == pytest.approx(-gp.dt * gp.rho_nw0 * lam_nw * kap * h, rel=1e-13)


def test_coupling_blocks_are_scaled_transposes():
    # App. B: A_up = -b int div(eta) chi and A_su = s rho_w b int div(eta) psi (no gravity),
    # so A_su = -s rho_w A_up^T and A_pu = -(1-s) rho_nw A_up^T cellwise.
    gp = oracle.default_params(0, flags=OR_ALL & ~(OR_GRAVITY | OR_SCALE | OR_DIRICHLET))
    s = oracle.System(gp)
    A = s.dense()
    nu = s.n_u
    Aup = A[:nu, nu + 1::2]
    Asu = A[nu::2, :nu]
    Apu = A[nu + 1::2, :nu]
    sw = s.fields["sw"]
    dp = s.fields["p"] - gp.p_ref
    rw = gp.rho_w0 * (1 + gp.c_w * dp)
    rnw = gp.rho_nw0 * (1 + gp.c_nw * dp)
    assert np.allclose(Asu, -(sw * rw)[:, None] * Aup.T, rtol=1e-13, atol=1e-13 * np.abs(Asu).max())
    assert np.allclose(Apu, -((1 - sw) * rnw)[:, None] * Aup.T, rtol=1e-13, atol=1e-13 * np.abs(Apu).max())


def test_fd_jacobian_matches_residual():
    # App. B Jacobian = derivative of the discrete weak form Eq. (5) with the App. B residuals,
    # TPFA fluxes Eq. (8)-(12), gravity, Corey-2 relperms and compressible phases.
    gp = oracle.default_params(0, nx=3, ny=3, nz=2, flags=OR_ALL & ~(OR_DIRICHLET | OR_SCALE))
    s = oracle.System(gp)
    J = s.dense()
    n, nu = s.n, s.n_u
    # the residual is at most quadratic in each unknown, so central differences are exact up to
    # round-off; steps are sized for round-off only
    eps = np.where(np.arange(n) < nu, 1e-5, np.where((np.arange(n) - nu) % 2 == 0, 1e-4, 1e3))
    Jfd = np.zeros_like(J)
    for j in range(n):
        dx = np.zeros(n); dx[j] = eps[j]
        Jfd[:, j] = (oracle.residual(gp, dx) - oracle.residual(gp, -dx)) / (2 * eps[j])
    rows = [slice(0, nu), slice(nu, n, 2), slice(nu + 1, n, 2)]
    cols = [slice(0, nu), slice(nu, n, 2), slice(nu + 1, n, 2)]
    for r in rows:
        for c in cols:
            a, b = J[r, c], Jfd[r, c]
            scale = max(np.abs(a).max(), np.abs(J[r]).max() * 1e-9)
            assert np.abs(a - b).max() <= 1e-6 * scale, (r, c, np.abs(a - b).max(), scale)
    assert np.abs(J[nu:, nu:]).max() > 0 and np.abs(J[:nu, nu:]).max() > 0


def test_scaling_rule():
    # §4 block-row scaling: mean A_uu diagonal over free dofs and mean |A_pp| diagonal become 1
    s = oracle.System(oracle.default_params(0))
    A = s.dense()
    d = np.diag(A)
    free = s.dirichlet == 0
    assert d[:s.n_u][free].mean() == pytest.approx(1.0, rel=1e-12)
    assert np.abs(d[s.n_u + 1::2]).mean() == pytest.approx(1.0, rel=1e-12)
    assert np.all(d[:s.n_u][~free] == 1.0)
    # constrained rows and columns are identity rows / zero columns
    dof = np.where(~free)[0]
    Ad = A.copy()
    Ad[dof, dof] = 0.0
    assert np.all(Ad[dof, :] == 0) and np.all(Ad[:, dof] == 0)
    assert np.all(s.rhs[:s.n_u][~free] == 0) and np.all(np.abs(s.rhs) <= 1)


def test_field_statistics():
    # synthetic stand-ins: ranges and first moments of the sampled fields
    s = oracle.System(oracle.default_params(0))
    f = s.fields
    assert 0.2 <= f["nu"].min() and f["nu"].max() <= 0.3
    assert 0.2 <= f["sw"].min() and f["sw"].max() <= 0.8
    assert 0.15 <= f["phi0"].min() and f["phi0"].max() <= 0.25
    assert abs(f["E"].mean() / 1e10 - 1) < 0.2
    assert abs(np.log(f["kh"]).std() - 1.0) < 0.2
    s1 = oracle.System(oracle.default_params(1, nx=64, ny=64, nz=16, flags=OR_ACCUM))
    assert np.allclose(s1.fields["kv"], 0.1 * s1.fields["kh"])
    E = s1.fields["E"].reshape(16, 64, 64)
    assert np.all(E == E[:, :1, :1]) and 1e9 <= E.min() and E.max() <= 50e9


def test_channel_fields():
    s = oracle.System(oracle.default_params(2, nx=60, ny=110, nz=20, flags=OR_ACCUM))
    kh = s.fields["kh"].reshape(20, 110, 60) / MD
    nlow = (20 * 50 + 42) // 85
    low = kh[:nlow]
    assert np.isclose(low.min(), 1e-2, rtol=1e-12)
    chan = low[low > 1.0]
    assert chan.size > 0 and chan.min() >= 1e3 * (1 - 1e-12) and chan.max() <= 1e4 * (1 + 1e-12)


def test_correlated_field_variance_and_autocorrelation():
    # white noise convolved with g(d) = exp(-(d/L)^2/2) and divided by ||g||_2 has unit variance and
    # autocorrelation exp(-d^2/(4 L^2)) along each axis
    L = 2
    f = oracle.correlated_field(77, 3, 96, 96, 48, L, L, 1)
    assert abs(f.mean()) < 0.05 and abs(f.std() - 1.0) < 0.05
    for d in (1, 2, 3):
        c = np.mean(f[:, :, d:] * f[:, :, :-d])
        assert abs(c - np.exp(-d * d / (4.0 * L * L))) < 0.05
    c = np.mean(f[1:] * f[:-1])
    assert abs(c - np.exp(-1 / 4.0)) < 0.05


def test_uniaxial_fixed_stress_modulus():
    # §5.1 remark: under one-dimensional loading the uniaxial (constrained) modulus K_v replaces K_dr in the
    # fixed-stress diagonal.  With K_dr = E / (3 (1 - 2 nu)) and K_v = E (1 - nu) / ((1 + nu) (1 - 2 nu)),
    # every cell's D_sp and D_pp scale by K_dr / K_v = (1 + nu) / (3 (1 - nu)); nothing else changes.
    kw = dict(nx=6, ny=5, nz=4)
    a = oracle.System(oracle.default_params(1, **kw))
    b = oracle.System(oracle.default_params(1, fs_modulus=1, **kw))
    nu = a.fields["nu"]
    ratio = (1.0 + nu) / (3.0 * (1.0 - nu))
    assert np.allclose(b.d_fs.reshape(-1, 2), a.d_fs.reshape(-1, 2) * ratio[:, None], rtol=1e-13, atol=0)
    for name in ("uu", "uf", "fu", "ff"):
        for x, y in zip(a.blocks[name], b.blocks[name]):
            assert np.array_equal(x, y)
    assert np.array_equal(a.rhs, b.rhs)
