"""Newton's method for one time step on the GPU against the oracle's (needs a GB300):

  * ps_assemble_at: the Jacobian values at a state away from the base one match the oracle's Jacobian there
    (or_generate_at) to the generator-parity tolerance, and the residual matches the oracle's residual;
  * ps_newton: the same number of Newton steps as the oracle's driver, the same iterate within 1e-6, a
    converged state whose residual (evaluated by the oracle) is below the nonlinear tolerance, with the
    paper's fixed Krylov tolerance and with Eisenstat-Walker forcing, in FP64 and in mixed precision."""
import numpy as np
import pytest

import oracle
import paper_1812_05540_gb300 as ps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [(0, {}), (1, dict(nx=12, ny=10, nz=6))]
WELLS = (1, dict(nx=12, ny=10, nz=6, flags=oracle.OR_ALL | oracle.OR_WELLS))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    ps.lib()


def _g():
    from tests import _gpu as g
    return g


def _offset(s0, seed):
    rng = np.random.default_rng(seed)
    dx = np.zeros(s0.n)
    dx[:s0.n_u] = 1e-3 * rng.standard_normal(s0.n_u)
    dx[:s0.n_u][s0.dirichlet.astype(bool)] = 0.0
    dx[s0.n_u::2] = 0.02 * rng.standard_normal(s0.n_cells)
    dx[s0.n_u + 1::2] = 2e5 * rng.standard_normal(s0.n_cells)
    return dx


@pytest.mark.parametrize("cfg,kw", CASES + [WELLS])
def test_assemble_at_matches_oracle(cfg, kw):
    from tests.test_gpu_parity import _rows_close
    g = _g()
    ogp = oracle.default_params(cfg, **kw)
    ggp = g.gen_params_like(ogp)
    s0 = oracle.System(ogp)
    dx = _offset(s0, 3)
    so = oracle.System(ogp, dx)
    sysp = ps.ps_generate(ggp)
    try:
        d = torch.from_numpy(dx).cuda()
        r = torch.empty_like(d)
        ps.ps_assemble_at(ggp, sysp, d.data_ptr(), r.data_ptr())
        torch.cuda.synchronize()
        got = g.system_to_numpy(sysp)
        r2 = torch.empty_like(d)
        ps.ps_residual_at(ggp, sysp, d.data_ptr(), r2.data_ptr())
        assert torch.equal(r, r2)  # the residual alone gives the same values
    finally:
        ps.ps_system_free(sysp)
    for name, bs in (("uu", 9), ("uf", 6), ("fu", 6), ("ff", 4)):
        orp, oci, ov = so.blocks[name]
        rp, ci, v = got[name]
        assert np.array_equal(rp, orp) and np.array_equal(ci, oci), name
        ok, worst = _rows_close(ov, v, bs, orp, 1e-13)
        assert ok, (name, worst)
    assert np.allclose(got["d_fs"], so.d_fs, rtol=1e-13, atol=0)
    assert got["alpha_u"] == pytest.approx(so.alpha_u, rel=1e-13)
    assert got["alpha_f"] == pytest.approx(so.alpha_f, rel=1e-13)
    ro = oracle.residual(ogp, dx)
    ro[:s0.n_u][s0.dirichlet.astype(bool)] = 0.0
    rg = r.cpu().numpy()
    nu = s0.n_u
    # the mechanics rows sum each element's Gauss points before the nodes' elements (the oracle adds every
    # Gauss point into the node): rounding only
    assert np.linalg.norm(rg[:nu] - ro[:nu]) <= 1e-12 * np.linalg.norm(ro[:nu])
    assert np.linalg.norm(rg[nu:] - ro[nu:]) <= 1e-12 * np.linalg.norm(ro[nu:])


@pytest.mark.parametrize("prec", [ps.PS_FP64, ps.PS_MIXED_FP32])
@pytest.mark.parametrize("forcing", [ps.PS_FORCING_FIXED, ps.PS_FORCING_EW])
@pytest.mark.parametrize("cfg,kw", CASES + [WELLS])
def test_newton_matches_oracle(cfg, kw, forcing, prec):
    ogp = oracle.default_params(cfg, **kw)
    ggp = _g().gen_params_like(ogp)
    # tight nonlinear tolerance on both sides, so that the two iterates can be compared within 1e-6
    onp = oracle.default_newton_params(forcing=forcing, rtol=1e-8)
    xo, so = oracle.newton(ogp, np_=onp)
    assert so["converged"]
    s0 = oracle.System(ogp)
    x = torch.zeros(s0.n, dtype=torch.float64, device="cuda")
    status, st = ps.ps_newton(ggp, ps.ps_params_default(precision=prec), ps.ps_newton_params_default(forcing=forcing, rtol=1e-8),
                              x.data_ptr())
    assert status == ps.PS_OK and st["converged"]
    xs = x.cpu().numpy()
    tol_steps = 0 if prec == ps.PS_FP64 else 1
    assert abs(st["newton_iters"] - so["newton_iters"]) <= tol_steps, (st["newton_iters"], so["newton_iters"])
    nu = s0.n_u
    for part in (slice(0, nu), slice(nu, None, 2), slice(nu + 1, None, 2)):
        assert np.linalg.norm(xs[part] - xo[part]) <= 1e-6 * np.linalg.norm(xo[part])
    # the oracle's residual at the GPU's iterate, in the base state's row scaling
    r = oracle.residual(ogp, xs)
    r[:nu][s0.dirichlet.astype(bool)] = 0.0
    rs = np.concatenate([r[:nu] / s0.alpha_u, r[nu:] / s0.alpha_f])
    assert np.linalg.norm(rs) <= onp.rtol * st["rnorm"][0] * 1.01
    assert st["rnorm"][0] == pytest.approx(so["rnorm"][0], rel=1e-10)
    if prec == ps.PS_FP64:
        for a, b in zip(st["lin_iters"], so["lin_iters"]):
            assert abs(a - b) <= max(1, int(0.1 * b) + 1), (st["lin_iters"], so["lin_iters"])
