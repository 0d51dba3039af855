"""Processor-local ILU(0) on the GPU (PS_ILU_LOCAL: the subdomains are the sweep tiles, columns of
PS_ILU_TILE_Y x PS_ILU_TILE_Z cells spanning x) against the oracle's ILU(0) with the same subdomains
(needs a GB300): the factor's inverse diagonal blocks within 1e-13, Algorithm 1 in FP64 within 1e-10, the
pencil sweeps and the level-by-level sweeps agreeing to rounding, and FGMRES with the north-star
tolerances, on grids with several tiles along y and z and ragged last tiles."""
import numpy as np
import pytest

import oracle
import paper_1812_05540_gb300 as ps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TY, TZ = 16, 8  # PS_ILU_TILE_Y, PS_ILU_TILE_Z of include/ps.h


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    ps.lib()


def _g():
    from tests import _gpu as g
    return g


def _local(**kw):
    return oracle.default_prec_params(ilu_tile_y=TY, ilu_tile_z=TZ, **kw)


@pytest.mark.parametrize("ilu", [ps.PS_ILU_PENCIL, ps.PS_ILU_LEVEL_LAUNCH])
@pytest.mark.parametrize("cfg,kw", [(1, dict(nx=12, ny=40, nz=20)), (2, dict(nx=21, ny=44, nz=17))])
def test_local_factor_and_apply_fp64(cfg, kw, ilu):
    g = _g()
    osys = oracle.System(oracle.default_params(cfg, **kw))
    P = oracle.Prec(osys, _local())
    dev = g.to_device(osys)
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(ilu_mode=ilu, ilu_scope=ps.PS_ILU_LOCAL))
    try:
        rp, ci, _ = P.spp()
        _, dinv = ps.ps_flow_copy(h, len(ci), osys.n_cells)
        do = P.ilu_dinv()
        assert np.allclose(dinv, do, rtol=1e-13, atol=1e-13 * np.abs(do).max())
        # the local factor differs from the global one on the tile faces
        dg = oracle.Prec(osys, oracle.default_prec_params(ilu_tile_y=0, ilu_tile_z=0)).ilu_dinv()
        assert np.abs(do - dg).max() > 1e-6 * np.abs(dg).max()
        for seed in range(2):
            vs = np.random.default_rng(seed).standard_normal(osys.n)
            v = torch.from_numpy(vs).cuda()
            z = torch.empty_like(v)
            ps.ps_apply_prec(h, v.data_ptr(), z.data_ptr())
            zo = P.apply(vs)
            assert np.linalg.norm(z.cpu().numpy() - zo) <= 1e-10 * np.linalg.norm(zo)
    finally:
        ps.ps_free(h)


@pytest.mark.parametrize("prec,rtol", [(ps.PS_FP64, 1e-12), (ps.PS_MIXED_FP32, 2e-5)])
def test_local_pencil_matches_level_launch(prec, rtol):
    g = _g()
    osys = oracle.System(oracle.default_params(1, nx=12, ny=40, nz=20))
    dev = g.to_device(osys)
    out = []
    for ilu in (ps.PS_ILU_PENCIL, ps.PS_ILU_LEVEL_LAUNCH):
        h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(precision=prec, ilu_mode=ilu,
                                                                 ilu_scope=ps.PS_ILU_LOCAL))
        try:
            v = torch.from_numpy(np.random.default_rng(7).standard_normal(osys.n)).cuda()
            z = torch.empty_like(v)
            ps.ps_apply_prec(h, v.data_ptr(), z.data_ptr())
            out.append(z.cpu().numpy())
        finally:
            ps.ps_free(h)
    assert np.linalg.norm(out[0] - out[1]) <= rtol * np.linalg.norm(out[1])


@pytest.mark.parametrize("prec", [ps.PS_FP64, ps.PS_MIXED_FP32])
@pytest.mark.parametrize("cfg,kw,cm", [(1, dict(nx=24, ny=20, nz=10), 60), (2, dict(nx=20, ny=44, nz=17), 100)])
def test_local_solve(cfg, kw, cm, prec):
    g = _g()
    osys = oracle.System(oracle.default_params(cfg, **kw))
    P = oracle.Prec(osys, _local(coarse_max_u=cm, coarse_max_p=cm))
    xo, _ = P.fgmres(tol=1e-12)
    _, sto8 = P.fgmres(tol=1e-8)
    dev = g.to_device(osys)
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(precision=prec, coarse_max_u=cm, coarse_max_p=cm,
                                                             ilu_scope=ps.PS_ILU_LOCAL))
    try:
        x = torch.zeros(osys.n, dtype=torch.float64, device="cuda")
        _, st = ps.ps_solve(h, dev.rhs.data_ptr(), x.data_ptr(), 1e-8)
    finally:
        ps.ps_free(h)
    xs = x.cpu().numpy()
    relres = np.linalg.norm(osys.rhs - osys.spmv(xs)) / np.linalg.norm(osys.rhs)
    assert relres <= 1e-8 and abs(st.true_relres - relres) <= 1e-10
    assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
    assert abs(st.iters - sto8.iters) <= max(1, int(0.1 * sto8.iters) + 1), (st.iters, sto8.iters)
