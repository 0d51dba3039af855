"""Block Gauss-Seidel local stage (§5.3 option 1, PS_LOCAL_HBGS) on the GPU against the oracle's (needs a
GB300): Algorithm 1 in FP64 within 1e-10, and the FGMRES solve in FP64 and mixed precision with the
spec tolerances (true relres <= 1e-8, solution within 1e-6 of the oracle at 1e-12, iterations
within 10 %).  Grids with odd nx exercise the empty colour slots."""
import numpy as np
import pytest

import oracle
import paper_1812_05540_gb300 as ps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    ps.lib()


CASES = [(0, {}), (0, dict(nx=7, ny=3, nz=2)), (1, dict(nx=24, ny=20, nz=10)), (2, dict(nx=21, ny=44, nz=17))]


@pytest.mark.parametrize("sweeps", [1, 3])
@pytest.mark.parametrize("cfg,kw", CASES)
def test_gs_algorithm1_fp64(cfg, kw, sweeps):
    from tests import _gpu as g
    osys = oracle.System(oracle.default_params(cfg, **kw))
    P = oracle.Prec(osys, oracle.default_prec_params(local_mode=oracle.LOCAL_GS, local_sweeps=sweeps))
    dev = g.to_device(osys)
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(local_stage=ps.PS_LOCAL_HBGS, local_sweeps=sweeps))
    try:
        for seed in range(2):
            vs = np.random.default_rng(seed).standard_normal(osys.n)
            v = torch.from_numpy(vs).cuda()
            z = torch.empty_like(v)
            ps.ps_apply_prec(h, v.data_ptr(), z.data_ptr())
            zo = P.apply(vs)
            assert np.linalg.norm(z.cpu().numpy() - zo) <= 1e-10 * np.linalg.norm(zo)
    finally:
        ps.ps_free(h)


@pytest.mark.parametrize("prec", [ps.PS_FP64, ps.PS_MIXED_FP32])
@pytest.mark.parametrize("cfg,kw", CASES[1:])
def test_gs_solve(cfg, kw, prec):
    from tests import _gpu as g
    osys = oracle.System(oracle.default_params(cfg, **kw))
    P = oracle.Prec(osys, oracle.default_prec_params(local_mode=oracle.LOCAL_GS))
    xo, _ = P.fgmres(tol=1e-12)
    _, sto8 = P.fgmres(tol=1e-8)
    dev = g.to_device(osys)
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(precision=prec, local_stage=ps.PS_LOCAL_HBGS))
    try:
        x = torch.zeros(osys.n, dtype=torch.float64, device="cuda")
        _, st = ps.ps_solve(h, dev.rhs.data_ptr(), x.data_ptr(), 1e-8)
    finally:
        ps.ps_free(h)
    xs = x.cpu().numpy()
    relres = np.linalg.norm(osys.rhs - osys.spmv(xs)) / np.linalg.norm(osys.rhs)
    assert relres <= 1e-8 and st.true_relres <= 1e-8
    assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
    assert abs(st.iters - sto8.iters) <= max(1, int(0.1 * sto8.iters) + 1), (st.iters, sto8.iters)


def test_gs_rejects_bad_sweep_count():
    from tests import _gpu as g
    osys = oracle.System(oracle.default_params(0))
    dev = g.to_device(osys)
    with pytest.raises(ps.PsError) as e:
        ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(local_stage=ps.PS_LOCAL_HBGS, local_sweeps=0))
    assert e.value.status == ps.PS_ERR_INVALID
