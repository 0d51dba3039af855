"""Rigid-body-mode smoothed aggregation for M_uu on the GPU (mech_amg = PS_MECH_RBM) against the oracle's
(MECH_AMG_RBM), needs a GB300: the hierarchy level by level (shapes, aggregates and block operators bit for
bit, the prolongator bit for bit), Algorithm 1 in FP64 within 1e-10, and FGMRES with the north-star
tolerances in both precisions."""
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


def _g():
    from tests import _gpu as g
    return g


CASES = [(0, {}, 20), (1, dict(nx=24, ny=20, nz=10), 60), (2, dict(nx=21, ny=44, nz=17), 200)]


@pytest.mark.parametrize("cfg,kw,cm", CASES)
def test_rbm_hierarchy_parity(cfg, kw, cm):
    g = _g()
    osys = oracle.System(oracle.default_params(cfg, **kw))
    P = oracle.Prec(osys, oracle.default_prec_params(mech_mode=oracle.MECH_AMG_RBM, coarse_max_u=cm))
    dev = g.to_device(osys)
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(mech_amg=ps.PS_MECH_RBM, coarse_max_u=cm))
    try:
        nl = P.rbm_nlevels()
        assert nl >= 2 and ps.ps_rbm_nlevels(h) == nl
        for l in range(nl):
            osh, sh = P.rbm_shape(l), ps.ps_rbm_level_shape(h, l)
            assert all(osh[k] == sh[k] for k in ("n", "b", "nnzb", "nagg", "pnnzb", "coarsest")), (l, osh, sh)
            orp, oci, ov = P.rbm_level(l)
            rp, ci, v, agg = ps.ps_rbm_level_copy(h, l)
            assert np.array_equal(rp, orp) and np.array_equal(ci, oci), l
            assert np.array_equal(v, ov), (l, np.abs(v - ov).max())
            if not sh["coarsest"]:
                oagg, _, _, _ = P.rbm_data(l)
                assert np.array_equal(agg, oagg), l
                prp, pci, pv = P.rbm_prolongator(l)
                grp, gci, gpv = ps.ps_rbm_prolongator_copy(h, l)
                assert np.array_equal(grp, prp) and np.array_equal(gci, pci), l
                assert np.array_equal(gpv, pv), (l, np.abs(gpv - pv).max())
    finally:
        ps.ps_free(h)


@pytest.mark.parametrize("cfg,kw,cm", CASES)
def test_rbm_apply_parity_fp64(cfg, kw, cm):
    g = _g()
    osys = oracle.System(oracle.default_params(cfg, **kw))
    P = oracle.Prec(osys, oracle.default_prec_params(mech_mode=oracle.MECH_AMG_RBM, coarse_max_u=cm))
    dev = g.to_device(osys)
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(mech_amg=ps.PS_MECH_RBM, coarse_max_u=cm))
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
@pytest.mark.parametrize("cfg,kw,cm", CASES[1:])
def test_rbm_solve(cfg, kw, cm, prec):
    g = _g()
    osys = oracle.System(oracle.default_params(cfg, **kw))
    P = oracle.Prec(osys, oracle.default_prec_params(mech_mode=oracle.MECH_AMG_RBM, coarse_max_u=cm))
    xo, _ = P.fgmres(tol=1e-12)
    _, sto8 = P.fgmres(tol=1e-8)
    dev = g.to_device(osys)
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(precision=prec, mech_amg=ps.PS_MECH_RBM,
                                                             coarse_max_u=cm))
    try:
        x = torch.zeros(osys.n, dtype=torch.float64, device="cuda")
        _, st = ps.ps_solve(h, dev.rhs.data_ptr(), x.data_ptr(), 1e-8)
        assert st.levels_u == P.rbm_nlevels()
    finally:
        ps.ps_free(h)
    xs = x.cpu().numpy()
    relres = np.linalg.norm(osys.rhs - osys.spmv(xs)) / np.linalg.norm(osys.rhs)
    assert relres <= 1e-8 and abs(st.true_relres - relres) <= 1e-10
    assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
    assert abs(st.iters - sto8.iters) <= max(1, int(0.1 * sto8.iters) + 1), (st.iters, sto8.iters)


def test_rbm_rejects_l1_smoothing():
    g = _g()
    osys = oracle.System(oracle.default_params(0))
    dev = g.to_device(osys)
    with pytest.raises(RuntimeError):
        ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(mech_amg=ps.PS_MECH_RBM, smoother=ps.PS_SMOOTH_L1JACOBI))
