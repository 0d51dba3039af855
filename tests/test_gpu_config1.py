"""The 64x64x32 workload (680,419 DoF, the size of the paper's 680,419-DoF staircase mesh of §6.1) with the
library's default parameters (coarse_max 500, Chebyshev smoothing, pencil-wavefront ILU(0)), against the
oracle at the same size and parameters (needs a GB300).  At this size every kernel family of the full
60x220x85 solve runs: multi-level hierarchies on both blocks, the stencil-slot level-0 kernels, the CSR
coarse-level kernels with every lane count, the SpGEMM capacity classes and the multi-CTA wavefront.

Checks:
  * both AMG hierarchies (§5.2, §5.3): aggregates and level operators bit-exact at every level; S_pp
    bit-exact; inv(U_ii) of block ILU(0) within 1e-13;
  * Algorithm 1 in FP64 within 1e-10 of the oracle's Algorithm 1 on the same vector;
  * FGMRES in FP64 and in mixed precision: true FP64 relres <= 1e-8 recomputed by the oracle, solution
    within 1e-6 relative 2-norm of the oracle solved to 1e-12, iterations within 10 % of the oracle's."""
import numpy as np
import pytest

import oracle
import paper_1812_05540_gb300 as ps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from tests import _gpu as g
    try:
        oracle.build(openmp=True)
        oracle.select(True)  # bit-identical to the serial build, on all host cores
    except Exception:
        oracle.select(False)
    try:
        osys = oracle.System(oracle.default_params(1))
        P = oracle.Prec(osys, oracle.default_prec_params())
    finally:
        oracle.select(False)
    assert osys.n == 680419
    xo, _ = P.fgmres(tol=1e-12)
    _, sto8 = P.fgmres(tol=1e-8)
    dev = g.to_device(osys)
    return osys, P, dev, xo, sto8


def test_config1_hierarchies_bit_exact(case):
    osys, P, dev, _, _ = case
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default())
    try:
        for which in (0, 1):
            nl = P.nlevels(which)
            assert nl >= 3, (which, nl)
            assert ps.ps_amg_nlevels(h, which) == nl
            for l in range(nl):
                orp, oci, ov = P.level(which, l)
                rp, ci, v, agg = ps.ps_amg_level_copy(h, which, l)
                assert np.array_equal(rp, orp) and np.array_equal(ci, oci), (which, l)
                assert np.array_equal(v, ov), (which, l, np.abs(v - ov).max())
                if l < nl - 1:
                    assert np.array_equal(agg, P.aggregates(which, l)[0]), (which, l)
        rp, ci, spp_o = P.spp()
        spp, dinv = ps.ps_flow_copy(h, len(ci), osys.n_cells)
        assert np.array_equal(spp, spp_o)
        do = P.ilu_dinv()
        assert np.allclose(dinv, do, rtol=1e-13, atol=1e-13 * np.abs(do).max())
    finally:
        ps.ps_free(h)


def test_config1_algorithm1_fp64(case):
    osys, P, dev, _, _ = case
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default())
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
def test_config1_solve(case, prec):
    osys, P, dev, xo, sto8 = case
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(precision=prec))
    try:
        x = torch.zeros(osys.n, dtype=torch.float64, device="cuda")
        _, st = ps.ps_solve(h, dev.rhs.data_ptr(), x.data_ptr(), 1e-8)
    finally:
        ps.ps_free(h)
    xs = x.cpu().numpy()
    relres = np.linalg.norm(osys.rhs - osys.spmv(xs)) / np.linalg.norm(osys.rhs)
    assert relres <= 1e-8 and st.true_relres <= 1e-8
    assert abs(st.true_relres - relres) <= 1e-10
    err = np.linalg.norm(xs - xo) / np.linalg.norm(xo)
    assert err <= 1e-6, err
    assert abs(st.iters - sto8.iters) <= max(1, int(0.1 * sto8.iters)), (st.iters, sto8.iters)
