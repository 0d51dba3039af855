"""Batched setup and lockstep solve of several uneven systems (ps_setup_batch / ps_solve_batch, needs a
GB300): each system's solution and iteration count equal those of ps_solve on the same system (the same
kernels in the same order, so the same bits), and the oracle's solution within the north-star
tolerance."""
import numpy as np
import pytest

import oracle
import paper_1812_05540_gb300 as ps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [(6, 5, 3), (12, 9, 5), (7, 3, 2), (16, 12, 8), (9, 14, 4)]


@pytest.mark.parametrize("prec", [ps.PS_FP64, ps.PS_MIXED_FP32])
def test_batch_equals_single_solves(prec):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from tests import _gpu as g
    torch.cuda.set_device(0)
    osys = [oracle.System(oracle.default_params(1, nx=a, ny=b, nz=c, seed=3100 + i))
            for i, (a, b, c) in enumerate(SIZES)]
    devs = [g.to_device(s) for s in osys]
    p = ps.ps_params_default(precision=prec)
    hs = ps.ps_setup_batch([d.jac for d in devs], [d.grid for d in devs], p)
    try:
        xs = [torch.zeros(s.n, dtype=torch.float64, device="cuda") for s in osys]
        status, stats = ps.ps_solve_batch(hs, [d.rhs.data_ptr() for d in devs], [x.data_ptr() for x in xs], 1e-8)
        assert status == ps.PS_OK
    finally:
        for h in hs:
            ps.ps_free(h)
    for i, (s, d) in enumerate(zip(osys, devs)):
        h = ps.ps_setup(d.jac, d.grid, p)
        try:
            x1 = torch.zeros(s.n, dtype=torch.float64, device="cuda")
            _, st1 = ps.ps_solve(h, d.rhs.data_ptr(), x1.data_ptr(), 1e-8)
        finally:
            ps.ps_free(h)
        assert stats[i].iters == st1.iters, i
        assert torch.equal(xs[i], x1), i
        xb = xs[i].cpu().numpy()
        assert np.linalg.norm(s.rhs - s.spmv(xb)) <= 1e-8 * np.linalg.norm(s.rhs)
        xo, _ = oracle.Prec(s).fgmres(tol=1e-12)
        assert np.linalg.norm(xb - xo) <= 1e-6 * np.linalg.norm(xo)


def test_batch_rejects_a_bad_system_and_frees_the_rest():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from tests import _gpu as g
    torch.cuda.set_device(0)
    good = g.to_device(oracle.System(oracle.default_params(0)))
    bad_grid = ps.ps_grid(good.grid.nx + 1, good.grid.ny, good.grid.nz, 10.0, 10.0, 10.0)
    with pytest.raises(ps.PsError) as e:
        ps.ps_setup_batch([good.jac, good.jac], [good.grid, bad_grid], ps.ps_params_default())
    assert e.value.status == ps.PS_ERR_INVALID
