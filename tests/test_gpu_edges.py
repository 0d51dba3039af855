"""Error paths and entry-point variants of the C ABI (needs a GB300)."""
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


@pytest.fixture(scope="module")
def sysd():
    from tests import _gpu as g
    osys = oracle.System(oracle.default_params(1, nx=8, ny=40, nz=20))
    return osys, g.to_device(osys)


def test_invalid_shapes_are_rejected(sysd):
    osys, dev = sysd
    bad = ps.ps_grid(osys.nx + 1, osys.ny, osys.nz, 10.0, 10.0, 10.0)
    with pytest.raises(ps.PsError) as e:
        ps.ps_setup(dev.jac, bad, ps.ps_params_default())
    assert e.value.status == ps.PS_ERR_INVALID
    with pytest.raises(ps.PsError) as e:
        ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(restart=0))
    assert e.value.status == ps.PS_ERR_INVALID


def test_zero_nan_and_iteration_cap(sysd):
    osys, dev = sysd
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(precision=ps.PS_MIXED_FP32, max_iters=3))
    try:
        x = torch.full((osys.n,), 7.0, dtype=torch.float64, device="cuda")
        b = torch.zeros_like(x)
        s, st = ps.ps_solve(h, b.data_ptr(), x.data_ptr(), 1e-8, raise_on_error=False)
        assert s == ps.PS_OK and torch.count_nonzero(x).item() == 0
        b = dev.rhs.clone()
        b[5] = float("nan")
        s, st = ps.ps_solve(h, b.data_ptr(), x.data_ptr(), 1e-8, raise_on_error=False)
        assert s == ps.PS_ERR_NAN
        s, st = ps.ps_solve(h, dev.rhs.data_ptr(), x.data_ptr(), 1e-8, raise_on_error=False)
        assert s == ps.PS_ERR_NOT_CONVERGED and st.iters == 3
        xs = x.cpu().numpy()
        rr = np.linalg.norm(osys.rhs - osys.spmv(xs)) / np.linalg.norm(osys.rhs)
        assert np.isfinite(rr) and rr < 1.0 and abs(rr - st.true_relres) < 1e-10
    finally:
        ps.ps_free(h)


def test_bounded_wait_times_out_and_handle_recovers(sysd):
    # a wavefront CTA that never publishes progress: its consumers give up after spin_limit polls,
    # the solve reports PS_ERR_TIMEOUT, and the same handle then solves normally
    osys, dev = sysd
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(spin_limit=20000, test_stall_wave=1,
                                                             ilu_scope=ps.PS_ILU_GLOBAL))
    try:
        x = torch.zeros(osys.n, dtype=torch.float64, device="cuda")
        s, st = ps.ps_solve(h, dev.rhs.data_ptr(), x.data_ptr(), 1e-8, raise_on_error=False)
        assert s == ps.PS_ERR_TIMEOUT
        assert "wavefront" in ps.ps_strerror(s)
        ps.ps_set_test_stall(h, 0)
        s, st = ps.ps_solve(h, dev.rhs.data_ptr(), x.data_ptr(), 1e-8, raise_on_error=False)
        assert s == ps.PS_OK and st.true_relres <= 1e-8
    finally:
        ps.ps_free(h)


def test_gram_schmidt_barrier_times_out_and_handle_recovers(sysd):
    # a Gram-Schmidt CTA that never reaches the grid barrier: the others give up after spin_limit
    # polls, the solve reports PS_ERR_TIMEOUT, and the same handle then solves normally
    osys, dev = sysd
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(spin_limit=20000, test_stall_gs=2))
    try:
        x = torch.zeros(osys.n, dtype=torch.float64, device="cuda")
        s, st = ps.ps_solve(h, dev.rhs.data_ptr(), x.data_ptr(), 1e-8, raise_on_error=False)
        assert s == ps.PS_ERR_TIMEOUT
        assert "Gram-Schmidt" in ps.ps_strerror(s)
        ps.ps_set_test_stall_gs(h, 0)
        s, st = ps.ps_solve(h, dev.rhs.data_ptr(), x.data_ptr(), 1e-8, raise_on_error=False)
        assert s == ps.PS_OK and st.true_relres <= 1e-8
    finally:
        ps.ps_free(h)


def test_host_pointer_path_matches_device_path(sysd):
    osys, dev = sysd
    import ctypes as C
    keep = []
    blocks = []
    dims = {"uu": (osys.n_nodes, osys.n_nodes, 3, 3), "uf": (osys.n_nodes, osys.n_cells, 3, 2),
            "fu": (osys.n_cells, osys.n_nodes, 2, 3), "ff": (osys.n_cells, osys.n_cells, 2, 2)}
    for name, (nb, ncol, br, bc) in dims.items():
        rp, ci, v = (np.ascontiguousarray(a) for a in osys.blocks[name])
        keep += [rp, ci, v]
        blocks.append(ps.ps_bsr(nb, ncol, len(ci), br, bc, rp.ctypes.data, ci.ctypes.data, v.ctypes.data))
    dfs = np.ascontiguousarray(osys.d_fs)
    keep.append(dfs)
    hjac = ps.ps_jacobian(blocks[0], blocks[1], blocks[2], blocks[3], dfs.ctypes.data, None)
    xh = np.zeros(osys.n)
    rhs = np.ascontiguousarray(osys.rhs)
    h = ps.ps_setup(hjac, dev.grid, ps.ps_params_default(host_ptrs=1))
    try:
        s, st = ps.ps_solve(h, rhs.ctypes.data, xh.ctypes.data, 1e-8)
    finally:
        ps.ps_free(h)
    xd = torch.zeros(osys.n, dtype=torch.float64, device="cuda")
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default())
    try:
        ps.ps_solve(h, dev.rhs.data_ptr(), xd.data_ptr(), 1e-8)
    finally:
        ps.ps_free(h)
    assert np.array_equal(xh, xd.cpu().numpy())


def test_setup_flow_rebuild_matches_fresh_setup(sysd):
    # per-Newton flow setup (§5.2: mechanics hierarchy kept, flow stage rebuilt) on the same values
    osys, dev = sysd
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default(precision=ps.PS_MIXED_FP32))
    try:
        x1 = torch.zeros(osys.n, dtype=torch.float64, device="cuda")
        x2 = torch.zeros_like(x1)
        ps.ps_solve(h, dev.rhs.data_ptr(), x1.data_ptr(), 1e-8)
        ps.ps_setup_flow(h, dev.jac)
        ps.ps_solve(h, dev.rhs.data_ptr(), x2.data_ptr(), 1e-8)
        assert torch.equal(x1, x2)
    finally:
        ps.ps_free(h)


@pytest.mark.parametrize("prec", [ps.PS_FP64, ps.PS_MIXED_FP32])
def test_setup_flow_with_the_next_newton_jacobian_matches_oracle(prec):
    # §5.4 flow-setup reuse against the oracle: the handle is set up on one Jacobian, then ps_setup_flow gets
    # the next Newton state's blocks (all four, so the outer SpMV is the new operator) and keeps the mechanics
    # AMG of the first; the oracle builds M_uu from the first Jacobian and the rest from the second
    from tests import _gpu as g
    import oracle
    kw = dict(nx=24, ny=20, nz=10)
    s1 = oracle.System(oracle.default_params(1, **kw))
    s2 = oracle.System(oracle.default_params(1, dp_amp=2e6, **kw))
    R = oracle.Prec(s2, mech_system=s1)
    xo, _ = R.fgmres(tol=1e-12)
    _, sto8 = R.fgmres(tol=1e-8)
    d1, d2 = g.to_device(s1), g.to_device(s2)
    h = ps.ps_setup(d1.jac, d1.grid, ps.ps_params_default(precision=prec))
    try:
        ps.ps_setup_flow(h, d2.jac)
        if prec == ps.PS_FP64:
            vs = np.random.default_rng(9).standard_normal(s2.n)
            v = torch.from_numpy(vs).cuda()
            z = torch.empty_like(v)
            ps.ps_apply_prec(h, v.data_ptr(), z.data_ptr())
            zo = R.apply(vs)
            assert np.linalg.norm(z.cpu().numpy() - zo) <= 1e-10 * np.linalg.norm(zo)
        x = torch.zeros(s2.n, dtype=torch.float64, device="cuda")
        _, st = ps.ps_solve(h, d2.rhs.data_ptr(), x.data_ptr(), 1e-8)
    finally:
        ps.ps_free(h)
    xs = x.cpu().numpy()
    relres = np.linalg.norm(s2.rhs - s2.spmv(xs)) / np.linalg.norm(s2.rhs)
    assert relres <= 1e-8 and abs(relres - st.true_relres) <= 1e-10
    assert np.linalg.norm(xs - xo) <= 1e-6 * np.linalg.norm(xo)
    assert abs(st.iters - sto8.iters) <= max(1, int(0.1 * sto8.iters) + 1), (st.iters, sto8.iters)
