"""ps_residual_noalloc: the residual entry point for callers that manage all
device memory themselves (a simulator that reserves its HBM at start-up, a
process with a capped allocator) and therefore cannot let the library
allocate.  It must give the same r = b - A x and ||r||^2 as the allocating
path (ps_spmv of a handle) on consecutive calls that share its static scratch.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
import paper_1812_05540_gb300 as ps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_residual_noalloc_matches_allocating_path():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from tests import _gpu as g
    torch.cuda.set_device(0)
    osys = oracle.System(oracle.default_params(1, nx=24, ny=20, nz=10))
    dev = g.to_device(osys)
    h = ps.ps_setup(dev.jac, dev.grid, ps.ps_params_default())
    try:
        b = dev.rhs
        r = torch.empty_like(b)
        rn2 = torch.empty(1, dtype=torch.float64, device="cuda")
        y = torch.empty_like(b)
        for seed in (0, 1):  # two calls in a row on the shared scratch
            x = torch.from_numpy(np.random.default_rng(seed).standard_normal(osys.n)).cuda()
            torch.cuda.synchronize()
            allocs = ps.ps_alloc_count()
            ps.ps_residual_noalloc(dev.jac, dev.grid, x.data_ptr(), b.data_ptr(), r.data_ptr(), rn2.data_ptr())
            torch.cuda.synchronize()
            assert ps.ps_alloc_count() == allocs  # the call made no device allocation
            ps.ps_spmv(h, x.data_ptr(), y.data_ptr())
            ref = (b - y).cpu().numpy()
            got = r.cpu().numpy()
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(y.cpu().numpy()).max()
            assert rn2.item() == pytest.approx(float(ref @ ref), rel=1e-12)
    finally:
        ps.ps_free(h)


def test_residual_noalloc_rejects_oversized_systems():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    # shapes are checked before any device work: a grid beyond the fixed scratch is refused
    grid = ps.ps_grid(400, 400, 40, 10.0, 10.0, 10.0)
    nn, nc = 401 * 401 * 41, 400 * 400 * 40
    blk = lambda r, c, br, bc: ps.ps_bsr(r, c, 0, br, bc, 1, 1, 1)
    jac = ps.ps_jacobian(blk(nn, nn, 3, 3), blk(nn, nc, 3, 2), blk(nc, nn, 2, 3), blk(nc, nc, 2, 2), 1, None)
    with pytest.raises(ps.PsError) as e:
        ps.ps_residual_noalloc(jac, grid, 8, 16, 24, 32)
    assert e.value.status == ps.PS_ERR_INVALID and "scratch" in str(e.value)


def test_residual_noalloc_rejects_bad_arguments_with_a_reason():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    grid = ps.ps_grid(4, 4, 2, 10.0, 10.0, 10.0)
    nn, nc = 5 * 5 * 3, 4 * 4 * 2
    blk = lambda r, c, br, bc: ps.ps_bsr(r, c, 0, br, bc, 1, 1, 1)
    jac = ps.ps_jacobian(blk(nn, nn, 3, 3), blk(nn, nc, 3, 2), blk(nc, nn, 2, 3), blk(nc, nc, 2, 2), 1, None)
    # r aliasing x or b is refused on the host
    with pytest.raises(ps.PsError) as e:
        ps.ps_residual_noalloc(jac, grid, 8, 16, 8, 24)
    assert e.value.status == ps.PS_ERR_INVALID and "same array" in str(e.value)
    # a block of the wrong shape is named
    bad = ps.ps_jacobian(blk(nn, nn, 3, 3), blk(nn, nc, 3, 2), blk(nc, nn, 2, 3), blk(nc, nc + 1, 2, 2), 1, None)
    with pytest.raises(ps.PsError) as e:
        ps.ps_residual_noalloc(bad, grid, 8, 16, 24, 32)
    assert e.value.status == ps.PS_ERR_INVALID and "A_ff" in str(e.value)
    # one row block past the scratch: ceil(nodes/8) + ceil(cells/8) = 2^19 + 1
    nx, ny, nz = 113, 189, 97
    nodes, cells = (nx + 1) * (ny + 1) * (nz + 1), nx * ny * nz
    assert -(-nodes // 8) + -(-cells // 8) == 2 ** 19 + 1
    big = ps.ps_grid(nx, ny, nz, 10.0, 10.0, 10.0)
    bj = ps.ps_jacobian(blk(nodes, nodes, 3, 3), blk(nodes, cells, 3, 2), blk(cells, nodes, 2, 3),
                        blk(cells, cells, 2, 2), 1, None)
    with pytest.raises(ps.PsError) as e:
        ps.ps_residual_noalloc(bj, big, 8, 16, 24, 32)
    assert e.value.status == ps.PS_ERR_INVALID and "scratch" in str(e.value)
