"""The request server admits a request when the bytes its handle is estimated to hold fit under the
budget (ps_setup_bytes_estimate, host arithmetic only, so it runs without a GPU).  The estimate must
cover the device arrays a handle is known to hold; here they are counted from the structured patterns
of the grid and the layout of each array: the Jacobian block copies, the FP64 stencil copy used by the
outer SpMV, the Krylov bases, and the ILU(0) sweep records ([tile][step][thread][20], 16 x 8 tiles,
steps padded to whole copy windows of 4 (FP32) or 2 (FP64) steps)."""
import pytest

import paper_1812_05540_gb300 as ps
from paper_1812_05540_gb300 import _build


def counts(nx, ny, nz):
    nn, nc = (nx + 1) * (ny + 1) * (nz + 1), nx * ny * nz
    uu = (3 * (nx + 1) - 2) * (3 * (ny + 1) - 2) * (3 * (nz + 1) - 2)   # 27-point node-node pattern
    uf = 8 * nc                                                          # a cell and its 8 corner nodes
    ff = nc + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1))  # 7-point TPFA pattern
    return nn, nc, uu, uf, ff


def jacobian(nx, ny, nz):
    nn, nc, uu, uf, ff = counts(nx, ny, nz)
    jac = ps.ps_jacobian(ps.ps_bsr(nn, nn, uu, 3, 3, None, None, None), ps.ps_bsr(nn, nc, uf, 3, 2, None, None, None),
                         ps.ps_bsr(nc, nn, uf, 2, 3, None, None, None), ps.ps_bsr(nc, nc, ff, 2, 2, None, None, None),
                         None, None)
    return jac, ps.ps_grid(nx, ny, nz, 1.0, 1.0, 1.0)


def lower_bound(nx, ny, nz, m, mixed):
    nn, nc, uu, uf, ff = counts(nx, ny, nz)
    n = 3 * nn + 2 * nc
    b = sum(nnzb * (8 * bs + 4) for nnzb, bs in ((uu, 9), (uf, 6), (uf, 6), (ff, 4)))  # values + column indices
    b += nn * (27 * 9 + 8 * 6) * 8 + nc * (8 * 6 + 7 * 4) * 8                         # FP64 stencil copy
    b += n * (2 * m + 1) * 8                                                           # V (m + 1) and Z (m)
    w = 4 if mixed else 2
    tiles = -(-ny // 16) * -(-nz // 8)
    steps = -(-(nx + 16 + 8 - 2) // w) * w
    b += 2 * tiles * steps * 128 * 20 * (4 if mixed else 8)                           # sweep records
    return b


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


@pytest.mark.parametrize("grid", [(60, 220, 85), (64, 64, 32), (8, 8, 4), (5, 33, 17), (48, 16, 24), (200, 1, 1), (300, 2, 1)])
@pytest.mark.parametrize("precision", [ps.PS_MIXED_FP32, ps.PS_FP64, ps.PS_MIXED_BF16P])
def test_estimate_covers_the_known_arrays(grid, precision):
    jac, g = jacobian(*grid)
    p = ps.ps_params_default(precision=precision)
    est = ps.ps_setup_bytes_estimate(jac, g, p)
    lb = lower_bound(*grid, p.restart, precision != ps.PS_FP64)
    assert est >= lb, (grid, est, lb)  # thin grids (200 x 1 x 1): the sweep records are half of the bound
    assert est <= 4 * lb, (grid, est, lb)  # an estimate far above the arrays would starve the server


def test_estimate_grows_with_the_restart_length():
    jac, g = jacobian(32, 40, 16)
    nn, nc = 33 * 41 * 17, 32 * 40 * 16
    n = 3 * nn + 2 * nc
    e50 = ps.ps_setup_bytes_estimate(jac, g, ps.ps_params_default(precision=ps.PS_MIXED_FP32, restart=50))
    e100 = ps.ps_setup_bytes_estimate(jac, g, ps.ps_params_default(precision=ps.PS_MIXED_FP32, restart=100))
    assert e100 - e50 >= 50 * 2 * n * 8
