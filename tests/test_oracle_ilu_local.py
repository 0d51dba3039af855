"""Pins of the oracle's processor-local ILU(0) (the paper's runs factor the rows each process owns, §6):
the ILU(0) of S_ff^(FS) without the blocks that couple cells of different subdomains, a subdomain being a
column of ty x tz cells in (y, z) spanning x.

  * one subdomain that holds the whole grid is the global ILU(0), bit for bit;
  * where every subdomain is a chain of cells (an x-pencil; a z-column or a y-row of a one-cell-wide grid),
    ILU(0) of each subdomain is its exact block LU factorisation, so the local stage is the exact solve with
    the block-diagonal part of S_ff^(FS) over the subdomains, formed densely with numpy;
  * a right-hand side supported in one subdomain gives a correction supported in that subdomain."""
import numpy as np
import pytest

import oracle
from tests.test_oracle_gs import dense_sff


def subdomain(s, ty, tz):
    c = np.arange(s.n_cells)
    y, z = (c // s.nx) % s.ny, c // (s.nx * s.ny)
    nby = (s.ny + ty - 1) // ty
    return y // ty + nby * (z // tz)


def local_exact(s, ty, tz, w):
    S = dense_sff(s)
    sub = np.repeat(subdomain(s, ty, tz), 2)
    S = np.where(sub[:, None] == sub[None, :], S, 0.0)
    return np.linalg.solve(S, w)


@pytest.mark.parametrize("cfg,kw", [(0, dict(nx=5, ny=4, nz=3)), (1, dict(nx=6, ny=7, nz=5))])
def test_one_subdomain_is_the_global_ilu(cfg, kw):
    s = oracle.System(oracle.default_params(cfg, **kw))
    Pg = oracle.Prec(s)
    Pl = oracle.Prec(s, oracle.default_prec_params(ilu_tile_y=s.ny, ilu_tile_z=s.nz))
    w = np.random.default_rng(3).standard_normal(2 * s.n_cells)
    assert np.array_equal(Pg.ilu_apply(w), Pl.ilu_apply(w))
    v = np.random.default_rng(4).standard_normal(s.n)
    assert np.array_equal(Pg.apply(v), Pl.apply(v))


@pytest.mark.parametrize("cfg,kw,ty,tz", [
    (0, dict(nx=5, ny=4, nz=3), 1, 1),     # x-pencils
    (1, dict(nx=6, ny=5, nz=4), 1, 1),
    (0, dict(nx=1, ny=4, nz=6), 1, 6),     # z-columns of a one-cell-wide grid
    (1, dict(nx=1, ny=5, nz=4), 1, 4),
    (0, dict(nx=1, ny=6, nz=3), 6, 1),     # y-rows of a one-cell-wide grid
    (1, dict(nx=1, ny=5, nz=4), 5, 1),
])
def test_chain_subdomains_are_solved_exactly(cfg, kw, ty, tz):
    s = oracle.System(oracle.default_params(cfg, **kw))
    P = oracle.Prec(s, oracle.default_prec_params(ilu_tile_y=ty, ilu_tile_z=tz))
    w = np.random.default_rng(5).standard_normal(2 * s.n_cells)
    expect = local_exact(s, ty, tz, w)
    got = P.ilu_apply(w)
    assert np.linalg.norm(got - expect) <= 1e-10 * np.linalg.norm(expect)
    # and the global ILU(0) is not that exact solve (the couplings between subdomains matter)
    g = oracle.Prec(s).ilu_apply(w)
    assert np.linalg.norm(g - expect) > 1e-6 * np.linalg.norm(expect)


@pytest.mark.parametrize("ty,tz", [(2, 2), (3, 1), (1, 2)])
def test_correction_stays_in_its_subdomain(ty, tz):
    s = oracle.System(oracle.default_params(1, nx=5, ny=6, nz=4))
    P = oracle.Prec(s, oracle.default_prec_params(ilu_tile_y=ty, ilu_tile_z=tz))
    sub = subdomain(s, ty, tz)
    rng = np.random.default_rng(6)
    for d in (0, sub.max() // 2, sub.max()):
        w = np.where(np.repeat(sub, 2) == d, rng.standard_normal(2 * s.n_cells), 0.0)
        dz = P.ilu_apply(w)
        assert np.any(dz[np.repeat(sub, 2) == d] != 0.0)
        assert np.all(dz[np.repeat(sub, 2) != d] == 0.0)
