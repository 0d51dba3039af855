"""The OpenMP build of the oracle (same source, -fopenmp, row loops on all host cores) returns the same
bits as the single-threaded build: generator, both AMG hierarchies, Algorithm 1 and the FGMRES solve.
The CPU baseline of the bench times the OpenMP build, so its numbers are those of the parity reference."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def both():
    try:
        oracle.build(openmp=True)
    except Exception as e:  # a host without an OpenMP runtime keeps the serial build only
        pytest.skip("no OpenMP build: %s" % e)
    out = {}
    for omp in (False, True):
        oracle.select(omp)
        try:
            s = oracle.System(oracle.default_params(1, nx=24, ny=20, nz=10))
            P = oracle.Prec(s)
        finally:
            oracle.select(False)
        out[omp] = (s, P)
    return out


def test_openmp_build_uses_threads():
    oracle.build(openmp=True)
    assert oracle.num_threads(False) == 1
    assert oracle.num_threads(True) >= 1


def test_generator_bitwise(both):
    (s0, _), (s1, _) = both[False], both[True]
    for name in ("uu", "uf", "fu", "ff"):
        for a, b in zip(s0.blocks[name], s1.blocks[name]):
            assert np.array_equal(a, b), name
    assert np.array_equal(s0.rhs, s1.rhs) and np.array_equal(s0.d_fs, s1.d_fs)


def test_hierarchies_bitwise(both):
    P0, P1 = both[False][1], both[True][1]
    for which in (0, 1):
        assert P0.nlevels(which) == P1.nlevels(which) > 1
        for l in range(P0.nlevels(which)):
            for a, b in zip(P0.level(which, l), P1.level(which, l)):
                assert np.array_equal(a, b), (which, l)
            if l < P0.nlevels(which) - 1:
                assert np.array_equal(P0.aggregates(which, l)[0], P1.aggregates(which, l)[0])
                for a, b in zip(P0.prolongator(which, l), P1.prolongator(which, l)):
                    assert np.array_equal(a, b), (which, l)
    assert np.array_equal(P0.spp()[2], P1.spp()[2])
    assert np.array_equal(P0.ilu_dinv(), P1.ilu_dinv())


def test_apply_and_solve_bitwise(both):
    (s0, P0), (s1, P1) = both[False], both[True]
    v = np.random.default_rng(3).standard_normal(s0.n)
    assert np.array_equal(P0.apply(v), P1.apply(v))
    assert np.array_equal(s0.spmv(v), s1.spmv(v))
    x0, st0 = P0.fgmres(tol=1e-8)
    x1, st1 = P1.fgmres(tol=1e-8)
    assert st0.iters == st1.iters and st0.true_relres == st1.true_relres
    assert np.array_equal(x0, x1)
