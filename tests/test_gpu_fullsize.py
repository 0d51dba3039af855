"""The 60x220x85 workload (5,722,098 DoF) that bench.py times, checked at full size (needs a GB300).
The oracle cannot solve it in test time, so the checks are the ones that hold at any size: the GPU
generator's Jacobian equals the oracle's on sampled rows, and the mixed-precision solve reaches a
true relative residual <= 1e-8 recomputed with the oracle's own FP64 SpMV on the oracle's Jacobian."""
import numpy as np
import pytest

import oracle
import paper_1812_05540_gb300 as ps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_full_size_workload_matches_oracle_and_converges():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from tests import _gpu as g
    torch.cuda.set_device(0)
    ogp = oracle.default_params(2)
    osys = oracle.System(ogp)
    sp = ps.ps_generate(g.gen_params_like(ogp))
    try:
        s = sp.contents
        assert s.n == osys.n == 5722098
        # sampled block rows of every Jacobian block: same pattern, values within 1e-13 of the row scale
        rng = np.random.default_rng(11)
        for name, bs, blk, nrow in (("uu", 9, s.jac.A_uu, osys.n_nodes), ("uf", 6, s.jac.A_uf, osys.n_nodes),
                                    ("fu", 6, s.jac.A_fu, osys.n_cells), ("ff", 4, s.jac.A_ff, osys.n_cells)):
            orp, oci, ov = osys.blocks[name]
            rp = g.dev_to_numpy(blk.rowptr, nrow + 1, np.int64)
            assert np.array_equal(rp, orp), name
            for r in rng.integers(0, nrow, 200):
                a, b = int(rp[r]), int(rp[r + 1])
                ci = g.dev_to_numpy(blk.colind + 4 * a, b - a, np.int32)
                v = g.dev_to_numpy(blk.val + 8 * a * bs, (b - a) * bs, np.float64)
                assert np.array_equal(ci, oci[a:b]), (name, r)
                ref = ov[a * bs:b * bs]
                assert np.abs(v - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1e-300), (name, r)
        # the bench's solve: mixed precision, FGMRES(100), tol 1e-8
        p = ps.ps_params_default(precision=ps.PS_MIXED_FP32)
        h = ps.ps_setup(s.jac, s.grid, p)
        try:
            x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
            _, st = ps.ps_solve(h, s.rhs, x.data_ptr(), 1e-8)
        finally:
            ps.ps_free(h)
        xs = x.cpu().numpy()
        relres = np.linalg.norm(osys.rhs - osys.spmv(xs)) / np.linalg.norm(osys.rhs)
        assert relres <= 1e-8 and abs(relres - st.true_relres) <= 1e-10, (relres, st.true_relres)
    finally:
        ps.ps_system_free(sp)
