"""The request server (batched and served workloads) through the C ABI (needs a GB300): every
request's result is the same alone and in the mix, and admission keeps the in-flight device bytes
under the budget."""
import numpy as np
import pytest

import paper_1812_05540_gb300 as ps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [(12, 10, 6), (16, 16, 8), (20, 14, 9), (9, 9, 5), (24, 20, 10), (8, 8, 4)]


@pytest.fixture(scope="module")
def systems():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    out = []
    for k, (nx, ny, nz) in enumerate(SIZES):
        gp = ps.ps_gen_default(1, nx=nx, ny=ny, nz=nz, seed=3000 + k)
        sp = ps.ps_generate(gp)
        n = sp.contents.n
        rhs2 = torch.from_numpy(np.random.default_rng(k).uniform(-1, 1, n)).cuda()
        out.append((sp, rhs2))
    torch.cuda.synchronize()
    yield out
    for sp, _ in out:
        ps.ps_system_free(sp)


def _params():
    return ps.ps_params_default(precision=ps.PS_MIXED_FP32)


def _alone(sp, rhs_ptrs):
    s = sp.contents
    h = ps.ps_setup(s.jac, s.grid, _params())
    xs = []
    try:
        for r in rhs_ptrs:
            x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
            _, st = ps.ps_solve(h, r, x.data_ptr(), 1e-8)
            assert st.true_relres <= 1e-8
            xs.append(x.cpu().numpy())
    finally:
        ps.ps_free(h)
    return xs


def test_requests_give_the_same_result_alone_and_in_the_mix(systems):
    alone = [_alone(sp, [sp.contents.rhs, r2.data_ptr()]) for sp, r2 in systems]
    srv = ps.ps_server_create(3, 0, _params())
    xs, tickets = [], []
    try:
        for sp, r2 in systems:
            s = sp.contents
            x = [torch.zeros(s.n, dtype=torch.float64, device="cuda") for _ in range(2)]
            xs.append(x)
            tickets.append(ps.ps_server_submit(srv, s.jac, s.grid, [s.rhs, r2.data_ptr()],
                                               [x[0].data_ptr(), x[1].data_ptr()], 1e-8))
        infos = []
        for t in tickets:
            st, info = ps.ps_server_wait(srv, t)
            assert st == ps.PS_OK
            infos.append(info)
        info = ps.ps_server_info_get(srv)
    finally:
        ps.ps_server_destroy(srv)
    assert info.completed == len(systems) and info.max_inflight_requests >= 2
    for (xa, xm, inf) in zip(alone, xs, infos):
        assert inf.worst_relres <= 1e-8 and inf.t_arrival <= inf.t_start <= inf.t_end
        for a, m in zip(xa, xm):
            m = m.cpu().numpy()
            assert np.linalg.norm(m - a) <= 1e-10 * np.linalg.norm(a)


def test_admission_keeps_inflight_bytes_under_budget(systems):
    p = _params()
    est = [ps.ps_setup_bytes_estimate(sp.contents.jac, sp.contents.grid, p) for sp, _ in systems]
    budget = int(1.2 * max(est))
    srv = ps.ps_server_create(4, budget, p)
    xs, tickets = [], []
    try:
        for sp, _ in systems:
            s = sp.contents
            x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
            xs.append(x)
            tickets.append(ps.ps_server_submit(srv, s.jac, s.grid, [s.rhs], [x.data_ptr()], 1e-8))
        for t in tickets:
            st, inf = ps.ps_server_wait(srv, t)
            assert st == ps.PS_OK and inf.worst_relres <= 1e-8
        info = ps.ps_server_info_get(srv)
    finally:
        ps.ps_server_destroy(srv)
    assert 0 < info.max_inflight_bytes <= budget


def test_request_above_budget_is_refused(systems):
    sp, _ = systems[4]
    s = sp.contents
    srv = ps.ps_server_create(1, 1 << 20, _params())
    try:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        with pytest.raises(ps.PsError) as e:
            ps.ps_server_submit(srv, s.jac, s.grid, [s.rhs], [x.data_ptr()], 1e-8)
        assert e.value.status == ps.PS_ERR_BUDGET
    finally:
        ps.ps_server_destroy(srv)
