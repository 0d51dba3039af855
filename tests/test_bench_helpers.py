"""Host arithmetic behind the bench's roofline fields (no GPU): the Arnoldi step indices of a solve, the
flop and compulsory-byte counts of one modified Gram-Schmidt step, the derived FP64 peak, and the DRAM
traffic records that are used only while the profiled source is unchanged."""
import hashlib
import json
import os

import bench


def mgs_step_counts(n, j):
    """Flops and distinct 8-byte words read / written by one modified Gram-Schmidt step, counted on a
    literal implementation: h_k = v_k . w, w -= h_k v_k for k = 0..j, then ||w|| and w /= ||w||."""
    flops = 0
    reads, writes = set(), set()
    for k in range(j + 1):
        for r in range(n):          # dot
            flops += 2
            reads.add(("v", k, r)); reads.add(("w", r))
        for r in range(n):          # update
            flops += 2
            reads.add(("v", k, r)); writes.add(("w", r))
    for r in range(n):              # norm
        flops += 2
    for r in range(n):              # scaling
        flops += 1
        writes.add(("w", r))
    return flops, len(reads), len(writes)


def test_mgs_flops_match_a_counted_step():
    for n, j in ((5, 0), (7, 3), (4, 9)):
        flops, _, _ = mgs_step_counts(n, j)
        assert bench.mgs_flops(n, j) == flops


def test_mgs_bytes_are_each_word_moved_once():
    for n, j in ((5, 0), (7, 3), (4, 9)):
        _, nread, nwrite = mgs_step_counts(n, j)
        assert bench.mgs_bytes_alg(n, j) == 8 * (nread + nwrite)


def test_arnoldi_steps_of_full_and_partial_cycles():
    assert bench.arnoldi_steps(93, 0, 100) == list(range(93))
    js = bench.arnoldi_steps(250, 2, 100)
    assert len(js) == 250 and js[:100] == list(range(100)) and js[100:200] == list(range(100))
    assert js[200:] == list(range(50))
    assert bench.arnoldi_steps(0, 0, 100) == [0]


def test_fp64_peak_from_units_and_clock():
    tf, src = bench.fp64_peak_tflops(152, {"sm_max_mhz": 2070.0})
    assert abs(tf - 152 * 2 * 2 * 2.07e9 / 1e12) < 1e-12  # 2 FP64 FMA per SM and clock
    assert "152 SMs" in src


def test_traffic_records_are_dropped_once_the_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"k_mgs": {"source": "kernel.cu", "source_sha1": hashlib.sha1(src.read_bytes()).hexdigest(),
                     "bytes_per_row_per_column": 17.0},
           "spmv": {"source": "kernel.cu", "source_sha1": "0" * 40, "bytes_per_launch": 3.5e9}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    t = bench.load_traffic()
    assert "k_mgs" in t and "spmv" not in t
    # scaled to a solve's steps: mean over j of bytes_per_row_per_column * n * (j + 3)
    n, js = 1000, [0, 1, 2]
    assert bench.traffic_per_launch(t, "k_mgs", n, js) == sum(17.0 * n * (j + 3) for j in js) / 3
    assert bench.traffic_per_launch(t, "spmv", n, None) is None
    src.write_text("__global__ void k() { }\n")
    assert bench.load_traffic() == {}


def test_vcycle_bytes_two_level_hand_count():
    # level 0: 10 rows, CSR with 28 entries, nc = 1, FP32 values; P has 12 entries onto 3 coarse rows;
    # level 1 (coarsest): 3 rows, dense FP64 inverse
    L0 = (10, 28, 3, 12, 0, 4, 4, 0)
    L1 = (3, 9, 0, 0, 0, 4, 4, 1)
    vec0, vec1 = 10 * 4, 3 * 4
    op = 28 * (4 + 4) + 4 * 11                     # values + column indices + row pointers, per pass
    # 4 operator passes; vectors: fused first two pre steps 4 (b, D^{-1}/theta, D in; x out), residual 3,
    # first post step 5 (x, b, D in; x, d out), second post step 5 (x, b, D, d in; x out)
    level0 = 4 * op + 17 * vec0
    level0 += 12 * 8 + 4 * 11 + vec1 + 2 * vec0    # x += P e
    level0 += 12 * 8 + 4 * 4 + vec0 + vec1         # b_c = R r
    level1 = 3 * 3 * 8 + 2 * vec1                  # dense inverse + b, x
    assert bench.vcycle_bytes([L0, L1], 1) == level0 + level1


def test_vcycle_bytes_stencil_level_has_no_indices():
    # a 7-point stencil level reads 7 values per row and no column index or row pointer per pass
    L0 = (100, 500, 10, 300, 7, 4, 4, 0)
    L0_csr = (100, 500, 10, 300, 0, 4, 4, 0)
    L1 = (10, 30, 0, 0, 0, 4, 4, 1)
    d = bench.vcycle_bytes([L0_csr, L1], 1) - bench.vcycle_bytes([L0, L1], 1)
    assert d == 4 * ((500 * 8 + 4 * 101) - 7 * 4 * 100)
