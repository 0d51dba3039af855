"""The C ABI library builds, loads and exports every entry point declared in
include/ps.h (no compute: no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ps_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1812_05540_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_abi():
    import paper_1812_05540_gb300 as ps
    for n in ("ps_setup", "ps_setup_flow", "ps_solve", "ps_free", "ps_generate", "ps_system_free", "ps_spmv",
              "ps_apply_prec", "ps_strerror", "ps_params_default", "ps_gen_default", "ps_server_create",
              "ps_server_submit", "ps_server_wait", "ps_server_destroy", "ps_setup_bytes_estimate",
              "ps_assemble_at", "ps_residual_at", "ps_newton", "ps_newton_params_default"):
        assert callable(getattr(ps, n))


def test_struct_layouts_match_header():
    # sizes of the ctypes mirrors against the C structs, via a tiny compiled probe
    import subprocess
    import tempfile
    import paper_1812_05540_gb300 as ps
    probe = r'''
#include <stdio.h>
#include "ps.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(ps_grid), sizeof(ps_bsr),
         sizeof(ps_jacobian), sizeof(ps_params), sizeof(ps_stats), sizeof(ps_gen_params), sizeof(ps_system),
         sizeof(ps_server_params), sizeof(ps_request_info), sizeof(ps_server_info), sizeof(ps_newton_params),
         sizeof(ps_newton_stats));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(v) for v in subprocess.check_output([exe]).split()]
    mine = [ctypes.sizeof(t) for t in (ps.ps_grid, ps.ps_bsr, ps.ps_jacobian, ps.ps_params, ps.ps_stats,
                                       ps.ps_gen_params, ps.ps_system, ps.ps_server_params, ps.ps_request_info,
                                       ps.ps_server_info, ps.ps_newton_params, ps.ps_newton_stats)]
    assert sizes == mine
