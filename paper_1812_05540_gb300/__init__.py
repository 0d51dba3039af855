"""Python binding of libps, the GB300 solver for linearised multiphase
poromechanics Jacobians under the two-stage preconditioner of arXiv 1812.05540.

Argument marshalling only: every step of the setup and solve runs in the CUDA
library (include/ps.h).  Device memory is passed as raw pointers
(``tensor.data_ptr()``); PyTorch is used by callers for allocation and streams.
Importing this module loads ``_build/libps.so`` and raises if it is missing;
there is no CPU fallback.
"""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libps.so")

PS_OK, PS_ERR_INVALID, PS_ERR_OOM, PS_ERR_CUDA, PS_ERR_NOT_CONVERGED, PS_ERR_BREAKDOWN, PS_ERR_NAN, \
    PS_ERR_TIMEOUT, PS_ERR_BUDGET = range(9)
PS_FP64, PS_MIXED_FP32, PS_MIXED_BF16P = 0, 1, 2
PS_SMOOTH_L1JACOBI, PS_SMOOTH_CHEBYSHEV = 0, 1
PS_ILU_LEVEL_LAUNCH, PS_ILU_PENCIL = 0, 1
PS_ORTHO_MGS, PS_ORTHO_CGS2 = 0, 1
PS_LOCAL_ILU0, PS_LOCAL_HBGS = 0, 1
PS_ILU_GLOBAL, PS_ILU_LOCAL = 0, 1
PS_MECH_SDC, PS_MECH_RBM = 0, 1
PS_ILU_TILE_Y, PS_ILU_TILE_Z = 16, 8
PS_CPR_QUASI_IMPES, PS_CPR_TRUE_IMPES = 0, 1
PS_SOLVER_FGMRES, PS_SOLVER_RICHARDSON = 0, 1
PS_FS_GIVEN, PS_FS_RSL = 0, 1
PS_FIELDS_LOGNORMAL, PS_FIELDS_LAYERED, PS_FIELDS_CHANNELS, PS_FIELDS_HOMOGENEOUS = range(4)
PS_GEN_GRAVITY, PS_GEN_DIRICHLET, PS_GEN_SCALE, PS_GEN_ACCUM, PS_GEN_FLUX, PS_GEN_FLUX_SAT, PS_GEN_COUPLING = \
    (1 << i for i in range(7))
PS_GEN_ALL = 0x7F
PS_GEN_WELLS = 1 << 7  # Peaceman wells (an option; not in PS_GEN_ALL)


class ps_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double)]


class ps_bsr(C.Structure):
    _fields_ = [("n_brow", C.c_int64), ("n_bcol", C.c_int64), ("nnzb", C.c_int64), ("br", C.c_int32),
                ("bc", C.c_int32), ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("val", C.c_void_p)]


class ps_jacobian(C.Structure):
    _fields_ = [("A_uu", ps_bsr), ("A_uf", ps_bsr), ("A_fu", ps_bsr), ("A_ff", ps_bsr),
                ("d_fs", C.c_void_p), ("dirichlet_u", C.c_void_p)]


class ps_params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("restart", C.c_int32), ("max_iters", C.c_int32),
                ("smoother", C.c_int32), ("pre", C.c_int32), ("post", C.c_int32), ("cheb_degree", C.c_int32),
                ("cheb_ratio", C.c_double), ("theta_u", C.c_double), ("theta_p", C.c_double),
                ("coarse_max_u", C.c_int32), ("coarse_max_p", C.c_int32), ("max_levels", C.c_int32),
                ("ilu_mode", C.c_int32), ("spin_limit", C.c_int64), ("host_ptrs", C.c_int32),
                ("hbm_budget", C.c_int64), ("stream", C.c_void_p), ("test_stall_wave", C.c_int32),
                ("ortho", C.c_int32), ("test_stall_gs", C.c_int32), ("ortho_sweep", C.c_int32),
                ("local_stage", C.c_int32), ("local_sweeps", C.c_int32), ("cpr_reduction", C.c_int32),
                ("solver", C.c_int32), ("fs_mode", C.c_int32), ("vcycle_tail", C.c_int32),
                ("pdl", C.c_int32), ("ilu_scope", C.c_int32), ("mech_amg", C.c_int32), ("autotune", C.c_int32)]


class ps_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("true_relres", C.c_double),
                ("est_relres", C.c_double), ("ms_setup_u", C.c_float), ("ms_setup_f", C.c_float),
                ("ms_solve", C.c_float), ("bytes_model", C.c_int64), ("handle_bytes", C.c_int64),
                ("levels_u", C.c_int32), ("levels_p", C.c_int32), ("ms_prec", C.c_float), ("ms_spmv", C.c_float),
                ("ms_orth", C.c_float), ("reorth", C.c_int32), ("ms_vcycle_u", C.c_float),
                ("ms_flow24", C.c_float), ("ms_vcycle_p", C.c_float), ("ms_ilu", C.c_float),
                ("ms_copy_in", C.c_float)]


class ps_server_params(C.Structure):
    _fields_ = [("slots", C.c_int32), ("hbm_budget", C.c_int64), ("params", ps_params)]


class ps_request_info(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("status", C.c_int32), ("nrhs", C.c_int32), ("iters", C.c_int32),
                ("worst_relres", C.c_double), ("t_arrival", C.c_double), ("t_start", C.c_double),
                ("t_end", C.c_double), ("bytes", C.c_int64)]


class ps_server_info(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("max_inflight_bytes", C.c_int64),
                ("max_inflight_requests", C.c_int64)]


class ps_newton_params(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_newton", C.c_int32), ("forcing", C.c_int32), ("eta_fixed", C.c_double),
                ("ew_gamma", C.c_double), ("ew_omega", C.c_double), ("ew_eta0", C.c_double),
                ("ew_eta_max", C.c_double), ("max_backtracks", C.c_int32)]


class ps_newton_stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("linear_iters", C.c_int32), ("backtracks", C.c_int32),
                ("converged", C.c_int32), ("rnorm", C.c_double * 33), ("eta", C.c_double * 32),
                ("lin_iters", C.c_int32 * 32), ("ms_assemble", C.c_float), ("ms_linear", C.c_float),
                ("ms_total", C.c_float)]


PS_FORCING_FIXED, PS_FORCING_EW = 0, 1


class ps_gen_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("h", C.c_double),
                ("seed", C.c_uint64), ("field_kind", C.c_int32), ("flags", C.c_uint32),
                ("dt", C.c_double), ("biot", C.c_double), ("c_w", C.c_double), ("c_nw", C.c_double),
                ("c_r", C.c_double), ("mu_w", C.c_double), ("mu_nw", C.c_double), ("rho_w0", C.c_double),
                ("rho_nw0", C.c_double), ("rho_s0", C.c_double), ("s_wr", C.c_double), ("s_nwr", C.c_double),
                ("grav", C.c_double), ("p_ref", C.c_double), ("dp_amp", C.c_double), ("corey", C.c_double),
                ("E0", C.c_double), ("nu0", C.c_double), ("kappa0", C.c_double), ("phi0", C.c_double),
                ("sw0", C.c_double), ("fs_modulus", C.c_int32)]


_PD = C.POINTER(C.c_double)


class ps_system(C.Structure):
    _fields_ = [("jac", ps_jacobian), ("grid", ps_grid), ("rhs", C.c_void_p), ("n_nodes", C.c_int64),
                ("n_cells", C.c_int64), ("n_u", C.c_int64), ("n_f", C.c_int64), ("n", C.c_int64),
                ("alpha_u", C.c_double), ("alpha_f", C.c_double),
                ("E", C.c_void_p), ("nu", C.c_void_p), ("kh", C.c_void_p), ("kv", C.c_void_p),
                ("phi0", C.c_void_p), ("sw", C.c_void_p), ("p", C.c_void_p)]


_lib = None


def lib():
    """Load libps.so (built in-tree by __graft_entry__.build()); raises when absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libps.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        H = C.c_void_p
        L.ps_params_default.argtypes = [C.POINTER(ps_params)]
        L.ps_params_default.restype = None
        L.ps_setup.argtypes = [C.POINTER(ps_jacobian), C.POINTER(ps_grid), C.POINTER(ps_params), C.POINTER(H)]
        L.ps_setup_flow.argtypes = [H, C.POINTER(ps_jacobian)]
        L.ps_set_test_stall.argtypes = [H, C.c_int32]
        L.ps_set_test_stall_gs.argtypes = [H, C.c_int32]
        L.ps_solve.argtypes = [H, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(ps_stats)]
        L.ps_spmv.argtypes = [H, C.c_void_p, C.c_void_p]
        L.ps_apply_prec.argtypes = [H, C.c_void_p, C.c_void_p]
        L.ps_amg_nlevels.argtypes = [H, C.c_int32]
        L.ps_amg_nlevels.restype = C.c_int32
        L.ps_amg_level_info.argtypes = [H, C.c_int32, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                        C.POINTER(C.c_int64)]
        L.ps_setup_batch.argtypes = [C.c_int32, C.POINTER(ps_jacobian), C.POINTER(ps_grid), C.POINTER(ps_params),
                                     C.POINTER(H)]
        L.ps_solve_batch.argtypes = [C.c_int32, C.POINTER(H), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                     C.c_double, C.POINTER(ps_stats)]
        L.ps_amg_level_shape.argtypes = [H, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]
        L.ps_rbm_nlevels.argtypes = [H]
        L.ps_rbm_level_shape.argtypes = [H, C.c_int32, C.POINTER(C.c_int64)]
        L.ps_rbm_level_copy.argtypes = [H, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.ps_rbm_prolongator_copy.argtypes = [H, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
        L.ps_amg_level_copy.argtypes = [H, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.ps_flow_copy.argtypes = [H, C.c_void_p, C.c_void_p]
        L.ps_free.argtypes = [H]
        L.ps_free.restype = None
        L.ps_gen_default.argtypes = [C.POINTER(ps_gen_params), C.c_int32]
        L.ps_gen_default.restype = None
        L.ps_generate.argtypes = [C.POINTER(ps_gen_params), C.c_void_p, C.POINTER(C.POINTER(ps_system))]
        L.ps_system_free.argtypes = [C.POINTER(ps_system)]
        L.ps_system_free.restype = None
        L.ps_assemble_at.argtypes = [C.POINTER(ps_gen_params), C.POINTER(ps_system), C.c_void_p, C.c_void_p,
                                     C.c_void_p]
        L.ps_residual_at.argtypes = [C.POINTER(ps_gen_params), C.POINTER(ps_system), C.c_void_p, C.c_void_p,
                                     C.c_void_p]
        L.ps_newton_params_default.argtypes = [C.POINTER(ps_newton_params)]
        L.ps_newton_params_default.restype = None
        L.ps_newton_eta.argtypes = [C.POINTER(ps_newton_params), C.c_int32, C.c_double, C.c_double, C.c_double,
                                    C.c_double]
        L.ps_newton_eta.restype = C.c_double
        L.ps_newton.argtypes = [C.POINTER(ps_gen_params), C.POINTER(ps_params), C.POINTER(ps_newton_params),
                                C.c_void_p, C.POINTER(ps_newton_stats)]
        L.ps_residual_noalloc.argtypes = [C.POINTER(ps_jacobian), C.POINTER(ps_grid), C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
        S = C.c_void_p
        L.ps_setup_bytes_estimate.argtypes = [C.POINTER(ps_jacobian), C.POINTER(ps_grid), C.POINTER(ps_params)]
        L.ps_setup_bytes_estimate.restype = C.c_int64
        L.ps_server_create.argtypes = [C.POINTER(ps_server_params), C.POINTER(S)]
        L.ps_server_clock.argtypes = [S]
        L.ps_server_clock.restype = C.c_double
        L.ps_server_submit.argtypes = [S, C.POINTER(ps_jacobian), C.POINTER(ps_grid), C.c_int32,
                                       C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_double, C.c_double,
                                       C.POINTER(C.c_uint64)]
        L.ps_server_wait.argtypes = [S, C.c_uint64, C.POINTER(ps_request_info)]
        L.ps_server_info_get.argtypes = [S, C.POINTER(ps_server_info)]
        L.ps_server_destroy.argtypes = [S]
        L.ps_server_destroy.restype = None
        L.ps_launch_count.argtypes = []
        L.ps_launch_count.restype = C.c_int64
        L.ps_pool_bytes.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.ps_alloc_count.argtypes = []
        L.ps_alloc_count.restype = C.c_int64
        L.ps_strerror.argtypes = [C.c_int]
        L.ps_strerror.restype = C.c_char_p
        _lib = L
    return _lib


class PsError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s: %s (status %d)" % (what, lib().ps_strerror(status).decode(), status))
        self.status = status


def _check(status, what):
    if status != PS_OK:
        raise PsError(status, what)


def ps_strerror(status):
    return lib().ps_strerror(status).decode()


def ps_launch_count():
    return lib().ps_launch_count()


def ps_alloc_count():
    return lib().ps_alloc_count()


def ps_pool_bytes():
    """(reserved, used) device bytes of the library's memory pool on the current device."""
    r, u = C.c_int64(), C.c_int64()
    _check(lib().ps_pool_bytes(C.byref(r), C.byref(u)), "ps_pool_bytes")
    return r.value, u.value


def ps_params_default(**kw):
    p = ps_params()
    lib().ps_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def ps_gen_default(config=0, **kw):
    gp = ps_gen_params()
    lib().ps_gen_default(C.byref(gp), config)
    for k, v in kw.items():
        setattr(gp, k, v)
    return gp


def ps_generate(gp, stream=None):
    """Seeded synthetic Jacobian on the device; returns a ctypes ps_system pointer."""
    out = C.POINTER(ps_system)()
    _check(lib().ps_generate(C.byref(gp), stream, C.byref(out)), "ps_generate")
    return out


def ps_system_free(sys_ptr):
    lib().ps_system_free(sys_ptr)


def ps_assemble_at(gp, sys_ptr, dx_ptr, r_ptr, stream=None):
    """Jacobian values of the generated system (and the residual into r_ptr, may be 0) at base + dx"""
    _check(lib().ps_assemble_at(C.byref(gp), sys_ptr, dx_ptr, r_ptr or None, stream), "ps_assemble_at")


def ps_residual_at(gp, sys_ptr, dx_ptr, r_ptr, stream=None):
    _check(lib().ps_residual_at(C.byref(gp), sys_ptr, dx_ptr, r_ptr, stream), "ps_residual_at")


def ps_newton_params_default(**kw):
    p = ps_newton_params()
    lib().ps_newton_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def ps_newton_eta(np_, k, rk, rkm1, eta_prev, r0):
    return lib().ps_newton_eta(C.byref(np_), k, rk, rkm1, eta_prev, r0)


def ps_newton(gp, lin, np_, x_ptr, raise_on_error=True):
    """Newton's method for one time step; returns (status, stats dict)"""
    st = ps_newton_stats()
    status = lib().ps_newton(C.byref(gp), C.byref(lin), C.byref(np_), x_ptr, C.byref(st))
    if raise_on_error and status != PS_OK:
        _check(status, "ps_newton")
    k = st.newton_iters
    return status, dict(newton_iters=k, linear_iters=st.linear_iters, backtracks=st.backtracks,
                        converged=bool(st.converged), rnorm=list(st.rnorm[:k + 1]), eta=list(st.eta[:k]),
                        lin_iters=list(st.lin_iters[:k]), ms_assemble=st.ms_assemble, ms_linear=st.ms_linear,
                        ms_total=st.ms_total)


def ps_setup(jac, grid, params):
    h = C.c_void_p()
    _check(lib().ps_setup(C.byref(jac), C.byref(grid), C.byref(params), C.byref(h)), "ps_setup")
    return h


def ps_set_test_stall(h, wave_cta_plus_one):
    _check(lib().ps_set_test_stall(h, wave_cta_plus_one), "ps_set_test_stall")


def ps_set_test_stall_gs(h, cta_plus_one):
    _check(lib().ps_set_test_stall_gs(h, cta_plus_one), "ps_set_test_stall_gs")


def ps_setup_flow(h, jac):
    _check(lib().ps_setup_flow(h, C.byref(jac)), "ps_setup_flow")


def ps_solve(h, rhs_ptr, x_ptr, tol, raise_on_error=True):
    """Returns (status, ps_stats); raises unless raise_on_error is False."""
    st = ps_stats()
    s = lib().ps_solve(h, rhs_ptr, x_ptr, tol, C.byref(st))
    if raise_on_error:
        _check(s, "ps_solve")
    return s, st


def ps_spmv(h, x_ptr, y_ptr):
    _check(lib().ps_spmv(h, x_ptr, y_ptr), "ps_spmv")


def ps_apply_prec(h, v_ptr, z_ptr):
    _check(lib().ps_apply_prec(h, v_ptr, z_ptr), "ps_apply_prec")


def ps_residual_noalloc(jac, grid, x_ptr, b_ptr, r_ptr, rnorm2_ptr, stream=None):
    """r = b - A x and ||r||^2 with no device allocation (all pointers device memory)."""
    _check(lib().ps_residual_noalloc(C.byref(jac), C.byref(grid), x_ptr, b_ptr, r_ptr, rnorm2_ptr, stream),
           "ps_residual_noalloc")


def ps_free(h):
    lib().ps_free(h)


def ps_amg_nlevels(h, which):
    return lib().ps_amg_nlevels(h, which)


def ps_amg_level_info(h, which, level):
    n, nnz, nagg = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().ps_amg_level_info(h, which, level, C.byref(n), C.byref(nnz), C.byref(nagg)), "ps_amg_level_info")
    return n.value, nnz.value, nagg.value


def ps_setup_batch(jacs, grids, params):
    """Handles of len(jacs) systems set up together; each handle owns a stream of its own."""
    n = len(jacs)
    JA = (ps_jacobian * n)(*jacs)
    GA = (ps_grid * n)(*grids)
    out = (C.c_void_p * n)()
    _check(lib().ps_setup_batch(n, JA, GA, C.byref(params), out), "ps_setup_batch")
    return list(out)


def ps_solve_batch(handles, rhs_ptrs, x_ptrs, tol, raise_on_error=True):
    """Lockstep FGMRES of every handle; returns (status, [ps_stats])."""
    n = len(handles)
    HA = (C.c_void_p * n)(*handles)
    RA = (C.c_void_p * n)(*rhs_ptrs)
    XA = (C.c_void_p * n)(*x_ptrs)
    st = (ps_stats * n)()
    s = lib().ps_solve_batch(n, HA, RA, XA, tol, st)
    if raise_on_error:
        _check(s, "ps_solve_batch")
    return s, list(st)


def ps_amg_level_shape(h, which, level):
    """(rows, entries, next rows, P entries, stencil slots, operator value bytes, P/R value bytes, coarsest)"""
    out = (C.c_int64 * 8)()
    _check(lib().ps_amg_level_shape(h, which, level, out), "ps_amg_level_shape")
    return tuple(int(v) for v in out)


def ps_amg_level_copy(h, which, level):
    """Host copies (numpy) of a level operator and its aggregates."""
    import numpy as np
    n, nnz, _ = ps_amg_level_info(h, which, level)
    nc = 3 if which == 0 else 1
    rp = np.empty(n + 1, np.int64)
    ci = np.empty(max(nnz, 1), np.int32)
    v = np.empty(max(nnz, 1) * nc)
    agg = np.empty(n, np.int32)
    _check(lib().ps_amg_level_copy(h, which, level, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, agg.ctypes.data),
           "ps_amg_level_copy")
    return rp, ci[:nnz], v[:nnz * nc].reshape(nnz, nc), agg


def ps_rbm_nlevels(h):
    return lib().ps_rbm_nlevels(h)


def ps_rbm_level_shape(h, level):
    out = (C.c_int64 * 6)()
    _check(lib().ps_rbm_level_shape(h, level, out), "ps_rbm_level_shape")
    return dict(n=out[0], b=out[1], nnzb=out[2], nagg=out[3], pnnzb=out[4], coarsest=bool(out[5]))


def ps_rbm_level_copy(h, level):
    """Host copies (numpy) of a rigid-body-mode level: rowptr, colind, blocks (nnzb, b, b), aggregates."""
    import numpy as np
    sh = ps_rbm_level_shape(h, level)
    n, b, nnz = sh["n"], sh["b"], sh["nnzb"]
    rp = np.empty(n + 1, np.int64)
    ci = np.empty(max(nnz, 1), np.int32)
    v = np.empty(max(nnz, 1) * b * b)
    agg = np.empty(n, np.int32)
    _check(lib().ps_rbm_level_copy(h, level, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, agg.ctypes.data),
           "ps_rbm_level_copy")
    return rp, ci[:nnz], v[:nnz * b * b].reshape(nnz, b, b), agg


def ps_rbm_prolongator_copy(h, level):
    import numpy as np
    sh = ps_rbm_level_shape(h, level)
    n, b, nnz = sh["n"], sh["b"], sh["pnnzb"]
    rp = np.empty(n + 1, np.int64)
    ci = np.empty(max(nnz, 1), np.int32)
    v = np.empty(max(nnz, 1) * b * 6)
    _check(lib().ps_rbm_prolongator_copy(h, level, rp.ctypes.data, ci.ctypes.data, v.ctypes.data),
           "ps_rbm_prolongator_copy")
    return rp, ci[:nnz], v[:nnz * b * 6].reshape(nnz, b, 6)


def ps_flow_copy(h, nnzb, ncells):
    import numpy as np
    spp = np.empty(nnzb)
    dinv = np.empty(4 * ncells)
    _check(lib().ps_flow_copy(h, spp.ctypes.data, dinv.ctypes.data), "ps_flow_copy")
    return spp, dinv


def bsr(n_brow, n_bcol, br, bc, rowptr, colind, val, nnzb):
    """ps_bsr from three pointers (ints)."""
    return ps_bsr(n_brow, n_bcol, nnzb, br, bc, rowptr, colind, val)


# ---- request server ----
def ps_setup_bytes_estimate(jac, grid, params):
    return lib().ps_setup_bytes_estimate(C.byref(jac), C.byref(grid), C.byref(params))


def ps_server_create(slots, hbm_budget=0, params=None):
    sp = ps_server_params(slots, hbm_budget, params if params is not None else ps_params_default())
    s = C.c_void_p()
    _check(lib().ps_server_create(C.byref(sp), C.byref(s)), "ps_server_create")
    return s


def ps_server_clock(s):
    return lib().ps_server_clock(s)


def ps_server_submit(s, jac, grid, rhs_ptrs, x_ptrs, tol, t_arrival=-1.0):
    """rhs_ptrs, x_ptrs: lists of device (or host) addresses, one per right-hand side."""
    k = len(rhs_ptrs)
    R = (C.c_void_p * k)(*rhs_ptrs)
    X = (C.c_void_p * k)(*x_ptrs)
    t = C.c_uint64()
    _check(lib().ps_server_submit(s, C.byref(jac), C.byref(grid), k, R, X, tol, t_arrival, C.byref(t)),
           "ps_server_submit")
    return t.value


def ps_server_wait(s, ticket):
    """Returns (status, ps_request_info)."""
    info = ps_request_info()
    st = lib().ps_server_wait(s, ticket, C.byref(info))
    return st, info


def ps_server_info_get(s):
    info = ps_server_info()
    _check(lib().ps_server_info_get(s, C.byref(info)), "ps_server_info_get")
    return info


def ps_server_destroy(s):
    lib().ps_server_destroy(s)
