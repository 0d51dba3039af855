"""ctypes binding of the plain FP64 CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package; the
product package never does.

The oracle restates arXiv 1812.05540 (two-stage fixed-stress / CPR
preconditioner for multiphase poromechanics) literally in FP64: the App. B
Jacobian, §5.1 fixed-stress Schur approximation, §5.2 SDC mechanics AMG,
§5.3 quasi-IMPES + pressure AMG + block ILU(0), Algorithm 1, and flexible
GMRES (§4).  Pins live in tests/test_oracle_*.py.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")

OR_GRAVITY, OR_DIRICHLET, OR_SCALE, OR_ACCUM, OR_FLUX, OR_FLUX_SAT, OR_COUPLING = (1 << i for i in range(7))
OR_ALL = 0x7F
OR_WELLS = 1 << 7  # Peaceman wells (an option; not in OR_ALL)
FIELDS_LOGNORMAL, FIELDS_LAYERED, FIELDS_CHANNELS, FIELDS_HOMOGENEOUS = range(4)
MECH_AMG, MECH_EXACT, MECH_AMG_RBM = 0, 1, 2
FLOW_CPR, FLOW_EXACT_FS, FLOW_EXACT_SCHUR = 0, 1, 2
LOCAL_ILU0, LOCAL_EXACT, LOCAL_GS = 0, 1, 2
PRESS_AMG, PRESS_EXACT = 0, 1
CPR_QUASI_IMPES, CPR_TRUE_IMPES = 0, 1
FS_GIVEN, FS_RSL, FS_RSL_EXACT = 0, 1, 2


def build(force=False, openmp=False):
    """Compile oracle.cpp with g++ (x86 here, aarch64 on the GPU host).  openmp=True builds the same
    source with -fopenmp (row loops on all host cores, results bit-identical to the serial build)."""
    src = os.path.join(_HERE, "oracle.cpp")
    hdr = os.path.join(_HERE, "oracle.h")
    out = _LIB_OMP if openmp else _LIB
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", src, "-o", tmp]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


class NewtonParams(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_newton", C.c_int32), ("forcing", C.c_int32), ("eta_fixed", C.c_double),
                ("ew_gamma", C.c_double), ("ew_omega", C.c_double), ("ew_eta0", C.c_double),
                ("ew_eta_max", C.c_double), ("max_backtracks", C.c_int32), ("restart", C.c_int32),
                ("max_linear", C.c_int32)]


class NewtonStats(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("linear_iters", C.c_int32), ("backtracks", C.c_int32),
                ("converged", C.c_int32), ("rnorm", C.c_double * 33), ("eta", C.c_double * 32),
                ("lin_iters", C.c_int32 * 32)]


class GenParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("h", C.c_double),
                ("seed", C.c_uint64), ("field_kind", C.c_int32), ("flags", C.c_uint32),
                ("dt", C.c_double), ("biot", C.c_double), ("c_w", C.c_double), ("c_nw", C.c_double),
                ("c_r", C.c_double), ("mu_w", C.c_double), ("mu_nw", C.c_double),
                ("rho_w0", C.c_double), ("rho_nw0", C.c_double), ("rho_s0", C.c_double),
                ("s_wr", C.c_double), ("s_nwr", C.c_double), ("grav", C.c_double),
                ("p_ref", C.c_double), ("dp_amp", C.c_double), ("corey", C.c_double),
                ("E0", C.c_double), ("nu0", C.c_double), ("kappa0", C.c_double),
                ("phi0", C.c_double), ("sw0", C.c_double), ("fs_modulus", C.c_int32)]


_PD, _PI64, _PI32, _PU8 = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_uint8)


class _System(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("h", C.c_double),
                ("n_nodes", C.c_int64), ("n_cells", C.c_int64), ("n_u", C.c_int64), ("n_f", C.c_int64),
                ("n", C.c_int64),
                ("nnzb_uu", C.c_int64), ("nnzb_uf", C.c_int64), ("nnzb_fu", C.c_int64), ("nnzb_ff", C.c_int64),
                ("uu_rp", _PI64), ("uu_ci", _PI32), ("uu_v", _PD),
                ("uf_rp", _PI64), ("uf_ci", _PI32), ("uf_v", _PD),
                ("fu_rp", _PI64), ("fu_ci", _PI32), ("fu_v", _PD),
                ("ff_rp", _PI64), ("ff_ci", _PI32), ("ff_v", _PD),
                ("d_fs", _PD), ("dirichlet", _PU8), ("rhs", _PD),
                ("alpha_u", C.c_double), ("alpha_f", C.c_double),
                ("E", _PD), ("nu", _PD), ("kh", _PD), ("kv", _PD), ("phi0", _PD), ("sw", _PD), ("p", _PD)]


class PrecParams(C.Structure):
    _fields_ = [("theta_u", C.c_double), ("theta_p", C.c_double), ("coarse_max_u", C.c_int32),
                ("coarse_max_p", C.c_int32), ("max_levels", C.c_int32), ("pre", C.c_int32),
                ("post", C.c_int32), ("smoother", C.c_int32), ("cheb_degree", C.c_int32),
                ("cheb_ratio", C.c_double), ("mech_mode", C.c_int32), ("flow_mode", C.c_int32),
                ("local_mode", C.c_int32), ("press_mode", C.c_int32), ("full_exact", C.c_int32),
                ("local_sweeps", C.c_int32), ("cpr_reduction", C.c_int32),
                ("fs_mode", C.c_int32), ("ilu_tile_y", C.c_int32), ("ilu_tile_z", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("breakdown", C.c_int32), ("true_relres", C.c_double), ("est_relres", C.c_double)]


class TerzaghiParams(C.Structure):
    _fields_ = [("nz", C.c_int32), ("h", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("biot", C.c_double), ("kappa", C.c_double), ("mu", C.c_double), ("phi0", C.c_double),
                ("rho0", C.c_double), ("sigma0", C.c_double), ("dt", C.c_double), ("nsteps", C.c_int32)]


_libs = {}
_use_openmp = False


def select(openmp):
    """Choose the build that new Systems (and their Precs) use: serial (False) or OpenMP (True)."""
    global _use_openmp
    _use_openmp = bool(openmp)


def lib(openmp=None):
    openmp = _use_openmp if openmp is None else bool(openmp)
    if openmp not in _libs:
        L = C.CDLL(build(openmp=openmp))
        L.or_num_threads.restype = C.c_int
        L.or_generate.argtypes = [C.POINTER(GenParams), C.POINTER(C.POINTER(_System))]
        L.or_generate_at.argtypes = [C.POINTER(GenParams), _PD, C.POINTER(C.POINTER(_System))]
        L.or_newton_params_default.argtypes = [C.POINTER(NewtonParams)]
        L.or_newton.argtypes = [C.POINTER(GenParams), C.POINTER(PrecParams), C.POINTER(NewtonParams), _PD,
                                C.POINTER(NewtonStats)]
        L.or_ew_eta.argtypes = [C.POINTER(NewtonParams), C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_ew_eta.restype = C.c_double
        L.or_system_free.argtypes = [C.POINTER(_System)]
        L.or_default_params.argtypes = [C.POINTER(GenParams), C.c_int]
        L.or_spmv.argtypes = [C.POINTER(_System), _PD, _PD]
        L.or_ref_integrals.argtypes = [C.c_double, _PD, _PD, _PD, _PD]
        L.or_residual.argtypes = [C.POINTER(GenParams), _PD, _PD]
        L.or_default_prec_params.argtypes = [C.POINTER(PrecParams)]
        L.or_prec_setup.argtypes = [C.POINTER(_System), C.POINTER(PrecParams), C.POINTER(C.c_void_p)]
        L.or_prec_setup_reuse.argtypes = [C.POINTER(_System), C.POINTER(_System), C.POINTER(PrecParams),
                                           C.POINTER(C.c_void_p)]
        L.or_prec_free.argtypes = [C.c_void_p]
        L.or_prec_apply.argtypes = [C.c_void_p, _PD, _PD]
        L.or_amg_nlevels.argtypes = [C.c_void_p, C.c_int]
        L.or_amg_level_n.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.or_amg_level_n.restype = C.c_int64
        L.or_amg_level_nnz.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.or_amg_level_nnz.restype = C.c_int64
        L.or_amg_level_matrix.argtypes = [C.c_void_p, C.c_int, C.c_int, _PI64, _PI32, _PD]
        L.or_amg_aggregates.argtypes = [C.c_void_p, C.c_int, C.c_int, _PI32]
        L.or_amg_aggregates.restype = C.c_int64
        L.or_amg_roots.argtypes = [C.c_void_p, C.c_int, C.c_int, _PU8]
        L.or_amg_roots.restype = C.c_int64
        L.or_aggregate.argtypes = [C.c_int64, C.c_int, _PI64, _PI32, _PD, C.c_double, C.c_int, _PI32, _PU8]
        L.or_aggregate.restype = C.c_int64
        L.or_amg_p_nnz.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.or_amg_p_nnz.restype = C.c_int64
        L.or_amg_prolongator.argtypes = [C.c_void_p, C.c_int, C.c_int, _PI64, _PI32, _PD]
        L.or_amg_vcycle.argtypes = [C.c_void_p, C.c_int, C.c_int, _PD, _PD]
        L.or_rbm_nlevels.argtypes = [C.c_void_p]
        L.or_rbm_level_shape.argtypes = [C.c_void_p, C.c_int, _PI64]
        L.or_rbm_level_matrix.argtypes = [C.c_void_p, C.c_int, _PI64, _PI32, _PD]
        L.or_rbm_level_data.argtypes = [C.c_void_p, C.c_int, _PI32, _PD, _PD, _PD]
        L.or_rbm_prolongator.argtypes = [C.c_void_p, C.c_int, _PI64, _PI32, _PD]
        L.or_rbm_vcycle.argtypes = [C.c_void_p, _PD, _PD]
        L.or_rigid_body_modes.argtypes = [C.c_int, C.c_int, C.c_int, _PD]
        L.or_spp_nnz.argtypes = [C.c_void_p]
        L.or_spp_nnz.restype = C.c_int64
        L.or_spp.argtypes = [C.c_void_p, _PI64, _PI32, _PD]
        L.or_ilu_dinv.argtypes = [C.c_void_p, _PD]
        L.or_fs_diag.argtypes = [C.c_void_p, _PD]
        L.or_ilu_apply.argtypes = [C.c_void_p, _PD, _PD]
        L.or_gs_apply.argtypes = [C.c_void_p, _PD, _PD, C.c_int]
        L.or_fgmres.argtypes = [C.POINTER(_System), C.c_void_p, _PD, _PD, C.c_double, C.c_int, C.c_int,
                                C.POINTER(Stats)]
        L.or_richardson.argtypes = [C.POINTER(_System), C.c_void_p, _PD, _PD, C.c_double, C.c_int,
                                    C.POINTER(Stats)]
        L.or_fgmres_diag.argtypes = [C.c_int64, _PD, _PD, _PD, C.c_double, C.c_int, C.c_int, C.POINTER(Stats)]
        L.or_dense_solve.argtypes = [C.POINTER(_System), _PD, _PD]
        L.or_lu_solve.argtypes = [C.c_int64, _PD, _PD, _PD]
        L.or_smoother_apply.argtypes = [C.c_int64, _PI64, _PI32, _PD, _PD, _PD, C.c_int, C.c_int, C.c_double,
                                        C.c_int]
        L.or_splitmix64.argtypes = [C.c_uint64]
        L.or_splitmix64.restype = C.c_uint64
        L.or_correlated_field.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_int, _PD]
        L.or_terzaghi.argtypes = [C.POINTER(TerzaghiParams), _PD, _PD, _PD, _PD, _PD]
        _libs[openmp] = L
    return _libs[openmp]


def rigid_body_modes(nx, ny, nz):
    B = np.empty(((nx + 1) * (ny + 1) * (nz + 1) * 3, 6))
    lib().or_rigid_body_modes(nx, ny, nz, _d(B))
    return B


def num_threads(openmp=None):
    return lib(openmp).or_num_threads()


def _d(a):
    return a.ctypes.data_as(_PD)


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype)
    return np.ctypeslib.as_array(ptr, shape=(int(n),)).astype(dtype, copy=True)


def default_params(config=0, **kw):
    gp = GenParams()
    lib().or_default_params(C.byref(gp), config)
    for k, v in kw.items():
        setattr(gp, k, v)
    return gp


class System:
    """A generated Jacobian held as numpy arrays (copied out of the oracle)."""

    def __init__(self, gp, dx=None):
        """dx: the Jacobian at the state base + dx (n values ordered as x); None: at the base state"""
        ptr = C.POINTER(_System)()
        self._L = lib()
        if dx is None:
            rc = self._L.or_generate(C.byref(gp), C.byref(ptr))
        else:
            dx = np.ascontiguousarray(dx, dtype=np.float64)
            rc = self._L.or_generate_at(C.byref(gp), _d(dx), C.byref(ptr))
        if rc:
            raise RuntimeError("or_generate failed: %d" % rc)
        self._ptr = ptr
        s = ptr.contents
        self.gp = gp
        self.nx, self.ny, self.nz, self.h = s.nx, s.ny, s.nz, s.h
        self.n_nodes, self.n_cells, self.n_u, self.n_f, self.n = s.n_nodes, s.n_cells, s.n_u, s.n_f, s.n
        self.alpha_u, self.alpha_f = s.alpha_u, s.alpha_f
        nn, nc = s.n_nodes, s.n_cells
        self.blocks = {}
        for name, nb, bs, nnzb in (("uu", nn, 9, s.nnzb_uu), ("uf", nn, 6, s.nnzb_uf),
                                   ("fu", nc, 6, s.nnzb_fu), ("ff", nc, 4, s.nnzb_ff)):
            rp = _arr(getattr(s, name + "_rp"), nb + 1, np.int64)
            ci = _arr(getattr(s, name + "_ci"), nnzb, np.int32)
            v = _arr(getattr(s, name + "_v"), nnzb * bs, np.float64)
            self.blocks[name] = (rp, ci, v)
        self.d_fs = _arr(s.d_fs, 2 * nc, np.float64)
        self.dirichlet = _arr(s.dirichlet, s.n_u, np.uint8)
        self.rhs = _arr(s.rhs, s.n, np.float64)
        self.fields = {k: _arr(getattr(s, k), nc, np.float64) for k in ("E", "nu", "kh", "kv", "phi0", "sw", "p")}

    def __del__(self):
        try:
            self._L.or_system_free(self._ptr)
        except Exception:
            pass

    def spmv(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n)
        self._L.or_spmv(self._ptr, _d(x), _d(y))
        return y

    def dense(self):
        """Dense Jacobian assembled in numpy from the BSR blocks (tiny systems)."""
        A = np.zeros((self.n, self.n))
        off = {"uu": (0, 0, 3, 3), "uf": (0, self.n_u, 3, 2), "fu": (self.n_u, 0, 2, 3),
               "ff": (self.n_u, self.n_u, 2, 2)}
        for name, (r0, c0, br, bc) in off.items():
            rp, ci, v = self.blocks[name]
            v = v.reshape(-1, br, bc)
            for i in range(len(rp) - 1):
                for q in range(rp[i], rp[i + 1]):
                    A[r0 + i * br:r0 + (i + 1) * br, c0 + ci[q] * bc:c0 + (ci[q] + 1) * bc] += v[q]
        return A

    def dense_solve(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty(self.n)
        rc = self._L.or_dense_solve(self._ptr, _d(b), _d(x))
        if rc:
            raise RuntimeError("or_dense_solve failed: %d" % rc)
        return x


def default_prec_params(**kw):
    pp = PrecParams()
    lib().or_default_prec_params(C.byref(pp))
    for k, v in kw.items():
        setattr(pp, k, v)
    return pp


class Prec:
    def __init__(self, system, pp=None, mech_system=None):
        """mech_system: build M_uu from that system's A_uu instead (flow-setup reuse of §5.4)."""
        self.system = system
        self.mech_system = mech_system
        self.pp = pp if pp is not None else default_prec_params()
        h = C.c_void_p()
        self._L = system._L
        if mech_system is not None:
            rc = self._L.or_prec_setup_reuse(system._ptr, mech_system._ptr, C.byref(self.pp), C.byref(h))
        else:
            rc = self._L.or_prec_setup(system._ptr, C.byref(self.pp), C.byref(h))
        if rc:
            raise RuntimeError("or_prec_setup failed: %d" % rc)
        self._h = h

    def __del__(self):
        try:
            self._L.or_prec_free(self._h)
        except Exception:
            pass

    def apply(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        z = np.empty(self.system.n)
        self._L.or_prec_apply(self._h, _d(v), z.ctypes.data_as(_PD))
        return z

    def nlevels(self, which):
        return self._L.or_amg_nlevels(self._h, which)

    def level(self, which, l):
        n = self._L.or_amg_level_n(self._h, which, l)
        nnz = self._L.or_amg_level_nnz(self._h, which, l)
        nc = 3 if which == 0 else 1
        rp = np.empty(n + 1, np.int64)
        ci = np.empty(nnz, np.int32)
        v = np.empty(nnz * nc)
        self._L.or_amg_level_matrix(self._h, which, l, rp.ctypes.data_as(_PI64), ci.ctypes.data_as(_PI32), _d(v))
        return rp, ci, v.reshape(nnz, nc)

    def aggregates(self, which, l):
        n = self._L.or_amg_level_n(self._h, which, l)
        agg = np.empty(n, np.int32)
        na = self._L.or_amg_aggregates(self._h, which, l, agg.ctypes.data_as(_PI32))
        return agg, na

    def roots(self, which, l):
        n = self._L.or_amg_level_n(self._h, which, l)
        r = np.zeros(n, np.uint8)
        self._L.or_amg_roots(self._h, which, l, r.ctypes.data_as(_PU8))
        return r.astype(bool)

    def prolongator(self, which, l):
        n = self._L.or_amg_level_n(self._h, which, l)
        nnz = self._L.or_amg_p_nnz(self._h, which, l)
        nc = 3 if which == 0 else 1
        rp = np.empty(n + 1, np.int64)
        ci = np.empty(nnz, np.int32)
        v = np.empty(nnz * nc)
        self._L.or_amg_prolongator(self._h, which, l, rp.ctypes.data_as(_PI64), ci.ctypes.data_as(_PI32), _d(v))
        return rp, ci, v.reshape(nnz, nc)

    def vcycle(self, which, comp, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        self._L.or_amg_vcycle(self._h, which, comp, _d(b), _d(x))
        return x

    # rigid-body-mode smoothed aggregation (mech_mode=MECH_AMG_RBM)
    def rbm_nlevels(self):
        return self._L.or_rbm_nlevels(self._h)

    def rbm_shape(self, l):
        sh = np.zeros(6, np.int64)
        assert self._L.or_rbm_level_shape(self._h, l, sh.ctypes.data_as(_PI64)) == 0
        return dict(n=int(sh[0]), b=int(sh[1]), nnzb=int(sh[2]), nagg=int(sh[3]), pnnzb=int(sh[4]),
                    coarsest=bool(sh[5]))

    def rbm_level(self, l):
        sh = self.rbm_shape(l)
        n, b, nnz = sh["n"], sh["b"], sh["nnzb"]
        rp = np.empty(n + 1, np.int64)
        ci = np.empty(nnz, np.int32)
        v = np.empty(nnz * b * b)
        self._L.or_rbm_level_matrix(self._h, l, rp.ctypes.data_as(_PI64), ci.ctypes.data_as(_PI32), _d(v))
        return rp, ci, v.reshape(nnz, b, b)

    def rbm_data(self, l):
        sh = self.rbm_shape(l)
        n, b = sh["n"], sh["b"]
        agg = np.empty(n, np.int32)
        B = np.empty((n * b, 6))
        Pt = np.empty((n * b, 6))
        lam = np.zeros(1)
        self._L.or_rbm_level_data(self._h, l, agg.ctypes.data_as(_PI32), _d(B), _d(Pt), _d(lam))
        return agg, B, Pt, float(lam[0])

    def rbm_prolongator(self, l):
        sh = self.rbm_shape(l)
        n, b, nnz = sh["n"], sh["b"], sh["pnnzb"]
        rp = np.empty(n + 1, np.int64)
        ci = np.empty(nnz, np.int32)
        v = np.empty(nnz * b * 6)
        assert self._L.or_rbm_prolongator(self._h, l, rp.ctypes.data_as(_PI64), ci.ctypes.data_as(_PI32),
                                          _d(v)) == 0
        return rp, ci, v.reshape(nnz, b, 6)

    def rbm_vcycle(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        assert self._L.or_rbm_vcycle(self._h, _d(b), _d(x)) == 0
        return x

    def spp(self):
        nc = self.system.n_cells
        nnz = self._L.or_spp_nnz(self._h)
        rp = np.empty(nc + 1, np.int64)
        ci = np.empty(nnz, np.int32)
        v = np.empty(nnz)
        self._L.or_spp(self._h, rp.ctypes.data_as(_PI64), ci.ctypes.data_as(_PI32), _d(v))
        return rp, ci, v

    def fs_diag(self):
        d = np.empty(2 * self.system.n_cells)
        self._L.or_fs_diag(self._h, _d(d))
        return d

    def ilu_dinv(self):
        d = np.empty(4 * self.system.n_cells)
        self._L.or_ilu_dinv(self._h, _d(d))
        return d

    def ilu_apply(self, w):
        w = np.ascontiguousarray(w, dtype=np.float64)
        dz = np.empty_like(w)
        self._L.or_ilu_apply(self._h, _d(w), _d(dz))
        return dz

    def richardson(self, b=None, tol=1e-8, max_iters=1000):
        s = self.system
        b = s.rhs if b is None else np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty(s.n)
        st = Stats()
        self._L.or_richardson(s._ptr, self._h, _d(b), _d(x), tol, max_iters, C.byref(st))
        return x, st

    def gs_apply(self, w, sweeps):
        w = np.ascontiguousarray(w, dtype=np.float64)
        dz = np.empty_like(w)
        self._L.or_gs_apply(self._h, _d(w), _d(dz), sweeps)
        return dz

    def fgmres(self, b=None, tol=1e-8, restart=100, max_iters=1000):
        s = self.system
        b = s.rhs if b is None else np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty(s.n)
        st = Stats()
        self._L.or_fgmres(s._ptr, self._h, _d(b), _d(x), tol, restart, max_iters, C.byref(st))
        return x, st


def fgmres_diag(diag, b, tol=1e-10, restart=100, max_iters=1000):
    diag = np.ascontiguousarray(diag, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty_like(b)
    st = Stats()
    lib().or_fgmres_diag(len(b), _d(diag), _d(b), _d(x), tol, restart, max_iters, C.byref(st))
    return x, st


def aggregate(rp, ci, v, nc=1, theta=0.08, level=0):
    """Aggregates and distance-2 MIS roots of a CSR level operator (nc values per entry)."""
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    n = len(rp) - 1
    agg = np.empty(n, np.int32)
    root = np.zeros(n, np.uint8)
    na = lib().or_aggregate(n, nc, rp.ctypes.data_as(_PI64), ci.ctypes.data_as(_PI32), _d(v), theta, level,
                            agg.ctypes.data_as(_PI32), root.ctypes.data_as(_PU8))
    return agg, root.astype(bool), na


def ref_integrals(h):
    G = np.empty(8 * 8 * 9)
    IN = np.empty(8)
    IdN = np.empty(24)
    INdN = np.empty(8 * 8 * 3)
    lib().or_ref_integrals(h, _d(G), _d(IN), _d(IdN), _d(INdN))
    return G.reshape(8, 8, 3, 3), IN, IdN.reshape(8, 3), INdN.reshape(8, 8, 3)


def correlated_field(seed, field, nx, ny, nz, Lx, Ly, Lz):
    out = np.empty(nx * ny * nz)
    lib().or_correlated_field(seed, field, nx, ny, nz, Lx, Ly, Lz, _d(out))
    return out.reshape(nz, ny, nx)


FORCING_FIXED, FORCING_EW = 0, 1


def default_newton_params(**kw):
    np_ = NewtonParams()
    lib().or_newton_params_default(C.byref(np_))
    for k, v in kw.items():
        setattr(np_, k, v)
    return np_


def newton(gp, pp=None, np_=None):
    """Newton's method for one time step from the base state: (x relative to the base state, stats dict)"""
    pp = pp or default_prec_params()
    np_ = np_ or default_newton_params()
    n = 3 * (gp.nx + 1) * (gp.ny + 1) * (gp.nz + 1) + 2 * gp.nx * gp.ny * gp.nz
    x = np.zeros(n)
    st = NewtonStats()
    rc = lib().or_newton(C.byref(gp), C.byref(pp), C.byref(np_), _d(x), C.byref(st))
    k = st.newton_iters
    return x, dict(rc=rc, newton_iters=k, linear_iters=st.linear_iters, backtracks=st.backtracks,
                   converged=bool(st.converged), rnorm=list(st.rnorm[:k + 1]), eta=list(st.eta[:k]),
                   lin_iters=list(st.lin_iters[:k]))


def ew_eta(np_, k, rk, rkm1, eta_prev, r0):
    return lib().or_ew_eta(C.byref(np_), k, rk, rkm1, eta_prev, r0)


def residual(gp, dx):
    dx = np.ascontiguousarray(dx, dtype=np.float64)
    r = np.empty_like(dx)
    if lib().or_residual(C.byref(gp), _d(dx), _d(r)) != 0:
        raise ValueError("or_residual: invalid parameters")
    return r


def lu_solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64).copy()
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty_like(b)
    rc = lib().or_lu_solve(len(b), _d(A), _d(b), _d(x))
    if rc:
        raise RuntimeError("singular")
    return x


def smoother_apply(rp, ci, v, b, kind, count, ratio=20.0, x0=None):
    """One V-cycle level smoother on a scalar CSR matrix: kind 1 = Chebyshev of degree count on
    D^{-1}A over [lambda_hat/ratio, lambda_hat], kind 0 = count l1-Jacobi sweeps; from x0 (or 0)."""
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    rc = lib().or_smoother_apply(len(b), rp.ctypes.data_as(_PI64), ci.ctypes.data_as(_PI32), _d(v), _d(b), _d(x),
                                 kind, count, ratio, 1 if x0 is None else 0)
    if rc:
        raise RuntimeError("row without a diagonal entry")
    return x


def terzaghi(**kw):
    tp = TerzaghiParams(**kw)
    nz, ns = tp.nz, tp.nsteps
    t = np.empty(ns)
    p = np.empty(ns * nz)
    p0 = C.c_double()
    cv = C.c_double()
    nr = C.c_double()
    lib().or_terzaghi(C.byref(tp), _d(t), _d(p), C.byref(p0), C.byref(cv), C.byref(nr))
    return t, p.reshape(ns, nz), p0.value, cv.value, nr.value
