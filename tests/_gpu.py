"""Helpers for the GPU tests: move an oracle system to device memory, and read
device arrays written by the library back into numpy."""
import ctypes as C

import numpy as np
import torch

import paper_1812_05540_gb300 as ps


class _CAI:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def dev_to_numpy(ptr, n, dtype):
    """Copy n elements of a raw device array to host numpy."""
    ts = {np.float64: "<f8", np.int64: "<i8", np.int32: "<i4", np.uint8: "|u1"}[dtype]
    if n == 0:
        return np.zeros(0, dtype)
    t = torch.as_tensor(_CAI(ptr, n, ts), device="cuda")
    return t.cpu().numpy().copy()


class DeviceSystem:
    """Device copies of an oracle-generated Jacobian as a ps_jacobian."""

    def __init__(self, osys):
        self.tensors = []
        dev = "cuda"

        def put(a):
            t = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
            self.tensors.append(t)
            return t

        blocks = {}
        dims = {"uu": (osys.n_nodes, osys.n_nodes, 3, 3), "uf": (osys.n_nodes, osys.n_cells, 3, 2),
                "fu": (osys.n_cells, osys.n_nodes, 2, 3), "ff": (osys.n_cells, osys.n_cells, 2, 2)}
        for name, (nb, ncol, br, bc) in dims.items():
            rp, ci, v = osys.blocks[name]
            trp, tci, tv = put(rp), put(ci), put(v)
            blocks[name] = ps.ps_bsr(nb, ncol, len(ci), br, bc, trp.data_ptr(), tci.data_ptr(), tv.data_ptr())
        self.dfs = put(osys.d_fs)
        self.dir = put(osys.dirichlet)
        self.rhs = put(osys.rhs)
        self.jac = ps.ps_jacobian(blocks["uu"], blocks["uf"], blocks["fu"], blocks["ff"], self.dfs.data_ptr(),
                                  self.dir.data_ptr())
        self.grid = ps.ps_grid(osys.nx, osys.ny, osys.nz, osys.h, osys.h, osys.h)
        self.n = osys.n


def to_device(osys):
    return DeviceSystem(osys)


def system_to_numpy(sp):
    """Host copy of a library-generated system (ps_system pointer)."""
    s = sp.contents
    out = {"n_nodes": s.n_nodes, "n_cells": s.n_cells, "n": s.n, "alpha_u": s.alpha_u, "alpha_f": s.alpha_f}
    for name, b, bs in (("uu", s.jac.A_uu, 9), ("uf", s.jac.A_uf, 6), ("fu", s.jac.A_fu, 6), ("ff", s.jac.A_ff, 4)):
        out[name] = (dev_to_numpy(b.rowptr, b.n_brow + 1, np.int64), dev_to_numpy(b.colind, b.nnzb, np.int32),
                     dev_to_numpy(b.val, b.nnzb * bs, np.float64))
    out["d_fs"] = dev_to_numpy(s.jac.d_fs, 2 * s.n_cells, np.float64)
    out["dirichlet"] = dev_to_numpy(s.jac.dirichlet_u, s.n_u, np.uint8)
    out["rhs"] = dev_to_numpy(s.rhs, s.n, np.float64)
    for k in ("E", "nu", "kh", "kv", "phi0", "sw", "p"):
        out[k] = dev_to_numpy(getattr(s, k), s.n_cells, np.float64)
    return out


def gen_params_like(ogp):
    """ps_gen_params with the same values as an oracle GenParams."""
    gp = ps.ps_gen_params()
    for name, _ in ps.ps_gen_params._fields_:
        setattr(gp, name, getattr(ogp, name))
    return gp
