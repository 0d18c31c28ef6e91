"""Python binding of the factor-graph C-ABI (argument marshalling only).

Every method maps to one ``fga_*`` entry point of include/fgadmm.h with the
same name; all computation happens in libfgadmm's CUDA kernels.  Arrays can
be NumPy (host) or torch CUDA tensors (device; passed by pointer).
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import check, fga_iter_opts, fga_iter_result


def _ptr(a):
    """Pointer + keep-alive for a float64/int64 host array or a CUDA tensor."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return ctypes.c_void_p(a.data_ptr()), a
    except ImportError:
        pass
    return ctypes.c_void_p(a.ctypes.data), a


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)   # torch.cuda.Stream


class FactorGraph:
    """One factor graph held by libfgadmm (fga_graph_create ... fga_destroy)."""

    def __init__(self, precision="f64", device=0, stream=None):
        self._lib = _lib.load()
        self._g = ctypes.c_void_p()
        prec = _lib.FGA_F64 if precision in ("f64", _lib.FGA_F64) else _lib.FGA_F32
        self.precision = "f64" if prec == _lib.FGA_F64 else "f32"
        check(self._lib.fga_graph_create(ctypes.byref(self._g), prec, int(device), _stream_handle(stream)),
              "fga_graph_create")

    def __del__(self):
        self.fga_destroy()

    # -- building -----------------------------------------------------------
    def fga_set_stream(self, stream):
        check(self._lib.fga_set_stream(self._g, _stream_handle(stream)), "fga_set_stream")

    def fga_set_option(self, option, value):
        check(self._lib.fga_set_option(self._g, int(option), int(value)), "fga_set_option")

    def fga_add_variables(self, count, dim):
        first = ctypes.c_int64()
        check(self._lib.fga_add_variables(self._g, int(count), int(dim), ctypes.byref(first)), "fga_add_variables")
        return first.value

    def fga_add_factors(self, ftype, var_ids, params=None, shared=False):
        var_ids = np.ascontiguousarray(var_ids, dtype=np.int64)
        if var_ids.ndim == 1:
            var_ids = var_ids[None, :]
        count, nv = var_ids.shape
        if params is None:
            params = np.zeros(0)
            npf = 0
        else:
            params = np.ascontiguousarray(params, dtype=np.float64)
            if shared:
                params = params.reshape(-1)
                npf = params.shape[0]
            else:
                params = params.reshape(count, -1)
                npf = params.shape[1]
        first = ctypes.c_int64()
        vp, _ = _ptr(var_ids)
        pp, _ = _ptr(params) if params.size else (None, None)
        check(self._lib.fga_add_factors(self._g, int(ftype), count, nv, vp, pp, npf, 1 if shared else 0,
                                        ctypes.byref(first)), "fga_add_factors")
        return first.value

    def fga_register_prox(self, cuda_source, function_name, arity, params_per_factor):
        """Compiles a user-supplied proximal operator (CUDA source of a
        function template, see include/fgadmm.h) and returns its type number
        for fga_add_factors."""
        t = ctypes.c_int32()
        check(self._lib.fga_register_prox(self._g, cuda_source.encode(), function_name.encode(), int(arity),
                                          int(params_per_factor), ctypes.byref(t)), "fga_register_prox")
        return t.value

    def fga_set_rho_alpha(self, rho, alpha):
        check(self._lib.fga_set_rho_alpha(self._g, float(rho), float(alpha)), "fga_set_rho_alpha")

    def fga_set_edge_rho_alpha(self, rho=None, alpha=None):
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        a = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64)
        rp, _ = _ptr(r)
        ap, _ = _ptr(a)
        check(self._lib.fga_set_edge_rho_alpha(self._g, rp, ap), "fga_set_edge_rho_alpha")

    def fga_finalize(self):
        check(self._lib.fga_finalize(self._g), "fga_finalize")

    def fga_graph_info(self):
        e, z, f, v = (ctypes.c_int64() for _ in range(4))
        check(self._lib.fga_graph_info(self._g, ctypes.byref(e), ctypes.byref(z), ctypes.byref(f),
                                       ctypes.byref(v)), "fga_graph_info")
        return dict(num_edges=e.value, num_scalar_vars=z.value, num_factors=f.value, num_vars=v.value)

    @property
    def num_edges(self):
        return self.fga_graph_info()["num_edges"]

    @property
    def num_scalar_vars(self):
        return self.fga_graph_info()["num_scalar_vars"]

    # -- running ------------------------------------------------------------
    def fga_init(self, z0=None, u0=None):
        if z0 is not None and not hasattr(z0, "data_ptr"):
            z0 = np.ascontiguousarray(z0, dtype=np.float64)
        if u0 is not None and not hasattr(u0, "data_ptr"):
            u0 = np.ascontiguousarray(u0, dtype=np.float64)
        zp, _z = _ptr(z0)
        up, _u = _ptr(u0)
        check(self._lib.fga_init(self._g, zp, up), "fga_init")

    def fga_iterate(self, max_iters, tol_pri=0.0, tol_dual=0.0, check_every=1, fused=True,
                    barrier_timeout_ns=0, fault_skip_block=-1, raise_on_error=True):
        o = fga_iter_opts(int(max_iters), float(tol_pri), float(tol_dual), int(check_every), 1 if fused else 0,
                          int(barrier_timeout_ns), int(fault_skip_block), 0)
        r = fga_iter_result()
        rc = self._lib.fga_iterate(self._g, ctypes.byref(o), ctypes.byref(r))
        out = dict(iters=r.iters, r_pri=r.r_pri, r_dual=r.r_dual, status=r.status, ms=r.ms, rc=rc)
        if raise_on_error and rc not in (_lib.FGA_OK,):
            check(rc, "fga_iterate")
        return out

    def fga_launch_info(self):
        info = (ctypes.c_int64 * 7)()
        check(self._lib.fga_launch_info(self._g, info, 7), "fga_launch_info")
        return dict(grid=info[0], block=info[1], smem=info[2], blocks_per_sm=info[3], chunks=info[4],
                    buckets=info[5], zorder=info[6])

    def fga_latency_floor(self, iters, mode=1):
        """Device ms of `iters` operator-free passes on the disk-tile grid."""
        ms = ctypes.c_float()
        check(self._lib.fga_latency_floor(self._g, int(iters), int(mode), ctypes.byref(ms)), "fga_latency_floor")
        return ms.value

    def fga_residuals(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        check(self._lib.fga_residuals(self._g, ctypes.byref(a), ctypes.byref(b)), "fga_residuals")
        return a.value, b.value

    def fga_read_z(self, out=None):
        n = self.num_scalar_vars
        if out is None:
            out = np.empty(n, dtype=np.float64)
        op, _ = _ptr(out)
        check(self._lib.fga_read_z(self._g, op, n), "fga_read_z")
        return out

    def fga_read_edge_state(self, which, out=None):
        n = self.num_edges
        if out is None:
            out = np.empty(n, dtype=np.float64)
        op, _ = _ptr(out)
        check(self._lib.fga_read_edge_state(self._g, int(which), op, n), "fga_read_edge_state")
        return out

    def fga_destroy(self):
        g = getattr(self, "_g", None)
        if g is not None and g.value:
            self._lib.fga_destroy(g)
            self._g = ctypes.c_void_p()


def graph_from_problem(problem, precision="f64", device=0, stream=None, options=None, init=True):
    """Builds, finalizes and (optionally) initialises a FactorGraph from a
    problem description of ``paper_1603_02526_gb300.inputs``."""
    g = FactorGraph(precision, device, stream)
    for opt, val in (options or {}).items():
        g.fga_set_option(opt, val)
    for count, dim in _merge_var_blocks(problem.var_blocks):
        g.fga_add_variables(count, dim)
    for blk in problem.factor_blocks:
        g.fga_add_factors(blk.ftype, blk.var_ids, blk.params if blk.params.size else None)
    g.fga_set_rho_alpha(problem.rho, problem.alpha)
    g.fga_finalize()
    if init:
        g.fga_init(problem.z0)
    return g


def _merge_var_blocks(blocks):
    """Consecutive blocks of equal dimension as one call each."""
    out = []
    for count, dim in blocks:
        if out and out[-1][1] == dim:
            out[-1][0] += count
        else:
            out.append([count, dim])
    return out
