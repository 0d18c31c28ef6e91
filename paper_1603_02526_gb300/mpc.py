"""Python binding of the batched MPC C-ABI (fga_mpc_batch_*), marshalling only."""
import ctypes

import numpy as np

from . import _lib
from ._lib import check, fga_mpc_opts, fga_mpc_result


def _p(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


class MpcBatch:
    """Ragged batch of linear MPC instances solved on the GPU in one launch."""

    def __init__(self, T, A, B, q, r, umax=1.0, rho=1.0, alpha=1.0, precision="f32", device=0, stream=None,
                 sys_of_inst=None):
        self._lib = _lib.load()
        self._b = ctypes.c_void_p()
        T = np.ascontiguousarray(T, dtype=np.int32)
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        r = np.ascontiguousarray(r, dtype=np.float64)
        if A.ndim == 2:
            A, B, q, r = A[None], B[None], q[None], r[None]
        nsys, nx, nu = A.shape[0], A.shape[1], B.shape[2]
        self.n, self.nx, self.nu = len(T), nx, nu
        self.T = T
        sp = None
        if sys_of_inst is not None:
            sys_of_inst = np.ascontiguousarray(sys_of_inst, dtype=np.int32)
            sp = _p(sys_of_inst)
        prec = _lib.FGA_F32 if precision == "f32" else _lib.FGA_F64
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream")
                                                         else int(stream))
        check(self._lib.fga_mpc_batch_create(ctypes.byref(self._b), prec, int(device), st, len(T), _p(T), nx, nu,
                                             nsys, sp, _p(A), _p(B), _p(q), _p(r), float(umax), float(rho),
                                             float(alpha)), "fga_mpc_batch_create")
        S = nx + nu
        self.V = S * T.astype(np.int64) + nx
        self.E = 2 * nx + (3 * nx + 3 * nu) * T.astype(np.int64)
        self.zoff = np.concatenate([[0], np.cumsum(self.V)[:-1]])
        self.eoff = np.concatenate([[0], np.cumsum(self.E)[:-1]])

    def __del__(self):
        b = getattr(self, "_b", None)
        if b is not None and b.value:
            self._lib.fga_mpc_batch_destroy(b)
            self._b = ctypes.c_void_p()

    def fga_mpc_batch_set_x0(self, x0):
        x0 = np.ascontiguousarray(x0, dtype=np.float64) if not hasattr(x0, "data_ptr") else x0
        check(self._lib.fga_mpc_batch_set_x0(self._b, _p(x0)), "fga_mpc_batch_set_x0")

    def fga_mpc_batch_init(self, z0=None, u0=None):
        z0 = None if z0 is None else np.ascontiguousarray(z0, dtype=np.float64)
        u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
        check(self._lib.fga_mpc_batch_init(self._b, _p(z0), _p(u0)), "fga_mpc_batch_init")

    def fga_mpc_batch_warm_start(self, pred, ld):
        check(self._lib.fga_mpc_batch_warm_start(self._b, _p(pred), int(ld)), "fga_mpc_batch_warm_start")

    def fga_mpc_batch_targets(self, out, ld):
        check(self._lib.fga_mpc_batch_targets(self._b, _p(out), int(ld)), "fga_mpc_batch_targets")

    def fga_mpc_batch_solve(self, max_iters, tol=1e-4, tol_dual=None, check_every=0, threads=0, use_graph=True):
        o = fga_mpc_opts(int(max_iters), float(tol), float(tol if tol_dual is None else tol_dual),
                         int(check_every), int(threads), 1 if use_graph else 0, 0)
        r = fga_mpc_result()
        check(self._lib.fga_mpc_batch_solve(self._b, ctypes.byref(o), ctypes.byref(r)), "fga_mpc_batch_solve")
        return dict(total_iters=r.total_iters, max_inst_iters=r.max_inst_iters, n_converged=r.n_converged,
                    n_budget=r.n_budget, n_nonfinite=r.n_nonfinite, ms=r.ms, threads=r.threads,
                    check_every=r.check_every)

    def fga_mpc_batch_read(self, state=True):
        """Readout; state=False skips z and u (per-instance counters only)."""
        z = np.empty(int(self.V.sum())) if state else None
        u = np.empty(int(self.E.sum())) if state else None
        it = np.empty(self.n, dtype=np.int64)
        st = np.empty(self.n, dtype=np.int32)
        rp = np.empty(self.n)
        rd = np.empty(self.n)
        check(self._lib.fga_mpc_batch_read(self._b, _p(z), _p(u), _p(it), _p(st), _p(rp), _p(rd)),
              "fga_mpc_batch_read")
        return dict(z=z, u=u, iters=it, status=st, r_pri=rp, r_dual=rd)

    def fga_mpc_batch_info(self):
        info = (ctypes.c_int64 * 6)()
        check(self._lib.fga_mpc_batch_info(self._b, info, 6), "fga_mpc_batch_info")
        return dict(n_inst=info[0], edges=info[1], scalar_vars=info[2], tmax=info[3], threads=info[4],
                    check_every=info[5])

    def fga_mpc_batch_autotune(self, max_iters, tol, cache_path=None):
        th, ce = ctypes.c_int32(), ctypes.c_int32()
        cp = None if cache_path is None else str(cache_path).encode()
        check(self._lib.fga_mpc_batch_autotune(self._b, cp, int(max_iters), float(tol), ctypes.byref(th),
                                               ctypes.byref(ce)), "fga_mpc_batch_autotune")
        return th.value, ce.value

    def instance_z(self, z, i):
        return z[self.zoff[i]: self.zoff[i] + self.V[i]]

    def instance_u(self, u, i):
        return u[self.eoff[i]: self.eoff[i] + self.E[i]]


def batch_from_inputs(d, precision="f32", rho=1.0, alpha=1.0, device=0, stream=None):
    """MpcBatch for a dict from inputs.mpc_batch_inputs, x0 set, cold start."""
    b = MpcBatch(d["T"], d["A"], d["B"], d["q"], d["r"], umax=d["umax"], rho=rho, alpha=alpha,
                 precision=precision, device=device, stream=stream)
    b.fga_mpc_batch_set_x0(d["x0"])
    b.fga_mpc_batch_init()
    return b
