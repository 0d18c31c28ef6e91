"""Python binding of the long-horizon MPC C-ABI (fga_horizon_*), marshalling
only."""
import ctypes

import numpy as np

from . import _lib
from ._lib import check, fga_iter_opts, fga_iter_result


class Horizon:
    """One MPC of horizon K (nx = 4, nu = 1) solved with the horizon laid
    along the grid; variable and edge order as in the C header."""

    def __init__(self, K, A, B, q, r, x0, rho=1.0, alpha=1.0, device=0, stream=None):
        self._lib = _lib.load()
        self._h = ctypes.c_void_p()
        arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (A, B, q, r, x0)]
        self._keep = arrs
        A, B, q, r, x0 = arrs
        nx, nu = B.shape
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream")
                                                         else stream)
        check(self._lib.fga_horizon_create(ctypes.byref(self._h), int(K), nx, nu, *(ctypes.c_void_p(a.ctypes.data)
                                                                                     for a in arrs),
                                           float(rho), float(alpha), int(device), st), "fga_horizon_create")
        info = (ctypes.c_int64 * 4)()
        check(self._lib.fga_horizon_info(self._h, info, 4), "fga_horizon_info")
        self.K, self.grid, self.block, self.num_edges, self.num_scalar_vars = K, info[0], info[1], info[2], info[3]

    @classmethod
    def from_problem(cls, p, **kw):
        """From an inputs.mpc_horizon_problem description (no input box)."""
        m = p.meta
        if m.get("umax") is not None:
            raise ValueError("the input box is not supported here")
        return cls(m["K"], m["A"], m["B"], m["q"], m["r"], m["x0"], rho=p.rho, alpha=p.alpha, **kw)

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fga_horizon_destroy(self._h)
            self._h = None

    def fga_horizon_init(self):
        check(self._lib.fga_horizon_init(self._h), "fga_horizon_init")

    def fga_horizon_solve(self, max_iters, tol_pri=0.0, tol_dual=0.0, check_every=1, barrier_timeout_ns=0,
                          fault_skip_block=-1, raise_on_error=True):
        o = fga_iter_opts(int(max_iters), float(tol_pri), float(tol_dual), int(check_every), 1,
                          int(barrier_timeout_ns), int(fault_skip_block), 0)
        r = fga_iter_result()
        rc = self._lib.fga_horizon_solve(self._h, ctypes.byref(o), ctypes.byref(r))
        if raise_on_error:
            check(rc, "fga_horizon_solve")
        return dict(iters=r.iters, r_pri=r.r_pri, r_dual=r.r_dual, status=r.status, ms=r.ms, rc=rc)

    def fga_horizon_read(self):
        """(z, x, u) in FP64: z in variable order, x and u in creation order."""
        z = np.empty(self.num_scalar_vars)
        x = np.empty(self.num_edges)
        u = np.empty(self.num_edges)
        check(self._lib.fga_horizon_read(self._h, ctypes.c_void_p(z.ctypes.data), ctypes.c_void_p(x.ctypes.data),
                                         ctypes.c_void_p(u.ctypes.data)), "fga_horizon_read")
        return z, x, u
