"""ctypes wrapper around the serial FP64 C oracle (``fga_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product library.

The oracle follows Algorithm 2 of the paper (Sec. II) literally: five loops
per iteration over factors, edges, variables, edges, edges, in FP64, with
edge arrays in creation order (Sec. III) and each z-sum taken over the
variable's edges in ascending creation order.
"""
import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fga_oracle.c")
_SO = os.path.join(_HERE, "_build", "libfga_oracle.so")
_lock = threading.Lock()
_lib = None

# Factor types: interface numbers agreed with the library, written down here
# independently of it.
T_PACK_PAIR = 0
T_PACK_WALL = 1
T_PACK_RADIUS_LIN = 2
T_PACK_RADIUS_QUAD = 3
T_SVM_HINGE = 4
T_SVM_L2 = 5
T_MPC_DYN = 6
T_MPC_QUAD = 7
T_MPC_BOX = 8
T_FIX = 9
T_SVM_MARGIN = 10
T_SVM_SLACK = 11
T_EQUAL = 12
T_USER0 = 64   # first type number of user-supplied operators (og_register_prox)

EDGE_X, EDGE_M, EDGE_U, EDGE_N = 0, 1, 2, 3


def build_oracle(force=False):
    """Compiles the oracle with gcc (-O2, no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = _declare(ctypes.CDLL(build_oracle()))
        return _lib


def build_variant(source_text, path):
    """Compiles `source_text` (a modified copy of the oracle's C source) with
    the oracle's flags into `path` and loads it.  For the planted-mistake
    tests only: they check that the pins fail on such builds."""
    src = path + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
                           "-fPIC", "-shared", "-o", path, src, "-lm"])
    return _declare(ctypes.CDLL(path))


@contextlib.contextmanager
def using_build(lib):
    """Routes every oracle call in the block to `lib` (a build_variant)."""
    global _lib
    _load()
    with _lock:
        saved = _lib
        _lib = lib
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def source_text():
    with open(_SRC) as fh:
        return fh.read()


def _declare(lib):
    """Argument and result types of the oracle's C entry points."""
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_int64)
    ip = ctypes.POINTER(ctypes.c_int32)
    lib.og_new.restype = P
    lib.og_free.argtypes = [P]
    lib.og_add_vars.argtypes = [P, i64, i32]
    lib.og_add_vars.restype = i64
    lib.og_add_factors.argtypes = [P, i32, i64, i32, lp, i32, dp]
    lib.og_add_factors.restype = i64
    lib.og_num_edges.argtypes = [P]
    lib.og_num_edges.restype = i64
    lib.og_num_scalar_vars.argtypes = [P]
    lib.og_num_scalar_vars.restype = i64
    lib.og_finalize.argtypes = [P]
    lib.og_set_rho_alpha.argtypes = [P, dp, dp, dbl, dbl]
    lib.og_init.argtypes = [P, dp, dp]
    lib.og_iterate.argtypes = [P, i64, dbl, dbl, i32, lp, dp, dp]
    lib.og_get_edge.argtypes = [P, i32, dp]
    lib.og_get_z.argtypes = [P, dp]
    lib.og_get_edge_var.argtypes = [P, lp]
    lib.og_prox.argtypes = [i32, i32, ip, dp, dp, dp, dp]
    lib.og_set_weights.argtypes = [P, i32]
    lib.og_register_prox.argtypes = [P, PROX_FN, P, i32, i32]
    lib.og_register_prox.restype = i32
    return lib


# og_prox_fn: (arity, n, rho, params, x, ctx), see og_register_prox
PROX_FN = ctypes.CFUNCTYPE(None, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def oracle_prox(ftype, dims, params, rho, n):
    """Evaluates one factor's proximal operator (Eq. PO) in the oracle."""
    lib = _load()
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    params = np.ascontiguousarray(params if params is not None else [0.0], dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    x = np.zeros_like(n)
    rc = lib.og_prox(ftype, len(dims), dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                     _dp(params), _dp(rho), _dp(n), _dp(x))
    if rc != 0:
        raise ValueError("oracle prox rejected the input (status %d)" % rc)
    return x


class OracleGraph:
    """A factor graph held by the oracle; mirrors the library's build calls."""

    def __init__(self):
        self._lib = _load()
        self._g = self._lib.og_new()
        self.finalized = False
        self._callbacks = []   # user operators: kept alive as long as the graph

    def __del__(self):
        try:
            if self._g:
                self._lib.og_free(self._g)
                self._g = None
        except Exception:
            pass

    def add_variables(self, count, dim):
        r = self._lib.og_add_vars(self._g, int(count), int(dim))
        if r < 0:
            raise ValueError("oracle: bad variables")
        return r

    def register_prox(self, fn, arity, n_params):
        """Registers a user-supplied proximal operator (the paper's addNode
        takes it as a function pointer, Sec. III): fn(n, rho, params) returns
        x = Prox_{f,rho}(n) for one factor, all FP64 arrays (n and rho of
        length `arity` in creation order, params of length `n_params`).
        Returns the new type number (T_USER0, T_USER0 + 1, ...)."""
        def call(arity_c, n, rho, prm, x, ctx):
            nn = np.ctypeslib.as_array(n, shape=(arity_c,)).copy()
            rr = np.ctypeslib.as_array(rho, shape=(arity_c,)).copy()
            pp = (np.ctypeslib.as_array(prm, shape=(n_params,)).copy() if n_params
                  else np.zeros(0))
            np.ctypeslib.as_array(x, shape=(arity_c,))[:] = np.asarray(fn(nn, rr, pp), dtype=np.float64)

        cb = PROX_FN(call)
        t = self._lib.og_register_prox(self._g, cb, None, int(arity), int(n_params))
        if t < 0:
            raise ValueError("oracle: operator not registered")
        self._callbacks.append(cb)
        return t

    def add_factors(self, ftype, var_ids, params=None):
        """var_ids: (count, nv) ids; params: (count, np), or (np,) shared by all."""
        var_ids = np.ascontiguousarray(var_ids, dtype=np.int64)
        if var_ids.ndim == 1:
            var_ids = var_ids[None, :]
        count, nv = var_ids.shape
        if params is None:
            params = np.zeros((count, 0))
        params = np.asarray(params, dtype=np.float64)
        if params.ndim == 1:
            params = np.broadcast_to(params, (count, params.shape[0]))
        params = np.ascontiguousarray(params)
        pbuf = params if params.size else np.zeros(1)
        r = self._lib.og_add_factors(self._g, ftype, count, nv, _lp(var_ids), params.shape[1], _dp(pbuf))
        if r < 0:
            raise ValueError("oracle: bad factors (type %d)" % ftype)
        return r

    def finalize(self, rho=1.0, alpha=1.0):
        rc = self._lib.og_finalize(self._g)
        if rc != 0:
            raise RuntimeError("oracle finalize failed: %d" % rc)
        self.finalized = True
        self.set_rho_alpha(rho, alpha)

    def set_rho_alpha(self, rho=1.0, alpha=1.0):
        E = self.num_edges
        rp = ap = None
        ru = au = 1.0
        if np.ndim(rho) == 0:
            ru = float(rho)
        else:
            rho = np.ascontiguousarray(rho, dtype=np.float64)
            assert rho.shape == (E,)
            rp = _dp(rho)
        if np.ndim(alpha) == 0:
            au = float(alpha)
        else:
            alpha = np.ascontiguousarray(alpha, dtype=np.float64)
            assert alpha.shape == (E,)
            ap = _dp(alpha)
        rc = self._lib.og_set_rho_alpha(self._g, rp, ap, ru, au)
        if rc != 0:
            raise ValueError("oracle: bad rho/alpha")

    def set_weights(self, mode):
        """0: fixed rho per edge (Algorithm 2 as printed); 1: three weights
        (weight classes zero / standard / infinite set by each x-update;
        see og_set_weights in fga_oracle.c)."""
        rc = self._lib.og_set_weights(self._g, int(mode))
        if rc != 0:
            raise ValueError("oracle: bad weight mode")

    @property
    def num_edges(self):
        return int(self._lib.og_num_edges(self._g))

    @property
    def num_scalar_vars(self):
        return int(self._lib.og_num_scalar_vars(self._g))

    def init(self, z0=None, u0=None):
        zp = up = None
        if z0 is not None:
            z0 = np.ascontiguousarray(z0, dtype=np.float64)
            assert z0.shape == (self.num_scalar_vars,)
            zp = _dp(z0)
        if u0 is not None:
            u0 = np.ascontiguousarray(u0, dtype=np.float64)
            assert u0.shape == (self.num_edges,)
            up = _dp(u0)
        rc = self._lib.og_init(self._g, zp, up)
        if rc != 0:
            raise RuntimeError("oracle init failed: %d" % rc)

    def iterate(self, max_iters, tol_pri=0.0, tol_dual=0.0, check_every=1):
        it = ctypes.c_int64(0)
        rp = ctypes.c_double(0)
        rd = ctypes.c_double(0)
        rc = self._lib.og_iterate(self._g, int(max_iters), float(tol_pri), float(tol_dual),
                                  int(check_every), ctypes.byref(it), ctypes.byref(rp), ctypes.byref(rd))
        return dict(status=rc, iters=it.value, r_pri=rp.value, r_dual=rd.value)

    def edge(self, which):
        out = np.empty(self.num_edges, dtype=np.float64)
        rc = self._lib.og_get_edge(self._g, int(which), _dp(out))
        if rc != 0:
            raise RuntimeError("oracle readout failed")
        return out

    def z(self):
        out = np.empty(self.num_scalar_vars, dtype=np.float64)
        self._lib.og_get_z(self._g, _dp(out))
        return out

    def edge_var(self):
        out = np.empty(self.num_edges, dtype=np.int64)
        self._lib.og_get_edge_var(self._g, _lp(out))
        return out


def from_problem(problem, z0=True, weights=0):
    """Loads a problem description (variable blocks, factor blocks, rho,
    alpha, start point) into a fresh oracle graph and initialises it;
    weights: the weight mode (set_weights)."""
    g = OracleGraph()
    for count, dim in problem.var_blocks:
        g.add_variables(count, dim)
    for blk in problem.factor_blocks:
        g.add_factors(blk.ftype, blk.var_ids, blk.params)
    g.finalize(problem.rho, problem.alpha)
    if weights:
        g.set_weights(weights)
    g.init(problem.z0 if z0 else None)
    return g
