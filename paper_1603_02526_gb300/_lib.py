"""ctypes loader for libfgadmm.so (the C-ABI of include/fgadmm.h).

The library is built in-tree by ``paper_1603_02526_gb300.build``.  If it is
missing, every entry point raises: there is no CPU fallback.
"""
import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfgadmm.so")

_lock = threading.Lock()
_lib = None

# status codes (include/fgadmm.h)
FGA_OK = 0
FGA_EINVAL = -1
FGA_ENOMEM = -2
FGA_ECUDA = -3
FGA_ESTATE = -4
FGA_ETIMEOUT = -5
FGA_ENONFINITE = -6
FGA_EBUDGET = -7
STATUS_NAMES = {0: "FGA_OK", -1: "FGA_EINVAL", -2: "FGA_ENOMEM", -3: "FGA_ECUDA", -4: "FGA_ESTATE",
                -5: "FGA_ETIMEOUT", -6: "FGA_ENONFINITE", -7: "FGA_EBUDGET"}

FGA_F32 = 0
FGA_F64 = 1
FGA_EDGE_X, FGA_EDGE_M, FGA_EDGE_U, FGA_EDGE_N = 0, 1, 2, 3
FGA_OPT_ZORDER, FGA_OPT_STORE_M, FGA_OPT_BLOCK, FGA_OPT_WEIGHTS = 0, 1, 2, 3
FGA_USER_TYPE0 = 64


class FgaError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__("%s failed: %s (%s)" % (where, msg, STATUS_NAMES.get(code, code)))
        self.code = code


class fga_iter_opts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int64), ("tol_pri", ctypes.c_double), ("tol_dual", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("fused", ctypes.c_int32),
                ("barrier_timeout_ns", ctypes.c_int64), ("fault_skip_block", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class fga_mpc_opts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int64), ("tol_pri", ctypes.c_double), ("tol_dual", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("threads", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class fga_mpc_result(ctypes.Structure):
    _fields_ = [("total_iters", ctypes.c_int64), ("max_inst_iters", ctypes.c_int64),
                ("n_converged", ctypes.c_int32), ("n_budget", ctypes.c_int32), ("n_nonfinite", ctypes.c_int32),
                ("ms", ctypes.c_float), ("threads", ctypes.c_int32), ("check_every", ctypes.c_int32)]


class fga_iter_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("r_pri", ctypes.c_double), ("r_dual", ctypes.c_double),
                ("status", ctypes.c_int32), ("ms", ctypes.c_float)]


def _declare(lib):
    P = ctypes.c_void_p
    PP = ctypes.POINTER(ctypes.c_void_p)
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    pi64 = ctypes.POINTER(ctypes.c_int64)
    pdbl = ctypes.POINTER(ctypes.c_double)
    sigs = {
        "fga_graph_create": [PP, i32, i32, P],
        "fga_set_stream": [P, P],
        "fga_set_option": [P, i32, i64],
        "fga_add_variables": [P, i64, i32, pi64],
        "fga_add_factors": [P, i32, i64, i32, P, P, i32, i32, pi64],
        "fga_register_prox": [P, ctypes.c_char_p, ctypes.c_char_p, i32, i32, ctypes.POINTER(ctypes.c_int32)],
        "fga_set_rho_alpha": [P, dbl, dbl],
        "fga_set_edge_rho_alpha": [P, P, P],
        "fga_finalize": [P],
        "fga_graph_info": [P, pi64, pi64, pi64, pi64],
        "fga_init": [P, P, P],
        "fga_iterate": [P, ctypes.POINTER(fga_iter_opts), ctypes.POINTER(fga_iter_result)],
        "fga_residuals": [P, pdbl, pdbl],
        "fga_launch_info": [P, pi64, i32],
        "fga_latency_floor": [P, i64, i32, ctypes.POINTER(ctypes.c_float)],
        "fga_read_z": [P, P, i64],
        "fga_read_edge_state": [P, i32, P, i64],
        "fga_destroy": [P],
        "fga_mpc_batch_create": [PP, i32, i32, P, i32, P, i32, i32, i32, P, P, P, P, P, dbl, dbl, dbl],
        "fga_mpc_batch_set_x0": [P, P],
        "fga_mpc_batch_init": [P, P, P],
        "fga_mpc_batch_warm_start": [P, P, i64],
        "fga_mpc_batch_targets": [P, P, i64],
        "fga_mpc_batch_solve": [P, ctypes.POINTER(fga_mpc_opts), ctypes.POINTER(fga_mpc_result)],
        "fga_mpc_batch_read": [P, P, P, P, P, P, P],
        "fga_mpc_batch_info": [P, pi64, i32],
        "fga_mpc_batch_autotune": [P, ctypes.c_char_p, i64, dbl, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32)],
        "fga_mpc_batch_destroy": [P],
        "fga_horizon_create": [PP, i32, i32, i32, P, P, P, P, P, dbl, dbl, i32, P],
        "fga_horizon_init": [P],
        "fga_horizon_solve": [P, ctypes.POINTER(fga_iter_opts), ctypes.POINTER(fga_iter_result)],
        "fga_horizon_read": [P, P, P, P],
        "fga_horizon_info": [P, pi64, i32],
        "fga_horizon_destroy": [P],
        "fga_mlp_create": [PP, i32, i32, i32, i32, i32, ctypes.c_uint64, i32, P],
        "fga_mlp_num_params": [P, pi64],
        "fga_mlp_set_params": [P, P, i64],
        "fga_mlp_get_params": [P, P, i64],
        "fga_mlp_fit_normalization": [P, P, i64],
        "fga_mlp_get_normalization": [P, P, P],
        "fga_mlp_gradients": [P, P, P, i32, P, pdbl],
        "fga_mlp_train_step": [P, P, P, i32, ctypes.c_float, pdbl],
        "fga_mlp_forward": [P, P, P, i32],
        "fga_mlp_destroy": [P],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.fga_last_error.restype = ctypes.c_char_p
    lib.fga_last_error.argtypes = []
    lib.fga_version.restype = ctypes.c_char_p
    lib.fga_version.argtypes = []


def load():
    """Returns the loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfgadmm.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_1603_02526_gb300.build" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        _declare(lib)
        _lib = lib
        return lib


def check(code, where):
    if code != FGA_OK:
        msg = load().fga_last_error().decode(errors="replace")
        raise FgaError(code, where, msg)
    return code
