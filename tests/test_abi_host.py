"""CPU checks of the C-ABI library: it loads, exports every declared entry
point, and its host-side validation rejects bad input (no GPU needed until
fga_finalize)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1603_02526_gb300 import build, _lib
    build.build()
    return _lib.load()


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fga_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    headers = [h for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]
    names = []
    for h in headers:
        names += _declared(h)
    assert "fga_iterate" in names and "fga_finalize" in names
    for n in names:
        assert hasattr(lib, n), "libfgadmm.so does not export %s" % n


def test_version(lib):
    assert b"sm_103a" in lib.fga_version()


def _new(lib, prec=1):
    g = ctypes.c_void_p()
    assert lib.fga_graph_create(ctypes.byref(g), prec, 0, None) == 0
    return g


def test_validation_errors(lib):
    from paper_1603_02526_gb300._lib import FGA_EINVAL, FGA_ESTATE
    g = _new(lib)
    first = ctypes.c_int64()
    assert lib.fga_add_variables(g, 2, 2, ctypes.byref(first)) == 0 and first.value == 0
    assert lib.fga_add_variables(g, 2, 1, ctypes.byref(first)) == 0 and first.value == 2
    assert lib.fga_add_variables(g, 1, 0, None) == FGA_EINVAL
    ids = np.array([[0, 2, 1, 3]], dtype=np.int64)
    P = ctypes.c_void_p
    # a valid pair factor
    assert lib.fga_add_factors(g, 0, 1, 4, P(ids.ctypes.data), None, 0, 0, None) == 0
    # out-of-range variable id
    bad = np.array([[0, 2, 1, 9]], dtype=np.int64)
    assert lib.fga_add_factors(g, 0, 1, 4, P(bad.ctypes.data), None, 0, 0, None) == FGA_EINVAL
    assert b"out of range" in lib.fga_last_error()
    # wrong shape for the type (radius on a 2-D variable)
    one = np.array([[0]], dtype=np.int64)
    w = np.array([1.0])
    assert lib.fga_add_factors(g, 2, 1, 1, P(one.ctypes.data), P(w.ctypes.data), 1, 0, None) == FGA_EINVAL
    # wrong parameter count for a wall
    wall = np.array([[0, 2]], dtype=np.int64)
    q = np.array([0.0, 1.0, 0.0])
    assert lib.fga_add_factors(g, 1, 1, 2, P(wall.ctypes.data), P(q.ctypes.data), 3, 0, None) == FGA_EINVAL
    # unknown type
    assert lib.fga_add_factors(g, 42, 1, 1, P(one.ctypes.data), None, 0, 0, None) == FGA_EINVAL
    # box with lo > hi
    box = np.array([[2]], dtype=np.int64)
    lohi = np.array([1.0, -1.0])
    assert lib.fga_add_factors(g, 8, 1, 1, P(box.ctypes.data), P(lohi.ctypes.data), 2, 0, None) == FGA_EINVAL
    # rho / alpha must be > 0
    assert lib.fga_set_rho_alpha(g, 0.0, 1.0) == FGA_EINVAL
    assert lib.fga_set_rho_alpha(g, 1.0, -1.0) == FGA_EINVAL
    assert lib.fga_set_rho_alpha(g, 2.0, 1.0) == 0
    # options: bad values
    assert lib.fga_set_option(g, 2, 100) == FGA_EINVAL
    assert lib.fga_set_option(g, 0, 5) == FGA_EINVAL
    assert lib.fga_set_option(g, 0, -1) == FGA_EINVAL
    assert lib.fga_set_option(g, 0, 1) == 0
    # calls that need a finalized / initialised graph
    out = np.zeros(6)
    assert lib.fga_read_z(g, P(out.ctypes.data), 6) == FGA_ESTATE
    assert lib.fga_init(g, None, None) == FGA_ESTATE
    # the latency floor: arguments first, then a finalized graph
    ms = ctypes.c_float()
    assert lib.fga_latency_floor(None, 10, 1, ctypes.byref(ms)) == FGA_EINVAL
    assert lib.fga_latency_floor(g, 0, 1, ctypes.byref(ms)) == FGA_EINVAL
    assert lib.fga_latency_floor(g, 10, 2, ctypes.byref(ms)) == FGA_EINVAL
    assert lib.fga_latency_floor(g, 10, 1, None) == FGA_EINVAL
    assert lib.fga_latency_floor(g, 10, 1, ctypes.byref(ms)) == FGA_ESTATE
    e, z, f, v = (ctypes.c_int64() for _ in range(4))
    assert lib.fga_graph_info(g, ctypes.byref(e), ctypes.byref(z), ctypes.byref(f), ctypes.byref(v)) == 0
    assert (e.value, z.value, f.value, v.value) == (6, 6, 1, 4)
    assert lib.fga_destroy(g) == 0


def test_create_rejects_bad_precision(lib):
    g = ctypes.c_void_p()
    assert lib.fga_graph_create(ctypes.byref(g), 7, 0, None) == -1
    assert lib.fga_graph_create(None, 0, 0, None) == -1


def test_binding_counts_match_problem(lib):
    """The binding registers a packing problem with the counts of Sec. V-A."""
    from paper_1603_02526_gb300 import inputs
    from paper_1603_02526_gb300.graph import FactorGraph, _merge_var_blocks
    p = inputs.packing_problem(20)
    g = FactorGraph("f32")
    for c, d in _merge_var_blocks(p.var_blocks):
        g.fga_add_variables(c, d)
    for b in p.factor_blocks:
        g.fga_add_factors(b.ftype, b.var_ids, b.params if b.params.size else None)
    info = g.fga_graph_info()
    assert info["num_edges"] == p.num_edges == 1340
    assert info["num_factors"] == inputs.packing_counts(20)["factors"]
    assert info["num_vars"] == 40


def test_paper_svm_types_validation(lib):
    """Shapes and parameters of the margin, minimal-error and equality types
    (Appendix C) are checked at registration."""
    from paper_1603_02526_gb300._lib import FGA_EINVAL
    from paper_1603_02526_gb300 import inputs
    g = _new(lib, 0)
    first = ctypes.c_int64()
    assert lib.fga_add_variables(g, 2, 3, ctypes.byref(first)) == 0            # w copies: ids 0, 1
    assert lib.fga_add_variables(g, 2, 1, ctypes.byref(first)) == 0            # b, xi: ids 2, 3
    P = ctypes.c_void_p
    eq_ok = np.array([[0, 1]], dtype=np.int64)
    eq_bad = np.array([[0, 2]], dtype=np.int64)                               # dims 3 and 1
    assert lib.fga_add_factors(g, inputs.EQUAL, 1, 2, P(eq_ok.ctypes.data), None, 0, 0, None) == 0
    assert lib.fga_add_factors(g, inputs.EQUAL, 1, 2, P(eq_bad.ctypes.data), None, 0, 0, None) == FGA_EINVAL
    mg = np.array([[0, 2, 3]], dtype=np.int64)
    xy = np.array([0.5, -1.0, 2.0, 1.0])                                      # x[3], y
    assert lib.fga_add_factors(g, inputs.SVM_MARGIN, 1, 3, P(mg.ctypes.data), P(xy.ctypes.data), 4, 0, None) == 0
    assert lib.fga_add_factors(g, inputs.SVM_MARGIN, 1, 3, P(mg.ctypes.data), P(xy.ctypes.data), 3, 0,
                               None) == FGA_EINVAL                            # parameter count
    mg_bad = np.array([[0, 2, 1]], dtype=np.int64)                            # xi of dimension 3
    assert lib.fga_add_factors(g, inputs.SVM_MARGIN, 1, 3, P(mg_bad.ctypes.data), P(xy.ctypes.data), 4, 0,
                               None) == FGA_EINVAL
    sl = np.array([[3]], dtype=np.int64)
    lam_ok, lam_bad = np.array([0.5]), np.array([-1.0])
    assert lib.fga_add_factors(g, inputs.SVM_SLACK, 1, 1, P(sl.ctypes.data), P(lam_ok.ctypes.data), 1, 0, None) == 0
    assert lib.fga_add_factors(g, inputs.SVM_SLACK, 1, 1, P(sl.ctypes.data), P(lam_bad.ctypes.data), 1, 0,
                               None) == FGA_EINVAL
    assert lib.fga_destroy(g) == 0


@pytest.mark.parametrize("which", ["svm_paper", "mpc_horizon"])
def test_binding_counts_match_new_workloads(lib, which):
    """The binding registers the paper-form SVM and the long-horizon MPC with
    the counts their generators state."""
    from paper_1603_02526_gb300 import inputs
    from paper_1603_02526_gb300.graph import FactorGraph, _merge_var_blocks
    if which == "svm_paper":
        p = inputs.svm_paper_problem(50, 4, seed=1)
        want = inputs.svm_paper_edges(50, 4)
    else:
        p = inputs.mpc_horizon_problem(300)
        want = inputs.mpc_horizon_edges(300)
    g = FactorGraph("f32")
    for c, d in _merge_var_blocks(p.var_blocks):
        g.fga_add_variables(c, d)
    for b in p.factor_blocks:
        g.fga_add_factors(b.ftype, b.var_ids, b.params if b.params.size else None)
    info = g.fga_graph_info()
    assert info["num_edges"] == p.num_edges == want
    assert info["num_factors"] == p.num_factors
    assert info["num_vars"] == p.num_vars


def test_factor_type_numbers_agree():
    """The factor-type numbers are an interface written down three times (the
    C header, the input generators, the oracle); they must agree."""
    import re
    from paper_1603_02526_gb300 import inputs
    import oracle.oracle as orc
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "fgadmm.h")).read()
    names = ["PACK_PAIR", "PACK_WALL", "PACK_RADIUS_LIN", "PACK_RADIUS_QUAD", "SVM_HINGE", "SVM_L2", "MPC_DYN",
             "MPC_QUAD", "MPC_BOX", "FIX", "SVM_MARGIN", "SVM_SLACK", "EQUAL"]
    for n in names:
        m = re.search(r"#define FGA_%s (\d+)" % n, hdr)
        assert m, n
        assert int(m.group(1)) == getattr(inputs, n) == getattr(orc, "T_" + n), n
    assert int(re.search(r"#define FGA_NUM_TYPES (\d+)", hdr).group(1)) == len(names)


def test_horizon_create_validation(lib):
    """fga_horizon_create refuses bad shapes and parameters before it touches
    a device."""
    from paper_1603_02526_gb300._lib import FGA_EINVAL
    P = ctypes.c_void_p
    h = ctypes.c_void_p()
    A, B = np.eye(4), np.ones((4, 1))
    q, r, x0 = np.ones(4), np.ones(1), np.zeros(4)
    ptrs = [P(v.ctypes.data) for v in (A, B, q, r, x0)]
    assert lib.fga_horizon_create(ctypes.byref(h), 10, 12, 4, *ptrs, 1.0, 1.0, 0, None) == FGA_EINVAL
    assert b"nx = 4" in lib.fga_last_error()
    assert lib.fga_horizon_create(ctypes.byref(h), 0, 4, 1, *ptrs, 1.0, 1.0, 0, None) == FGA_EINVAL
    assert lib.fga_horizon_create(ctypes.byref(h), 10, 4, 1, *ptrs, 0.0, 1.0, 0, None) == FGA_EINVAL
    assert lib.fga_horizon_create(ctypes.byref(h), 10, 4, 1, None, *ptrs[1:], 1.0, 1.0, 0, None) == FGA_EINVAL
    qn = -np.ones(4)
    assert lib.fga_horizon_create(ctypes.byref(h), 10, 4, 1, ptrs[0], ptrs[1], P(qn.ctypes.data), ptrs[3], ptrs[4],
                                  1.0, 1.0, 0, None) == FGA_EINVAL
    assert lib.fga_horizon_init(None) == FGA_EINVAL
    assert lib.fga_horizon_destroy(None) == 0


def test_register_prox_argument_checks(lib):
    """Host-side checks of fga_register_prox and of user type numbers (the
    compilation itself needs the GPU and is covered by the GPU tests)."""
    from paper_1603_02526_gb300._lib import FGA_EINVAL, FGA_USER_TYPE0
    g = _new(lib)
    t = ctypes.c_int32()
    assert lib.fga_register_prox(g, None, b"f", 1, 0, ctypes.byref(t)) == FGA_EINVAL
    assert lib.fga_register_prox(g, b"src", None, 1, 0, ctypes.byref(t)) == FGA_EINVAL
    assert lib.fga_register_prox(g, b"src", b"f", 0, 0, ctypes.byref(t)) == FGA_EINVAL
    assert lib.fga_register_prox(g, b"src", b"f", 65, 0, ctypes.byref(t)) == FGA_EINVAL
    assert lib.fga_register_prox(g, b"src", b"f", 1, -1, ctypes.byref(t)) == FGA_EINVAL
    assert lib.fga_add_variables(g, 1, 1, None) == 0
    one = np.array([[0]], dtype=np.int64)
    # no operator registered: user type numbers are unknown types
    assert lib.fga_add_factors(g, FGA_USER_TYPE0, 1, 1, ctypes.c_void_p(one.ctypes.data), None, 0, 0,
                               None) == FGA_EINVAL
    assert lib.fga_destroy(g) == 0


def test_batch_network_and_handle_validation(lib):
    """Entry points outside the graph object reject bad input on the host
    with FGA_EINVAL and a message naming the call; NULL handles are
    rejected, NULL destroys are no-ops, and a graph not yet finalized gives
    FGA_ESTATE.  Every call here fails its checks before any device work."""
    from paper_1603_02526_gb300._lib import FGA_EINVAL, FGA_ESTATE, fga_iter_opts, fga_iter_result
    P = ctypes.c_void_p
    ptr = lambda a: P(a.ctypes.data)
    nx, nu, n = 3, 1, 2
    T = np.array([5, 7], dtype=np.int32)
    A = np.eye(nx)
    B = np.ones((nx, nu))
    q = np.ones(nx)
    r = np.ones(nu)
    out = P()

    def batch(**kw):
        a = dict(out=ctypes.byref(out), prec=1, n=n, T=ptr(T), nx=nx, nu=nu, nsys=1, sys=None, A=ptr(A),
                 B=ptr(B), q=ptr(q), r=ptr(r), umax=1.0, rho=1.0, alpha=1.0)
        a.update(kw)
        return lib.fga_mpc_batch_create(a["out"], a["prec"], 0, None, a["n"], a["T"], a["nx"], a["nu"],
                                        a["nsys"], a["sys"], a["A"], a["B"], a["q"], a["r"], a["umax"],
                                        a["rho"], a["alpha"])

    qneg = -np.ones(nx)
    for kw in (dict(out=None), dict(prec=5), dict(nx=0), dict(nx=30, nu=5), dict(rho=0.0), dict(umax=-1.0),
               dict(nsys=2, n=3), dict(q=ptr(qneg)), dict(T=None)):
        assert batch(**kw) == FGA_EINVAL, kw
        assert b"fga_mpc_batch_create" in lib.fga_last_error(), kw

    m = P()
    assert lib.fga_mlp_create(None, 12, 64, 64, 16, 64, 1, 0, None) == FGA_EINVAL
    for shape in ((12, 60, 64, 16, 64), (12, 64, 64, 16, 4), (0, 64, 64, 16, 64), (12, 64, 64, 12, 64)):
        assert lib.fga_mlp_create(ctypes.byref(m), *shape, 1, 0, None) == FGA_EINVAL, shape
        assert b"fga_mlp_create" in lib.fga_last_error()

    f = lib.fga_mpc_solve_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, ctypes.c_float, ctypes.c_float,
                  ctypes.c_float, ctypes.c_int64, ctypes.c_double, ctypes.c_int32, P, P, P, P]
    buf = np.zeros(64, dtype=np.float32)
    b = ptr(buf)

    def noalloc(**kw):
        a = dict(n=n, T=ptr(T), nx=nx, nu=nu, umax=1.0, rho=1.0, alpha=1.0, iters=100, tol=1e-4, ce=1, z=b)
        a.update(kw)
        return f(a["n"], a["T"], a["nx"], a["nu"], b, b, b, b, b, a["umax"], a["rho"], a["alpha"], a["iters"],
                 a["tol"], a["ce"], a["z"], b, b, None)

    T0 = np.array([5, 0], dtype=np.int32)
    Tbig = np.array([5, 100001], dtype=np.int32)
    for kw in (dict(n=0), dict(n=4097), dict(nx=33), dict(nx=0), dict(nu=0), dict(rho=0.0), dict(ce=0),
               dict(iters=-1), dict(tol=-1.0), dict(z=None), dict(T=None), dict(T=ptr(T0)), dict(T=ptr(Tbig))):
        assert noalloc(**kw) == FGA_EINVAL, kw
        assert b"fga_mpc_solve_noalloc" in lib.fga_last_error(), kw

    info = (ctypes.c_int64 * 8)()
    d = ctypes.c_double()
    opts, res = fga_iter_opts(), fga_iter_result()
    assert lib.fga_residuals(None, ctypes.byref(d), ctypes.byref(d)) == FGA_EINVAL
    assert lib.fga_read_edge_state(None, 0, None, 0) == FGA_EINVAL
    assert lib.fga_launch_info(None, info, 8) == FGA_EINVAL
    assert lib.fga_set_edge_rho_alpha(None, None, None) == FGA_EINVAL
    assert lib.fga_set_stream(None, None) == FGA_EINVAL
    assert lib.fga_horizon_solve(None, ctypes.byref(opts), ctypes.byref(res)) == FGA_EINVAL
    assert lib.fga_horizon_read(None, None, None, None) == FGA_EINVAL
    assert lib.fga_horizon_info(None, info, 8) == FGA_EINVAL
    assert lib.fga_mpc_batch_info(None, info, 8) == FGA_EINVAL
    assert lib.fga_mlp_num_params(None, info) == FGA_EINVAL
    assert lib.fga_mpc_batch_destroy(None) == 0 and lib.fga_mlp_destroy(None) == 0

    g = _new(lib)
    assert lib.fga_add_variables(g, 2, 1, None) == 0
    ids = np.array([[0], [1]], dtype=np.int64)
    lohi = np.array([-1.0, 1.0])
    assert lib.fga_add_factors(g, 8, 2, 1, P(ids.ctypes.data), P(lohi.ctypes.data), 2, 1, None) == 0
    out2 = np.zeros(2)
    assert lib.fga_read_edge_state(g, 0, P(out2.ctypes.data), 2) == FGA_ESTATE
    assert lib.fga_launch_info(g, info, 8) == FGA_ESTATE
    bad = np.array([1.0, 0.0])
    assert lib.fga_set_edge_rho_alpha(g, P(bad.ctypes.data), None) == FGA_EINVAL
    nan = np.array([1.0, np.nan])
    assert lib.fga_set_edge_rho_alpha(g, None, P(nan.ctypes.data)) == FGA_EINVAL
    good = np.array([1.0, 2.0])
    assert lib.fga_set_edge_rho_alpha(g, P(good.ctypes.data), P(good.ctypes.data)) == 0
    assert lib.fga_destroy(g) == 0
