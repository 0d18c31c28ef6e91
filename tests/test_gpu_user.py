"""GPU parity of user-supplied proximal operators (fga_register_prox).

The paper's addNode takes a factor's operator as a function pointer
(Sec. III); the library takes it as CUDA source, compiles it at run time and
runs it in its own x-update kernel.  The oracle runs the same operators as
Python functions through its function-pointer path (tests/test_oracle_user.py
pins that path).  FP64 graphs (canonical z order, no multiply-add
contraction on either side) must agree with the oracle bit for bit; FP32
graphs by the FP32 rules of the other parity tests.
"""
import numpy as np
import pytest

from oracle import OracleGraph
from oracle.oracle import EDGE_M, EDGE_N, EDGE_U, EDGE_X, T_EQUAL, T_MPC_BOX, T_MPC_QUAD
from paper_1603_02526_gb300 import _lib
from paper_1603_02526_gb300._lib import FGA_EDGE_M, FGA_EDGE_N, FGA_EDGE_U, FGA_EDGE_X, FgaError
from paper_1603_02526_gb300.graph import FactorGraph
from tests import test_oracle_user as uo

pytestmark = pytest.mark.gpu

# CUDA versions of the operators of tests/test_oracle_user.py, written with
# the same operations in the same order.
CUDA_SHIFTED_QUAD = r"""
template <typename R>
void shifted_quad(int d, const R *n, const R *rho, const R *p, R *x) {
    for (int k = 0; k < d; ++k) x[k] = (p[d + k] * p[k] + rho[k] * n[k]) / (p[d + k] + rho[k]);
}
"""
CUDA_L1 = r"""
template <typename R>
void soft_l1(int d, const R *n, const R *rho, const R *p, R *x) {
    for (int k = 0; k < d; ++k) {
        const R t = p[0] / rho[k];
        x[k] = n[k] > t ? n[k] - t : (n[k] < -t ? n[k] + t : R(0));
    }
}
"""
CUDA_QUAD0 = r"""
template <typename R>
void quad0(int d, const R *n, const R *rho, const R *p, R *x) {
    for (int k = 0; k < d; ++k) x[k] = (rho[k] * n[k]) / (p[k] + rho[k]);
}
"""
CUDA_BOX = r"""
template <typename R>
__device__ void box(int d, const R *n, const R *rho, const R *p, R *x) {
    for (int k = 0; k < d; ++k) x[k] = fmin(fmax(n[k], p[0]), p[1]);
}
"""

PAIRS_GPU = dict(x=FGA_EDGE_X, m=FGA_EDGE_M, u=FGA_EDGE_U, n=FGA_EDGE_N)
PAIRS_OR = dict(x=EDGE_X, m=EDGE_M, u=EDGE_U, n=EDGE_N)


def lasso_gpu(a, q, lam, rho, precision, zorder=None):
    N, d = a.shape
    g = FactorGraph(precision, 0)
    if zorder is not None:
        g.fga_set_option(_lib.FGA_OPT_ZORDER, zorder)
    if precision == "f64":
        g.fga_set_option(_lib.FGA_OPT_STORE_M, 1)
    g.fga_add_variables(1, d)
    tq = g.fga_register_prox(CUDA_SHIFTED_QUAD, "shifted_quad", d, 2 * d)
    tl = g.fga_register_prox(CUDA_L1, "soft_l1", d, 1)
    assert (tq, tl) == (_lib.FGA_USER_TYPE0, _lib.FGA_USER_TYPE0 + 1)
    g.fga_add_factors(tq, np.zeros((N, 1), dtype=np.int64), np.concatenate([a, q], axis=1))
    g.fga_add_factors(tl, np.zeros((1, 1), dtype=np.int64), [[lam]])
    g.fga_set_edge_rho_alpha(rho, None)
    g.fga_finalize()
    return g


def assert_bit_equal(g, o, which=("x", "m", "u", "n")):
    np.testing.assert_array_equal(g.fga_read_z(), o.z())
    for w in which:
        np.testing.assert_array_equal(g.fga_read_edge_state(PAIRS_GPU[w]), o.edge(PAIRS_OR[w]), err_msg=w)


@pytest.mark.parametrize("N,zorder", [(6, None), (40, 4)])
def test_lasso_f64_bit_exact_and_closed_form(N, zorder):
    """Canonical order (N = 6) and the scatter order with an overflow row
    (N = 40 edges per coordinate > the column count): the messages after
    200 iterations checked every 7, then the stop rule at 1e-12."""
    a, q, lam = uo.lasso_data(4, N, 2)
    rng = np.random.default_rng(9)
    E = N * 4 + 4
    rho = rng.uniform(0.5, 2.0, E)
    g = lasso_gpu(a, q, lam, rho, "f64", zorder)
    o = uo.build_lasso_oracle(a, q, lam, rho)
    g.fga_init()
    o.init()
    rg = g.fga_iterate(200, check_every=7)
    ro = o.iterate(200, check_every=7)
    assert rg["iters"] == ro["iters"] == 200
    if zorder is None:
        assert_bit_equal(g, o)
        assert rg["r_pri"] == pytest.approx(ro["r_pri"], rel=1e-12)
    else:
        for w in ("x", "u"):
            np.testing.assert_allclose(g.fga_read_edge_state(PAIRS_GPU[w]), o.edge(PAIRS_OR[w]), rtol=1e-10,
                                       atol=1e-12)
        np.testing.assert_allclose(g.fga_read_z(), o.z(), rtol=1e-10, atol=1e-12)
    rg = g.fga_iterate(20000, tol_pri=1e-12, tol_dual=1e-12)
    ro = o.iterate(20000, tol_pri=1e-12, tol_dual=1e-12)
    assert rg["status"] == 0 and rg["iters"] < 20000
    if zorder is None:
        assert rg["iters"] == ro["iters"]
        assert_bit_equal(g, o, which=("x", "u"))
    np.testing.assert_allclose(g.fga_read_z(), uo.lasso_minimiser(a, q, lam), rtol=0, atol=1e-9)


def test_lasso_f32_converges_to_the_closed_form():
    a, q, lam = uo.lasso_data(4, 6, 3)
    E = 6 * 4 + 4
    g = lasso_gpu(a, q, lam, np.full(E, 1.0), "f32")
    assert g.fga_launch_info()["zorder"] in (0, 4)
    g.fga_init()
    r = g.fga_iterate(20000, tol_pri=1e-6, tol_dual=1e-6, check_every=10)
    assert r["status"] == 0
    np.testing.assert_allclose(g.fga_read_z(), uo.lasso_minimiser(a, q, lam), rtol=0, atol=2e-5)


def chain_gpu(T, d, seed, user, precision, zorder=None):
    """tests/test_oracle_user.py cost_box_chain on the GPU (same seeds)."""
    rng = np.random.default_rng(seed)
    g = FactorGraph(precision, 0)
    if zorder is not None:
        g.fga_set_option(_lib.FGA_OPT_ZORDER, zorder)
    g.fga_add_variables(T, d)
    q = rng.uniform(0.1, 10.0, (T, d))
    box = np.array([-0.4, 0.6])
    if user:
        tq = g.fga_register_prox(CUDA_QUAD0, "quad0", d, d)
        tb = g.fga_register_prox(CUDA_BOX, "box", d, 2)
    else:
        tq, tb = T_MPC_QUAD, T_MPC_BOX
    ids = np.arange(T)[:, None]
    g.fga_add_factors(tq, ids, q)
    g.fga_add_factors(tb, ids, np.broadcast_to(box, (T, 2)))
    g.fga_add_factors(T_EQUAL, np.stack([np.arange(T - 1), np.arange(1, T)], axis=1))
    E = g.num_edges
    rho = rng.uniform(0.5, 2.0, E)
    alpha = rng.uniform(0.5, 1.0, E)
    g.fga_set_edge_rho_alpha(rho, alpha)
    g.fga_finalize()
    g.fga_init(rng.normal(0.0, 1.0, T * d))
    return g


@pytest.mark.parametrize("T", [8, 3000])
def test_restated_builtins_f64_equal_builtin_and_oracle(T):
    gu = chain_gpu(T, 3, 7, True, "f64")
    gb = chain_gpu(T, 3, 7, False, "f64")
    o = uo.cost_box_chain(T, 3, 7, user=True)
    ru = gu.fga_iterate(30, check_every=5)
    rb = gb.fga_iterate(30, check_every=5)
    ro = o.iterate(30, check_every=5)
    assert ru["iters"] == rb["iters"] == ro["iters"] == 30
    np.testing.assert_array_equal(gu.fga_read_z(), gb.fga_read_z())
    np.testing.assert_array_equal(gu.fga_read_z(), o.z())
    for w in ("x", "u"):
        np.testing.assert_array_equal(gu.fga_read_edge_state(PAIRS_GPU[w]), o.edge(PAIRS_OR[w]), err_msg=w)
        np.testing.assert_array_equal(gu.fga_read_edge_state(PAIRS_GPU[w]), gb.fga_read_edge_state(PAIRS_GPU[w]))


@pytest.mark.parametrize("zorder", [None, 0])
def test_restated_builtins_f32_against_oracle(zorder):
    """FP32 (scatter order by default, or canonical): 30 iterations of the
    3000-block chain within FP32 rounding of the oracle (|g - o| <= 2e-5 S,
    S the largest |z|), and the same as the built-in types' run to the same
    bound."""
    T = 3000
    gu = chain_gpu(T, 3, 7, True, "f32", zorder)
    gb = chain_gpu(T, 3, 7, False, "f32", zorder)
    o = uo.cost_box_chain(T, 3, 7, user=True)
    if zorder is None:
        assert gu.fga_launch_info()["zorder"] == 4
    gu.fga_iterate(30, check_every=5)
    gb.fga_iterate(30, check_every=5)
    o.iterate(30, check_every=5)
    zo = o.z()
    S = np.max(np.abs(zo))
    assert np.max(np.abs(gu.fga_read_z() - zo)) <= 2e-5 * S
    assert np.max(np.abs(gu.fga_read_z() - gb.fga_read_z())) <= 2e-5 * S
    for w in ("x", "u"):
        assert np.max(np.abs(gu.fga_read_edge_state(PAIRS_GPU[w]) - o.edge(PAIRS_OR[w]))) <= 2e-5 * S, w


def test_stop_rule_and_resume_f64():
    a, q, lam = uo.lasso_data(3, 5, 1)
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.5, 2.0, 5 * 3 + 3)
    g1 = lasso_gpu(a, q, lam, rho, "f64")
    g2 = lasso_gpu(a, q, lam, rho, "f64")
    o = uo.build_lasso_oracle(a, q, lam, rho)
    for x in (g1, g2):
        x.fga_init()
    o.init()
    r1 = g1.fga_iterate(5000, tol_pri=1e-9, tol_dual=1e-9, check_every=3)
    ro = o.iterate(5000, tol_pri=1e-9, tol_dual=1e-9, check_every=3)
    assert r1["iters"] == ro["iters"] and r1["status"] == 0
    # the same iterates in two calls: about half (a multiple of the check
    # interval), then the rest of the solve
    half = 3 * (r1["iters"] // 6)
    assert half > 0
    ra = g2.fga_iterate(half, check_every=3)
    rb = g2.fga_iterate(5000, tol_pri=1e-9, tol_dual=1e-9, check_every=3)
    assert ra["iters"] + rb["iters"] == r1["iters"]
    np.testing.assert_array_equal(g2.fga_read_z(), g1.fga_read_z())
    np.testing.assert_array_equal(g1.fga_read_z(), o.z())


def test_registration_errors():
    g = FactorGraph("f64", 0)
    g.fga_add_variables(2, 2)
    with pytest.raises(FgaError) as e:
        g.fga_register_prox("template <typename R> void bad(int d, const R *n) { x = ; }", "bad", 2, 0)
    assert e.value.code == _lib.FGA_EINVAL and "error" in str(e.value)
    with pytest.raises(FgaError):
        g.fga_register_prox(CUDA_BOX, "box;", 2, 2)   # not an identifier
    t = g.fga_register_prox(CUDA_BOX, "box", 2, 2)
    with pytest.raises(FgaError):
        g.fga_add_factors(t, [[0, 1]], [[0.0, 1.0]])   # arity 4, registered 2
    with pytest.raises(FgaError):
        g.fga_add_factors(t, [[0]], [[0.0, 1.0, 2.0]])   # 3 parameters
    g.fga_add_factors(t, [[0]], [[0.0, 1.0]])
    g.fga_set_option(_lib.FGA_OPT_ZORDER, 1)
    with pytest.raises(FgaError) as e:
        g.fga_finalize()
    assert e.value.code == _lib.FGA_EINVAL
