"""GPU parity of the long-horizon MPC (Sec. V-B: one inverted-pendulum
instance, A 4 x 4, B 4 x 1 sampled at 40 ms, horizon K up to 10^5) as a
single factor graph, against the FP64 oracle through the C-ABI.

FP64 runs use the canonical z order and must match the oracle to 1e-9
relative per message (floor 1e-3 of the array's scale): the z sums are the
oracle's, but the dynamics operator is applied here as a precomputed
projection matrix and in the oracle by a Cholesky solve per call, which
round differently (a few ulps per iteration, not amplified).  FP32 runs
use the chunked fast order here (the scatter order, the FP32 default for
this graph, has its own tests with the same bounds).  Tolerance: one iteration rounds each message
by a few FP32 ulps of the variables' scale S (the dynamics operator is a
9-term dot product: at most about 9 * 2^-24 * S = 5.4e-7 S); the method on
this convex problem does not amplify earlier errors (each iteration is a
nonexpansive map), so after k iterations the error is at most k times that
if every rounding added up with the same sign: 300 iterations -> 1.6e-4 S,
20 iterations -> 1.1e-5 S."""
import numpy as np
import pytest

from oracle import from_problem as oracle_from_problem
from paper_1603_02526_gb300 import inputs
from paper_1603_02526_gb300 import _lib
from paper_1603_02526_gb300.graph import graph_from_problem
from tests.helpers import assert_messages_close_scaled, assert_messages_match

pytestmark = pytest.mark.gpu

F32_PER_ITER = 9 * 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


@pytest.mark.parametrize("fused", [True, False])
def test_horizon_f64(fused):
    """K = 500 (7,008 scalar edges: several chunks and a ragged tail), 300
    iterations, every message within 1e-9 of the oracle's."""
    p = inputs.mpc_horizon_problem(500)
    g = graph_from_problem(p, "f64")
    r = g.fga_iterate(300, fused=fused)
    o = oracle_from_problem(p)
    ro = o.iterate(300)
    assert r["iters"] == ro["iters"] == 300
    assert_messages_match(g, o, 1e-9)


@pytest.mark.parametrize("K", [1, 37, 500])
def test_horizon_f32_chunked_order(K):
    """FP32 fast order, 300 iterations, every message within the bound of
    the module docstring (300 iterations: 1.6e-4 S)."""
    p = inputs.mpc_horizon_problem(K)
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1, _lib.FGA_OPT_ZORDER: 1})
    g.fga_iterate(300)
    o = oracle_from_problem(p)
    o.iterate(300)
    assert_messages_close_scaled(g, o, 300 * F32_PER_ITER)


def test_horizon_full_size_f64_and_f32():
    """K = 10^5 (1,400,008 scalar edges), the size the benchmark times: 20
    iterations in FP64 (1e-9 per message) and in FP32 (20 iterations:
    1.1e-5 S)."""
    K = 100000
    p = inputs.mpc_horizon_problem(K)
    o = oracle_from_problem(p)
    o.iterate(20)
    g = graph_from_problem(p, "f64")
    g.fga_iterate(20)
    assert_messages_match(g, o, 1e-9)
    del g
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1, _lib.FGA_OPT_ZORDER: 1})
    g.fga_iterate(20)
    assert_messages_close_scaled(g, o, 20 * F32_PER_ITER)


def test_horizon_converges_to_lqr():
    """K = 2000 in FP64 to RMS residual 1e-12 (the RMS runs over 28,008
    edges, so single messages may sit a hundred times above it): the
    finite-horizon LQR trajectory (backward Riccati recursion) to 1e-6."""
    K = 2000
    p = inputs.mpc_horizon_problem(K)
    g = graph_from_problem(p, "f64")
    r = g.fga_iterate(400000, 1e-12, 1e-12, check_every=1)
    assert r["status"] == 0
    m = p.meta
    Q, R, A, B = np.diag(m["q"]), np.diag(m["r"]), m["A"], m["B"]
    P = Q.copy()
    gains = []
    for _ in range(K):
        Kt = np.linalg.solve(R + B.T @ P @ B, B.T @ P @ A)
        P = Q + A.T @ P @ (A - B @ Kt)
        gains.append(Kt)
    gains = gains[::-1]
    xl, ul = [m["x0"]], []
    for t in range(K):
        ul.append(-gains[t] @ xl[-1])
        xl.append(A @ xl[-1] + B @ ul[-1])
    xs, us = inputs.mpc_horizon_split(g.fga_read_z(), K)
    np.testing.assert_allclose(xs, np.array(xl), atol=1e-6)
    np.testing.assert_allclose(us, np.array(ul), atol=1e-6)


@pytest.mark.parametrize("zorder", [1, 4])
def test_horizon_full_size_f32_stop_rule(zorder):
    """K = 10^5 in FP32 (chunked and scatter orders) to residual 1e-5 (checked every 10; 1e-4 is met
    after about 10 iterations, the RMS running over 1.4M edges of which most
    stay near zero): the stop is
    reported with both residuals at or below the tolerance, the primal
    residual recomputed in FP64 from the read-back state agrees, and z meets
    the dynamics to within a few primal residuals (z averages copies of
    which the dynamics factor's satisfy x' = A x + B u exactly: RMS defect
    <= (1 + |A| + |B|) r_pri, about 2.4 r_pri)."""
    K = 100000
    p = inputs.mpc_horizon_problem(K)
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1, _lib.FGA_OPT_ZORDER: zorder})
    r = g.fga_iterate(50000, 1e-5, 1e-5, check_every=10)
    assert r["status"] == 0 and r["iters"] % 10 == 0 and r["iters"] > 100
    assert r["r_pri"] <= 1e-5 and r["r_dual"] <= 1e-5
    x = g.fga_read_edge_state(_lib.FGA_EDGE_X)
    z = g.fga_read_z()
    bvar = oracle_from_problem(p).edge_var()
    r_pri = np.sqrt(np.mean((x - z[bvar]) ** 2))
    assert abs(r_pri - r["r_pri"]) <= 1e-6 + 1e-3 * r["r_pri"]
    xs, us = inputs.mpc_horizon_split(z, K)
    A, B = p.meta["A"], p.meta["B"]
    defect = xs[1:] - xs[:-1] @ A.T - us @ B.T
    assert np.sqrt(np.mean(defect ** 2)) <= 5 * r["r_pri"]
