"""GPU parity of the scatter z-order (FGA_OPT_ZORDER 4) against the FP64
oracle, through the C-ABI.

In this order every edge's rho*m goes straight to a per-variable column
(column k holds the variable's k-th edge in creation order, k < W) or, past
the W columns, to the variable's overflow row; a variable's z is the sum of
its columns in column order, then of its overflow row (a warp's shuffle
tree, hub rows in pieces added in piece order).  A variable whose degree is
at most W therefore gets the serial creation-order sum of Algorithm 2's
z-update, the oracle's own: on graphs without overflow rows an FP64 run
takes exactly the canonical order's operations.  Overflow rows change the
order of the additions only: FP64 runs stay within 1e-10 relative of the
oracle.  FP32 runs get the bounds of the fast-order tests (the same
operators, rounded in FP32)."""
import numpy as np
import pytest

from oracle import from_problem as oracle_from_problem
from paper_1603_02526_gb300 import inputs
from paper_1603_02526_gb300 import _lib
from paper_1603_02526_gb300.graph import graph_from_problem
from tests.helpers import assert_messages_match, assert_messages_close_scaled

pytestmark = pytest.mark.gpu

SCATTER = {_lib.FGA_OPT_ZORDER: 4}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


def _edge_state(g):
    return [g.fga_read_edge_state(w) for w in (_lib.FGA_EDGE_X, _lib.FGA_EDGE_U, _lib.FGA_EDGE_N)]


@pytest.mark.parametrize("fused", [True, False])
def test_horizon_f64_equals_canonical_order(fused):
    """MPC horizon K = 500 (variables of degree 2 and 3: no overflow row),
    FP64, 300 iterations: within 1e-9 of the oracle (the dynamics projector
    rounds differently from the oracle's Cholesky solve, as in the canonical
    order) and bit for bit the canonical order's messages."""
    p = inputs.mpc_horizon_problem(500)
    g = graph_from_problem(p, "f64", options=SCATTER)
    info = g.fga_launch_info()
    assert info["zorder"] == 4 and info["chunks"] == 3      # three columns
    r = g.fga_iterate(300, fused=fused)
    o = oracle_from_problem(p)
    o.iterate(300)
    assert r["iters"] == 300
    assert_messages_match(g, o, 1e-9)
    c = graph_from_problem(p, "f64")
    c.fga_iterate(300, fused=fused)
    assert np.array_equal(g.fga_read_z(), c.fga_read_z())
    for a, b in zip(_edge_state(g), _edge_state(c)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("npts,d", [(1, 2), (200, 3), (5000, 2)])
def test_svm_paper_f64_with_hub(npts, d):
    """Paper-form SVM, FP64, 200 iterations: the offset b is on every margin
    factor (degree N: an overflow row past the columns; N = 5000 splits it
    into pieces of 2048).  Every message within 1e-10 of the oracle."""
    p = inputs.svm_paper_problem(npts, d, seed=3300 + npts, C=1.0)
    g = graph_from_problem(p, "f64", options=SCATTER)
    g.fga_iterate(200)
    o = oracle_from_problem(p)
    o.iterate(200)
    assert_messages_match(g, o, 1e-10)


@pytest.mark.parametrize("fused", [True, False])
def test_rows_of_every_length_f64(fused):
    """Variables of degree 0, 1, 31, 32, 33, 63, 64, 65, 97, 200 (a few in
    columns, most with overflow rows of every length), quadratic costs,
    boxes and fixed values interleaved in creation order, FP64, 40
    iterations: every message within 1e-10 of the oracle, and z equal bit
    for bit for the variables whose edges all sit in columns."""
    degrees = [0, 1, 31, 32, 33, 63, 64, 65, 97, 200] * 4 + [2, 3]
    rng = np.random.default_rng(12)
    p = inputs.Problem("degrees")
    v0 = p.add_vars(len(degrees), 1)
    for rep in range(max(degrees)):
        live = [i for i, dg in enumerate(degrees) if rep < dg]
        ids = [[v0 + i] for i in live]
        if rep % 3 == 0:
            p.add_factors(7, ids, [[0.5 + rng.random()] for _ in live])
        elif rep % 3 == 1:
            p.add_factors(8, ids, [[-0.5, 0.5 + rng.random()] for _ in live])
        else:
            p.add_factors(9, ids, [[rng.standard_normal()] for _ in live])
    p.z0 = rng.standard_normal(p.num_scalar_vars)
    g = graph_from_problem(p, "f64", options=SCATTER)
    W = g.fga_launch_info()["chunks"]
    assert 1 <= W <= 15
    g.fga_iterate(40, fused=fused)
    o = oracle_from_problem(p)
    o.iterate(40)
    assert_messages_match(g, o, 1e-10)
    cols = np.array(degrees) <= W
    assert np.array_equal(g.fga_read_z()[cols], o.z()[cols])


@pytest.mark.parametrize("K", [1, 37, 500])
def test_horizon_f32(K):
    """FP32 scatter order (the FP32 default for this graph), 300 iterations:
    every message within 300 iterations x 9 x 2^-24 of the scale (the bound
    of the fast-order test: a 9-term dot product per iteration, not
    amplified by the nonexpansive iteration)."""
    p = inputs.mpc_horizon_problem(K)
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1})
    assert g.fga_launch_info()["zorder"] == 4
    g.fga_iterate(300)
    o = oracle_from_problem(p)
    o.iterate(300)
    assert_messages_close_scaled(g, o, 300 * 9 * 2.0 ** -24)


@pytest.mark.parametrize("npts,d", [(1, 2), (37, 5), (500, 3)])
def test_svm_paper_f32(npts, d):
    """FP32 scatter order, 300 iterations, every message within 300 x
    4 (D + 2) 2^-24 of the scale (the margin's dot product over D + 2 edges
    with data values up to about 4)."""
    p = inputs.svm_paper_problem(npts, d, seed=3200 + npts, C=1.0)
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1})
    assert g.fga_launch_info()["zorder"] == 4
    g.fga_iterate(300)
    o = oracle_from_problem(p)
    o.iterate(300)
    assert_messages_close_scaled(g, o, 300 * 4 * (d + 2) * 2.0 ** -24)


def test_full_size_f32():
    """The two benchmarked general-sweep graphs at full size in the scatter
    order: the K = 10^5 horizon (1.4M edges, 20 iterations, bound 20 x 9 x
    2^-24) and the paper-form SVM 100,000 x 64 (25.9M edges, 3 iterations,
    bound 3 x 4 x 66 x 2^-24)."""
    p = inputs.mpc_horizon_problem(100000)
    o = oracle_from_problem(p)
    o.iterate(20)
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1})
    assert g.fga_launch_info()["zorder"] == 4
    g.fga_iterate(20)
    assert_messages_close_scaled(g, o, 20 * 9 * 2.0 ** -24)
    del g, o
    p = inputs.svm_paper_problem(100000, 64, seed=3000, C=1.0)
    o = oracle_from_problem(p)
    o.iterate(3)
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1})
    assert g.fga_launch_info()["zorder"] == 4
    g.fga_iterate(3)
    assert_messages_close_scaled(g, o, 3 * 4 * 66 * 2.0 ** -24)


def test_chained_calls_and_stop_rule():
    """Resume: 70 + 130 iterations equal one call of 200 bit for bit (FP32
    paper-form SVM); the stop rule (checked every 7) stops the FP64 horizon
    K = 200 at the oracle's iteration."""
    p = inputs.svm_paper_problem(300, 4, seed=3400, C=1.0)
    a = graph_from_problem(p, "f32", options=SCATTER)
    a.fga_iterate(70)
    a.fga_iterate(130)
    b = graph_from_problem(p, "f32", options=SCATTER)
    b.fga_iterate(200)
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())
    q = inputs.mpc_horizon_problem(200)
    g = graph_from_problem(q, "f64", options=SCATTER)
    r = g.fga_iterate(100000, 1e-7, 1e-7, check_every=7)
    o = oracle_from_problem(q)
    ro = o.iterate(100000, tol_pri=1e-7, tol_dual=1e-7, check_every=7)
    assert r["status"] == 0 and r["iters"] == ro["iters"]


def test_default_order_choice():
    """FP32 defaults: low-degree graphs (the horizon, the paper-form SVM)
    take the scatter order; a packing graph the disk tiles do not take (m
    kept per edge), whose disk coordinates sit on N - 1 pair factors each,
    keeps the chunked fast order; FP64 keeps the canonical order."""
    assert graph_from_problem(inputs.mpc_horizon_problem(50), "f32").fga_launch_info()["zorder"] == 4
    assert graph_from_problem(inputs.svm_paper_problem(50, 4), "f32").fga_launch_info()["zorder"] == 4
    assert graph_from_problem(inputs.mpc_horizon_problem(50), "f64").fga_launch_info()["zorder"] == 0
    p = inputs.packing_problem(40, seed=1)
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1}, init=False)
    assert g.fga_launch_info()["zorder"] == 1


def test_refusals():
    """Three weights and shards run other orders: asking for the scatter
    order with them is refused at finalize / shard begin."""
    p = inputs.mpc_horizon_problem(20)
    with pytest.raises(Exception):
        graph_from_problem(p, "f64", options={_lib.FGA_OPT_ZORDER: 4, _lib.FGA_OPT_WEIGHTS: 1})
