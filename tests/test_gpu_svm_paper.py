"""GPU parity of the soft-margin SVM in the paper's own factor-graph form
(Sec. V-C, Appendix C: a copy of w per point, chained by equality factors;
one-point margin, minimal-error and split-norm factors) against the FP64
oracle, through the C-ABI.

FP64 runs use the canonical z order; the margin, slack and equality
operators take the same operations in the same order as the oracle's, so
every message must equal the oracle's bit for bit.  FP32 runs use the
chunked fast order here (the scatter order, the FP32 default for this graph,
has its own tests with the same bound).  Tolerance: one iteration rounds a message by a few FP32 ulps of the
variables' scale S, the largest term being the margin's dot product over
D + 2 edges with data values of magnitude up to about 4: about
4 (D + 2) 2^-24 S; the method on this convex problem does not amplify
earlier errors (each iteration is a nonexpansive map), so k iterations stay
within k times that if every rounding added up with the same sign."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import from_problem as oracle_from_problem
from paper_1603_02526_gb300 import inputs
from paper_1603_02526_gb300 import _lib
from paper_1603_02526_gb300.graph import graph_from_problem
from tests.helpers import assert_messages_close_scaled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


def _f32_bound(D, iters):
    return iters * 4 * (D + 2) * 2.0 ** -24


def _edges_equal(g, o):
    from oracle.oracle import EDGE_X, EDGE_M, EDGE_U, EDGE_N
    for a, b in ((_lib.FGA_EDGE_X, EDGE_X), (_lib.FGA_EDGE_M, EDGE_M), (_lib.FGA_EDGE_U, EDGE_U),
                 (_lib.FGA_EDGE_N, EDGE_N)):
        assert np.array_equal(g.fga_read_edge_state(a), o.edge(b)), a


@pytest.mark.parametrize("fused", [True, False])
def test_svm_paper_f64_bit_exact(fused):
    """N = 200 points in d = 3 (2,994 scalar edges), C = 1, 300 iterations."""
    p = inputs.svm_paper_problem(200, 3, seed=3100, C=1.0)
    g = graph_from_problem(p, "f64")
    r = g.fga_iterate(300, fused=fused)
    o = oracle_from_problem(p)
    ro = o.iterate(300)
    assert r["iters"] == ro["iters"] == 300
    assert np.array_equal(g.fga_read_z(), o.z())
    _edges_equal(g, o)


@pytest.mark.parametrize("npts,d", [(1, 2), (37, 5), (500, 3)])
def test_svm_paper_f32_chunked_order(npts, d):
    """FP32 fast order, 300 iterations, every message within the module
    docstring's bound; N = 1 has no equality factor."""
    p = inputs.svm_paper_problem(npts, d, seed=3200 + npts, C=1.0)
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1, _lib.FGA_OPT_ZORDER: 1})
    g.fga_iterate(300)
    o = oracle_from_problem(p)
    o.iterate(300)
    assert_messages_close_scaled(g, o, _f32_bound(d, 300))


def test_svm_paper_full_size():
    """100,000 points in d = 64 (25.9M scalar edges, the size the benchmark
    times), 3 iterations: FP64 bit-exact, FP32 within the bound."""
    p = inputs.svm_paper_problem(100000, 64, seed=3000, C=1.0)
    assert p.num_edges == inputs.svm_paper_edges(100000, 64)
    o = oracle_from_problem(p)
    o.iterate(3)
    g = graph_from_problem(p, "f64")
    g.fga_iterate(3)
    assert np.array_equal(g.fga_read_z(), o.z())
    _edges_equal(g, o)
    del g
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1, _lib.FGA_OPT_ZORDER: 1})
    g.fga_iterate(3)
    assert_messages_close_scaled(g, o, _f32_bound(64, 3))


def test_svm_paper_converges_to_qp():
    """12 points in d = 2, C = 2, FP64 to residual 1e-11: every copy of w
    equal, and (w, b) the soft-margin QP's solution (SLSQP, epigraph form)."""
    X, y = inputs.svm_data(12, 2, seed=11)
    C = 2.0
    p = inputs.svm_paper_problem(12, 2, C=C, X=X, y=y)
    g = graph_from_problem(p, "f64")
    r = g.fga_iterate(2000000, 1e-11, 1e-11, check_every=10)
    assert r["status"] == 0
    z = g.fga_read_z()
    W, bz, xi = z[:24].reshape(12, 2), z[24], z[25:]
    np.testing.assert_allclose(W, np.broadcast_to(W[0], W.shape), atol=1e-7)
    cons = [dict(type="ineq", fun=lambda s: s[3:]),
            dict(type="ineq", fun=lambda s: s[3:] - (1 - y * (X @ s[:2] + s[2])))]
    sol = minimize(lambda s: 0.5 * s[:2] @ s[:2] + C * s[3:].sum(), np.concatenate([W[0], [bz], xi]),
                   constraints=cons, method="SLSQP", options=dict(ftol=1e-15, maxiter=2000))
    np.testing.assert_allclose(W[0], sol.x[:2], atol=1e-5)
    np.testing.assert_allclose(bz, sol.x[2], atol=1e-5)

