"""GPU parity of the hinge-bank sweep (FGA_OPT_ZORDER 3: a linear
soft-margin SVM in FP32 with alpha = 1, one scalar of state per hinge
factor, the data rows in shared memory, the z exchange through
count-and-sum words, a grid barrier on checked passes only) against the
FP64 oracle and against the chunked order, through the C-ABI.

FP32 rule: z and the edge messages are compared on the scale S of the
variables; a hinge whose margin sits at a rounding-level distance from 1
may switch between active and inactive, moving its edges by up to the
step, so edge messages are bounded at the 99.9th percentile."""
import numpy as np
import pytest

from oracle import from_problem as oracle_from_problem
from oracle.oracle import EDGE_X, EDGE_U, EDGE_N
from paper_1603_02526_gb300 import inputs, _lib
from paper_1603_02526_gb300.graph import graph_from_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


def _hinge(p, **opt):
    g = graph_from_problem(p, "f32", options=opt or None)
    assert g.fga_launch_info()["zorder"] == 3
    return g


def _edges(g):
    return [g.fga_read_edge_state(w) for w in (_lib.FGA_EDGE_X, _lib.FGA_EDGE_U, _lib.FGA_EDGE_N)]


def _primal(z, p):
    X, y, lam, c = p.meta["X"], p.meta["y"], p.meta["lam"], p.meta["c"]
    w, b = z[:-1], z[-1]
    return float(c * np.maximum(0.0, 1.0 - y * (X @ w + b)).sum() + 0.5 * lam * w @ w)


def test_hinge_order_is_the_f32_svm_default():
    p = inputs.svm_problem(100000, 64, seed=3000)
    g = graph_from_problem(p, "f32")
    info = g.fga_launch_info()
    assert info["zorder"] == 3 and info["block"] % 32 == 0
    assert graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1}).fga_launch_info()["zorder"] == 1


def test_hinge_full_size_first_iterations_against_oracle():
    """100,000 points x 64 after 3 iterations: z to 1e-5 S, x / u / n at the
    99.9th percentile to 1e-4 S; residuals to 1e-3 relative."""
    p = inputs.svm_problem(100000, 64, seed=3000)
    g = _hinge(p)
    r = g.fga_iterate(3)
    o = oracle_from_problem(p)
    ro = o.iterate(3)
    S = max(1.0, float(np.abs(o.z()).max()))
    assert np.abs(g.fga_read_z() - o.z()).max() <= 1e-5 * S
    for got, w in zip(_edges(g), (EDGE_X, EDGE_U, EDGE_N)):
        err = np.abs(got - o.edge(w))
        assert np.percentile(err, 99.9) <= 1e-4 * S, (w, np.percentile(err, 99.9))
    np.testing.assert_allclose([r["r_pri"], r["r_dual"]], [ro["r_pri"], ro["r_dual"]], rtol=1e-3)


@pytest.mark.parametrize("npts,d", [(300, 8), (2000, 64), (5000, 17)])
def test_hinge_small_against_oracle(npts, d):
    """Dimensions below 64 (rows padded), CTAs with uneven slices: 20
    iterations, z within 1e-4 S of the oracle."""
    p = inputs.svm_problem(npts, d, seed=3300 + d)
    g = _hinge(p)
    g.fga_iterate(20)
    o = oracle_from_problem(p)
    o.iterate(20)
    S = max(1.0, float(np.abs(o.z()).max()))
    err = np.abs(g.fga_read_z() - o.z()).max()
    print("N=%d d=%d: max |dz| = %.3e S" % (npts, d, err / S))
    assert err <= 1e-4 * S


def test_hinge_against_chunked_order():
    p = inputs.svm_problem(10000, 64, seed=3200)
    a = _hinge(p)
    a.fga_iterate(20)
    b = graph_from_problem(p, "f32", options={_lib.FGA_OPT_ZORDER: 1})
    b.fga_iterate(20)
    S = max(1.0, float(np.abs(b.fga_read_z()).max()))
    assert np.abs(a.fga_read_z() - b.fga_read_z()).max() <= 1e-4 * S


def test_hinge_objective_10k_matches_oracle():
    """Both run to residual 1e-4 (checked every 10 iterations): primal
    objectives within 1e-4 relative."""
    p = inputs.svm_problem(10000, 64, seed=3200)
    g = _hinge(p)
    rg = g.fga_iterate(100000, 1e-4, 1e-4, check_every=10)
    o = oracle_from_problem(p)
    ro = o.iterate(100000, 1e-4, 1e-4, check_every=10)
    assert rg["status"] == 0 and ro["status"] == 0
    fg, fo = _primal(g.fga_read_z(), p), _primal(o.z(), p)
    assert abs(fg - fo) <= 1e-4 * abs(fo), (fg, fo, rg, ro)


def test_hinge_chained_calls_and_resume_after_stop():
    p = inputs.svm_problem(5000, 64, seed=3400)
    a = _hinge(p)
    a.fga_iterate(300)
    b = _hinge(p)
    for _ in range(3):
        b.fga_iterate(100, check_every=7)
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())
    for x, y in zip(_edges(a), _edges(b)):
        assert np.array_equal(x, y)
    c = _hinge(p)
    r = c.fga_iterate(20000, 1e-3, 1e-3, check_every=5)
    assert r["status"] == 0 and 0 < r["iters"] < 20000
    c.fga_iterate(50, check_every=50)
    d = _hinge(p)
    d.fga_iterate(r["iters"] + 50, check_every=10**6)
    assert np.array_equal(c.fga_read_z(), d.fga_read_z())
    for x, y in zip(_edges(c), _edges(d)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("ce", [1, 7])
def test_hinge_stop_rule_state(ce):
    p = inputs.svm_problem(3000, 32, seed=3500)
    a = _hinge(p)
    r = a.fga_iterate(20000, 1e-4, 1e-4, check_every=ce)
    assert r["status"] == 0 and r["iters"] % ce == 0
    b = _hinge(p)
    rb = b.fga_iterate(r["iters"], check_every=r["iters"])
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())
    for x, y in zip(_edges(a), _edges(b)):
        assert np.array_equal(x, y)
    assert (rb["r_pri"], rb["r_dual"]) == (r["r_pri"], r["r_dual"])


def test_hinge_full_size_converges_and_is_deterministic():
    p = inputs.svm_problem(100000, 64, seed=3000)
    a = _hinge(p)
    r = a.fga_iterate(50000, 1e-4, 1e-4, check_every=10)
    assert r["status"] == 0 and r["iters"] < 50000, r
    b = _hinge(p)
    b.fga_iterate(r["iters"], check_every=10)
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())


def test_hinge_rejections():
    p = inputs.svm_problem(300, 8, seed=3100)
    with pytest.raises(_lib.FgaError):
        graph_from_problem(p, "f64", options={_lib.FGA_OPT_ZORDER: 3})
    q = inputs.svm_problem(300, 8, seed=3100, alpha=0.7)
    with pytest.raises(_lib.FgaError):
        graph_from_problem(q, "f32", options={_lib.FGA_OPT_ZORDER: 3})
    assert graph_from_problem(q, "f32").fga_launch_info()["zorder"] == 1
    with pytest.raises(_lib.FgaError):
        graph_from_problem(inputs.packing_problem(20), "f32", options={_lib.FGA_OPT_ZORDER: 3})
    g = _hinge(p)
    with pytest.raises(_lib.FgaError):
        g.fga_iterate(10, fused=False)


def test_hinge_latency_floor_leaves_the_solve_unchanged():
    """The operator-free floor (both modes) runs on the hinge bank's own
    grid and count-and-sum words: positive device times, and a solve split
    around floor calls bit-equal to one without them (the words are zeroed
    again); other orders and modes are refused."""
    p = inputs.svm_problem(5000, 64, seed=3400)
    a = _hinge(p)
    a.fga_iterate(200, check_every=10)
    b = _hinge(p)
    b.fga_iterate(100, check_every=10)
    ms1 = b.fga_latency_floor(500, 1)
    ms0 = b.fga_latency_floor(500, 0)
    assert ms1 > 0 and ms0 > 0
    b.fga_iterate(100, check_every=10)
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())
    for x, y in zip(_edges(a), _edges(b)):
        assert np.array_equal(x, y)
    c = graph_from_problem(p, "f32", options={_lib.FGA_OPT_ZORDER: 1})
    with pytest.raises(_lib.FgaError):
        c.fga_latency_floor(10, 1)
    with pytest.raises(_lib.FgaError):
        b.fga_latency_floor(10, 2)
