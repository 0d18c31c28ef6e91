"""GPU parity of the disk-tile sweep (FGA_OPT_ZORDER 2: FP32 circle packing,
disk-pair state in registers, x recomputed, the z exchange through
count-and-sum words, a grid barrier on checked passes only) against the
FP64 oracle and against the chunked fast order,
through the C-ABI.

FP32 rule (as for the chunked order): z and the edge messages are compared
with the oracle on the scale S of the variables; the disk-pair operator
divides by the distance of two incoming centres, so FP32 rounding is
amplified on the few pairs whose messages come close, and the edge
messages are bounded by percentile and maximum separately."""
import numpy as np
import pytest

from oracle import from_problem as oracle_from_problem
from oracle.oracle import EDGE_X, EDGE_U, EDGE_N
from paper_1603_02526_gb300 import inputs
from paper_1603_02526_gb300 import _lib
from paper_1603_02526_gb300.graph import graph_from_problem
from tests.helpers import packing_objective

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


def _tile(p, **opt):
    g = graph_from_problem(p, "f32", options=opt or None)
    assert g.fga_launch_info()["zorder"] == 2
    return g


def _edges(g):
    return [g.fga_read_edge_state(w) for w in (_lib.FGA_EDGE_X, _lib.FGA_EDGE_U, _lib.FGA_EDGE_N)]


def test_tile_order_is_the_f32_packing_default():
    p = inputs.packing_problem(1000)
    g = graph_from_problem(p, "f32")
    info = g.fga_launch_info()
    assert info["zorder"] == 2
    # 2016 units of 32 x 8 disks, one per warp, at most 16 warps per CTA
    assert info["chunks"] == 2016
    assert info["grid"] * info["block"] // 32 >= 2016
    # m kept, or per-edge rho, or FP64: the chunked / canonical orders
    assert graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1}).fga_launch_info()["zorder"] == 1
    q = inputs.packing_problem(20)
    assert graph_from_problem(q, "f64").fga_launch_info()["zorder"] == 0


@pytest.mark.parametrize("iters", [3, 10])
def test_tile_n1000_first_iterations_against_oracle(iters):
    """The benchmark graph after 3 and 10 iterations, against the FP64
    oracle, with bounds set by what FP32 rounding alone does: the FP32
    emulation (tests/fp32_emulation.py) with each z sum exact and rounded
    once -- the tile order's fixed-point sums are exact too.  z, and every
    edge message at the 99.9th percentile and at the maximum, within 2x the
    emulation's own distance from the oracle (measured on GB300: at most
    1.1x).  The disk-pair operator divides by the distance of two incoming
    centres, so the few pairs whose messages come close amplify rounding:
    hence percentile and maximum apart."""
    from tests.fp32_emulation import PackingFP32
    p = inputs.packing_problem(1000)
    g = _tile(p)
    r = g.fga_iterate(iters)
    assert r["iters"] == iters
    o = oracle_from_problem(p)
    ro = o.iterate(iters)
    em = PackingFP32(p, sums="exact")
    em.iterate(iters)
    S = float(np.max(np.abs(o.z())))
    ez = np.abs(g.fga_read_z() - o.z()).max()
    assert ez <= 2 * np.abs(em.z - o.z()).max(), (ez / S, np.abs(em.z - o.z()).max() / S)
    for got, w, ref in zip(_edges(g), (EDGE_X, EDGE_U, EDGE_N), (em.x, em.u, em.n)):
        err = np.abs(got - o.edge(w))
        eref = np.abs(ref.astype(np.float64) - o.edge(w))
        for q in (99.9, 100):
            assert np.percentile(err, q) <= 2 * np.percentile(eref, q), (w, q, np.percentile(err, q) / S,
                                                                            np.percentile(eref, q) / S)
    # residuals of the last iteration agree with the oracle's to FP32 level
    np.testing.assert_allclose([r["r_pri"], r["r_dual"]], [ro["r_pri"], ro["r_dual"]], rtol=1e-3)


@pytest.mark.parametrize("n", [5, 20, 200])
def test_tile_small_graphs_against_oracle(n):
    """Ragged tiles (N not a multiple of 32 or 8, diagonal tiles half
    empty): 10 iterations, z within 1e-4 S of the oracle."""
    p = inputs.packing_problem(n)
    g = _tile(p)
    g.fga_iterate(10)
    o = oracle_from_problem(p)
    o.iterate(10)
    S = float(np.max(np.abs(o.z())))
    err = np.max(np.abs(g.fga_read_z() - o.z()))
    print("N=%d: max |dz| = %.3e S" % (n, err / S))
    assert err <= 1e-4 * S


def test_tile_against_chunked_order():
    """The two FP32 fast orders differ only in summation order: after 10
    iterations of N=200 their z agree to 1e-4 S."""
    p = inputs.packing_problem(200)
    a = _tile(p)
    a.fga_iterate(10)
    b = graph_from_problem(p, "f32", options={_lib.FGA_OPT_ZORDER: 1})
    assert b.fga_launch_info()["zorder"] == 1
    b.fga_iterate(10)
    S = float(np.max(np.abs(b.fga_read_z())))
    err = np.max(np.abs(a.fga_read_z() - b.fga_read_z()))
    print("tile vs chunked: max |dz| = %.3e S" % (err / S))
    assert err <= 1e-4 * S


def test_tile_chained_calls_equal_one_call():
    """Resume: x is recomputed from u and the previous z, so a call that
    starts from a stored state must continue with the same bits."""
    p = inputs.packing_problem(200)
    a = _tile(p)
    a.fga_iterate(500)
    b = _tile(p)
    for _ in range(5):
        b.fga_iterate(100, check_every=7)
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())
    for x, y in zip(_edges(a), _edges(b)):
        assert np.array_equal(x, y)


def test_tile_resume_after_stop_and_alpha():
    """Resume after a call that stopped at its tolerance (the state of the
    checked iteration, not the last one computed) continues with the bits of
    an unbroken run; the same for the u form (alpha 0.7)."""
    p = inputs.packing_problem(20)
    p.factor_blocks[-1].params[:] = 0.01
    a = _tile(p)
    r = a.fga_iterate(20000, 1e-3, 1e-3, check_every=5)
    assert r["status"] == 0 and 0 < r["iters"] < 20000
    a.fga_iterate(300, check_every=300)
    b = _tile(p)
    b.fga_iterate(r["iters"] + 300, check_every=10**6)
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())
    for x, y in zip(_edges(a), _edges(b)):
        assert np.array_equal(x, y)
    q = inputs.packing_problem(200)
    q.alpha = 0.7
    c = _tile(q)
    c.fga_iterate(300)
    d = _tile(q)
    for _ in range(3):
        d.fga_iterate(100, check_every=7)
    assert np.array_equal(c.fga_read_z(), d.fga_read_z())
    for x, y in zip(_edges(c), _edges(d)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("alpha", [1.0, 0.7])
def test_tile_several_units_per_warp_bit_exact(alpha):
    """More units than warps in a CTA: with FGA_OPT_BLOCK 64 two warps take
    each CTA's fourteen units of N = 1000 in turn, their pair state in device
    memory between passes.  The same CTAs hold the same units, so every
    operator, staged value and fixed-point sum is the same, and the iterates
    equal those of one unit per warp bit for bit (the FP64 residual sums to
    rounding: a thread's partial now spans several units): through checks every 7
    iterations, then a solve stopping at its tolerance, then a resumed call
    (the u form for alpha 0.7)."""
    p = inputs.packing_problem(1000)
    p.alpha = alpha
    a = _tile(p)
    b = graph_from_problem(p, "f32", options={_lib.FGA_OPT_BLOCK: 64})
    ia, ib = a.fga_launch_info(), b.fga_launch_info()
    assert ib["zorder"] == 2 and ib["block"] == 64 and ia["block"] > 64 and ia["grid"] == ib["grid"]
    for ce in (7, 10):
        ra = a.fga_iterate(60, 1e-3, 1e-3, check_every=ce)
        rb = b.fga_iterate(60, 1e-3, 1e-3, check_every=ce)
        # the residual partials are grouped by thread, and a thread now holds
        # several units: the FP64 sums agree to rounding, the iterates exactly
        assert (ra["iters"], ra["status"]) == (rb["iters"], rb["status"])
        np.testing.assert_allclose([rb["r_pri"], rb["r_dual"]], [ra["r_pri"], ra["r_dual"]], rtol=1e-12)
        assert np.array_equal(a.fga_read_z(), b.fga_read_z())
        for x, y in zip(_edges(a), _edges(b)):
            assert np.array_equal(x, y)


def test_tile_n2000_several_units_per_warp():
    """N = 2000 (12M scalar edges): more units per CTA than warps, the disk
    tiles with their state in device memory between passes.  After 10
    iterations z agrees with the chunked order and with the FP64 oracle to
    1e-4 of the variables' scale."""
    p = inputs.packing_problem(2000)
    g = _tile(p)
    info = g.fga_launch_info()
    assert info["chunks"] > info["grid"] * (info["block"] // 32)
    r = g.fga_iterate(10)
    assert r["iters"] == 10 and r["status"] == 0
    b = graph_from_problem(p, "f32", options={_lib.FGA_OPT_ZORDER: 1})
    b.fga_iterate(10)
    o = oracle_from_problem(p)
    o.iterate(10)
    S = float(np.max(np.abs(o.z())))
    zg = g.fga_read_z()
    e_ch = np.max(np.abs(zg - b.fga_read_z()))
    e_or = np.max(np.abs(zg - o.z()))
    print("N=2000 tiles: max |dz| vs chunked %.3e S, vs oracle %.3e S" % (e_ch / S, e_or / S))
    assert e_ch <= 1e-4 * S and e_or <= 1e-4 * S


@pytest.mark.parametrize("ce", [1, 7])
def test_tile_stop_rule_state(ce):
    """A call that stops at the first checked iteration meeting the
    tolerances leaves exactly the state of a plain call of that many
    iterations."""
    p = inputs.packing_problem(20)
    p.factor_blocks[-1].params[:] = 0.01
    a = _tile(p)
    r = a.fga_iterate(20000, 1e-4, 1e-4, check_every=ce)
    assert r["status"] == 0 and r["iters"] < 20000 and r["iters"] % ce == 0
    assert r["r_pri"] <= 1e-4 and r["r_dual"] <= 1e-4
    b = _tile(p)
    rb = b.fga_iterate(r["iters"], check_every=r["iters"])
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())
    for x, y in zip(_edges(a), _edges(b)):
        assert np.array_equal(x, y)
    assert (rb["r_pri"], rb["r_dual"]) == (r["r_pri"], r["r_dual"])


def test_tile_objective_matches_oracle():
    """N=20 run to residual 1e-4 (reward 0.01): objective within 1e-4
    relative of the oracle's under the same stop rule."""
    p = inputs.packing_problem(20)
    p.factor_blocks[-1].params[:] = 0.01
    g = _tile(p)
    rg = g.fga_iterate(50000, 1e-4, 1e-4)
    o = oracle_from_problem(p)
    ro = o.iterate(50000, 1e-4, 1e-4)
    assert rg["status"] == 0 and ro["status"] == 0
    fg, fo = packing_objective(g.fga_read_z()), packing_objective(o.z())
    assert abs(fg - fo) <= 1e-4 * abs(fo), (fg, fo, rg, ro)


def test_tile_deterministic():
    p = inputs.packing_problem(1000)
    a = _tile(p)
    a.fga_iterate(50)
    b = _tile(p)
    b.fga_iterate(50)
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())
    assert np.array_equal(a.fga_read_edge_state(_lib.FGA_EDGE_U), b.fga_read_edge_state(_lib.FGA_EDGE_U))


@pytest.mark.parametrize("alpha", [1.0, 0.7])
def test_tile_area_reward_and_alpha(alpha):
    """The area reward -r^2/2 (rho 25) through the tile kernel, in the
    displacement form (alpha 1) and the u form (alpha 0.7): 200 iterations
    in calls of 70, 70 and 60 (resume, a check every 9), z within 1e-4 S of
    the oracle, and the same bits as one call."""
    p = inputs.packing_problem(30, reward="quad", rho=25.0)
    p.alpha = alpha
    g = _tile(p)
    g.fga_iterate(200)
    o = oracle_from_problem(p)
    o.iterate(200)
    S = float(np.max(np.abs(o.z())))
    assert np.max(np.abs(g.fga_read_z() - o.z())) <= 1e-4 * S
    h = _tile(p)
    for k in (70, 70, 60):
        h.fga_iterate(k, check_every=9)
    assert np.array_equal(g.fga_read_z(), h.fga_read_z())
    for x, y in zip(_edges(g), _edges(h)):
        assert np.array_equal(x, y)


def test_tile_rejections():
    p = inputs.packing_problem(20)
    with pytest.raises(_lib.FgaError):
        graph_from_problem(p, "f64", options={_lib.FGA_OPT_ZORDER: 2})
    with pytest.raises(_lib.FgaError):
        graph_from_problem(p, "f32", options={_lib.FGA_OPT_ZORDER: 2, _lib.FGA_OPT_STORE_M: 1})
    g = _tile(p)
    with pytest.raises(_lib.FgaError):
        g.fga_iterate(10, fused=False)


def test_tile_latency_floor_leaves_the_solve_unchanged():
    """The operator-free floor (both modes) on the disk-tile grid: positive
    device times, and a solve split around floor calls bit-equal to one
    without them (the count-and-sum words are zeroed again)."""
    p = inputs.packing_problem(200)
    a = _tile(p)
    a.fga_iterate(200, check_every=10)
    b = _tile(p)
    b.fga_iterate(100, check_every=10)
    ms1 = b.fga_latency_floor(500, 1)
    ms0 = b.fga_latency_floor(500, 0)
    assert ms1 > 0 and ms0 > 0
    b.fga_iterate(100, check_every=10)
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())
    for x, y in zip(_edges(a), _edges(b)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("iters", [3, 10])
def test_tile_n1000_area_reward_against_oracle(iters):
    """The paper's area reward -r^2/2 on the N = 1000 graph (rho 25, the
    prox needs rho > 1), under the same bounds as the linear reward's
    benchmark graph: z and the edge messages at the 99.9th percentile and
    at the maximum within 2x the FP32 emulation's own distance from the
    FP64 oracle; residuals to 1e-3 relative."""
    from tests.fp32_emulation import PackingFP32
    p = inputs.packing_problem(1000, reward="quad", rho=25.0)
    g = _tile(p)
    r = g.fga_iterate(iters)
    assert r["iters"] == iters
    o = oracle_from_problem(p)
    ro = o.iterate(iters)
    em = PackingFP32(p, sums="exact")
    em.iterate(iters)
    S = float(np.max(np.abs(o.z())))
    ez = np.abs(g.fga_read_z() - o.z()).max()
    assert ez <= 2 * np.abs(em.z - o.z()).max(), (ez / S, np.abs(em.z - o.z()).max() / S)
    for got, w, ref in zip(_edges(g), (EDGE_X, EDGE_U, EDGE_N), (em.x, em.u, em.n)):
        err = np.abs(got - o.edge(w))
        eref = np.abs(ref.astype(np.float64) - o.edge(w))
        for q in (99.9, 100):
            assert np.percentile(err, q) <= 2 * np.percentile(eref, q), (w, q, np.percentile(err, q) / S,
                                                                            np.percentile(eref, q) / S)
    np.testing.assert_allclose([r["r_pri"], r["r_dual"]], [ro["r_pri"], ro["r_dual"]], rtol=1e-3)
