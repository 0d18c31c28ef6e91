"""GPU parity of the three-weight mode (FGA_OPT_WEIGHTS 1) against the
oracle's (og_set_weights 1), through the C-ABI.  FP64 in the canonical
order reproduces the oracle's weight classes, sums and resets, so z and
every edge message must be bit-equal (MPC to 1e-9: the GPU applies a
precomputed projector, the oracle solves); FP32 is compared by the
objective after converging (a weight class decided by x == n can fall the
other way under FP32 rounding)."""
import numpy as np
import pytest

from oracle import from_problem as oracle_from_problem
from oracle.oracle import EDGE_X, EDGE_M, EDGE_U, EDGE_N
from paper_1603_02526_gb300 import inputs, _lib
from paper_1603_02526_gb300.graph import graph_from_problem
from tests.helpers import assert_messages_match

pytestmark = pytest.mark.gpu

TWA = {_lib.FGA_OPT_WEIGHTS: 1}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


def _pair(p, iters, precision="f64", fused=True, check_every=1, tol=0.0, rho_e=None):
    g = graph_from_problem(p, precision, options=TWA, init=False) if rho_e is None else None
    if rho_e is not None:
        from paper_1603_02526_gb300.graph import FactorGraph, _merge_var_blocks
        g = FactorGraph(precision)
        g.fga_set_option(_lib.FGA_OPT_WEIGHTS, 1)
        for count, dim in _merge_var_blocks(p.var_blocks):
            g.fga_add_variables(count, dim)
        for blk in p.factor_blocks:
            g.fga_add_factors(blk.ftype, blk.var_ids, blk.params if blk.params.size else None)
        g.fga_set_edge_rho_alpha(rho_e, None)
        g.fga_finalize()
    g.fga_init(p.z0)
    assert g.fga_launch_info()["zorder"] == 0
    rg = g.fga_iterate(iters, tol, tol, check_every=check_every, fused=fused)
    o = oracle_from_problem(p, weights=1, z0=False)
    if rho_e is not None:
        o.set_rho_alpha(rho_e, p.alpha)
    o.init(p.z0)
    ro = o.iterate(iters, tol, tol, check_every=check_every)
    return g, o, rg, ro


def _bit_equal(g, o):
    assert np.array_equal(g.fga_read_z(), o.z())
    for w, ow in ((_lib.FGA_EDGE_X, EDGE_X), (_lib.FGA_EDGE_M, EDGE_M), (_lib.FGA_EDGE_U, EDGE_U),
                  (_lib.FGA_EDGE_N, EDGE_N)):
        assert np.array_equal(g.fga_read_edge_state(w), o.edge(ow)), w


@pytest.mark.parametrize("fused", [True, False])
def test_packing_n20_f64_bit_exact(fused):
    """Disk pairs and walls switch between zero and standard weight as
    they touch and separate: 1000 iterations, checks every 7."""
    p = inputs.packing_problem(20)
    g, o, rg, ro = _pair(p, 1000, fused=fused, check_every=7)
    assert rg["iters"] == ro["iters"] == 1000
    _bit_equal(g, o)
    np.testing.assert_allclose([rg["r_pri"], rg["r_dual"]], [ro["r_pri"], ro["r_dual"]], rtol=1e-12)


def test_packing_stop_rule_matches_oracle():
    p = inputs.packing_problem(20)
    p.factor_blocks[-1].params[:] = 0.01
    g, o, rg, ro = _pair(p, 50000, check_every=5, tol=1e-6)
    assert rg["status"] == 0 and rg["iters"] == ro["iters"] < 50000
    _bit_equal(g, o)


def test_fixed_value_and_box_f64_bit_exact():
    """A scalar with a quadratic, a linear reward, a box and a fixed value
    (infinite weight), plus a second scalar with an inactive box: the
    infinite weight decides the first z at once."""
    p = inputs.Problem("twa_scalar")
    p.var_blocks = [(2, 1)]
    p.add_factors(inputs.MPC_QUAD, [[0], [1]], [[1.0], [2.0]])
    p.add_factors(inputs.PACK_RADIUS_LIN, [[0], [1]], [[2.0], [1.0]])
    p.add_factors(inputs.MPC_BOX, [[0], [1]], [[-10.0, 10.0], [-0.2, 0.2]])
    p.add_factors(inputs.FIX, [[0]], [[4.0]])
    p.z0 = np.array([0.0, 0.0])
    g, o, rg, ro = _pair(p, 60)
    _bit_equal(g, o)
    assert g.fga_read_z()[0] == 4.0


def test_per_edge_rho_f64_bit_exact():
    """Per-edge rho (the two coordinates of a disk centre share one): the
    standard-weight mean uses each edge's rho."""
    p = inputs.packing_problem(6)
    rng = np.random.default_rng(77)
    E = p.num_edges
    rho = rng.uniform(0.5, 2.0, E)
    # edges of a centre (two coordinates) share one rho: pairs c1(0,1), c2(3,4); walls c(0,1)
    npair = 15
    for f in range(npair):
        rho[6 * f + 1] = rho[6 * f]
        rho[6 * f + 4] = rho[6 * f + 3]
    for w in range(18):
        e0 = 6 * npair + 3 * w
        rho[e0 + 1] = rho[e0]
    g, o, rg, ro = _pair(p, 300, rho_e=rho)
    _bit_equal(g, o)


def test_svm_f64_bit_exact():
    p = inputs.svm_problem(300, 8, seed=3100)
    g, o, rg, ro = _pair(p, 200)
    _bit_equal(g, o)


def test_mpc_f64_against_oracle():
    d = inputs.mpc_batch_inputs(1, seed=4100, T_fixed=15)
    p = inputs.mpc_problem(d["A"][0], d["B"][0], d["q"][0], d["r"][0], 2.0 * d["x0"][0], 15)
    g, o, rg, ro = _pair(p, 150)
    assert_messages_match(g, o, 1e-9)


def test_packing_f32_against_oracle():
    """FP32 messages: a weight class decided by x == n can fall the other
    way under FP32 rounding, so FP32 is compared by its result: N=20
    (reward 0.01) run to residual 1e-4 by GPU and oracle in the same mode,
    objectives -sum r within 1e-4 relative; and the first 5 iterations (no
    class near a switch yet) within 1e-5 of the variables' scale."""
    from tests.helpers import packing_objective
    p = inputs.packing_problem(20)
    g, o, rg, ro = _pair(p, 5, precision="f32")
    S = float(np.abs(o.z()).max())
    assert np.abs(g.fga_read_z() - o.z()).max() <= 1e-5 * S
    p.factor_blocks[-1].params[:] = 0.01
    g, o, rg, ro = _pair(p, 50000, precision="f32", tol=1e-4)
    assert rg["status"] == 0 and ro["status"] == 0
    fg, fo = packing_objective(g.fga_read_z(), 0.01), packing_objective(o.z(), 0.01)
    print("three weights, N=20 to 1e-4: FP32 %d iterations, oracle %d; objectives %.8f / %.8f"
          % (rg["iters"], ro["iters"], fg, fo))
    assert abs(fg - fo) <= 1e-4 * abs(fo)


def test_three_weights_reach_a_feasible_packing():
    """N=20, reward 0.01, to residual 1e-6: the three-weight run converges
    to a packing without overlap; the iteration counts of both modes are
    printed."""
    p = inputs.packing_problem(20)
    p.factor_blocks[-1].params[:] = 0.01
    g = graph_from_problem(p, "f64", options=TWA)
    r = g.fga_iterate(50000, 1e-6, 1e-6, check_every=10)
    h = graph_from_problem(p, "f64")
    rh = h.fga_iterate(50000, 1e-6, 1e-6, check_every=10)
    print("N=20 to 1e-6: three weights %d iterations, fixed weights %d" % (r["iters"], rh["iters"]))
    assert r["status"] == 0
    z = g.fga_read_z()
    c = np.stack([z[0::3], z[1::3]], 1)
    rr = z[2::3]
    dd = np.linalg.norm(c[:, None] - c[None], axis=2)
    # an RMS residual of 1e-6 over 1,340 edges allows overlaps of a few 1e-5
    assert (rr[:, None] + rr[None] - dd)[np.triu_indices(20, 1)].max() <= 1e-4
    assert r["iters"] < rh["iters"]


def test_rejections():
    p = inputs.packing_problem(5)
    with pytest.raises(_lib.FgaError):
        graph_from_problem(p, "f32", options={_lib.FGA_OPT_WEIGHTS: 1, _lib.FGA_OPT_ZORDER: 2})
    with pytest.raises(_lib.FgaError):
        graph_from_problem(p, "f64", options={_lib.FGA_OPT_WEIGHTS: 2})
    # the FP32 default with three weights is the canonical order
    assert graph_from_problem(p, "f32", options=TWA).fga_launch_info()["zorder"] == 0
