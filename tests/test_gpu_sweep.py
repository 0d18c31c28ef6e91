"""GPU parity of the factor-graph sweep against the FP64 oracle (through the
C-ABI).  FP64 runs use the canonical z-order and must match the oracle to
1e-10 relative per message (floor 1e-3 of the array scale); in practice
they agree bit for bit.  FP32 runs use the fast order; their tolerances are
derived from FP32 rounding (see each test)."""
import numpy as np
import pytest

from oracle import from_problem as oracle_from_problem
from paper_1603_02526_gb300 import inputs
from paper_1603_02526_gb300 import _lib
from paper_1603_02526_gb300.graph import graph_from_problem, FactorGraph
from tests.helpers import (assert_messages_match, assert_messages_close_scaled, packing_objective,
                           rel_close_floor)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


def _both(problem, iters, precision="f64", fused=True, options=None, **kw):
    g = graph_from_problem(problem, precision, options=options)
    rg = g.fga_iterate(iters, fused=fused, **kw)
    o = oracle_from_problem(problem)
    ro = o.iterate(iters, **{k: v for k, v in kw.items() if k in ("tol_pri", "tol_dual", "check_every")})
    return g, o, rg, ro


@pytest.mark.parametrize("fused", [True, False])
def test_packing_n20_f64_5000_iterations(fused):
    """Circle packing N=20, rho = alpha = 1, 5000 iterations, FP64."""
    p = inputs.packing_problem(20)
    g, o, rg, ro = _both(p, 5000, fused=fused)
    assert rg["iters"] == ro["iters"] == 5000
    assert_messages_match(g, o, 1e-10)
    # the canonical order reproduces the serial sums exactly
    assert np.array_equal(g.fga_read_z(), o.z())
    np.testing.assert_allclose([rg["r_pri"], rg["r_dual"]], [ro["r_pri"], ro["r_dual"]], rtol=1e-12)


def test_packing_chained_calls_equal_one_call():
    """Resume: five calls of 1000 iterations reproduce one call of 5000."""
    p = inputs.packing_problem(20)
    a = graph_from_problem(p, "f64")
    a.fga_iterate(5000)
    b = graph_from_problem(p, "f64")
    for _ in range(5):
        b.fga_iterate(1000, check_every=7)
    for w in range(4):
        assert np.array_equal(a.fga_read_edge_state(w), b.fga_read_edge_state(w))
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())


def test_packing_n1000_f64_full_size():
    """The N=1000 graph (3,007,000 scalar edges) at FP64, a few iterations,
    every message compared."""
    p = inputs.packing_problem(1000)
    g, o, rg, ro = _both(p, 3)
    assert_messages_match(g, o, 1e-10)


def test_packing_stop_rule_matches_oracle():
    p = inputs.packing_problem(3)
    p.factor_blocks[-1].params[:] = 0.1
    for ce in (1, 5):
        g, o, rg, ro = _both(p, 5000, tol_pri=1e-7, tol_dual=1e-7, check_every=ce)
        assert rg["iters"] == ro["iters"] < 5000
        assert rg["status"] == 0
        assert_messages_match(g, o, 1e-10)


def test_budget_status():
    p = inputs.packing_problem(20)
    g = graph_from_problem(p, "f64")
    r = g.fga_iterate(10, tol_pri=1e-12, tol_dual=1e-12)
    assert r["iters"] == 10 and r["status"] == _lib.FGA_EBUDGET


def test_fast_order_f64_drift():
    """The fast (tree) z-order in FP64: reported drift vs the canonical
    order after 200 iterations of N=20 (non-convex, so differences of one
    ulp may grow; bound 1e-8 relative with the floor)."""
    p = inputs.packing_problem(20)
    g = graph_from_problem(p, "f64", options={_lib.FGA_OPT_ZORDER: 1})
    g.fga_iterate(200)
    o = oracle_from_problem(p)
    o.iterate(200)
    ok, emax, _ = rel_close_floor(g.fga_read_z(), o.z(), 1e-8)
    assert ok, emax


def test_fig1_readout_in_creation_order():
    p = inputs.fig1_problem()
    g, o, rg, ro = _both(p, 25)
    assert_messages_match(g, o, 1e-10)


def test_per_edge_rho_alpha():
    """Non-uniform rho and alpha per scalar edge (one rho per disk centre)."""
    p = inputs.packing_problem(6)
    rng = np.random.default_rng(3)
    o0 = oracle_from_problem(p)
    E = o0.num_edges
    ev = o0.edge_var()
    alpha = 0.5 + rng.random(E)
    rho = (1.2 + rng.random(p.num_scalar_vars))
    rho[1::3] = rho[0::3]
    rho_e = rho[ev]
    g = FactorGraph("f64")
    from paper_1603_02526_gb300.graph import _merge_var_blocks
    for c, d in _merge_var_blocks(p.var_blocks):
        g.fga_add_variables(c, d)
    for b in p.factor_blocks:
        g.fga_add_factors(b.ftype, b.var_ids, b.params if b.params.size else None)
    g.fga_set_edge_rho_alpha(rho_e, alpha)
    g.fga_finalize()
    g.fga_init(p.z0)
    g.fga_iterate(300)
    o = oracle_from_problem(p)
    o.set_rho_alpha(rho_e, alpha)
    o.init(p.z0)
    o.iterate(300)
    assert_messages_match(g, o, 1e-10)


def test_area_reward():
    """The paper's area reward -r^2/2 (Appendix A), whose prox needs rho > 1;
    at rho = 25 the iteration stays bounded (at rho ~ 1-2 both the oracle and
    the GPU diverge and report a non-finite residual)."""
    p = inputs.packing_problem(6, reward="quad", rho=25.0)
    g, o, rg, ro = _both(p, 300)
    assert_messages_match(g, o, 1e-10)
    q = inputs.packing_problem(6, reward="quad", rho=1.5)
    g = graph_from_problem(q, "f64")
    r = g.fga_iterate(2000, raise_on_error=False)
    assert r["rc"] == _lib.FGA_ENONFINITE
    with pytest.raises(_lib.FgaError):
        graph_from_problem(inputs.packing_problem(2, reward="quad", rho=1.0), "f64")


def test_f32_packing_n20_objective():
    """FP32 messages, FP64 residuals: N=20 (converging setting, reward 0.01)
    run to residual 1e-4 by GPU and oracle; objective -sum r within 1e-4
    relative of the oracle's."""
    p = inputs.packing_problem(20)
    p.factor_blocks[-1].params[:] = 0.01
    g = graph_from_problem(p, "f32")
    rg = g.fga_iterate(50000, 1e-4, 1e-4)
    o = oracle_from_problem(p)
    ro = o.iterate(50000, 1e-4, 1e-4)
    assert rg["status"] == 0 and ro["status"] == 0
    fg, fo = packing_objective(g.fga_read_z()), packing_objective(o.z())
    assert abs(fg - fo) <= 1e-4 * abs(fo), (fg, fo, rg, ro)


@pytest.mark.parametrize("iters", [3, 10])
def test_f32_n1000_chunked_order_first_iterations(iters):
    """N=1000 in FP32 through the chunked fast order (fused, m kept) against
    the FP64 oracle after 3 and 10 iterations.  Its z sums are FP32 trees
    (chunk partials, then warp and hub trees), so the yardstick is the FP32
    emulation (tests/fp32_emulation.py) with pairwise FP32 sums: z, and every
    edge message at the 99.9th percentile and at the maximum, within 4x the
    emulation's own distance from the oracle (measured on GB300: at most
    2.4x, the maximum after 10 iterations; 1.8x after 3).  The disk-pair operator divides by the distance of two incoming
    centres, so the few pairs whose messages come close amplify rounding:
    hence percentile and maximum apart."""
    from oracle.oracle import EDGE_X, EDGE_U, EDGE_N
    from tests.fp32_emulation import PackingFP32
    p = inputs.packing_problem(1000)
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 1})
    assert g.fga_launch_info()["zorder"] == 1
    g.fga_iterate(iters)
    o = oracle_from_problem(p)
    o.iterate(iters)
    em = PackingFP32(p, sums="tree")
    em.iterate(iters)
    S = float(np.max(np.abs(o.z())))
    ez = np.abs(g.fga_read_z() - o.z()).max()
    assert ez <= 4 * np.abs(em.z - o.z()).max(), (ez / S, np.abs(em.z - o.z()).max() / S)
    for a, b, ref in ((_lib.FGA_EDGE_X, EDGE_X, em.x), (_lib.FGA_EDGE_U, EDGE_U, em.u),
                      (_lib.FGA_EDGE_N, EDGE_N, em.n)):
        err = np.abs(g.fga_read_edge_state(a) - o.edge(b))
        eref = np.abs(ref.astype(np.float64) - o.edge(b))
        for q in (99.9, 100):
            assert np.percentile(err, q) <= 4 * np.percentile(eref, q), (a, q, np.percentile(err, q) / S,
                                                                            np.percentile(eref, q) / S)


def test_f32_is_deterministic():
    p = inputs.packing_problem(200)
    a = graph_from_problem(p, "f32")
    a.fga_iterate(100)
    b = graph_from_problem(p, "f32")
    b.fga_iterate(100)
    assert np.array_equal(a.fga_read_z(), b.fga_read_z())
    assert np.array_equal(a.fga_read_edge_state(_lib.FGA_EDGE_U), b.fga_read_edge_state(_lib.FGA_EDGE_U))


@pytest.mark.parametrize("kind,zorder", [("packing", 1), ("packing", 2), ("svm", 3)])
def test_barrier_time_limit_returns_timeout_and_recovers(kind, zorder):
    """Fault injection, in each fused kernel (chunked order, disk tiles,
    hinge bank): one CTA skips its first barrier arrival; the bounded wait
    runs out (50 ms) and fga_iterate returns FGA_ETIMEOUT.  The context
    stays usable: after fga_init the same graph iterates normally."""
    p = inputs.packing_problem(200) if kind == "packing" else inputs.svm_problem(3000, 32, seed=3600)
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_ZORDER: zorder})
    assert g.fga_launch_info()["zorder"] == zorder
    r = g.fga_iterate(10, barrier_timeout_ns=50_000_000, fault_skip_block=0, raise_on_error=False)
    assert r["rc"] == _lib.FGA_ETIMEOUT and r["status"] == _lib.FGA_ETIMEOUT
    with pytest.raises(_lib.FgaError):
        g.fga_iterate(1)                       # state undefined until re-initialised
    g.fga_init(p.z0)
    r = g.fga_iterate(10)
    assert r["iters"] == 10 and np.isfinite(r["r_pri"])


def test_nonfinite_residual_reported():
    """A start point that overflows FP32 makes the residual non-finite."""
    p = inputs.packing_problem(5)
    g = graph_from_problem(p, "f32", init=False)
    z0 = p.z0.copy()
    z0[0] = 1e300
    g.fga_init(z0)
    r = g.fga_iterate(5, raise_on_error=False)
    assert r["rc"] == _lib.FGA_ENONFINITE and r["status"] == _lib.FGA_ENONFINITE


def test_device_pointer_io():
    torch = pytest.importorskip("torch")
    p = inputs.packing_problem(20)
    g = graph_from_problem(p, "f64", init=False)
    z0 = torch.tensor(p.z0, dtype=torch.float64, device="cuda")
    g.fga_init(z0)
    g.fga_iterate(50)
    zd = torch.empty(g.num_scalar_vars, dtype=torch.float64, device="cuda")
    g.fga_read_z(zd)
    assert np.array_equal(zd.cpu().numpy(), g.fga_read_z())


@pytest.mark.parametrize("fused", [True, False])
def test_canonical_z_rows_of_every_length(fused):
    """FP64 canonical z order over variables whose degrees straddle the
    32-value blocks in which the z sums are staged (0, 1, 31, 32, 33, 63, 64,
    65, 97, 200) and more than 32 variables (groups of 32 with an uneven
    tail); quadratic costs, boxes and fixed values interleaved in creation
    order.  Every message against the oracle to 1e-10 after 40 iterations."""
    degrees = [0, 1, 31, 32, 33, 63, 64, 65, 97, 200] * 4 + [2, 3]
    rng = np.random.default_rng(11)
    p = inputs.Problem("degrees")
    v0 = p.add_vars(len(degrees), 1)
    for rep in range(max(degrees)):
        live = [i for i, d in enumerate(degrees) if rep < d]
        kind = rep % 3
        ids = [[v0 + i] for i in live]
        if kind == 0:
            p.add_factors(7, ids, [[0.5 + rng.random()] for _ in live])          # quadratic cost
        elif kind == 1:
            p.add_factors(8, ids, [[-0.5, 0.5 + rng.random()] for _ in live])    # box
        else:
            p.add_factors(9, ids, [[rng.standard_normal()] for _ in live])       # fixed value
    p.z0 = rng.standard_normal(p.num_scalar_vars)
    g, o, rg, ro = _both(p, 40, fused=fused)
    assert_messages_match(g, o, 1e-10)
    assert np.array_equal(g.fga_read_z(), o.z())
