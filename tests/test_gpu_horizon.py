"""GPU parity of the horizon-along-the-grid MPC solver (fga_horizon_*, the
long-horizon pendulum of Sec. V-B) against the FP64 oracle on the same
factor graph (inputs.mpc_horizon_problem), through the C-ABI.

FP32 tolerance as for the general path (tests/test_gpu_mpc_horizon.py): a
9-term dot product per iteration, about 9 * 2^-24 of the variables' scale S
per message, not amplified by the nonexpansive iteration: k iterations stay
within k times that."""
import numpy as np
import pytest

from oracle import from_problem as oracle_from_problem
from oracle.oracle import EDGE_X, EDGE_U
from paper_1603_02526_gb300 import inputs, _lib
from paper_1603_02526_gb300.horizon import Horizon

pytestmark = pytest.mark.gpu

F32_PER_ITER = 9 * 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


def _compare(h, o, iters):
    z, x, u = h.fga_horizon_read()
    S = float(np.max(np.abs(o.z())))
    bound = iters * F32_PER_ITER * S
    for name, g, w in (("z", z, o.z()), ("x", x, o.edge(EDGE_X)), ("u", u, o.edge(EDGE_U))):
        err = float(np.max(np.abs(g - w)))
        assert err <= bound, "%s: max abs err %.3e > %.3e" % (name, err, bound)


@pytest.mark.parametrize("K", [1, 2, 37, 223, 224, 225, 448, 500, 1000])
def test_horizon_grid_matches_oracle(K):
    """300 iterations; K around the 224-step CTA size (one CTA, a full CTA,
    a second CTA with one step, several CTAs with a ragged last one)."""
    p = inputs.mpc_horizon_problem(K)
    h = Horizon.from_problem(p)
    assert h.num_edges == p.num_edges and h.num_scalar_vars == p.num_scalar_vars
    h.fga_horizon_init()
    r = h.fga_horizon_solve(300)
    assert r["iters"] == 300 and r["status"] == 0
    o = oracle_from_problem(p)
    ro = o.iterate(300)
    _compare(h, o, 300)
    assert abs(r["r_pri"] - ro["r_pri"]) <= 1e-3 * ro["r_pri"] + 1e-6


def test_horizon_grid_full_size():
    """K = 10^5 (1,400,008 scalar edges, 447 CTAs), 20 iterations."""
    p = inputs.mpc_horizon_problem(100000)
    h = Horizon.from_problem(p)
    h.fga_horizon_init()
    h.fga_horizon_solve(20)
    o = oracle_from_problem(p)
    o.iterate(20)
    _compare(h, o, 20)


def test_horizon_grid_chained_calls():
    """Resume: three calls of 100 iterations equal one call of 300, bit for
    bit (one deterministic order of operations)."""
    p = inputs.mpc_horizon_problem(700)
    a = Horizon.from_problem(p)
    a.fga_horizon_init()
    a.fga_horizon_solve(300, check_every=7)
    b = Horizon.from_problem(p)
    b.fga_horizon_init()
    for _ in range(3):
        b.fga_horizon_solve(100, check_every=7)
    for va, vb in zip(a.fga_horizon_read(), b.fga_horizon_read()):
        assert np.array_equal(va, vb)


def test_horizon_grid_stop_rule():
    """K = 2000 to RMS residual 1e-5, checked every 10: the stop lands on
    the oracle's checked iteration (or the next check, FP32 near the
    threshold), with both residuals at or below the tolerance."""
    p = inputs.mpc_horizon_problem(2000)
    h = Horizon.from_problem(p)
    h.fga_horizon_init()
    r = h.fga_horizon_solve(50000, 1e-5, 1e-5, check_every=10)
    o = oracle_from_problem(p)
    ro = o.iterate(50000, 1e-5, 1e-5, check_every=10)
    assert r["status"] == 0 and ro["status"] == 0
    assert r["iters"] % 10 == 0 and abs(r["iters"] - ro["iters"]) <= 10
    assert r["r_pri"] <= 1e-5 and r["r_dual"] <= 1e-5


def test_horizon_grid_budget_status():
    p = inputs.mpc_horizon_problem(300)
    h = Horizon.from_problem(p)
    h.fga_horizon_init()
    r = h.fga_horizon_solve(5, 1e-12, 1e-12)
    assert r["iters"] == 5 and r["status"] == _lib.FGA_EBUDGET


def test_horizon_grid_barrier_time_limit():
    """A CTA that skips its first barrier arrival: the other CTAs' waits run
    out, the call returns FGA_ETIMEOUT, and after fga_horizon_init the
    object solves again (the GPU context stays usable)."""
    p = inputs.mpc_horizon_problem(2000)
    h = Horizon.from_problem(p)
    h.fga_horizon_init()
    r = h.fga_horizon_solve(10, barrier_timeout_ns=50_000_000, fault_skip_block=3, raise_on_error=False)
    assert r["rc"] == _lib.FGA_ETIMEOUT
    h.fga_horizon_init()
    r = h.fga_horizon_solve(10)
    assert r["iters"] == 10 and r["status"] == 0


def test_horizon_grid_rejects():
    """Shapes other than the pendulum's and horizons beyond one co-resident
    grid are refused at creation."""
    p = inputs.mpc_horizon_problem(10)
    m = p.meta
    with pytest.raises(_lib.FgaError):
        Horizon(10, np.eye(12), np.ones((12, 4)), np.ones(12), np.ones(4), np.zeros(12))
    with pytest.raises(_lib.FgaError):
        Horizon(10 ** 7, m["A"], m["B"], m["q"], m["r"], m["x0"])
