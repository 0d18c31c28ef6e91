"""Pins for the oracle's three-weight mode (og_set_weights, mode 1): every
x-update gives each edge a weight class -- infinite for a fixed value,
zero for a constraint-type factor that left the edge's message unchanged,
standard otherwise; z averages the infinite-weight messages if any, else
the standard ones, else all; u resets to 0 on non-standard edges.

  * a small example worked by hand (zero weight: an inactive box does not
    pull z; the box edge's u stays 0);
  * an infinite weight decides z at once and for good;
  * the minimiser is the one of the problem, as with fixed weights: a
    clipped quadratic in closed form, an MPC with an active box against the
    QP solution, the one-disk packing against the incircle;
  * a converged packing under three weights is feasible."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import OracleGraph, from_problem
from oracle.oracle import EDGE_X, EDGE_M, EDGE_U, EDGE_N
from paper_1603_02526_gb300 import inputs


def _scalar_graph(box, fix=None, rho=(1.0, 1.0, 2.0), alpha=1.0):
    """w with f1 = 1/2 w^2 (edge 0), f2 = -2 w (edge 1), a box on w (edge 2),
    optionally FIX(w) (edge 3)."""
    g = OracleGraph()
    g.add_variables(1, 1)
    g.add_factors(inputs.MPC_QUAD, [[0]], [[1.0]])
    g.add_factors(inputs.PACK_RADIUS_LIN, [[0]], [[2.0]])
    g.add_factors(inputs.MPC_BOX, [[0]], [list(box)])
    if fix is not None:
        g.add_factors(inputs.FIX, [[0]], [[fix]])
        rho = tuple(rho) + (1.0,)
    g.finalize(np.array(rho), alpha)
    g.set_weights(1)
    g.init(np.array([0.0]))
    return g


def test_inactive_box_by_hand():
    """rho = (1, 1, 2), alpha = 1, start z = 0, u = 0, n = 0.
    Iteration 1: x = (0 / 2, 0 + 2 / 1, clamp(0)) = (0, 2, 0); the box left
      its message unchanged: zero weight.  m = (0, 2, 0); z = (1*0 + 1*2) /
      (1 + 1) = 1 (with fixed weights: (0 + 2 + 2*0) / 4 = 1/2);
      u = (0 - 1, 2 - 1, reset) = (-1, 1, 0); n = z - u = (2, 0, 1).
    Iteration 2: x = (2 / 2, 0 + 2, clamp(1)) = (1, 2, 1), box zero again;
      m = (0, 3, 1); z = 3 / 2; u = (-1 + (1 - 3/2), 1 + (2 - 3/2), 0)
      = (-3/2, 3/2, 0); n = (3, 0, 3/2).
    Minimiser of 1/2 w^2 - 2 w on |w| <= 10: w = 2."""
    g = _scalar_graph((-10.0, 10.0))
    want = [dict(x=[0, 2, 0], m=[0, 2, 0], z=[1], u=[-1, 1, 0], n=[2, 0, 1]),
            dict(x=[1, 2, 1], m=[0, 3, 1], z=[1.5], u=[-1.5, 1.5, 0], n=[3, 0, 1.5])]
    for w in want:
        g.iterate(1)
        assert list(g.edge(EDGE_X)) == w["x"]
        assert list(g.edge(EDGE_M)) == w["m"]
        assert list(g.z()) == w["z"]
        assert list(g.edge(EDGE_U)) == w["u"]
        assert list(g.edge(EDGE_N)) == w["n"]
    r = g.iterate(5000, 1e-12, 1e-12)
    assert r["status"] == 0
    np.testing.assert_allclose(g.z(), [2.0], atol=1e-10)


def test_infinite_weight_decides_z():
    """A FIX(w = 4) edge: from the first iteration on z = 4 exactly, and the
    fixed edge's u stays 0."""
    g = _scalar_graph((-10.0, 10.0), fix=4.0)
    for _ in range(20):
        g.iterate(1)
        assert list(g.z()) == [4.0]
        assert g.edge(EDGE_U)[3] == 0.0


@pytest.mark.parametrize("box,want", [((-1.0, 1.0), 1.0), ((-10.0, 10.0), 2.0), ((2.5, 3.0), 2.5)])
def test_clipped_quadratic_minimiser(box, want):
    """argmin 1/2 w^2 - 2 w on lo <= w <= hi = clamp(2): reached with three
    weights as with fixed ones."""
    for mode in (0, 1):
        g = _scalar_graph(box)
        g.set_weights(mode)
        g.init(np.array([0.0]))
        r = g.iterate(20000, 1e-12, 1e-12)
        assert r["status"] == 0
        np.testing.assert_allclose(g.z(), [want], atol=1e-9)


def test_mpc_active_box_same_minimiser():
    """An MPC instance whose box is active: three weights converge to the
    QP solution (SciPy SLSQP on the condensed problem) like fixed weights."""
    d = inputs.mpc_batch_inputs(1, seed=4321, nx=3, nu=1, T_fixed=6, umax=0.3)
    A, B, q, r, x0 = d["A"][0], d["B"][0], d["q"][0], d["r"][0], 3.0 * d["x0"][0]
    p = inputs.mpc_problem(A, B, q, r, x0, 6, umax=0.3)
    g = from_problem(p, weights=1)
    res = g.iterate(200000, 1e-11, 1e-11)
    assert res["status"] == 0

    def cost(useq):
        x, J = x0.copy(), 0.0
        for t in range(6):
            J += 0.5 * (x @ (q * x)) + 0.5 * r[0] * useq[t] ** 2
            x = A @ x + B[:, 0] * useq[t]
        return J + 0.5 * (x @ (q * x))
    sol = minimize(cost, np.zeros(6), method="SLSQP", bounds=[(-0.3, 0.3)] * 6,
                   options=dict(ftol=1e-14, maxiter=500))
    z = g.z()
    S = 3 + 1
    u = np.array([z[t * S + 3] for t in range(6)])
    assert np.abs(np.abs(sol.x) - 0.3).min() < 1e-9       # the box is active at the optimum
    np.testing.assert_allclose(u, sol.x, atol=1e-6)


def test_one_disk_packing_is_the_incircle():
    g = from_problem(inputs.packing_problem(1), weights=1)
    r = g.iterate(20000, 1e-12, 1e-12)
    assert r["status"] == 0 and r["iters"] < 20000
    np.testing.assert_allclose(g.z(), [0.5, np.sqrt(3) / 6, np.sqrt(3) / 6], atol=1e-9)


def test_converged_packing_is_feasible():
    N = 20
    p = inputs.packing_problem(N)
    p.factor_blocks[-1].params[:] = 0.01
    g = from_problem(p, weights=1)
    r = g.iterate(50000, 1e-9, 1e-9)
    assert r["status"] == 0 and r["iters"] < 50000, r
    z = g.z()
    c = np.stack([z[0::3], z[1::3]], 1)
    rr = z[2::3]
    d = np.linalg.norm(c[:, None] - c[None], axis=2)
    ov = (rr[:, None] + rr[None] - d)[np.triu_indices(N, 1)].max()
    Q, V = inputs.triangle_walls()
    wall = (rr[:, None] - np.einsum("sk,isk->is", Q, c[:, None, :] - V[None])).max()
    assert ov <= 1e-6 and wall <= 1e-6 and rr.min() > 0
