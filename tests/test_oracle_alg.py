"""Pins for the oracle's Algorithm 2 as a whole.

  * Algorithm 1 (classical x/z/u ADMM, Sec. I) written here in its general
    matrix form equals Algorithm 2 iterate for iterate on consensus problems.
  * Closed forms: N=1 packing converges to the incircle; the two-point SVM
    converges to w = (1/a, 0), b = 0; MPC with an inactive box converges to
    finite-horizon LQR (backward Riccati recursion).
  * Library solutions: MPC with an active box and a small SVM vs SciPy.
  * Geometry: a converged packing has no overlap and stays in the triangle.
  * Counts of Sec. V-A and the edge-storage order of the Sec. II/III example.
"""
import os

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import from_problem, OracleGraph
from oracle.oracle import EDGE_X, EDGE_M, EDGE_U, EDGE_N
from paper_1603_02526_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Algorithm 1 in matrix form: f(w1) = 1/2 w1' H w1 + g' w1 s.t. C w1 = d,
# g-part of the objective = 0; constraint A w1 + B w2 = c.
# ---------------------------------------------------------------------------
def admm_alg1(H, gvec, C, d, A, B, c, rho, z0, iters):
    nw = H.shape[0]
    u = np.zeros(A.shape[0])
    z = z0.copy()
    xs, zs, us = [], [], []
    for _ in range(iters):
        # x <- argmin f(s) + rho/2 |A s + B z - c + u|^2  (KKT solve with C s = d)
        K = H + rho * A.T @ A
        rhs = -gvec - rho * A.T @ (B @ z - c + u)
        if C is not None and C.shape[0]:
            m = C.shape[0]
            KK = np.zeros((nw + m, nw + m))
            KK[:nw, :nw] = K
            KK[:nw, nw:] = C.T
            KK[nw:, :nw] = C
            x = np.linalg.solve(KK, np.concatenate([rhs, d]))[:nw]
        else:
            x = np.linalg.solve(K, rhs)
        # z <- argmin rho/2 |A x + B r - c + u|^2  (least squares)
        z = np.linalg.lstsq(B, -(A @ x - c + u), rcond=None)[0]
        # u <- u + A x + B z - c
        u = u + A @ x + B @ z - c
        xs.append(x); zs.append(z); us.append(u)
    return xs, zs, us


def test_alg1_equals_alg2_scalar_consensus():
    """f(w) = 1/2 q w^2 - a w + (lam/2) w^2 split into three factors on one
    scalar variable: Alg. 1 with A = I, B = -1, c = 0 vs Alg. 2."""
    q, a, lam, rho = 2.0, 0.7, 0.5, 1.3
    g = OracleGraph()
    g.add_variables(1, 1)
    g.add_factors(inputs.MPC_QUAD, [[0]], [[q]])
    g.add_factors(inputs.PACK_RADIUS_LIN, [[0]], [[a]])
    g.add_factors(inputs.SVM_L2, [[0]], [[lam]])
    g.finalize(rho, 1.0)
    z0 = np.array([0.9])
    g.init(z0)
    H = np.diag([q, 0.0, lam]); gv = np.array([0.0, -a, 0.0])
    xs, zs, us = admm_alg1(H, gv, None, None, np.eye(3), -np.ones((3, 1)), np.zeros(3), rho, z0, 40)
    for k in range(40):
        g.iterate(1)
        np.testing.assert_allclose(g.edge(EDGE_X), xs[k], rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(g.z(), zs[k], rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(g.edge(EDGE_U), us[k], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(g.z(), [a / (q + lam)], rtol=1e-9)


def test_alg1_equals_alg2_mpc_without_box():
    """One-step-horizon MPC (FIX, DYN, stage and terminal QUAD) as a
    consensus problem: A = I on the stacked factor copies, B = -S (S selects
    each copy's variable component), c = 0; indicator factors become the
    equality block C w1 = d of the x-update."""
    rng = np.random.default_rng(5)
    nx, nu, T = 3, 2, 2
    A_, B_, q, r = inputs.mpc_system(nx, nu, rng)
    x0 = rng.standard_normal(nx)
    prob = inputs.mpc_problem(A_, B_, q, r, x0, T, umax=1e9)
    prob.factor_blocks = prob.factor_blocks[:4]          # drop the box factors
    rho = 1.7
    prob.rho = rho
    g = from_problem(prob)
    ev = g.edge_var()
    E, Z = g.num_edges, g.num_scalar_vars
    S = np.zeros((E, Z)); S[np.arange(E), ev] = 1.0
    # stacked factor copies in creation order: FIX(12?) DYN... built from the blocks
    H = np.zeros((E, E)); gv = np.zeros(E)
    Crows, drows = [], []
    e = 0
    dims = prob.var_dims()
    for blk in prob.factor_blocks:
        for f in range(blk.var_ids.shape[0]):
            ar = int(dims[blk.var_ids[f]].sum())
            sl = slice(e, e + ar)
            if blk.ftype == inputs.FIX:
                for k in range(ar):
                    row = np.zeros(E); row[e + k] = 1.0
                    Crows.append(row); drows.append(blk.params[f, k])
            elif blk.ftype == inputs.MPC_DYN:
                M = np.concatenate([A_, B_, -np.eye(nx)], axis=1)
                for k in range(nx):
                    row = np.zeros(E); row[sl] = M[k]
                    Crows.append(row); drows.append(0.0)
            elif blk.ftype == inputs.MPC_QUAD:
                H[sl, sl] = np.diag(blk.params[f])
            e += ar
    C = np.array(Crows); d = np.array(drows)
    xs, zs, us = admm_alg1(H, gv, C, d, np.eye(E), -S, np.zeros(E), rho, np.zeros(Z), 30)
    for k in range(30):
        g.iterate(1)
        np.testing.assert_allclose(g.edge(EDGE_X), xs[k], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(g.z(), zs[k], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(g.edge(EDGE_U), us[k], rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------
# Packing
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 20, 1000])
def test_packing_counts(N):
    p = inputs.packing_problem(N)
    cnt = inputs.packing_counts(N)
    var_edges = sum(b.var_ids.size for b in p.factor_blocks)
    assert var_edges == cnt["edges"]
    assert p.num_vars == cnt["var_nodes"]
    assert p.num_factors == cnt["factors"]
    assert p.num_edges == (N * (N - 1) // 2) * 6 + 3 * N * 3 + N


def test_packing_one_disk_is_the_incircle():
    g = from_problem(inputs.packing_problem(1))
    r = g.iterate(20000, 1e-12, 1e-12)
    assert r["status"] == 0 and r["iters"] < 20000
    np.testing.assert_allclose(g.z(), [0.5, np.sqrt(3) / 6, np.sqrt(3) / 6], atol=1e-10)


def _packing_violation(z, N):
    c = np.stack([z[0::3], z[1::3]], 1); rr = z[2::3]
    d = np.linalg.norm(c[:, None] - c[None], axis=2)
    ov = (rr[:, None] + rr[None] - d)[np.triu_indices(N, 1)].max()
    Q, V = inputs.triangle_walls()
    wall = (rr[:, None] - np.einsum("sk,isk->is", Q, c[:, None, :] - V[None])).max()
    return ov, wall, rr


def test_converged_packing_is_feasible():
    """With a small radius reward the N=20 run converges; brute-force O(N^2)
    geometry check: no overlap and every disk inside the triangle."""
    N = 20
    p = inputs.packing_problem(N)
    p.factor_blocks[-1].params[:] = 0.01
    g = from_problem(p)
    r = g.iterate(50000, 1e-9, 1e-9)
    assert r["iters"] < 50000
    ov, wall, rr = _packing_violation(g.z(), N)
    assert ov <= 1e-6 and wall <= 1e-6
    assert rr.min() > 0 and rr.sum() > np.sqrt(3) / 6      # beats one incircle


def test_fig1_edge_storage_order():
    """Sec. III: x is stored in edge-creation order
    [x11 x12 x13 x21 x24 x25 x32 x35 x45]; z in variable order."""
    want = []
    with open(os.path.join(GOLDEN, "fig1_edge_order.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                a, b = line.split()
                want.append((int(a), int(b)))
    p = inputs.fig1_problem()
    g = from_problem(p)
    got = []
    for fi, blk in enumerate(p.factor_blocks):
        for v in blk.var_ids[0]:
            got.append((fi + 1, int(v) + 1))
    assert got == want
    np.testing.assert_array_equal(g.edge_var() + 1, [b for _, b in want])
    g.iterate(3)
    assert g.z().shape == (5,)


def test_residual_definition_and_stop_rule():
    """RMS residuals after each iteration recomputed from the readouts, and
    the stop at the first checked iteration meeting both tolerances."""
    p = inputs.packing_problem(3)
    p.factor_blocks[-1].params[:] = 0.1
    g = from_problem(p)
    ev = g.edge_var()
    zprev = g.z()
    for _ in range(5):
        r = g.iterate(1)
        x, z = g.edge(EDGE_X), g.z()
        rp = np.sqrt(np.mean((x - z[ev]) ** 2))
        rd = np.sqrt(np.mean((z[ev] - zprev[ev]) ** 2))
        np.testing.assert_allclose([r["r_pri"], r["r_dual"]], [rp, rd], rtol=1e-12)
        np.testing.assert_allclose(g.edge(EDGE_M), x + (g.edge(EDGE_U) - (x - z[ev])), rtol=0, atol=1e-15)
        np.testing.assert_array_equal(g.edge(EDGE_N), z[ev] - g.edge(EDGE_U))
        zprev = z
    g2 = from_problem(p)
    hist = []
    for k in range(3000):
        r = g2.iterate(1)
        hist.append((r["r_pri"], r["r_dual"]))
    tol = 1e-6
    first = next(k + 1 for k, (a, b) in enumerate(hist) if a <= tol and b <= tol)
    g3 = from_problem(p)
    r = g3.iterate(3000, tol, tol)
    assert r["iters"] == first
    g4 = from_problem(p)
    r = g4.iterate(3000, tol, tol, check_every=7)
    assert r["iters"] % 7 == 0 and r["iters"] >= first
    assert r["iters"] == next(k for k in range(7, 3001, 7) if hist[k - 1][0] <= tol and hist[k - 1][1] <= tol)


def test_oracle_is_deterministic():
    p = inputs.packing_problem(20)
    a = from_problem(p); a.iterate(500)
    b = from_problem(p); b.iterate(500)
    assert np.array_equal(a.z(), b.z()) and np.array_equal(a.edge(EDGE_U), b.edge(EDGE_U))


# ---------------------------------------------------------------------------
# MPC
# ---------------------------------------------------------------------------
def _lqr(A, B, q, r, x0, T):
    """Finite-horizon LQR by the backward Riccati recursion, terminal Q_f = Q."""
    Q = np.diag(q); R = np.diag(r)
    P = Q.copy()
    Ks = []
    for _ in range(T):
        K = np.linalg.solve(R + B.T @ P @ B, B.T @ P @ A)
        P = Q + A.T @ P @ (A - B @ K)
        Ks.append(K)
    Ks = Ks[::-1]
    xs, us = [x0], []
    for t in range(T):
        u = -Ks[t] @ xs[-1]
        us.append(u)
        xs.append(A @ xs[-1] + B @ u)
    return np.array(xs), np.array(us)


def _mpc_split(z, nx, nu, T):
    xs = np.array([z[t * (nx + nu): t * (nx + nu) + nx] for t in range(T + 1)])
    us = np.array([z[t * (nx + nu) + nx: (t + 1) * (nx + nu)] for t in range(T)])
    return xs, us


def test_mpc_inactive_box_is_lqr():
    rng = np.random.default_rng(21)
    nx, nu, T = 12, 4, 10
    A, B, q, r = inputs.mpc_system(nx, nu, rng)
    x0 = rng.standard_normal(nx)
    g = from_problem(inputs.mpc_problem(A, B, q, r, x0, T, umax=1e6))
    res = g.iterate(200000, 1e-11, 1e-11)
    assert res["iters"] < 200000
    xs, us = _mpc_split(g.z(), nx, nu, T)
    xl, ul = _lqr(A, B, q, r, x0, T)
    np.testing.assert_allclose(xs, xl, atol=1e-8)
    np.testing.assert_allclose(us, ul, atol=1e-8)


def test_mpc_active_box_matches_qp():
    rng = np.random.default_rng(22)
    nx, nu, T = 4, 2, 6
    A, B, q, r = inputs.mpc_system(nx, nu, rng)
    x0 = 3.0 * rng.standard_normal(nx)
    umax = 0.2
    g = from_problem(inputs.mpc_problem(A, B, q, r, x0, T, umax=umax))
    res = g.iterate(200000, 1e-11, 1e-11)
    assert res["iters"] < 200000
    xs, us = _mpc_split(g.z(), nx, nu, T)
    assert np.abs(us).max() <= umax + 1e-9
    assert np.abs(us).max() >= umax - 1e-9                  # the box is active

    def cost(U):
        U = U.reshape(T, nu)
        x = x0.copy(); c = 0.0
        for t in range(T):
            c += 0.5 * (np.sum(q * x * x) + np.sum(r * U[t] * U[t]))
            x = A @ x + B @ U[t]
        return c + 0.5 * np.sum(q * x * x)
    sol = minimize(cost, np.zeros(T * nu), method="L-BFGS-B", bounds=[(-umax, umax)] * (T * nu),
                   options=dict(ftol=1e-15, gtol=1e-12, maxiter=10000))
    np.testing.assert_allclose(us.ravel(), sol.x, atol=2e-5)
    assert cost(us.ravel()) <= sol.fun + 1e-9


def test_pendulum_sampling_closed_form():
    """The sampled inverted pendulum of the long-horizon MPC (Sec. V-B: A
    4 x 4, B 4 x 1, 40 ms) against the zero-order-hold solution written out
    by hand: the angle obeys th'' = w^2 th - F/(M l), w^2 = (M + m) g / (M l)
    (hyperbolic sines and cosines), and the cart integrates F/M - (m g/M) th
    twice."""
    h, M, m, l, g = 0.04, 1.0, 0.1, 0.5, 9.81
    A, B = inputs.pendulum_system(h, M, m, l, g)
    w = np.sqrt((M + m) * g / (M * l))
    ch, sh = np.cosh(w * h), np.sinh(w * h)
    c = m * g / M
    A_ref = np.array([
        [1.0, h, -c * (ch - 1) / w**2, -c * (sh / w - h) / w**2],
        [0.0, 1.0, -c * sh / w, -c * (ch - 1) / w**2],
        [0.0, 0.0, ch, sh / w],
        [0.0, 0.0, w * sh, ch]])
    k = 1.0 / (M * l)
    B_ref = np.array([h * h / (2 * M) + c * k * ((ch - 1) / w**2 - h * h / 2) / w**2,
                      h / M + c * k * (sh / w - h) / w**2,
                      -k * (ch - 1) / w**2,
                      -k * sh / w])
    np.testing.assert_allclose(A, A_ref, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(B.ravel(), B_ref, rtol=1e-12, atol=1e-15)
    assert np.max(np.abs(np.linalg.eigvals(A))) > 1.2     # open-loop unstable


def test_mpc_horizon_pendulum_is_lqr():
    """The long-horizon pendulum graph (two variable blocks, no box),
    converged by the oracle, is the finite-horizon LQR trajectory."""
    K = 60
    p = inputs.mpc_horizon_problem(K)
    assert p.num_edges == inputs.mpc_horizon_edges(K)
    g = from_problem(p)
    res = g.iterate(200000, 1e-10, 1e-10)
    assert res["status"] == 0
    xs, us = inputs.mpc_horizon_split(g.z(), K)
    m = p.meta
    xl, ul = _lqr(m["A"], m["B"], m["q"], m["r"], m["x0"], K)
    np.testing.assert_allclose(xs, xl, atol=1e-6)
    np.testing.assert_allclose(us, ul, atol=1e-6)


# ---------------------------------------------------------------------------
# SVM
# ---------------------------------------------------------------------------
def test_svm_two_points_closed_form():
    """Points (+-a, 0) with labels +-1: for lam < 2 a^2 the optimum is
    w = (1/a, 0), b = 0 (both hinges exactly at the margin)."""
    a = 2.0
    X = np.array([[a, 0.0], [-a, 0.0]]); y = np.array([1.0, -1.0])
    p = inputs.svm_problem(2, 2, lam=1e-3, X=X, y=y)
    g = from_problem(p)
    res = g.iterate(200000, 1e-12, 1e-12)
    assert res["iters"] < 200000
    np.testing.assert_allclose(g.z(), [1 / a, 0.0, 0.0], atol=1e-8)


def test_svm_paper_form_matches_qp():
    """The paper's SVM form (a copy of w per point chained by equality
    factors, margin, slack and split-norm factors), converged by the oracle:
    the soft-margin QP's solution min 1/2 |w|^2 + C sum xi (SLSQP on the
    epigraph form), every copy of w equal, and the slacks the hinge losses."""
    X, y = inputs.svm_data(12, 2, seed=11)
    C = 2.0
    p = inputs.svm_paper_problem(12, 2, C=C, X=X, y=y)
    assert p.num_edges == inputs.svm_paper_edges(12, 2)
    g = from_problem(p)
    res = g.iterate(2000000, 1e-11, 1e-11, check_every=10)
    assert res["status"] == 0
    z = g.z()
    W = z[:24].reshape(12, 2)
    bz = z[24]
    xi = z[25:]
    np.testing.assert_allclose(W, np.broadcast_to(W[0], W.shape), atol=1e-7)
    cons = [dict(type="ineq", fun=lambda s: s[3:]),
            dict(type="ineq", fun=lambda s: s[3:] - (1 - y * (X @ s[:2] + s[2])))]
    s0 = np.concatenate([W[0], [bz], xi])
    sol = minimize(lambda s: 0.5 * s[:2] @ s[:2] + C * s[3:].sum(), s0, constraints=cons,
                   method="SLSQP", options=dict(ftol=1e-15, maxiter=2000))
    np.testing.assert_allclose(W[0], sol.x[:2], atol=1e-5)
    np.testing.assert_allclose(bz, sol.x[2], atol=1e-5)
    np.testing.assert_allclose(xi, np.maximum(0.0, 1 - y * (X @ W[0] + bz)), atol=1e-6)


def test_svm_small_matches_qp():
    X, y = inputs.svm_data(30, 3, seed=9)
    lam = 0.1
    g = from_problem(inputs.svm_problem(30, 3, lam=lam, X=X, y=y))
    res = g.iterate(400000, 1e-10, 1e-10)
    assert res["iters"] < 400000
    z = g.z()

    def F(v):
        return np.maximum(0, 1 - y * (X @ v[:3] + v[3])).sum() + 0.5 * lam * v[:3] @ v[:3]
    # epigraph QP
    nv = 4 + 30
    cons = [dict(type="ineq", fun=lambda s: s[4:]),
            dict(type="ineq", fun=lambda s: s[4:] - (1 - y * (X @ s[:3] + s[3])))]
    s0 = np.concatenate([z, np.maximum(0, 1 - y * (X @ z[:3] + z[3]))])
    sol = minimize(lambda s: s[4:].sum() + 0.5 * lam * s[:3] @ s[:3], s0, constraints=cons,
                   method="SLSQP", options=dict(ftol=1e-14, maxiter=2000))
    assert F(z) <= sol.fun + 1e-7
    np.testing.assert_allclose(z[:3], sol.x[:3], atol=1e-4)


def test_two_factor_weighted_rho_and_alpha_by_hand():
    """Per-edge rho and alpha, worked by hand (Algorithm 2's update rules,
    Sec. II).  One scalar variable w; factor 1 is f = 1/2 w^2 (cost q = 1)
    on an edge with rho 1, factor 2 fixes w = 4 on an edge with rho 3; both
    edges take alpha = 1/2.  Start z = 0, u = 0, so n = 0.

    Iteration 1: x = (rho n / (q + rho), 4) = (0, 4); m = x + u = (0, 4);
      z = (1*0 + 3*4) / (1 + 3) = 3;  u = 0 + 1/2 (x - 3) = (-3/2, 1/2);
      n = z - u = (9/2, 5/2).
    Iteration 2: x = (1 * 9/2 / 2, 4) = (9/4, 4); m = (3/4, 9/2);
      z = (3/4 + 27/2) / 4 = 57/16;  u = (-3/2 + 1/2 (9/4 - 57/16),
      1/2 + 1/2 (4 - 57/16)) = (-69/32, 23/32);  n = (183/32, 91/32).
    Every value is a dyadic rational, so FP64 holds it exactly.  An
    unweighted mean would give z = 2 after iteration 1, and alpha taken as 1
    would give u = (-3, 1).

    Residuals (RMS over the two edges): iteration 1, x - z = (-3, 1) and
    rho (z - z_prev) = (3, 9), so r_pri = sqrt(10 / 2) and r_dual =
    sqrt(90 / 2); iteration 2, x - z = (-21/16, 7/16) and rho (z - z_prev) =
    (9/16, 27/16), so r_pri = sqrt(490 / 512) and r_dual = sqrt(810 / 512).
    Without rho in the dual residual it would be sqrt(9) after iteration 1."""
    g = OracleGraph()
    g.add_variables(1, 1)
    g.add_factors(inputs.MPC_QUAD, [[0]], [[1.0]])
    g.add_factors(inputs.FIX, [[0]], [[4.0]])
    g.finalize(np.array([1.0, 3.0]), np.array([0.5, 0.5]))
    g.init(np.array([0.0]))
    want = [
        dict(x=[0.0, 4.0], m=[0.0, 4.0], z=[3.0], u=[-1.5, 0.5], n=[4.5, 2.5], r=(10 / 2, 90 / 2)),
        dict(x=[2.25, 4.0], m=[0.75, 4.5], z=[57 / 16], u=[-69 / 32, 23 / 32], n=[183 / 32, 91 / 32],
             r=(490 / 512, 810 / 512)),
    ]
    for w in want:
        r = g.iterate(1)
        np.testing.assert_allclose([r["r_pri"], r["r_dual"]], np.sqrt(w["r"]), rtol=1e-15)
        assert list(g.edge(EDGE_X)) == w["x"]
        assert list(g.edge(EDGE_M)) == w["m"]
        assert list(g.z()) == w["z"]
        assert list(g.edge(EDGE_U)) == w["u"]
        assert list(g.edge(EDGE_N)) == w["n"]
    # the fixed point does not depend on rho or alpha: z -> 4, and the
    # quadratic edge's x -> 4 as well (its u carries the cost's gradient)
    g.iterate(2000)
    np.testing.assert_allclose(g.z(), [4.0], rtol=1e-12)
    np.testing.assert_allclose(g.edge(EDGE_X), [4.0, 4.0], rtol=1e-9)
    # at the fixed point the cost edge has x = rho n / (q + rho) = z, so
    # u_1 = z - n = -q z / rho_1 = -4; with one alpha and u0 = 0 the sum
    # rho_1 u_1 + rho_2 u_2 stays 0 (next test)
    u = g.edge(EDGE_U)
    np.testing.assert_allclose(u[0], -4.0, rtol=1e-9)
    np.testing.assert_allclose(1.0 * u[0] + 3.0 * u[1], 0.0, atol=1e-9)


def test_weighted_dual_sum_decays_by_one_minus_alpha():
    """With one alpha on every edge of a variable, sum_e rho_e u_e after an
    iteration is (1 - alpha) times its value before (the z-update makes the
    rho-weighted mean of x + u equal z); with u0 = 0 it stays 0.  Checked
    on a three-factor scalar graph with unequal rho and alpha = 0.3."""
    g = OracleGraph()
    g.add_variables(1, 1)
    g.add_factors(inputs.MPC_QUAD, [[0]], [[2.0]])
    g.add_factors(inputs.PACK_RADIUS_LIN, [[0]], [[0.7]])
    g.add_factors(inputs.FIX, [[0]], [[-1.25]])
    rho = np.array([0.5, 2.0, 1.5])
    g.finalize(rho, 0.3)
    u0 = np.array([0.4, -0.1, 0.2])
    g.init(np.array([0.25]), u0)
    s = float(rho @ u0)
    for _ in range(5):
        g.iterate(1)
        s *= 0.7
        np.testing.assert_allclose(float(rho @ g.edge(EDGE_U)), s, rtol=1e-12, atol=1e-15)
