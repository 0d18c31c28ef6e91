"""Pins for the oracle's proximal operators (Eq. PO; Appendices A-C).

Each operator is checked against something other than itself: a numerical
minimiser of the defining problem argmin_s h(s) + sum rho_k/2 (s_k - n_k)^2
(SciPy's SLSQP, multi-start for the non-convex disk pair), library
projections (null space / KKT solve) and closed forms.  A dropped term, a
wrong sign or a transposed operand in any oracle formula fails one of them.
"""
import numpy as np
import pytest
from scipy.linalg import null_space
from scipy.optimize import minimize

from oracle import (oracle_prox, T_PACK_PAIR, T_PACK_WALL, T_PACK_RADIUS_LIN,
                    T_PACK_RADIUS_QUAD, T_SVM_HINGE, T_SVM_L2, T_MPC_DYN, T_MPC_QUAD,
                    T_MPC_BOX, T_FIX, T_SVM_MARGIN, T_SVM_SLACK, T_EQUAL)


def _quad(s, n, rho):
    return 0.5 * np.sum(rho * (s - n) ** 2)


def _pair_constraint(v):
    c1, r1, c2, r2 = v[0:2], v[2], v[3:5], v[5]
    return np.linalg.norm(c1 - c2) - r1 - r2


def _best_constrained(n, rho, cons, starts):
    best = None
    for s0 in starts:
        res = minimize(lambda s: _quad(s, n, rho), s0, jac=lambda s: rho * (s - n),
                       constraints=cons, method="SLSQP",
                       options=dict(ftol=1e-15, maxiter=500))
        ok = all(c["fun"](res.x) >= -1e-9 for c in cons)
        if ok and (best is None or res.fun < best.fun):
            best = res
    return best


@pytest.mark.parametrize("seed", range(12))
def test_pack_pair_matches_bruteforce(seed):
    """Appendix A no-collision operator vs a multi-start constrained minimiser
    (random overlapping inputs, random per-disk rho)."""
    rng = np.random.default_rng(seed)
    n = np.concatenate([rng.random(2), [0.3 + 0.3 * rng.random()],
                        rng.random(2), [0.3 + 0.3 * rng.random()]])
    r1, r2 = rng.uniform(0.5, 3.0, 2)
    rho = np.array([r1, r1, r1, r2, r2, r2]) if seed % 2 else rng.uniform(0.5, 3.0, 6)
    rho[1] = rho[0]
    rho[4] = rho[3]
    x = oracle_prox(T_PACK_PAIR, [2, 1, 2, 1], None, rho, n)
    assert _pair_constraint(x) >= -1e-12
    cons = [dict(type="ineq", fun=_pair_constraint)]
    starts = [n + 0.3 * rng.standard_normal(6) for _ in range(12)] + [x]
    best = _best_constrained(n, rho, cons, starts)
    assert best is not None
    assert _quad(x, n, rho) <= best.fun + 1e-9
    np.testing.assert_allclose(x, best.x, atol=2e-5)


def test_pack_pair_identity_when_feasible():
    n = np.array([0.0, 0.0, 0.2, 1.0, 0.0, 0.3])
    x = oracle_prox(T_PACK_PAIR, [2, 1, 2, 1], None, np.ones(6), n)
    assert np.array_equal(x, n)


def test_pack_pair_radii_shrink_and_equal_rho_closed_form():
    """Equal rho: each component moves by D/4 with the radii decreasing
    (reading of the printed radius sign)."""
    n = np.array([0.0, 0.0, 0.5, 0.6, 0.0, 0.5])
    x = oracle_prox(T_PACK_PAIR, [2, 1, 2, 1], None, np.ones(6), n)
    D = 0.5 + 0.5 - 0.6
    np.testing.assert_allclose(x, [-D / 4, 0, 0.5 - D / 4, 0.6 + D / 4, 0, 0.5 - D / 4], atol=1e-15)


def test_pack_pair_coincident_centres():
    n = np.array([0.3, 0.4, 0.1, 0.3, 0.4, 0.1])
    x = oracle_prox(T_PACK_PAIR, [2, 1, 2, 1], None, np.ones(6), n)
    assert _pair_constraint(x) >= -1e-12
    assert x[0] < n[0] and x[3] > n[3]      # nhat = (1, 0)


@pytest.mark.parametrize("seed", range(10))
def test_pack_wall_matches_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    ang = rng.uniform(0, 2 * np.pi)
    scale = 1.0 if seed % 2 == 0 else rng.uniform(0.5, 2.0)   # non-unit normal too
    Q = scale * np.array([np.cos(ang), np.sin(ang)])
    V = rng.standard_normal(2)
    n = rng.standard_normal(3)
    rc, rr = rng.uniform(0.5, 3.0, 2)
    rho = np.array([rc, rc, rr])
    p = np.concatenate([Q, V])
    x = oracle_prox(T_PACK_WALL, [2, 1], p, rho, n)
    g = lambda v: Q @ (v[:2] - V) - v[2]
    assert g(x) >= -1e-12
    best = _best_constrained(n, rho, [dict(type="ineq", fun=g)], [n, x, np.zeros(3)])
    np.testing.assert_allclose(x, best.x, atol=1e-6)
    if g(n) >= 0:
        assert np.array_equal(x, n)


def test_pack_wall_printed_equal_rho_form():
    """Unit Q, equal rho: (c, r) = n + E(-Q, 1), E = min(0, (Q.(n_c - V) - n_r)/2)."""
    Q = np.array([0.0, 1.0]); V = np.zeros(2)
    n = np.array([0.3, 0.1, 0.4])
    x = oracle_prox(T_PACK_WALL, [2, 1], np.concatenate([Q, V]), np.ones(3), n)
    E = min(0.0, 0.5 * (Q @ (n[:2] - V) - n[2]))
    np.testing.assert_allclose(x, n + E * np.array([-Q[0], -Q[1], 1.0]), atol=1e-15)


@pytest.mark.parametrize("rho", [0.5, 1.0, 3.0])
def test_radius_rewards(rho):
    n = np.array([0.37])
    w = 0.25
    x = oracle_prox(T_PACK_RADIUS_LIN, [1], [w], [rho], n)
    res = minimize(lambda s: -w * s[0] + 0.5 * rho * (s[0] - n[0]) ** 2, n, method="BFGS",
                   options=dict(gtol=1e-12))
    np.testing.assert_allclose(x, res.x, atol=1e-7)
    if rho > 1.0:
        x2 = oracle_prox(T_PACK_RADIUS_QUAD, [1], None, [rho], n)
        res = minimize(lambda s: -0.5 * s[0] ** 2 + 0.5 * rho * (s[0] - n[0]) ** 2, n,
                       method="BFGS", options=dict(gtol=1e-12))
        np.testing.assert_allclose(x2, res.x, atol=1e-7)
    else:
        with pytest.raises(ValueError):
            oracle_prox(T_PACK_RADIUS_QUAD, [1], None, [rho], n)


@pytest.mark.parametrize("seed", range(10))
def test_svm_hinge_matches_bruteforce(seed):
    rng = np.random.default_rng(200 + seed)
    D = 3
    xi = rng.standard_normal(D)
    y = 1.0 if seed % 2 else -1.0
    c = [0.05, 0.3, 1.0, 10.0][seed % 4]
    n = rng.standard_normal(D + 1) * 0.5
    rho = rng.uniform(0.5, 2.0, D + 1)
    x = oracle_prox(T_SVM_HINGE, [D, 1], np.concatenate([xi, [y, c]]), rho, n)

    # epigraph form: min c t + sum rho/2 (v - n)^2, t >= 0, t >= 1 - y (w.x + b)
    def obj(v):
        return c * v[-1] + _quad(v[:-1], n, rho)
    cons = [dict(type="ineq", fun=lambda v: v[-1]),
            dict(type="ineq", fun=lambda v: v[-1] - (1 - y * (v[:D] @ xi + v[D])))]
    best = None
    for s0 in [np.concatenate([n, [2.0]]), np.concatenate([x, [0.5]])]:
        r = minimize(obj, s0, constraints=cons, method="SLSQP", options=dict(ftol=1e-15, maxiter=1000))
        if best is None or r.fun < best.fun:
            best = r
    np.testing.assert_allclose(x, best.x[:-1], atol=1e-6)


def test_svm_hinge_inactive_is_identity():
    xi = np.array([1.0, 2.0]); n = np.array([1.0, 1.0, 0.0])
    x = oracle_prox(T_SVM_HINGE, [2, 1], np.concatenate([xi, [1.0, 1.0]]), np.ones(3), n)
    assert np.array_equal(x, n)


@pytest.mark.parametrize("seed", range(10))
def test_svm_margin_matches_bruteforce(seed):
    """Appendix C one-point margin: the projection of n onto
    {y (w.x + b) >= 1 - xi} in the rho-weighted norm, against SLSQP on the
    defining problem (per-edge rho, both labels, active and inactive)."""
    rng = np.random.default_rng(300 + seed)
    D = 3
    xv = rng.standard_normal(D)
    y = 1.0 if seed % 2 else -1.0
    n = rng.standard_normal(D + 2) * (0.3 if seed < 7 else 2.0)
    rho = rng.uniform(0.5, 2.0, D + 2)
    x = oracle_prox(T_SVM_MARGIN, [D, 1, 1], np.concatenate([xv, [y]]), rho, n)
    cons = [dict(type="ineq", fun=lambda v: y * (v[:D] @ xv + v[D]) - 1.0 + v[D + 1])]
    best = _best_constrained(n, rho, cons, [n, n + 1.0, x])
    np.testing.assert_allclose(x, best.x, atol=1e-6)
    assert y * (x[:D] @ xv + x[D]) - 1.0 + x[D + 1] >= -1e-12


def test_svm_margin_inactive_is_identity():
    n = np.array([1.0, 1.0, 0.5, 0.0])      # y (w.x + b) = 1.5 + 0.5 >= 1
    x = oracle_prox(T_SVM_MARGIN, [2, 1, 1], [1.0, 0.5, 1.0], np.ones(4), n)
    assert np.array_equal(x, n)


@pytest.mark.parametrize("lam", [0.0, 0.3, 2.0])
def test_svm_slack_matches_bruteforce(lam):
    """Appendix C minimal error: argmin lam xi + rho/2 (xi - n)^2, xi >= 0,
    against a bounded scalar minimiser per component."""
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(17)
    n = rng.standard_normal(6)
    rho = rng.uniform(0.5, 2.0, 6)
    x = oracle_prox(T_SVM_SLACK, [6], [lam], rho, n)
    for j in range(6):
        r = minimize_scalar(lambda t: lam * t + 0.5 * rho[j] * (t - n[j]) ** 2, bounds=(0.0, 10.0),
                            method="bounded", options=dict(xatol=1e-12))
        assert abs(x[j] - r.x) <= 1e-8
    assert np.all(x >= 0.0)


def test_equal_matches_constrained_minimiser():
    """Appendix C equality: argmin sum rho/2 (v - n)^2 subject to v1 = v2, as
    a projection onto the null space of [I  -I] in the rho-weighted norm
    (SciPy null space, weighted least squares)."""
    rng = np.random.default_rng(23)
    d = 4
    n = rng.standard_normal(2 * d)
    rho = rng.uniform(0.5, 2.0, 2 * d)
    x = oracle_prox(T_EQUAL, [d, d], None, rho, n)
    N = null_space(np.hstack([np.eye(d), -np.eye(d)]))
    Wh = np.diag(np.sqrt(rho))
    c, *_ = np.linalg.lstsq(Wh @ N, Wh @ n, rcond=None)
    np.testing.assert_allclose(x, N @ c, atol=1e-12)


@pytest.mark.parametrize("lam", [1e-3, 1.0, 5.0])
def test_svm_l2_and_quad(lam):
    rng = np.random.default_rng(7)
    n = rng.standard_normal(4)
    rho = rng.uniform(0.5, 2, 4)
    x = oracle_prox(T_SVM_L2, [4], [lam], rho, n)
    res = minimize(lambda s: 0.5 * lam * s @ s + _quad(s, n, rho), n, method="BFGS", options=dict(gtol=1e-13))
    np.testing.assert_allclose(x, res.x, atol=1e-7)
    q = rng.uniform(0.1, 10, 4)
    x = oracle_prox(T_MPC_QUAD, [3, 1], q, rho, n)
    res = minimize(lambda s: 0.5 * np.sum(q * s * s) + _quad(s, n, rho), n, method="BFGS",
                   options=dict(gtol=1e-13))
    np.testing.assert_allclose(x, res.x, atol=1e-7)


def test_box_and_fix():
    n = np.array([-3.0, -0.5, 0.2, 4.0])
    x = oracle_prox(T_MPC_BOX, [4], [-1.0, 1.0], np.ones(4), n)
    np.testing.assert_array_equal(x, [-1.0, -0.5, 0.2, 1.0])
    v = np.array([0.1, 0.2, 0.3])
    x = oracle_prox(T_FIX, [3], v, np.ones(3), np.zeros(3))
    np.testing.assert_array_equal(x, v)


@pytest.mark.parametrize("uniform", [True, False])
def test_mpc_dyn_projection(uniform):
    """Appendix B dynamics operator = rho-weighted projection onto
    {x' = A x + B u}: compared with a null-space projection (uniform rho) and
    a KKT solve (weighted), and checked for feasibility."""
    rng = np.random.default_rng(11)
    nx, nu = 4, 2
    A = rng.standard_normal((nx, nx)) * 0.4
    B = rng.standard_normal((nx, nu))
    n = rng.standard_normal(2 * nx + nu)
    rho = np.full(2 * nx + nu, 1.7) if uniform else rng.uniform(0.5, 3.0, 2 * nx + nu)
    x = oracle_prox(T_MPC_DYN, [nx, nu, nx], np.concatenate([A.ravel(), B.ravel()]), rho, n)
    M = np.concatenate([A, B, -np.eye(nx)], axis=1)
    np.testing.assert_allclose(M @ x, 0.0, atol=1e-12)
    if uniform:
        N_ = null_space(M)
        np.testing.assert_allclose(x, N_ @ (N_.T @ n), atol=1e-12)
    else:
        k = 2 * nx + nu
        K = np.zeros((k + nx, k + nx))
        K[:k, :k] = np.diag(rho)
        K[:k, k:] = M.T
        K[k:, :k] = M
        sol = np.linalg.solve(K, np.concatenate([rho * n, np.zeros(nx)]))
        np.testing.assert_allclose(x, sol[:k], atol=1e-12)
