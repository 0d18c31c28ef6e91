"""Pins for user-supplied proximal operators in the oracle.

The paper's addNode takes each factor's proximal operator as a function
pointer (Sec. III); the oracle's og_register_prox does the same, and its
Algorithm 2 then calls that pointer in the x-update.  What the pins fix:

  * the operator receives its factor's messages n, weights rho and
    parameters in creation order (the factor's variables in the order given,
    each variable's components in order), checked on the first call;
  * user operators that restate built-in types (cost, box) give the built-in
    types' iterates bit for bit, with per-edge rho and alpha != 1;
  * a consensus lasso built from user operators (shifted quadratics and an
    l1 term) converges to its closed-form minimiser, a soft-threshold of the
    weighted mean, whatever the per-edge rho;
  * registration rejects a factor whose arity or parameter count differs.

The operators below are used by the GPU parity tests as well (the GPU side
compiles its own CUDA versions of them).
"""
import numpy as np
import pytest

from oracle import OracleGraph
from oracle.oracle import EDGE_U, EDGE_X, T_EQUAL, T_MPC_BOX, T_MPC_QUAD, T_USER0


# ---------------------------------------------------------------------------
# operators, x = argmin_s f(s) + sum_k rho_k / 2 (s_k - n_k)^2 (Eq. PO)
# ---------------------------------------------------------------------------
def prox_shifted_quad(n, rho, p):
    """f(v) = 1/2 sum_k q_k (v_k - a_k)^2, params (a_1..a_d, q_1..q_d):
    setting the gradient q (x - a) + rho (x - n) to zero."""
    d = n.size
    a, q = p[:d], p[d:]
    return (q * a + rho * n) / (q + rho)


def prox_l1(n, rho, p):
    """f(v) = lam sum_k |v_k|, params (lam): soft threshold at lam / rho_k."""
    t = p[0] / rho
    return np.where(n > t, n - t, np.where(n < -t, n + t, 0.0))


def prox_quad0(n, rho, p):
    """f(v) = 1/2 sum_k q_k v_k^2 (the built-in cost type, restated)."""
    return (rho * n) / (p + rho)


def prox_box(n, rho, p):
    """indicator of lo <= v <= hi (the built-in box type, restated)."""
    return np.minimum(np.maximum(n, p[0]), p[1])


def lasso_data(d, N, seed):
    """min_w sum_i 1/2 sum_k q_ik (w_k - a_ik)^2 + lam |w|_1 on one variable
    w of dimension d: the centres a and weights q of N shifted quadratics,
    and lam."""
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, 1.0, (N, d))
    q = rng.uniform(0.5, 2.0, (N, d))
    lam = 0.8
    return a, q, lam


def lasso_minimiser(a, q, lam):
    """Per coordinate: N (w - weighted mean) Q + lam sign(w) = 0, i.e. the
    weighted mean soft-thresholded at lam / Q, Q = sum_i q_ik."""
    Q = q.sum(axis=0)
    mean = (q * a).sum(axis=0) / Q
    return np.sign(mean) * np.maximum(np.abs(mean) - lam / Q, 0.0)


def build_lasso_oracle(a, q, lam, rho):
    N, d = a.shape
    g = OracleGraph()
    g.add_variables(1, d)
    tq = g.register_prox(prox_shifted_quad, d, 2 * d)
    tl = g.register_prox(prox_l1, d, 1)
    g.add_factors(tq, np.zeros((N, 1), dtype=np.int64), np.concatenate([a, q], axis=1))
    g.add_factors(tl, np.zeros((1, 1), dtype=np.int64), [[lam]])
    g.finalize(rho, 1.0)
    return g


# ---------------------------------------------------------------------------
def test_operator_sees_its_messages_in_creation_order():
    calls = []

    def record(n, rho, p):
        calls.append((n.copy(), rho.copy(), p.copy()))
        return n

    g = OracleGraph()
    g.add_variables(1, 2)   # v0 = (z0, z1)
    g.add_variables(1, 1)   # v1 = z2
    t = g.register_prox(record, 3, 2)
    assert t == T_USER0
    g.add_factors(t, [[0, 1], ], [[7.0, 8.0]])
    g.add_factors(t, [[1, 0], ], [[9.0, 10.0]])
    rho = np.array([1.5, 2.5, 3.5, 4.5, 5.5, 6.5])
    g.finalize(rho, 1.0)
    g.init(np.array([1.0, 2.0, 3.0]))
    g.iterate(1)
    assert len(calls) == 2
    np.testing.assert_array_equal(calls[0][0], [1.0, 2.0, 3.0])
    np.testing.assert_array_equal(calls[0][1], [1.5, 2.5, 3.5])
    np.testing.assert_array_equal(calls[0][2], [7.0, 8.0])
    np.testing.assert_array_equal(calls[1][0], [3.0, 1.0, 2.0])
    np.testing.assert_array_equal(calls[1][1], [4.5, 5.5, 6.5])
    np.testing.assert_array_equal(calls[1][2], [9.0, 10.0])


def cost_box_chain(T, d, seed, user):
    """A chain of T blocks of dimension d: a quadratic cost and a box on
    each block, an equality between neighbours; the cost and the box either
    built in or as user types that restate them."""
    rng = np.random.default_rng(seed)
    g = OracleGraph()
    g.add_variables(T, d)
    q = rng.uniform(0.1, 10.0, (T, d))
    box = np.array([-0.4, 0.6])
    if user:
        tq = g.register_prox(prox_quad0, d, d)
        tb = g.register_prox(prox_box, d, 2)
    else:
        tq, tb = T_MPC_QUAD, T_MPC_BOX
    ids = np.arange(T)[:, None]
    g.add_factors(tq, ids, q)
    g.add_factors(tb, ids, box)
    g.add_factors(T_EQUAL, np.stack([np.arange(T - 1), np.arange(1, T)], axis=1))
    E = g.num_edges
    rho = rng.uniform(0.5, 2.0, E)
    alpha = rng.uniform(0.5, 1.0, E)
    g.finalize(rho, alpha)
    g.init(rng.normal(0.0, 1.0, T * d))
    return g


def test_user_operators_restating_builtins_match_bit_for_bit():
    gb = cost_box_chain(8, 3, 7, user=False)
    gu = cost_box_chain(8, 3, 7, user=True)
    rb = gb.iterate(40, check_every=5)
    ru = gu.iterate(40, check_every=5)
    assert rb == ru
    np.testing.assert_array_equal(gu.z(), gb.z())
    np.testing.assert_array_equal(gu.edge(EDGE_X), gb.edge(EDGE_X))
    np.testing.assert_array_equal(gu.edge(EDGE_U), gb.edge(EDGE_U))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_user_lasso_converges_to_the_closed_form(seed):
    a, q, lam = lasso_data(4, 6, seed)
    rng = np.random.default_rng(100 + seed)
    E = a.shape[0] * a.shape[1] + a.shape[1]
    g = build_lasso_oracle(a, q, lam, rng.uniform(0.5, 2.0, E))
    g.init()
    r = g.iterate(20000, tol_pri=1e-13, tol_dual=1e-13)
    assert r["status"] == 0 and r["iters"] < 20000, r
    w = lasso_minimiser(a, q, lam)
    np.testing.assert_allclose(g.z(), w, rtol=0, atol=1e-10)
    # seeds 1 and 3 threshold a coordinate to zero (both branches of the l1
    # operator decide the minimiser); seed 2 thresholds none
    assert bool(np.any(w == 0.0)) == (seed != 2)


def test_registration_rejects_other_shapes():
    g = OracleGraph()
    g.add_variables(2, 2)
    t = g.register_prox(prox_box, 2, 2)
    with pytest.raises(ValueError):
        g.add_factors(t, [[0, 1]], [[0.0, 1.0]])   # arity 4, registered 2
    with pytest.raises(ValueError):
        g.add_factors(t, [[0]], [[0.0, 1.0, 2.0]])   # 3 parameters, registered 2
    with pytest.raises(ValueError):
        g.add_factors(T_USER0 + 1, [[0]], [[0.0, 1.0]])   # not registered
    g.add_factors(t, [[0]], [[0.0, 1.0]])
