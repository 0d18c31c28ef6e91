"""Pins for the MLP oracle: its analytic gradients against central finite
differences of its own loss (FP64, no rounding), the BF16 rounding helper
against exhaustive properties, and Adam against its closed form on a
quadratic."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo


def _net(shape, seed):
    rng = np.random.default_rng(seed)
    n_in, h1, h2, n_out = shape
    parts = [rng.standard_normal((h1, n_in)) * 0.5, rng.standard_normal(h1) * 0.1,
             rng.standard_normal((h2, h1)) * 0.3, rng.standard_normal(h2) * 0.1,
             rng.standard_normal((n_out, h2)) * 0.3, rng.standard_normal(n_out) * 0.1]
    return mo.pack(parts)


def test_gradients_match_finite_differences():
    shape = (5, 8, 8, 6)
    p = _net(shape, 0)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((7, 5))
    T = rng.standard_normal((7, 6))
    loss, g = mo.loss_and_grads(p, shape, X, T, bf16=False)
    assert loss == pytest.approx(mo.loss_only(p, shape, X, T), rel=1e-14)
    h = 1e-6
    idx = rng.choice(p.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mo.loss_only(p + e, shape, X, T) - mo.loss_only(p - e, shape, X, T)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i


def test_bf16_rounding():
    # exactly representable values are unchanged; others go to a neighbour
    vals = np.array([0.0, 1.0, -2.0, 0.5, 3.0, 1.0 + 2 ** -7, 65280.0])
    assert np.array_equal(mo.to_bf16(vals), vals)
    x = np.array([1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -8])
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1
    np.testing.assert_array_equal(mo.to_bf16(x), [1.0, 1.0 + 2 ** -7, 1.0])
    r = np.random.default_rng(2).standard_normal(10000)
    q = mo.to_bf16(r)
    assert np.all(np.abs(q - r) <= np.abs(r) * 2 ** -8 + 1e-300)


def test_adam_closed_form_first_step():
    """First Adam step moves every coordinate by lr * sign(g) (up to eps)."""
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    p1, m, v = mo.adam_step(p, np.zeros(3), np.zeros(3), g, 1, 0.01)
    np.testing.assert_allclose(p1, p - 0.01 * np.sign(g), rtol=1e-6)
