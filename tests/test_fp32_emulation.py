"""The FP32 emulation used as the yardstick of the GPU's FP32 tolerances
(tests/fp32_emulation.py) against the FP64 oracle: with its three ways of
summing z it must stay within FP32 rounding of the oracle on a small
packing, and in FP64-like conditions (tiny graph, few iterations) its
distance from the oracle must be of the order of FP32's unit roundoff."""
import numpy as np
import pytest

from oracle import from_problem
from oracle.oracle import EDGE_X, EDGE_U, EDGE_N
from paper_1603_02526_gb300 import inputs
from tests.fp32_emulation import PackingFP32


@pytest.mark.parametrize("sums", ["serial", "tree", "exact"])
def test_emulation_tracks_the_oracle(sums):
    """20 iterations of N=20: every value within 2e-4 of the variables'
    scale (the non-convex pair operator amplifies rounding by about 10^3
    over these iterations; a wrong operator or update would be off by
    O(1))."""
    p = inputs.packing_problem(20)
    e = PackingFP32(p, sums=sums)
    e.iterate(20)
    o = from_problem(p)
    o.iterate(20)
    S = float(np.abs(o.z()).max())
    assert np.abs(e.z - o.z()).max() <= 2e-4 * S
    for arr, w in ((e.x, EDGE_X), (e.u, EDGE_U), (e.n, EDGE_N)):
        assert np.abs(arr.astype(np.float64) - o.edge(w)).max() <= 2e-4 * S


@pytest.mark.parametrize("reward,rho", [("lin", 1.0), ("quad", 25.0)])
def test_one_iteration_is_fp32_rounding_of_the_oracle(reward, rho):
    """After one iteration from an FP32-representable start every value is
    a handful of roundings away from the FP64 result: within 8 ulps of
    FP32 at the variables' scale (linear reward, and the area reward at
    rho 25)."""
    p = inputs.packing_problem(20, reward=reward, rho=rho)
    p.z0 = p.z0.astype(np.float32).astype(np.float64)
    e = PackingFP32(p, sums="exact")
    e.iterate(1)
    o = from_problem(p)
    o.iterate(1)
    S = float(np.abs(o.z()).max())
    tol = 8 * np.finfo(np.float32).eps * S
    assert np.abs(e.z - o.z()).max() <= tol
    for arr, w in ((e.x, EDGE_X), (e.u, EDGE_U), (e.n, EDGE_N)):
        assert np.abs(arr.astype(np.float64) - o.edge(w)).max() <= tol


def test_area_reward_emulation_tracks_the_oracle():
    """The area reward (rho 25), 20 iterations of N = 20: within 2e-4 of the
    variables' scale, as for the linear reward; the reward's edges follow
    x = rho n / (rho - 1) (a wrong factor, e.g. n + 1 / (rho - 1), or the
    linear reward's operator, is off by far more)."""
    p = inputs.packing_problem(20, reward="quad", rho=25.0)
    e = PackingFP32(p, sums="exact")
    e.iterate(20)
    o = from_problem(p)
    o.iterate(20)
    S = float(np.abs(o.z()).max())
    assert np.abs(e.z - o.z()).max() <= 2e-4 * S
    for arr, w in ((e.x, EDGE_X), (e.u, EDGE_U), (e.n, EDGE_N)):
        assert np.abs(arr.astype(np.float64) - o.edge(w)).max() <= 2e-4 * S
