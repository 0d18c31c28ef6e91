"""Shared test helpers (comparison rules, problem loaders)."""
import numpy as np

from oracle import from_problem as oracle_from_problem
from oracle.oracle import EDGE_X, EDGE_M, EDGE_U, EDGE_N


def rel_close_floor(got, want, rtol):
    """Per-message rule for FP64 parity: |g - o| <= rtol * max(|o|, 1e-3 |o|_inf)
    (relative error with a floor at a thousandth of the array's scale)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.max(np.abs(want)) if want.size else 0.0
    bound = rtol * np.maximum(np.abs(want), 1e-3 * scale)
    err = np.abs(got - want)
    bad = np.nonzero(err > bound)[0]
    return bad.size == 0, (float(err.max()) if err.size else 0.0), bad[:10]


def assert_messages_match(gpu_graph, oracle_graph, rtol, which=("x", "m", "u", "n", "z")):
    from paper_1603_02526_gb300._lib import FGA_EDGE_X, FGA_EDGE_M, FGA_EDGE_U, FGA_EDGE_N
    pairs = dict(x=(FGA_EDGE_X, EDGE_X), m=(FGA_EDGE_M, EDGE_M), u=(FGA_EDGE_U, EDGE_U), n=(FGA_EDGE_N, EDGE_N))
    for name in which:
        if name == "z":
            g, o = gpu_graph.fga_read_z(), oracle_graph.z()
        else:
            a, b = pairs[name]
            g, o = gpu_graph.fga_read_edge_state(a), oracle_graph.edge(b)
        ok, emax, bad = rel_close_floor(g, o, rtol)
        assert ok, "%s differs from the oracle: max abs err %.3e at %s" % (name, emax, bad)


def packing_objective(z, w=1.0):
    """Linear radius reward: f = -w sum r (constraints reported separately)."""
    return -w * float(np.sum(z[2::3]))


def assert_messages_close_scaled(gpu_graph, oracle_graph, rtol, which=("x", "m", "u", "n", "z")):
    """FP32 rule: |g - o| <= rtol * S for every message, S = the largest
    |z| of the oracle (the variables' scale).  FP32 rounding errors in
    u = u + alpha (x - z) and n = z - u are a few ulps of |x| ~ |z|, not of
    the (possibly tiny) message itself."""
    from paper_1603_02526_gb300._lib import FGA_EDGE_X, FGA_EDGE_M, FGA_EDGE_U, FGA_EDGE_N
    pairs = dict(x=(FGA_EDGE_X, EDGE_X), m=(FGA_EDGE_M, EDGE_M), u=(FGA_EDGE_U, EDGE_U), n=(FGA_EDGE_N, EDGE_N))
    S = float(np.max(np.abs(oracle_graph.z())))
    for name in which:
        if name == "z":
            g, o = gpu_graph.fga_read_z(), oracle_graph.z()
        else:
            a, b = pairs[name]
            g, o = gpu_graph.fga_read_edge_state(a), oracle_graph.edge(b)
        err = float(np.max(np.abs(g - o))) if o.size else 0.0
        assert err <= rtol * S, "%s: max abs err %.3e > %.1e * %.3g" % (name, err, rtol, S)
