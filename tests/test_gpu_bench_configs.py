"""GPU parity at the benchmarked configurations, at their full length and in
the launch configuration the benchmark times, through the C-ABI:

  * circle packing N = 1000 (Sec. V-A; 3,007,000 scalar edges, linear
    radius reward of weight 1), 2000 iterations in one call:
      - FP32 through the disk-tile kernel: objective -sum r against the FP64
        oracle after the same 2000 iterations, 1e-4 relative;
      - FP64 in the canonical z-order: z and every edge message bit-equal to
        the oracle's;
  * the linear SVM 100,000 x 64 (Sec. V-C, hinge form) through the hinge
    bank, FP32, run to RMS residual 1e-4 checked every 10 iterations: the
    primal objective within 1e-4 relative of the oracle's under the same
    stop rule.

The oracle runs take about a minute of one host core in all."""
import numpy as np
import pytest

from oracle import from_problem as oracle_from_problem
from oracle.oracle import EDGE_X, EDGE_M, EDGE_U, EDGE_N
from paper_1603_02526_gb300 import inputs, _lib
from paper_1603_02526_gb300.graph import graph_from_problem
from tests.helpers import packing_objective

pytestmark = pytest.mark.gpu

N_DISKS = 1000
ITERS = 2000


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def packing():
    p = inputs.packing_problem(N_DISKS, seed=1000)
    o = oracle_from_problem(p)
    ro = o.iterate(ITERS, check_every=ITERS)
    assert ro["iters"] == ITERS
    state = dict(z=o.z(), x=o.edge(EDGE_X), m=o.edge(EDGE_M), u=o.edge(EDGE_U), n=o.edge(EDGE_N),
                 r_pri=ro["r_pri"], r_dual=ro["r_dual"])
    return p, state


def _violations(z, N):
    """Largest pairwise overlap r_i + r_j - |c_i - c_j| and largest wall
    violation r - Q.(c - V) (brute force, O(N^2))."""
    c = np.stack([z[0::3], z[1::3]], 1)
    r = z[2::3]
    iu = np.triu_indices(N, 1)
    d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))[iu]
    ov = float((r[iu[0]] + r[iu[1]] - d).max())
    Q, V = inputs.triangle_walls()
    wall = float((r[:, None] - np.einsum("sk,isk->is", Q, c[:, None, :] - V[None])).max())
    return ov, wall


def test_packing_n1000_f32_tile_2000_iterations_objective(packing):
    """The headline solve: FP32 messages, disk-tile kernel, one call of 2000
    iterations (residuals checked only at the end, as timed).  The objective
    -sum r must be within 1e-4 relative of the oracle's after the same 2000
    iterations from the same start."""
    p, o = packing
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_STORE_M: 0})
    assert g.fga_launch_info()["zorder"] == 2
    r = g.fga_iterate(ITERS, check_every=ITERS)
    assert r["iters"] == ITERS and r["status"] == 0
    z = g.fga_read_z()
    fg, fo = packing_objective(z), packing_objective(o["z"])
    ovg, wg = _violations(z, N_DISKS)
    ovo, wo = _violations(o["z"], N_DISKS)
    S = float(np.abs(o["z"]).max())
    print("N=1000 FP32 tile, 2000 iterations: objective %.9f (oracle %.9f), rel gap %.3e; "
          "max overlap %.3e (oracle %.3e), max wall violation %.3e (oracle %.3e); max |dz| %.3e S; "
          "r_pri %.4e / %.4e, r_dual %.4e / %.4e"
          % (fg, fo, abs(fg - fo) / abs(fo), ovg, ovo, wg, wo, np.abs(z - o["z"]).max() / S,
             r["r_pri"], o["r_pri"], r["r_dual"], o["r_dual"]))
    assert abs(fg - fo) <= 1e-4 * abs(fo)


def test_packing_n1000_f64_canonical_2000_iterations_bit_exact(packing):
    """FP64, canonical z-order (the order the FP64 benchmark times): after
    2000 iterations z and every edge message equal the oracle's bit for
    bit."""
    p, o = packing
    g = graph_from_problem(p, "f64")
    assert g.fga_launch_info()["zorder"] == 0
    r = g.fga_iterate(ITERS, check_every=ITERS)
    assert r["iters"] == ITERS
    assert np.array_equal(g.fga_read_z(), o["z"])
    for w, name in ((_lib.FGA_EDGE_X, "x"), (_lib.FGA_EDGE_M, "m"), (_lib.FGA_EDGE_U, "u"),
                    (_lib.FGA_EDGE_N, "n")):
        got = g.fga_read_edge_state(w)
        assert np.array_equal(got, o[name]), "%s: %d messages differ, max %.3e" % (
            name, int(np.count_nonzero(got != o[name])), float(np.abs(got - o[name]).max()))
    # the residual sums are FP64 in another order than the oracle's loop
    np.testing.assert_allclose([r["r_pri"], r["r_dual"]], [o["r_pri"], o["r_dual"]], rtol=1e-12)


def _svm_primal(z, p):
    X, y, lam, c = p.meta["X"], p.meta["y"], p.meta["lam"], p.meta["c"]
    w, b = z[:-1], z[-1]
    return float(c * np.maximum(0.0, 1.0 - y * (X @ w + b)).sum() + 0.5 * lam * w @ w)


def test_svm_100k_hinge_bank_to_tolerance_objective():
    """The SVM as benchmarked: 100,000 points in d = 64, FP32 hinge bank, run
    to RMS residual 1e-4 checked every 10 iterations.  The oracle runs the
    same stop rule; primal objectives within 1e-4 relative."""
    p = inputs.svm_problem(100000, 64, seed=3000)
    g = graph_from_problem(p, "f32")
    assert g.fga_launch_info()["zorder"] == 3
    rg = g.fga_iterate(50000, 1e-4, 1e-4, check_every=10)
    o = oracle_from_problem(p)
    ro = o.iterate(50000, 1e-4, 1e-4, check_every=10)
    assert rg["status"] == 0 and ro["status"] == 0, (rg, ro)
    fg, fo = _svm_primal(g.fga_read_z(), p), _svm_primal(o.z(), p)
    print("SVM 100k x 64 hinge bank: %d iterations (oracle %d), objective %.9g (oracle %.9g), rel gap %.3e"
          % (rg["iters"], ro["iters"], fg, fo, abs(fg - fo) / abs(fo)))
    assert abs(fg - fo) <= 1e-4 * abs(fo)
