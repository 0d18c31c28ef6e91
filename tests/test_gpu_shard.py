"""GPU parity of the shard path (fga_shard_*): a graph cut into contiguous
factor slices, each slice a graph of its own, the slices' sums of rho m
exchanged between them.  Here every shard runs on the one GPU, one after
another in rank order (LocalGroup: no kernel waits on another), which
exercises the same kernels and the same hand-over as one process per GPU.

FP64 with the chain exchange keeps the serial creation-order sums, so z and
every edge message (the shards' edges concatenated in rank order) must
equal the one-GPU canonical run and the FP64 oracle bit for bit; the stop
rule must stop at the oracle's iteration.  FP32 with the gather exchange is
compared with the one-GPU fast-order run by the variables' scale."""
import numpy as np
import pytest

from oracle import from_problem as oracle_from_problem
from oracle.oracle import EDGE_X, EDGE_M, EDGE_U, EDGE_N
from paper_1603_02526_gb300 import inputs, _lib
from paper_1603_02526_gb300.graph import graph_from_problem
from paper_1603_02526_gb300.shard import LocalGroup, ShardGraph, ShardedSweep, split_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


def _sharded(p, G, precision="f64", zorder=0, exchange="chain"):
    parts, first = split_problem(p, G)
    shards = [ShardGraph(q, precision, zorder=zorder) for q in parts]
    assert sum(s.ne for s in shards) == p.num_edges
    sw = ShardedSweep(LocalGroup(shards), p.num_edges, exchange=exchange)
    sw.init()
    return sw, shards


def _edges(shards, which):
    return np.concatenate([s.read_edges(which) for s in shards])


@pytest.mark.parametrize("G", [1, 2, 3])
def test_packing_f64_chain_bit_exact(G):
    """N=20, 300 iterations checked every 7: the shards reproduce the oracle
    (and so the one-GPU canonical run) bit for bit."""
    p = inputs.packing_problem(20)
    sw, shards = _sharded(p, G)
    r = sw.iterate(300, check_every=7)
    assert r["iters"] == 300 and r["status"] == 0
    o = oracle_from_problem(p)
    ro = o.iterate(300, check_every=7)
    for s in shards:
        assert np.array_equal(s.read_z(), o.z())
    for w, ow in ((_lib.FGA_EDGE_X, EDGE_X), (_lib.FGA_EDGE_M, EDGE_M), (_lib.FGA_EDGE_U, EDGE_U),
                  (_lib.FGA_EDGE_N, EDGE_N)):
        assert np.array_equal(_edges(shards, w), o.edge(ow)), w
    np.testing.assert_allclose([r["r_pri"], r["r_dual"]], [ro["r_pri"], ro["r_dual"]], rtol=1e-12)


def test_packing_f64_chain_stop_rule_and_resume():
    """A run to tolerance stops at the oracle's iteration with the oracle's
    state; a second call continues like one unbroken oracle run."""
    p = inputs.packing_problem(3)
    p.factor_blocks[-1].params[:] = 0.1
    sw, shards = _sharded(p, 2)
    r = sw.iterate(5000, 1e-7, 1e-7, check_every=5)
    o = oracle_from_problem(p)
    ro = o.iterate(5000, 1e-7, 1e-7, check_every=5)
    assert r["status"] == 0 and r["iters"] == ro["iters"] < 5000
    assert np.array_equal(shards[0].read_z(), o.z())
    assert np.array_equal(_edges(shards, _lib.FGA_EDGE_U), o.edge(EDGE_U))
    sw.iterate(40, check_every=40)
    o.iterate(40, check_every=40)
    assert np.array_equal(shards[1].read_z(), o.z())
    assert np.array_equal(_edges(shards, _lib.FGA_EDGE_X), o.edge(EDGE_X))


def test_packing_n1000_f64_chain_two_shards():
    """The N=1000 graph (3,007,000 edges, every variable a hub of degree
    about 1000 split between the shards): 3 iterations bit-equal to the
    oracle."""
    p = inputs.packing_problem(1000)
    sw, shards = _sharded(p, 2)
    sw.iterate(3)
    o = oracle_from_problem(p)
    o.iterate(3)
    assert np.array_equal(shards[0].read_z(), o.z())
    assert np.array_equal(_edges(shards, _lib.FGA_EDGE_U), o.edge(EDGE_U))
    assert np.array_equal(_edges(shards, _lib.FGA_EDGE_X), o.edge(EDGE_X))


def test_svm_f64_chain_bit_exact():
    """Hinge factors on a shared (w, b) (the hub of Sec. V-C) cut across
    three shards: 200 iterations, bit-equal to the oracle."""
    p = inputs.svm_problem(300, 8, seed=3100)
    sw, shards = _sharded(p, 3)
    sw.iterate(200)
    o = oracle_from_problem(p)
    o.iterate(200)
    assert np.array_equal(shards[2].read_z(), o.z())
    assert np.array_equal(_edges(shards, _lib.FGA_EDGE_U), o.edge(EDGE_U))


def test_mpc_f64_chain_equals_one_gpu():
    """An MPC instance (dynamics factors through the precomputed projector)
    in two shards: bit-equal to the same graph on one GPU, and within 1e-9
    per message of the oracle (its Cholesky solves round differently)."""
    d = inputs.mpc_batch_inputs(1, seed=4100, T_fixed=20)
    p = inputs.mpc_problem(d["A"][0], d["B"][0], d["q"][0], d["r"][0], d["x0"][0], 20)
    sw, shards = _sharded(p, 2)
    sw.iterate(150, check_every=10)
    g = graph_from_problem(p, "f64")
    g.fga_iterate(150, check_every=10)
    assert np.array_equal(shards[0].read_z(), g.fga_read_z())
    assert np.array_equal(_edges(shards, _lib.FGA_EDGE_U), g.fga_read_edge_state(_lib.FGA_EDGE_U))
    o = oracle_from_problem(p)
    o.iterate(150)
    np.testing.assert_allclose(shards[0].read_z(), o.z(), rtol=1e-9, atol=1e-9 * np.abs(o.z()).max())


def test_packing_f32_gather_fast_order():
    """FP32, fast z-order, gather exchange (every shard sums its own terms,
    the sums are added in rank order): N=200 in 3 shards, 10 iterations,
    within 1e-4 of the variables' scale of the one-GPU fast-order run, and
    deterministic."""
    p = inputs.packing_problem(200)
    zs = []
    for _ in range(2):
        sw, shards = _sharded(p, 3, precision="f32", zorder=1, exchange="gather")
        sw.iterate(10)
        zs.append(shards[0].read_z())
        for s in shards[1:]:
            assert np.array_equal(s.read_z(), zs[-1])
    assert np.array_equal(zs[0], zs[1])
    g = graph_from_problem(p, "f32", options={_lib.FGA_OPT_ZORDER: 1})
    g.fga_iterate(10)
    S = float(np.abs(g.fga_read_z()).max())
    assert np.abs(zs[0] - g.fga_read_z()).max() <= 1e-4 * S


def test_shard_graph_refuses_the_one_gpu_calls():
    p = inputs.packing_problem(5)
    parts, _ = split_problem(p, 2)
    s = ShardGraph(parts[0], "f64")
    s.begin(*s.rho_chain(None, None))
    s.init()
    with pytest.raises(_lib.FgaError):
        s.g.fga_iterate(1)
    with pytest.raises(_lib.FgaError):
        s.finish()                          # nothing pending before the first z-step
