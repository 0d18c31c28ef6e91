"""The synthetic workloads (paper_1603_02526_gb300/inputs.py) against the
recipe they are stated to follow: the shapes, counts and value
distributions of the paper's packing (Sec. V-A), MPC (Sec. V-B) and SVM
(Sec. V-C) workloads.  The counts are checked against the paper's own formulas or against the graph
written out by definition; the distributions by their moments on samples
large enough that the bounds are many standard errors wide."""
import numpy as np
import pytest

from paper_1603_02526_gb300 import inputs


def _edges_by_definition(p):
    """Scalar edges: per factor, the dimensions of the variables it touches."""
    dims = p.var_dims()
    return sum(int(dims[b.var_ids].sum()) for b in p.factor_blocks)


@pytest.mark.parametrize("N", [3, 20, 1000])
def test_packing_counts_are_the_papers(N):
    """Sec. V-A counts edges between factors and variable nodes (a centre
    is one node): 2N^2 - N + 2NS of them, with 2N variable nodes and
    N(N - 1)/2 + N + NS factors; the scalar edges are 3N^2 + 7N."""
    p = inputs.packing_problem(N)
    c = inputs.packing_counts(N)
    assert sum(b.var_ids.size for b in p.factor_blocks) == c["edges"]
    assert p.num_factors == c["factors"] and p.num_vars == c["var_nodes"]
    assert p.num_edges == _edges_by_definition(p) == 3 * N * N + 7 * N
    if N == 1000:
        assert (p.num_edges, p.num_factors) == (3007000, 503500)


def test_packing_start_is_uniform_in_the_triangle():
    N = 40000
    c, r = inputs.packing_start(N, 1000)
    Q, V = inputs.triangle_walls()
    for s in range(3):
        assert np.all((c - V[s]) @ Q[s] >= -1e-12)          # inside every wall
    assert np.all((r >= 0.0) & (r < 0.05))
    assert abs(r.mean() - 0.025) < 0.001
    # uniform in the triangle: the centroid and the second moments of the
    # area measure (side 1: E[x] = 1/2, E[y] = sqrt(3)/6, Var x = Var y = 1/24)
    assert np.allclose(c.mean(axis=0), [0.5, np.sqrt(3) / 6], atol=0.005)
    assert np.allclose(c.var(axis=0), [1 / 24, 1 / 24], atol=0.002)
    c2, r2 = inputs.packing_start(N, 1000)
    assert np.array_equal(c, c2) and np.array_equal(r, r2)
    c3, _ = inputs.packing_start(N, 1001)
    assert not np.array_equal(c, c3)


def test_svm_data_and_graph():
    X, y = inputs.svm_data(100000, 64, 3000)
    assert X.shape == (100000, 64) and set(np.unique(y)) == {-1.0, 1.0}
    # balanced classes at +-0.5 (1, ..., 1) with 5% of the labels flipped:
    # E[y x_j] = 0.5 (1 - 2 * 0.05) = 0.45, E[x_j] = 0, unit variance around
    # the class means, so E[x_j^2] = 1.25
    assert abs(np.mean(y[:, None] * X) - 0.45) < 0.003
    assert abs(np.mean(X)) < 0.003
    assert abs(np.mean(X * X) - 1.25) < 0.005                    # 1 + 0.5^2 per component
    assert abs(np.mean(y)) <= 0.05 + 1e-12
    p = inputs.svm_problem(100000, 64, seed=3000)
    assert p.num_edges == 6500064 == _edges_by_definition(p)
    # w and b are hubs: every hinge factor touches both
    hinge = [b for b in p.factor_blocks if b.ftype == inputs.SVM_HINGE][0]
    assert hinge.var_ids.shape[0] == 100000 and np.unique(hinge.var_ids, axis=0).shape[0] == 1


@pytest.mark.parametrize("npts,d", [(100000, 64), (100000, 2), (57, 5)])
def test_svm_paper_form_counts(npts, d):
    want = {(100000, 64): 25899872, (100000, 2): 1099996}.get((npts, d))
    assert inputs.svm_paper_edges(npts, d) == npts * (4 * d + 3) - 2 * d
    if want is not None:
        assert inputs.svm_paper_edges(npts, d) == want
    if npts < 1000:
        p = inputs.svm_paper_problem(npts, d, seed=3000)
        assert p.num_edges == inputs.svm_paper_edges(npts, d) == _edges_by_definition(p)


def test_mpc_batch_recipe():
    d = inputs.mpc_batch_inputs(4096, seed=4000)
    T = d["T"]
    assert T.min() == 10 and T.max() == 50 and set(np.unique(T)) == set(range(10, 51))
    assert abs(T.mean() - 30.0) < 0.5
    A, B, q, r, x0 = d["A"], d["B"], d["q"], d["r"], d["x0"]
    assert A.shape == (4096, 12, 12) and B.shape == (4096, 12, 4)
    rad = np.array([np.max(np.abs(np.linalg.eigvals(a))) for a in A[:256]])
    np.testing.assert_allclose(rad, 0.95, rtol=1e-12)
    assert np.all((q >= 0.1) & (q <= 10.0)) and np.all((r >= 0.1) & (r <= 10.0))
    assert abs(np.mean(B * B) * 12 - 1.0) < 0.05                     # B Gaussian / sqrt(nx)
    assert abs(x0.mean()) < 0.02 and abs(x0.std() - 1.0) < 0.02
    assert d["umax"] == 1.0


def test_warm_start_sets_share_the_system_not_the_states():
    a = inputs.mpc_warmstart_inputs(1000, x0_seed=5001)
    b = inputs.mpc_warmstart_inputs(1000, x0_seed=5002)
    for k in ("A", "B", "q", "r"):
        assert np.array_equal(a[k], b[k])
    assert not np.array_equal(a["x0"], b["x0"])
    assert np.all(a["T"] == 30)


@pytest.mark.parametrize("K", [1, 200, 1000])
def test_mpc_horizon_counts(K):
    p = inputs.mpc_horizon_problem(K)
    assert p.num_edges == inputs.mpc_horizon_edges(K) == _edges_by_definition(p)
    pb = inputs.mpc_horizon_problem(K, umax=1.0)
    assert pb.num_edges == inputs.mpc_horizon_edges(K, box=True)
    A, B = inputs.pendulum_system()
    assert A.shape == (4, 4) and B.shape == (4, 1)


def test_mpc_instance_counts():
    d = inputs.mpc_batch_inputs(3, seed=4000)
    for i in range(3):
        p = inputs.mpc_problem(d["A"][i], d["B"][i], d["q"][i], d["r"][i], d["x0"][i], int(d["T"][i]))
        assert p.num_edges == inputs.mpc_edges(int(d["T"][i])) == _edges_by_definition(p)
