"""GPU MLP kernels (BF16 tensor cores, FP32 accumulation) against the FP64
oracle.  With BF16 rounding emulated at the same points the two agree to
accumulation order (rare BF16 rounding-boundary flips of an activation
aside): gradients within 1e-2 relative in norm per tensor.  Against the
unrounded FP64 network the gap is BF16 precision (2^-8): 5e-2."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo

pytestmark = pytest.mark.gpu

SHAPE = (12, 256, 256, 960)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


def _setup(seed=0, batch=128):
    import torch
    from paper_1603_02526_gb300.mlp import MLP
    rng = np.random.default_rng(seed)
    m = MLP(*SHAPE, max_batch=1024, seed=seed)
    p = m.fga_mlp_get_params().astype(np.float64)
    # non-zero biases so that every gradient path is exercised
    W1, b1, W2, b2, W3, b3 = mo.unpack(p, SHAPE)
    p = mo.pack([W1, rng.standard_normal(b1.size) * 0.1, W2, rng.standard_normal(b2.size) * 0.1, W3,
                 rng.standard_normal(b3.size) * 0.1])
    m.fga_mlp_set_params(p.astype(np.float32))
    X = rng.standard_normal((batch, SHAPE[0])).astype(np.float32)
    T = rng.standard_normal((batch, SHAPE[3])).astype(np.float32)
    Xd = torch.tensor(X, device="cuda")
    Td = torch.tensor(T, device="cuda")
    return m, p.astype(np.float32).astype(np.float64), X.astype(np.float64), T.astype(np.float64), Xd, Td


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_params_roundtrip_and_init_scale():
    from paper_1603_02526_gb300.mlp import MLP
    m = MLP(*SHAPE, max_batch=64, seed=11)
    p = m.fga_mlp_get_params()
    assert p.size == 12 * 256 + 256 + 256 * 256 + 256 + 960 * 256 + 960
    W1 = mo.unpack(p, SHAPE)[0]
    assert abs(W1.std() - np.sqrt(2 / 12)) < 0.02       # He initialisation
    m2 = MLP(*SHAPE, max_batch=64, seed=11)
    assert np.array_equal(m2.fga_mlp_get_params(), p)   # seeded


def test_gradients_match_bf16_oracle():
    m, p, X, T, Xd, Td = _setup(0)
    loss, g = m.fga_mlp_gradients(Xd, Td)
    lo, go = mo.loss_and_grads(p, SHAPE, X, T, bf16=True)
    assert loss == pytest.approx(lo, rel=1e-4)
    gg, gr = mo.unpack(g.astype(np.float64), SHAPE), mo.unpack(go, SHAPE)
    for a, b in zip(gg, gr):
        assert _rel(a, b) < 1e-2, _rel(a, b)
    lf, gf = mo.loss_and_grads(p, SHAPE, X, T, bf16=False)
    assert loss == pytest.approx(lf, rel=2e-2)
    for a, b in zip(gg, mo.unpack(gf, SHAPE)):
        assert _rel(a, b) < 5e-2, _rel(a, b)


def test_forward_matches_oracle():
    import torch
    m, p, X, T, Xd, Td = _setup(1, batch=256)
    Y = torch.empty((256, SHAPE[3]), device="cuda")
    m.fga_mlp_forward(Xd, Y)
    yo = mo.forward(p, SHAPE, X, bf16=True)["Y"]
    assert _rel(Y.cpu().numpy().astype(np.float64), yo) < 5e-3


def test_adam_step_matches_oracle():
    m, p, X, T, Xd, Td = _setup(2)
    _, g = m.fga_mlp_gradients(Xd, Td)
    m.fga_mlp_train_step(Xd, Td, 1e-3)
    p1 = m.fga_mlp_get_params().astype(np.float64)
    po, _, _ = mo.adam_step(p, np.zeros_like(p), np.zeros_like(p), g.astype(np.float64), 1, 1e-3)
    np.testing.assert_allclose(p1, po, atol=2e-6, rtol=1e-5)


def test_training_reduces_loss():
    """A learnable target (a fixed random 2-layer map of the input)."""
    import torch
    from paper_1603_02526_gb300.mlp import MLP
    rng = np.random.default_rng(3)
    X = rng.standard_normal((1024, 12)).astype(np.float32)
    A1 = rng.standard_normal((12, 64)) / np.sqrt(12)
    A2 = rng.standard_normal((64, 960)) / 8
    T = (np.tanh(X @ A1) @ A2).astype(np.float32)
    m = MLP(*SHAPE, max_batch=1024, seed=4)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    m.fga_mlp_fit_normalization(Td)
    first = m.fga_mlp_train_step(Xd, Td, 1e-3, want_loss=True)
    for _ in range(300):
        last = m.fga_mlp_train_step(Xd, Td, 1e-3, want_loss=True)
    assert last < 0.1 * first, (first, last)


def test_normalization_stats():
    import torch
    from paper_1603_02526_gb300.mlp import MLP
    rng = np.random.default_rng(5)
    Y = (rng.standard_normal((4096, 960)) * rng.uniform(0.1, 5, 960) + rng.uniform(-3, 3, 960)).astype(np.float32)
    m = MLP(*SHAPE, max_batch=64, seed=6)
    Yd = torch.tensor(Y, device="cuda")
    m.fga_mlp_fit_normalization(Yd)
    mu, sd = m.fga_mlp_get_normalization()
    np.testing.assert_allclose(mu, Y.astype(np.float64).mean(0), rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(sd, Y.astype(np.float64).std(0), rtol=1e-5)
    Z = Yd.cpu().numpy()
    np.testing.assert_allclose(Z.mean(0), 0, atol=1e-4)
    np.testing.assert_allclose(Z.std(0), 1, rtol=1e-4)


RAGGED = (5, 24, 40, 72)


@pytest.mark.parametrize("batch", [8, 200])
def test_ragged_network_matches_oracle(batch):
    """Sizes that fill no GEMM tile (128 x 128 outputs, blocks of 64 k):
    the tensor maps' zero fill past the edges, partial tiles and the scalar
    tails of the epilogue, in every product of the forward and backward."""
    import torch
    from paper_1603_02526_gb300.mlp import MLP
    rng = np.random.default_rng(batch)
    m = MLP(*RAGGED, max_batch=256, seed=21)
    W1, b1, W2, b2, W3, b3 = mo.unpack(m.fga_mlp_get_params().astype(np.float64), RAGGED)
    p = mo.pack([W1, rng.standard_normal(b1.size) * 0.1, W2, rng.standard_normal(b2.size) * 0.1, W3,
                 rng.standard_normal(b3.size) * 0.1])
    m.fga_mlp_set_params(p.astype(np.float32))
    p = p.astype(np.float32).astype(np.float64)
    X = rng.standard_normal((batch, RAGGED[0])).astype(np.float32)
    T = rng.standard_normal((batch, RAGGED[3])).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    loss, g = m.fga_mlp_gradients(Xd, Td)
    lo, go = mo.loss_and_grads(p, RAGGED, X.astype(np.float64), T.astype(np.float64), bf16=True)
    assert loss == pytest.approx(lo, rel=1e-4)
    for a, b in zip(mo.unpack(g.astype(np.float64), RAGGED), mo.unpack(go, RAGGED)):
        assert _rel(a, b) < 1e-2, _rel(a, b)
    Y = torch.empty((batch, RAGGED[3]), device="cuda")
    m.fga_mlp_forward(Xd, Y)
    yo = mo.forward(p, RAGGED, X.astype(np.float64), bf16=True)["Y"]
    assert _rel(Y.cpu().numpy().astype(np.float64), yo) < 5e-3


def test_forward_evaluation_batch_sampled_rows():
    """The 16,384-row inference batch (multi-wave GEMM grids): 512 sampled
    rows against the oracle (rows are independent)."""
    import torch
    from paper_1603_02526_gb300.mlp import MLP
    rng = np.random.default_rng(5)
    m = MLP(*SHAPE, max_batch=16384, seed=5)
    p = m.fga_mlp_get_params().astype(np.float64)
    X = rng.standard_normal((16384, SHAPE[0])).astype(np.float32)
    Y = torch.empty((16384, SHAPE[3]), device="cuda")
    m.fga_mlp_forward(torch.tensor(X, device="cuda"), Y)
    rows = np.sort(rng.choice(16384, 512, replace=False))
    yo = mo.forward(p, SHAPE, X[rows].astype(np.float64), bf16=True)["Y"]
    assert _rel(Y.cpu().numpy()[rows].astype(np.float64), yo) < 5e-3
