"""The learned warm start end to end at reduced size: solver-generated
training data, BF16 MLP training on the GPU, then cold vs warm batched
solves of fresh instances to residual 1e-4.  The network must cut the mean
iteration count, every instance must still converge (cold fallback on a
budget miss), and the warm solutions must equal the cold ones up to the
tolerance (the network only changes the start point)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1603_02526_gb300 import build
    build.build()


def test_warm_start_reduces_iterations():
    from paper_1603_02526_gb300 import warmstart
    X, Y, res = warmstart.generate(16384, x0_seed=7001)
    assert X.shape[0] >= 16000
    net, info = warmstart.train(X, Y, epochs=40, batch=1024, lr=2e-3)
    assert info["losses"][-1] < 0.2 * info["losses"][0]
    ev = warmstart.evaluate(net, n_eval=2048, x0_seed=7003, calib=512)
    assert ev["cold"]["converged"] == ev["n"]
    assert ev["warm"]["iters_mean"] < 0.8 * ev["cold"]["iters_mean"], ev
    if ev["max_abs_dz_warm_vs_cold"] is not None:
        # both stop at RMS residual 1e-4; the iterates agree to that scale
        assert ev["max_abs_dz_warm_vs_cold"] < 5e-2, ev
