"""Python binding of the warm-start MLP C-ABI (fga_mlp_*), marshalling only."""
import ctypes

import numpy as np

from . import _lib
from ._lib import check


def _p(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


class MLP:
    """ReLU MLP in -> h1 -> h2 -> out on BF16 tensor cores (FP32 accumulate)."""

    def __init__(self, n_in=12, h1=256, h2=256, n_out=960, max_batch=16384, seed=5000, device=0, stream=None):
        self._lib = _lib.load()
        self._m = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream")
                                                         else int(stream))
        check(self._lib.fga_mlp_create(ctypes.byref(self._m), n_in, h1, h2, n_out, max_batch, seed, device, st),
              "fga_mlp_create")
        self.shape = (n_in, h1, h2, n_out)

    def __del__(self):
        m = getattr(self, "_m", None)
        if m is not None and m.value:
            self._lib.fga_mlp_destroy(m)
            self._m = ctypes.c_void_p()

    def fga_mlp_num_params(self):
        n = ctypes.c_int64()
        check(self._lib.fga_mlp_num_params(self._m, ctypes.byref(n)), "fga_mlp_num_params")
        return n.value

    def fga_mlp_get_params(self):
        out = np.empty(self.fga_mlp_num_params(), dtype=np.float32)
        check(self._lib.fga_mlp_get_params(self._m, _p(out), out.size), "fga_mlp_get_params")
        return out

    def fga_mlp_set_params(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        check(self._lib.fga_mlp_set_params(self._m, _p(params), params.size), "fga_mlp_set_params")

    def fga_mlp_fit_normalization(self, Y):
        check(self._lib.fga_mlp_fit_normalization(self._m, _p(Y), int(Y.shape[0])), "fga_mlp_fit_normalization")

    def fga_mlp_get_normalization(self):
        n = self.shape[3]
        mu = np.empty(n, dtype=np.float32)
        sd = np.empty(n, dtype=np.float32)
        check(self._lib.fga_mlp_get_normalization(self._m, _p(mu), _p(sd)), "fga_mlp_get_normalization")
        return mu, sd

    def fga_mlp_gradients(self, X, Y):
        g = np.empty(self.fga_mlp_num_params(), dtype=np.float32)
        loss = ctypes.c_double()
        check(self._lib.fga_mlp_gradients(self._m, _p(X), _p(Y), int(X.shape[0]), _p(g), ctypes.byref(loss)),
              "fga_mlp_gradients")
        return loss.value, g

    def fga_mlp_train_step(self, X, Y, lr, want_loss=False):
        loss = ctypes.c_double()
        check(self._lib.fga_mlp_train_step(self._m, _p(X), _p(Y), int(X.shape[0]), float(lr),
                                           ctypes.byref(loss) if want_loss else None), "fga_mlp_train_step")
        return loss.value if want_loss else None

    def fga_mlp_forward(self, X, Y):
        check(self._lib.fga_mlp_forward(self._m, _p(X), _p(Y), int(X.shape[0])), "fga_mlp_forward")
        return Y


def unpack(params, shape):
    """Split a packed parameter vector into (W1, b1, W2, b2, W3, b3)."""
    n_in, h1, h2, n_out = shape
    out, off = [], 0
    for r, c in ((h1, n_in), (h2, h1), (n_out, h2)):
        out.append(params[off: off + r * c].reshape(r, c))
        off += r * c
        out.append(params[off: off + r])
        off += r
    return out
