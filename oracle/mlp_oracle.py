"""FP64 reference for the warm-start MLP (test infrastructure only).

The network is in -> h1 -> h2 -> out with ReLU after the two hidden
layers, mean-squared-error loss L = sum (Y - T)^2 / (rows * out), and Adam
(beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  Written as plain
matrix products; the backward pass is the chain rule layer by layer.

`bf16=True` rounds to bfloat16 (round to nearest even) exactly where the
GPU stores a BF16 value: the input, the weights, both hidden activations,
the output gradient used by the matrix products and both hidden-layer
gradients.  Everything else stays FP64.
"""
import numpy as np


def to_bf16(a):
    """Rounds to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, shape):
    n_in, h1, h2, n_out = shape
    p = np.asarray(params, dtype=np.float64)
    out, off = [], 0
    for r, c in ((h1, n_in), (h2, h1), (n_out, h2)):
        out.append(p[off: off + r * c].reshape(r, c))
        off += r * c
        out.append(p[off: off + r])
        off += r
    return out


def pack(parts):
    return np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in parts])


def forward(params, shape, X, bf16=False):
    W1, b1, W2, b2, W3, b3 = unpack(params, shape)
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Xq = r(X)
    W1q, W2q, W3q = r(W1), r(W2), r(W3)
    H1 = r(np.maximum(Xq @ W1q.T + b1, 0.0))
    H2 = r(np.maximum(H1 @ W2q.T + b2, 0.0))
    Y = H2 @ W3q.T + b3
    return dict(Xq=Xq, W1q=W1q, W2q=W2q, W3q=W3q, H1=H1, H2=H2, Y=Y)


def loss_and_grads(params, shape, X, T, bf16=False):
    """Loss and the gradient of every parameter (packed like the params)."""
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    f = forward(params, shape, X, bf16)
    n = f["Y"].size
    D = f["Y"] - T
    loss = float(np.sum(D * D) / n)
    dY = 2.0 * D / n
    dYq = r(dY)
    gW3 = dYq.T @ f["H2"]
    gb3 = dY.sum(axis=0)
    dH2 = r((dYq @ f["W3q"]) * (f["H2"] > 0))
    gW2 = dH2.T @ f["H1"]
    gb2 = dH2.sum(axis=0)
    dH1 = r((dH2 @ f["W2q"]) * (f["H1"] > 0))
    gW1 = dH1.T @ f["Xq"]
    gb1 = dH1.sum(axis=0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3])


def loss_only(params, shape, X, T):
    Y = forward(params, shape, X, False)["Y"]
    return float(np.sum((Y - T) ** 2) / Y.size)


def adam_step(params, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
