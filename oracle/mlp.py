"""Warm-start network in FP64 (oracle; test infrastructure).

3-layer perceptron x -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> W3 h2 + b3, mean-squared-error
loss over batch and outputs, gradients by the chain rule, Adam (Kingma & Ba, ICLR 2015).  The
device keeps BF16 copies of the weights for its products; the oracle is given those rounded
values (bf16_round) so both differentiate the same function.  Feature and target maps sample
grid profiles at z_j = (j + 1/2) Lz / n by linear interpolation (0 on the grounded planes).
"""
from __future__ import annotations

import numpy as np

Q_E = 1.602176634e-19


def split(params, sizes):
    """Views W1, b1, W2, b2, W3, b3 of the flat parameter vector (W row-major [out][in])."""
    out, off = [], 0
    for l in range(3):
        nw = sizes[l + 1] * sizes[l]
        out.append(params[off:off + nw].reshape(sizes[l + 1], sizes[l]))
        off += nw
        out.append(params[off:off + sizes[l + 1]])
        off += sizes[l + 1]
    return out


def bf16_round(w):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    b = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def forward(params, sizes, X):
    W1, b1, W2, b2, W3, b3 = split(np.asarray(params, float), sizes)
    H1 = np.tanh(X @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    Y = H2 @ W3.T + b3
    return H1, H2, Y


def loss_and_grads(params, sizes, X, T):
    params = np.asarray(params, float)
    W1, b1, W2, b2, W3, b3 = split(params, sizes)
    H1, H2, Y = forward(params, sizes, X)
    n = Y.size
    loss = ((Y - T) ** 2).sum() / n
    G3 = 2.0 * (Y - T) / n
    gW3, gb3 = G3.T @ H2, G3.sum(0)
    G2 = (G3 @ W3) * (1 - H2 ** 2)
    gW2, gb2 = G2.T @ H1, G2.sum(0)
    G1 = (G2 @ W2) * (1 - H1 ** 2)
    gW1, gb1 = G1.T @ X, G1.sum(0)
    return loss, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def adam_step(w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return w, m, v


def _profile(grid, f3d, n):
    """Lateral mean of the interior planes sampled at z_j = (j + 1/2) Lz / n."""
    prof = np.concatenate([[0.0], np.asarray(f3d, float).reshape(grid.nz - 1, -1).mean(axis=1), [0.0]])
    t = (np.arange(n) + 0.5) * grid.nz / n
    return np.interp(t, np.arange(grid.nz + 1), prof)


def features(grid, donor_rho, n=256, shift=21.0, scale=6.0):
    nd = _profile(grid, donor_rho, n) / Q_E
    return (np.log10(np.maximum(nd, 1e15)) - shift) / scale


def targets(grid, phi, n=256, scale=0.2):
    return _profile(grid, phi, n) / scale


def inject(grid, y, scale=0.2):
    """Grid potential from the n-point profile: linear between sample points, 0 V at the ends."""
    n = len(y)
    zs = np.concatenate([[0.0], (np.arange(n) + 0.5) / n, [1.0]])
    vs = np.concatenate([[0.0], np.asarray(y, float), [0.0]])
    zk = np.arange(1, grid.nz) / grid.nz
    prof = np.interp(zk, zs, vs) * scale
    return np.broadcast_to(prof[:, None, None], (grid.nz - 1, grid.ny, grid.nx)).copy()
