"""Oracle of the learned-guess network (test infrastructure only).

Plain numpy FP64 forward and backward of the per-cell MLP
n_in -> h -> h -> h -> n_out with SiLU, with the network's quantisation
points written out: inputs, weights and hidden activations rounded to
bfloat16, error gradients rounded to bfloat16 before each product (the
numerics the library states for its BF16-in/FP32-accumulate kernels).
quantize=False gives the exact FP64 network, pinned by finite differences.
Parameters are packed W1 [h x n_in], b1, W2 [h x h], b2, W3, b3,
W4 [n_out x h], b4.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Nearest bfloat16 (ties to even) of the float32 value of x, as float64:
    keep the upper 16 bits of the float32 pattern after adding half an ulp of
    the kept part (plus one when the kept part is odd, for ties to even)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def dims_of(n_in, hidden, n_out):
    return [n_in, hidden, hidden, hidden, n_out]


def unpack(w, n_in, hidden, n_out):
    d = dims_of(n_in, hidden, n_out)
    Ws, bs, o = [], [], 0
    for l in range(4):
        n = d[l + 1] * d[l]
        Ws.append(np.asarray(w[o:o + n], dtype=np.float64).reshape(d[l + 1], d[l]))
        o += n
        bs.append(np.asarray(w[o:o + d[l + 1]], dtype=np.float64))
        o += d[l + 1]
    return Ws, bs


def n_params(n_in, hidden, n_out):
    d = dims_of(n_in, hidden, n_out)
    return sum(d[l + 1] * d[l] + d[l + 1] for l in range(4))


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(w, X, n_in, hidden, n_out, quantize=True):
    q = bf16_round if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    Ws, bs = unpack(w, n_in, hidden, n_out)
    H, Z = [q(X)], []
    for l in range(4):
        z = H[-1] @ q(Ws[l]).T + bs[l]
        Z.append(z)
        if l < 3:
            H.append(q(silu(z)))
    return Z[3], H, Z


def forward_backward(w, X, T, n_in, hidden, n_out, quantize=True):
    """Returns Y, loss = mean((Y - T)^2), packed gradient of the loss."""
    q = bf16_round if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    Ws, _ = unpack(w, n_in, hidden, n_out)
    Y, H, Z = forward(w, X, n_in, hidden, n_out, quantize)
    E = Y - np.asarray(T, dtype=np.float64)
    loss = float(np.mean(E * E))
    dz = 2.0 * E / E.size
    gW, gb = [None] * 4, [None] * 4
    for l in range(3, -1, -1):
        dzq = q(dz)
        gW[l] = dzq.T @ H[l]
        gb[l] = dz.sum(axis=0)
        if l > 0:
            dz = (dzq @ q(Ws[l])) * dsilu(Z[l - 1])
    g = np.concatenate([np.concatenate([gW[l].reshape(-1), gb[l]]) for l in range(4)])
    return Y, loss, g
