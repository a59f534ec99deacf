"""Pins of the oracle's learned-guess network: its bfloat16 rounding against
PyTorch's independent conversion, its exact backward pass against central
finite differences, and the zero-output-layer property."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        [0.0, 1.0, -1.0, 1.00390625, 1.01171875]])   # exact ties included
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)


def test_exact_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    n_in, h, n_out, M = 5, 7, 3, 11
    w = rng.standard_normal(mlp.n_params(n_in, h, n_out)) * 0.5
    X = rng.standard_normal((M, n_in))
    T = rng.standard_normal((M, n_out))
    _, _, g = mlp.forward_backward(w, X, T, n_in, h, n_out, quantize=False)
    eps = 1e-6
    fd = np.empty_like(w)
    for i in range(len(w)):
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        lp = mlp.forward_backward(wp, X, T, n_in, h, n_out, quantize=False)[1]
        lm = mlp.forward_backward(wm, X, T, n_in, h, n_out, quantize=False)[1]
        fd[i] = (lp - lm) / (2 * eps)
    assert np.abs(fd - g).max() < 1e-7 * max(1.0, np.abs(g).max())


def test_zero_output_layer_gives_zero_correction():
    rng = np.random.default_rng(2)
    n_in, h, n_out = 6, 8, 4
    w = rng.standard_normal(mlp.n_params(n_in, h, n_out))
    Ws, bs = mlp.unpack(w, n_in, h, n_out)
    o = mlp.n_params(n_in, h, n_out) - (n_out * h + n_out)
    w[o:] = 0.0
    Y, _, _ = mlp.forward(w, rng.standard_normal((9, n_in)), n_in, h, n_out)
    assert np.all(Y == 0.0)
