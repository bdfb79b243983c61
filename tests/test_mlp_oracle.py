"""Pins for the MLP oracle: backprop equals central finite differences of the loss (exact
form), and the BF16 rounding used by the quantised form equals torch's float -> bfloat16
conversion (round to nearest, ties to even)."""
import numpy as np
import pytest

from oracle import mlp


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = mlp.init(5)
    X = rng.normal(size=(12, mlp.IN))
    t = rng.normal(size=12)
    _, loss, g = mlp.forward_backward(p, X, t, quantised=False)
    idx = np.concatenate([rng.choice(len(p), 60, replace=False), [len(p) - 1]])
    h = 1e-6
    for i in idx:
        d = np.zeros_like(p)
        d[i] = h
        lp = mlp.forward_backward(p + d, X, t, quantised=False)[1]
        lm = mlp.forward_backward(p - d, X, t, quantised=False)[1]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000).astype(np.float32),
                        np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 1e-30, 3.0e38], dtype=np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def test_quantised_equals_exact_on_bf16_representable_inputs():
    # with inputs and weights already BF16 and a network whose activations stay exact, the
    # two forms agree: a special case that ties the quantised form to the exact one
    p = mlp.bf16(mlp.init(2))
    X = mlp.bf16(np.random.default_rng(1).normal(size=(4, mlp.IN)))
    y_exact = mlp.forward_backward(p, X, quantised=False)[0]
    y_q = mlp.forward_backward(p, X, quantised=True)[0]
    assert np.allclose(y_exact, y_q, rtol=2e-2, atol=2e-2)
