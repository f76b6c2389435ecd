"""Pins of the FP64 surrogate-MLP oracle."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_parameter_count_and_packing():
    theta = M.init_params(0)
    assert theta.size == M.n_params() == 64 * 256 + 256 + 3 * (256 * 256 + 256) + 257
    layers, w5, b5 = M.unpack(theta)
    np.testing.assert_array_equal(M.pack(layers, w5, b5), theta.astype(np.float64))


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 65504.0]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(M.bf16(a), ref.astype(np.float64))


def test_silu_grad_is_the_derivative():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    np.testing.assert_allclose(M.silu_grad(z), (M.silu(z + h) - M.silu(z - h)) / (2 * h), rtol=1e-7,
                               atol=1e-9)


def test_features_closed_form():
    freqs = np.random.default_rng(1).normal(0, 4, (32, 2))
    f = M.features(freqs, np.zeros((3, 2)))
    np.testing.assert_allclose(f[:, :32], 0.0, atol=1e-15)
    np.testing.assert_allclose(f[:, 32:], 1.0)
    x = np.array([[0.25, 0.5]])
    v = 2 * np.pi * (freqs @ x[0])
    np.testing.assert_allclose(M.features(freqs, x)[0], np.concatenate([np.sin(v), np.cos(v)]))


def test_zero_hidden_weights_give_a_constant():
    layers, w5, b5 = M.unpack(M.init_params(2).astype(np.float64))
    layers = [(np.zeros_like(W), np.full(W.shape[0], 0.1 * (i + 1))) for i, (W, _) in enumerate(layers)]
    theta = M.pack(layers, w5, 0.3)
    x = np.random.default_rng(3).uniform(0, 1, (5, 2))
    y, _ = M.forward(theta, np.ones((32, 2)), x, emulate_bf16=False)
    np.testing.assert_allclose(y, M.silu(0.4) * w5.sum() + 0.3, rtol=1e-14)


def test_gradient_by_central_differences():
    rng = np.random.default_rng(4)
    theta = M.init_params(5).astype(np.float64) * 0.5
    freqs = rng.normal(0, 2, (32, 2))
    x = rng.uniform(0, 1, (16, 2))
    t = rng.normal(size=16)
    _, g = M.loss_grad(theta, freqs, x, t, emulate_bf16=False)
    h = 1e-6
    for i in list(rng.choice(theta.size, 25, replace=False)) + [theta.size - 1, theta.size - 2]:
        e = np.zeros_like(theta)
        e[i] = h
        lp, _ = M.loss_grad(theta + e, freqs, x, t, emulate_bf16=False)
        lm, _ = M.loss_grad(theta - e, freqs, x, t, emulate_bf16=False)
        assert g[i] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-10)
