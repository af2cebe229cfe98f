"""Pins for the CPU reference of the router network (oracle/router.py)."""
import numpy as np
import pytest

from oracle import router as R


def rand_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    theta = (rng.standard_normal(R.NPARAM) * scale).astype(np.float32)
    mu = rng.standard_normal(16).astype(np.float32)
    isd = (0.5 + rng.random(16)).astype(np.float32)
    X = rng.standard_normal((300, R.NIN)).astype(np.float32)
    y = rng.standard_normal(300).astype(np.float32)
    return theta, mu, isd, X, y


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.00390625, 1.005859375, 1.0078125, -3.14159], dtype=np.float32)
    r = R.bf16_round(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: rounds to the even mantissa (1)
    assert r[0] == 1.0 and r[1] == 1.0
    assert r[2] == 1.0078125 and r[3] == 1.0078125
    assert abs(r[4] - (-3.140625)) < 1e-12


def test_only_output_bias_closed_form():
    theta, mu, isd, X, y = rand_params(1)
    theta[:] = 0.0
    theta[R.OFF_B3] = 0.25
    pred = R.forward(theta, mu, isd, X)
    assert np.all(pred == 0.25)
    q = 0.8
    loss, g = R.pinball_grad(theta, mu, isd, X, y, q)
    u = y.astype(np.float64) - 0.25
    assert loss == pytest.approx(np.mean(np.where(u >= 0, q * u, (q - 1) * u)), rel=1e-12)
    assert g[R.OFF_B3] == pytest.approx(np.mean(u < 0) - q, rel=1e-12)
    assert np.all(g[:R.OFF_B3] == 0.0)


@pytest.mark.parametrize("q", [0.5, 0.9])
def test_gradient_against_finite_differences(q):
    theta, mu, isd, X, y = rand_params(2)
    # unrounded weights make the loss a smooth function away from kinks
    loss, g = R.pinball_grad(theta.astype(np.float64), mu, isd, X, y, q, round_weights=False)
    rng = np.random.default_rng(3)
    picks = np.concatenate([rng.integers(R.OFF_W1, R.OFF_W1 + 12 * 64, 6), rng.integers(R.OFF_W2, R.OFF_B2, 6),
                            rng.integers(R.OFF_W3, R.OFF_B3, 4), [R.OFF_B3], rng.integers(R.OFF_B1, R.OFF_W2, 3)])
    th64 = theta.astype(np.float64)
    for i in picks:
        h = 1e-6   # small enough that no sample crosses a pinball or ReLU kink
        tp = th64.copy(); tp[i] += h
        tm = th64.copy(); tm[i] -= h
        fp = R.pinball_loss(tp, mu, isd, X, y, q, round_weights=False)
        fm = R.pinball_loss(tm, mu, isd, X, y, q, round_weights=False)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[i]) <= 2e-3 * max(1e-3, abs(g[i])) + 2e-5, (i, fd, g[i])


def test_padded_inputs_have_no_gradient():
    theta, mu, isd, X, y = rand_params(4)
    _, g = R.pinball_grad(theta, mu, isd, X, y, 0.7)
    W1g = g[R.OFF_W1:R.OFF_B1].reshape(16, 64)
    assert np.all(W1g[12:] == 0.0)


def test_layer_inputs_are_bf16_rounded():
    """A network that passes normalised feature 0 straight through (unit
    weights, zero biases) returns that feature rounded to BF16 once (the
    rounding is idempotent), and the unrounded value without rounding."""
    th = np.zeros(R.NPARAM, np.float32)
    th[R.OFF_W1 + 0 * R.NH + 0] = 1.0
    th[R.OFF_W2 + 0 * R.NH + 0] = 1.0
    th[R.OFF_W3 + 0] = 1.0
    mu = np.zeros(16, np.float32)
    isd = np.ones(16, np.float32)
    x0 = np.array([1.0 + 2.0 ** -10, 3.0 + 2.0 ** -9, 0.75], np.float64)
    X = np.zeros((3, 12), np.float32)
    X[:, 0] = x0
    y = R.forward(th, mu, isd, X)
    assert np.array_equal(y, R.bf16_round(x0))
    assert y[0] == 1.0 and y[1] == 3.0 and y[2] == 0.75
    assert np.array_equal(R.forward(th, mu, isd, X, round_weights=False), X[:, 0].astype(np.float64))
