"""CPU reference of the learned precision router's network (FP64, numpy).

TEST INFRASTRUCTURE (same rules as the rest of ``oracle/``).

The router is a 12 -> 64 -> 64 -> 1 ReLU MLP whose weights are used in BF16
(round to nearest even from the FP32 master copy) with the features
normalised as (x - mu) * isd. The input of every layer (the normalised
features, the two hidden activations) is rounded to BF16 as well, since the
GPU evaluates the layers as BF16 tensor-core products; everything else is
exact here (FP64). It is trained with the pinball (quantile) loss
rho_q(u) = u (q - [u < 0]), u = y - prediction. This module evaluates the
network and the loss gradient in FP64 from the same BF16-rounded weights, so
that the GPU forward and backward kernels can be checked against it.
The parameter layout is the library's: W1[16][64] b1[64] W2[64][64] b2[64]
W3[64] b3, inputs padded to 16 (rows 12..15 of W1 unused).

Pinned by tests/test_oracle_router.py: finite differences of the loss, and
closed forms (a network with only b3 non-zero).
"""
from __future__ import annotations

import numpy as np

NIN, NINP, NH = 12, 16, 64
OFF_W1 = 0
OFF_B1 = NINP * NH
OFF_W2 = OFF_B1 + NH
OFF_B2 = OFF_W2 + NH * NH
OFF_W3 = OFF_B2 + NH
OFF_B3 = OFF_W3 + NH
NPARAM = OFF_B3 + 1


def bf16_round(a: np.ndarray) -> np.ndarray:
    """float32 -> bf16 (nearest even) -> float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    finite = (u & 0x7F800000) != 0x7F800000
    r = np.where(finite, (u + 0x7FFF + ((u >> 16) & 1)) >> 16, u >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(theta: np.ndarray, round_weights: bool = True):
    t = np.asarray(theta, dtype=np.float32 if round_weights else np.float64)
    rw = bf16_round if round_weights else (lambda x: np.asarray(x, dtype=np.float64))
    W1 = rw(t[OFF_W1:OFF_B1]).reshape(NINP, NH)[:NIN]
    b1 = t[OFF_B1:OFF_W2].astype(np.float64)
    W2 = rw(t[OFF_W2:OFF_B2]).reshape(NH, NH)
    b2 = t[OFF_B2:OFF_W3].astype(np.float64)
    W3 = rw(t[OFF_W3:OFF_B3])
    b3 = float(t[OFF_B3])
    return W1, b1, W2, b2, W3, b3


def _layers(theta, mu, isd, X, round_weights):
    """Forward pass; returns (xn, a1, h1, a2, h2, out, weights). With
    round_weights the layer inputs xn, h1, h2 are BF16-rounded too."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, round_weights)
    ra = bf16_round if round_weights else (lambda x: x)
    xn = ra((np.asarray(X, np.float64) - np.asarray(mu, np.float64)[:NIN]) * np.asarray(isd, np.float64)[:NIN])
    a1 = xn @ W1 + b1
    h1 = ra(np.maximum(a1, 0.0))
    a2 = h1 @ W2 + b2
    h2 = ra(np.maximum(a2, 0.0))
    return xn, a1, h1, a2, h2, h2 @ W3 + b3, (W1, b1, W2, b2, W3, b3)


def forward(theta, mu, isd, X, round_weights=True):
    """Prediction per row (without the routing margin), FP64."""
    return _layers(theta, mu, isd, X, round_weights)[5]


def pinball_loss(theta, mu, isd, X, y, q, round_weights=True):
    u = np.asarray(y, np.float64) - forward(theta, mu, isd, X, round_weights)
    return float(np.mean(np.where(u >= 0, q * u, (q - 1.0) * u)))


def pinball_grad(theta, mu, isd, X, y, q, round_weights=True):
    """(loss, gradient w.r.t. the flat parameters), backpropagation in FP64.

    The derivative is taken with respect to the weights as used (the BF16
    rounding is treated as the identity, a straight-through estimate), which
    is what the GPU training kernels do; the same holds for the rounding of
    the layer inputs."""
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    xn, a1, h1, a2, h2, out, (W1, b1, W2, b2, W3, b3) = _layers(theta, mu, isd, X, round_weights)
    u = np.asarray(y, np.float64) - out
    loss = float(np.mean(np.where(u >= 0, q * u, (q - 1.0) * u)))
    g = ((u < 0).astype(np.float64) - q) / n           # d loss / d out, per row
    gW3 = h2.T @ g
    gb3 = g.sum()
    d2 = np.outer(g, W3) * (a2 > 0)
    gW2 = h1.T @ d2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (a1 > 0)
    gW1 = xn.T @ d1
    gb1 = d1.sum(axis=0)
    grad = np.zeros(NPARAM)
    W1p = np.zeros((NINP, NH))
    W1p[:NIN] = gW1
    grad[OFF_W1:OFF_B1] = W1p.ravel()
    grad[OFF_B1:OFF_W2] = gb1
    grad[OFF_W2:OFF_B2] = gW2.ravel()
    grad[OFF_B2:OFF_W3] = gb2
    grad[OFF_W3:OFF_B3] = gW3
    grad[OFF_B3] = gb3
    return loss, grad
