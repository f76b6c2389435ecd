"""FP64 CPU oracle of the surrogate MLP (test infrastructure only).

The surrogate maps a transmitter position x in [0, 1]^2 to a scalar:
Fourier features (32 frequencies B_j, features sin(2 pi B_j . x) and
cos(2 pi B_j . x)), four Linear(256) + SiLU layers, and Linear(1).  This
module computes it in float64, optionally rounding to bfloat16 at exactly the
points where the GPU network stores bfloat16 values (weights, features,
hidden activations, pre-activation gradients), so that the GPU's FP32
accumulation is the only remaining difference.

Parameter layout (flat float32/float64 vector): W1 [256][64], b1 [256],
W2..W4 [256][256] with b2..b4 [256], w5 [256], b5 [1].
"""
from __future__ import annotations

import numpy as np

N_FREQ = 32
N_FEAT = 2 * N_FREQ
WIDTH = 256
HIDDEN = 4


def layer_shapes():
    shapes = [(WIDTH, N_FEAT)] + [(WIDTH, WIDTH)] * (HIDDEN - 1)
    return shapes


def n_params() -> int:
    return sum(n * k + n for n, k in layer_shapes()) + WIDTH + 1


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, o = [], 0
    for n, k in layer_shapes():
        W = theta[o:o + n * k].reshape(n, k); o += n * k
        b = theta[o:o + n]; o += n
        out.append((W, b))
    w5 = theta[o:o + WIDTH]; o += WIDTH
    b5 = theta[o]; o += 1
    assert o == theta.size
    return out, w5, b5


def pack(layers, w5, b5):
    parts = []
    for W, b in layers:
        parts += [np.ravel(W), np.ravel(b)]
    parts += [np.ravel(w5), np.atleast_1d(b5)]
    return np.concatenate(parts)


def bf16(a):
    """Round float64/float32 values to bfloat16 (round to nearest even), returned as float64."""
    a32 = np.asarray(a, np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a32)
    out[nan] = np.nan
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def features(freqs, x):
    """[B, 64]: sin(2 pi x B^T), cos(2 pi x B^T)."""
    v = 2.0 * np.pi * (np.asarray(x, np.float64) @ np.asarray(freqs, np.float64).T)
    return np.concatenate([np.sin(v), np.cos(v)], axis=1)


def init_params(seed: int = 0) -> np.ndarray:
    """He-style uniform initialisation (float32 values)."""
    rng = np.random.default_rng(seed)
    layers = []
    for n, k in layer_shapes():
        lim = np.sqrt(6.0 / k)
        layers.append((rng.uniform(-lim, lim, (n, k)), np.zeros(n)))
    w5 = rng.uniform(-np.sqrt(3.0 / WIDTH), np.sqrt(3.0 / WIDTH), WIDTH)
    return pack(layers, w5, 0.0).astype(np.float32)


def forward(theta, freqs, x, emulate_bf16=True):
    """(y [B], cache) of the network."""
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    layers, w5, b5 = unpack(theta)
    h = r(features(freqs, x))
    cache = {"h": [h], "z": []}
    for W, b in layers:
        z = h @ r(W).T + b
        h = r(silu(z))
        cache["z"].append(z)
        cache["h"].append(h)
    y = h @ r(w5) + b5
    return y, cache


def loss_grad(theta, freqs, x, target, emulate_bf16=True):
    """(loss, grad): loss = mean (y - target)^2, grad w.r.t. the flat parameters."""
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    layers, w5, b5 = unpack(theta)
    y, c = forward(theta, freqs, x, emulate_bf16)
    B = y.shape[0]
    d = y - np.asarray(target, np.float64)
    loss = float(np.mean(d * d))
    dy = 2.0 * d / B
    grads = [None] * HIDDEN
    dw5 = c["h"][HIDDEN].T @ dy
    db5 = dy.sum()
    dh = np.outer(dy, r(w5))
    for l in range(HIDDEN - 1, -1, -1):
        dz = r(dh * silu_grad(c["z"][l]))
        dW = dz.T @ c["h"][l]
        db = dz.sum(axis=0)
        grads[l] = (dW, db)
        if l > 0:
            dh = dz @ r(layers[l][0])
    return loss, pack(grads, dw5, db5)
