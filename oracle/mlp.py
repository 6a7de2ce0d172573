"""Oracle MLP reconstructor (slopes -> modal coefficients), FP64.

The paper's reconstructor is linear (Table 1 ``modalrec``); the learned nonlinear
reconstructor is an extension of this project. Readings (stated here because no
source defines them):

  * input: slopes standardised per feature, x = (s - mean) * inv_std;
  * layers: z_l = W_l h_{l-1} + b_l, h_l = gelu(z_l) for the hidden layers,
    out = W_L h_{L-1} + b_L; gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2;
  * loss: mean squared error over the batch and the outputs,
    L = sum (out - y)^2 / (B n_out);
  * Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected), FP32/FP64 master weights;
  * parameters are listed layer by layer, W_l (out x in, row-major) then b_l.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def layer_sizes(n_in, n_hidden, n_hidden_layers, n_out):
    return [n_in] + [n_hidden] * n_hidden_layers + [n_out]


def init_params(sizes, rng):
    """He-normal weights (std sqrt(2/in)), zero biases; rng: numpy Generator."""
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        params.append(rng.standard_normal((b, a)) * math.sqrt(2.0 / a))
        params.append(np.zeros(b))
    return params


def flatten(params):
    return np.concatenate([p.ravel() for p in params])


def unflatten(vec, sizes):
    out, o = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        out.append(vec[o:o + a * b].reshape(b, a))
        o += a * b
        out.append(vec[o:o + b])
        o += b
    return out


def forward(params, x):
    """x: (B, n_in) standardised input. Returns output and the cache of (z, h)."""
    h = np.asarray(x, dtype=np.float64)
    cache = [(None, h)]
    n = len(params) // 2
    for l in range(n):
        W, b = params[2 * l], params[2 * l + 1]
        z = h @ W.T + b
        h = gelu(z) if l < n - 1 else z
        cache.append((z, h))
    return h, cache


def loss(out, y):
    d = out - y
    return float(np.sum(d * d) / d.size)


def backward(params, cache, out, y):
    """Gradients of the MSE loss w.r.t. every parameter (same order as params)."""
    n = len(params) // 2
    grads = [None] * len(params)
    dz = 2.0 * (out - y) / out.size
    for l in range(n - 1, -1, -1):
        h_prev = cache[l][1]
        grads[2 * l] = dz.T @ h_prev
        grads[2 * l + 1] = dz.sum(axis=0)
        if l > 0:
            dh = dz @ params[2 * l]
            dz = dh * gelu_grad(cache[l][0])
    return grads


def adam_update(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); updates params, m, v in place."""
    for i, g in enumerate(grads):
        m[i] = beta1 * m[i] + (1 - beta1) * g
        v[i] = beta2 * v[i] + (1 - beta2) * g * g
        mh = m[i] / (1 - beta1 ** t)
        vh = v[i] / (1 - beta2 ** t)
        params[i] = params[i] - lr * mh / (np.sqrt(vh) + eps)
    return params
