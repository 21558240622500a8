"""Oracle of the lnL emulator network (float64).  TEST INFRASTRUCTURE ONLY.

A multilayer perceptron x -> (GELU hidden layers) -> scalar, the learned
part that pre-screens prior points for the nested sampler.  Exact GELU,
g(z) = z * Phi(z) with Phi the standard normal CDF; mean squared error loss in
normalised units, L = mean((y_net - (t - y_shift) / y_scale)^2).  Forward and
backward passes are written out layer by layer; pinned by finite differences
of the loss and by tabulated values of Phi.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    # d/dz [z Phi(z)] = Phi(z) + z phi(z)
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, x, x_shift, x_scale):
    """params: list of (W [out, in], b [out]).  Returns (y_net [n], cache)."""
    h = (np.asarray(x, np.float64) - x_shift) * x_scale
    hs, zs = [h], []
    for l, (W, b) in enumerate(params):
        z = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        zs.append(z)
        if l + 1 < len(params):
            h = gelu(z)
            hs.append(h)
    return zs[-1][:, 0], (hs, zs)


def loss_and_grads(params, x, t, x_shift, x_scale, y_shift, y_scale):
    """Mean squared error of the normalised output and its gradient for every
    (W, b).  Returns (loss, [(dW, db), ...])."""
    y, (hs, zs) = forward(params, x, x_shift, x_scale)
    n = y.shape[0]
    r = y - (np.asarray(t, np.float64) - y_shift) / y_scale
    loss = float(np.mean(r * r))
    dz = (2.0 * r / n)[:, None]                     # dL/dz of the output layer
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W = np.asarray(params[l][0], np.float64)
        grads[l] = (dz.T @ hs[l], dz.sum(axis=0))
        if l > 0:
            dh = dz @ W
            dz = dh * gelu_grad(zs[l - 1])
    return loss, grads
