"""Power-spectrum posterior products from a nested-sampling run.

The sampler's parameters are the per-k-bin power-spectrum coefficients
phi_i (log10 of the prior variance of the EoR amplitudes in bin i, Fig. 1
caption).  From the weighted posterior samples this module gives, per bin:

* the posterior of phi_i (weighted mean, standard deviation, quantiles);
* P(k_i) = 10^phi_i and the dimensionless power
  Delta^2(k_i) = k_i^3 P(k_i) / (2 pi^2) (Sec. "Statement of need", the
  equation after the spherical average P(k_i)), each with quantiles;
* a check of an injected spectrum against those intervals;
* Bayes factors between models from their evidences (Sec. "Summary": the
  evidence makes the package usable for model selection), including a
  point-null model whose evidence is its likelihood at one parameter value.

k is in whatever units the caller's bin centres use (the synthetic
instruments use uv-eta grid units).  Host-side post-processing of sampler
output: no likelihood arithmetic happens here.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def weighted_quantiles(x, w, qs):
    """Quantiles of the distribution placing weight w_i on x_i.

    Midpoint rule: the sorted x_(j) sits at cumulative probability
    sum_{i<j} w_(i) + w_(j)/2 (weights normalised), and quantiles are read
    off by linear interpolation, clamped to the extreme samples.  With equal
    weights this is the (i - 1/2)/n ("Hazen") plotting position.
    """
    x = np.asarray(x, float)
    w = np.asarray(w, float)
    if x.ndim != 1 or x.shape != w.shape or len(x) == 0:
        raise ValueError("x and w must be non-empty 1-D arrays of equal length")
    if np.any(w < 0) or not np.isfinite(w).all() or w.sum() <= 0:
        raise ValueError("weights must be finite, non-negative and not all zero")
    order = np.argsort(x, kind="stable")
    xs, ws = x[order], w[order] / w.sum()
    pos = np.cumsum(ws) - 0.5 * ws
    return np.interp(np.asarray(qs, float), pos, xs)


def delta_squared(k, p):
    """Dimensionless power Delta^2(k) = k^3 P(k) / (2 pi^2)."""
    k = np.asarray(k, float)
    return k ** 3 * np.asarray(p, float) / (2.0 * math.pi ** 2)


@dataclass
class BinSummary:
    k: float
    phi_mean: float
    phi_std: float
    phi_q: np.ndarray       # quantiles of phi at `qs`
    p_q: np.ndarray         # quantiles of P(k) = 10^phi
    delta2_q: np.ndarray    # quantiles of Delta^2(k)


def power_spectrum_posterior(samples, weights, k_centres, qs=(0.16, 0.5, 0.84)):
    """Per-bin posterior summaries.  samples: (n, n_k) phi values, weights:
    (n,) posterior weights (any positive scale), k_centres: (n_k,)."""
    s = np.asarray(samples, float)
    w = np.asarray(weights, float)
    k_centres = np.asarray(k_centres, float)
    if s.ndim != 2 or s.shape[1] != len(k_centres) or s.shape[0] != len(w):
        raise ValueError("samples must be (n, n_k) with n weights and n_k bin centres")
    wn = w / w.sum()
    out = []
    for i, k in enumerate(k_centres):
        x = s[:, i]
        mean = float(np.sum(wn * x))
        std = float(math.sqrt(max(np.sum(wn * (x - mean) ** 2), 0.0)))
        phq = weighted_quantiles(x, wn, qs)
        pq = 10.0 ** phq                                  # monotone map: quantiles carry over
        out.append(BinSummary(k=float(k), phi_mean=mean, phi_std=std, phi_q=phq, p_q=pq,
                              delta2_q=delta_squared(k, pq)))
    return out


def injected_within(summary, phi_true, n_sigma=4.0):
    """Per bin: |posterior mean - phi_true| <= n_sigma * posterior std (with
    a floor of 0.05 in phi for bins the data pin down very tightly)."""
    phi_true = np.asarray(phi_true, float)
    return np.array([abs(b.phi_mean - t) <= n_sigma * max(b.phi_std, 0.05) for b, t in zip(summary, phi_true)])


def format_table(summary, qs=(0.16, 0.5, 0.84)):
    lines = [f"{'k':>10} {'phi mean':>9} {'phi std':>8}  P(k) [{qs[0]:.2f}, {qs[1]:.2f}, {qs[2]:.2f}]"
             f"   Delta^2 [{qs[0]:.2f}, {qs[1]:.2f}, {qs[2]:.2f}]"]
    for b in summary:
        lines.append(f"{b.k:10.4g} {b.phi_mean:9.4f} {b.phi_std:8.4f}  "
                     + " ".join(f"{v:.4g}" for v in b.p_q) + "   "
                     + " ".join(f"{v:.4g}" for v in b.delta2_q))
    return "\n".join(lines)


def log_bayes_factor(logz_a: float, logz_b: float) -> float:
    """ln K = ln Z_a - ln Z_b: K > 1 favours model a."""
    return float(logz_a) - float(logz_b)


def point_null_logz(loglike, phi) -> float:
    """Evidence of a model with no free parameters (phi fixed): Z = L(phi)."""
    return float(np.asarray(loglike(np.atleast_2d(np.asarray(phi, float))), float)[0])
