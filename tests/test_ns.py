"""Nested sampler on analytic toys (CPU): evidence against closed forms,
seed-matched emulator screening, and checkpoint/resume."""

import math
import os

import numpy as np
from scipy.special import erf

from paper_2501_12928_gb300.ns import NestedSampler

MU = np.array([0.3, -0.5, 0.1, 0.7, -1.0, 0.0, 0.4, -0.2, 1.1])
S = 0.5


def gauss9(x):
    return -0.5 * np.sum((np.atleast_2d(x) - MU) ** 2, axis=1) / S ** 2


def gauss9_logz():
    # Z = prod_d (1/4) int_{-2}^{2} exp(-(x - mu_d)^2 / (2 s^2)) dx
    a = S * math.sqrt(math.pi / 2) * (erf((2 - MU) / (S * math.sqrt(2))) + erf((2 + MU) / (S * math.sqrt(2))))
    return float(np.sum(np.log(a / 4.0)))


def test_gaussian_9d_evidence():
    ns = NestedSampler(gauss9, 9, n_live=300, batch=16, seed=11)
    r = ns.run()
    ref = gauss9_logz()
    assert abs(r.logz - ref) <= 3 * r.logz_err + 0.05, (r.logz, ref, r.logz_err)
    # posterior mean close to MU (box truncation is negligible at 2/0.5 = 4 sigma... except dim 5)
    xs, w = r.posterior()
    mean = (xs * w[:, None]).sum(axis=0)
    assert np.abs(mean[:4] - MU[:4]).max() < 0.15


def bimodal(x):
    x = np.atleast_2d(x)
    a = -0.5 * np.sum((x - np.array([-1.0, -1.0])) ** 2, axis=1) / 0.2 ** 2
    b = -0.5 * np.sum((x - np.array([1.2, 0.8])) ** 2, axis=1) / 0.3 ** 2 + math.log(0.5)
    return np.logaddexp(a, b)


def test_bimodal_2d_evidence():
    # Z = (1/16) [2 pi 0.2^2 + 0.5 * 2 pi 0.3^2] (both modes well inside the box)
    ref = math.log((2 * math.pi * 0.04 + 0.5 * 2 * math.pi * 0.09) / 16.0)
    vals = []
    for seed in (1, 2, 3):
        r = NestedSampler(bimodal, 2, n_live=400, batch=16, seed=seed).run()
        vals.append(r.logz)
        assert abs(r.logz - ref) <= 4 * r.logz_err + 0.05, (r.logz, ref, r.logz_err)
    assert abs(np.mean(vals) - ref) <= 0.1


def test_screen_seed_matched_is_identical_and_cheaper():
    a = NestedSampler(gauss9, 9, n_live=150, batch=32, k_remove=4, seed=7).run()
    # a perfect screen (the likelihood itself) never rejects an acceptable point
    b = NestedSampler(gauss9, 9, n_live=150, batch=32, k_remove=4, seed=7, screen=gauss9, screen_delta=0.0).run()
    assert a.n_iter == b.n_iter
    assert abs(a.logz - b.logz) < 1e-12
    assert b.n_exact < 0.5 * a.n_exact, (a.n_exact, b.n_exact)


def test_checkpoint_resume(tmp_path):
    ck = os.path.join(tmp_path, "ns")
    full = NestedSampler(gauss9, 9, n_live=100, batch=16, seed=3).run()
    part = NestedSampler(gauss9, 9, n_live=100, batch=16, seed=3, checkpoint=ck)
    assert part.run(stop_after=120) is None
    resumed = NestedSampler(gauss9, 9, n_live=100, batch=16, seed=999, checkpoint=ck).run(resume=True)
    assert resumed.n_iter == full.n_iter
    assert abs(resumed.logz - full.logz) < 1e-9
    assert resumed.n_exact == full.n_exact


def test_adaptive_screen_is_ticked_on_every_block():
    """An adaptive screen must hear of every candidate block, also while L_min
    is above its support limit (else it could never move that limit)."""
    import math

    from paper_2501_12928_gb300.ns import NestedSampler

    class Owner:
        def __init__(self):
            self.ticks = 0
            self.support_limit = -math.inf     # never consulted

        def tick(self):
            self.ticks += 1

    calls = []

    def loglike(x):
        calls.append(len(x))
        return -0.5 * np.sum(np.asarray(x) ** 2, axis=1)

    owner = Owner()
    ns = NestedSampler(loglike, 2, n_live=40, k_remove=4, batch=16, seed=3, screen=lambda c: np.zeros(len(c)),
                       max_iter=30)
    ns._screen_owner = owner
    ns.run()
    blocks = len(calls) - math.ceil(40 / 16)     # the initial live points come in ceil(40/16) calls
    assert owner.ticks == blocks > 0
    assert ns.n_screened == 0
