"""Separate EoR and foreground fields of view on the GPU (`synth/fov2.py`:
the foreground model on a uv grid of half the cell size, i.e. twice the
EoR FoV): the library's lnL and posterior mean from the dense T against the
oracle (mixed and float64 paths), and the evidence-based comparison with
the single-FoV model on data drawn from the wide-FoV model: nested sampling
on the exact GPU likelihood of each model gives ln K = ln Z_wide - ln Z_single
far above 0 (the oracle's lnL difference at the same points is ~260)."""

import numpy as np
import pytest

import oracle as O
from synth import draw_phi
from synth.fov2 import build_fov2, single_fov_T

pytestmark = pytest.mark.gpu


def _like(P, inst, T, precision):
    lk = P.Likelihood(precision)
    lk.set_T(T, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
    lk.set_data(inst.d, inst.noise_var)
    lk.precompute()
    return lk


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_two_fov_lnl_and_posterior_mean_match_the_oracle(precision):
    import paper_2501_12928_gb300 as P

    inst = build_fov2("C0", 2.0)
    lv = inst.spec.lssm_prior_var
    M, db = O.herm_dense(inst.T, inst.noise_var), O.dbar_dense(inst.T, inst.noise_var, inst.d)
    ph = draw_phi(inst.spec, 16, stream=7)
    lk = _like(P, inst, inst.T, precision)
    got, st = lk.lnl(ph)
    assert np.all(st == 0), st
    refs = [O.evaluate(M, db, inst.kbin, p, lv) for p in ph]
    ref = np.array([r["lnl"] for r in refs])
    if precision == "mixed":
        assert np.abs(got - ref).max() <= 1e-2, np.abs(got - ref).max()
    else:
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    a, sa = lk.posterior_mean(ph[0])
    assert sa == 0
    assert np.linalg.norm(a - refs[0]["abar"]) <= 1e-6 * np.linalg.norm(refs[0]["abar"])
    lk.close()


def test_evidence_prefers_the_wide_foreground_fov():
    import paper_2501_12928_gb300 as P
    from paper_2501_12928_gb300.emulated_sampler import ExactLikelihood
    from paper_2501_12928_gb300.ns import NestedSampler
    from paper_2501_12928_gb300.posterior import log_bayes_factor

    inst = build_fov2("C0", 2.0)
    logz = {}
    for name, T in (("wide", inst.T), ("single", single_fov_T(inst))):
        lk = _like(P, inst, T, "mixed")
        res = NestedSampler(ExactLikelihood(lk, max_batch=256), inst.spec.n_k, n_live=100, k_remove=8,
                            batch=64, seed=3).run()
        logz[name] = (res.logz, res.logz_err)
        lk.close()
    lnk = log_bayes_factor(logz["wide"][0], logz["single"][0])
    print("ln K (wide foreground FoV vs single FoV)", lnk, logz)
    assert lnk > 100.0
