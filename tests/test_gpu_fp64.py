"""GPU float64 path against the CPU oracle (tolerance 1e-10 relative)."""

import json
import os

import numpy as np
import pytest

import oracle as O
from synth.instrument import random_problem
from tests.gpu_common import instrument, make_like, oracle_eval, oracle_pre, phis

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def P():
    import paper_2501_12928_gb300 as P
    return P


@pytest.mark.parametrize("dense", [True, False])
def test_precompute_C0(P, dense):
    lk = make_like(P, "C0", dense=dense)
    M, db = oracle_pre("C0", dense=True)
    Mg = lk.get_M()
    assert np.abs(Mg - M).max() <= 1e-13 * np.abs(M).max()
    assert np.abs(lk.get_dbar() - db).max() <= 1e-13 * np.abs(db).max()


def test_lnl_fp64_C0_golden(P):
    lk = make_like(P, "C0")
    with open(os.path.join(os.path.dirname(__file__), "golden", "c0_oracle.json")) as f:
        g = json.load(f)
    phi = np.array([r["phi"] for r in g["rows"]])
    ref = np.array([r["lnl"] for r in g["rows"]])
    got, st = lk.lnl(phi)
    assert np.all(st == 0)
    assert np.all(np.abs(got - ref) <= RTOL * np.abs(ref))
    t = lk.terms(len(phi))
    for key in ("logdet_phi", "logdet_sigma", "q"):
        r = np.array([row[key] for row in g["rows"]])
        assert np.all(np.abs(t[key] - r) <= RTOL * np.abs(r).max()), key


def test_lnl_fp64_C0_many(P):
    lk = make_like(P, "C0")
    ph = phis("C0", 64, stream=13)
    got, st = lk.lnl(ph)
    assert np.all(st == 0)
    for i in range(0, 64, 9):
        ref = oracle_eval("C0", ph[i])["lnl"]
        assert abs(got[i] - ref) <= RTOL * abs(ref)


def test_posterior_mean_fp64_C0(P):
    lk = make_like(P, "C0")
    ph = phis("C0", 2, stream=21)
    for p in ph:
        a, st = lk.posterior_mean(p)
        ref = oracle_eval("C0", p)["abar"]
        assert st == 0
        assert np.linalg.norm(a - ref) <= RTOL * np.linalg.norm(ref)


@pytest.mark.parametrize("nvis,n,nk", [(12, 5, 2), (300, 130, 3), (260, 256, 4), (400, 383, 5)])
def test_lnl_fp64_random_shapes(P, nvis, n, nk):
    p = random_problem(nvis, n, nk, seed=n)
    lk = P.Likelihood("fp64")
    lk.set_T(p["T"], p["kbin"], nk, 2.0)
    lk.set_data(p["d"], p["noise_var"])
    lk.precompute()
    M = O.herm_dense(p["T"], p["noise_var"])
    db = O.dbar_dense(p["T"], p["noise_var"], p["d"])
    ph = np.random.default_rng(n).uniform(-2, 2, (3, nk))
    got, st = lk.lnl(ph)
    for i in range(3):
        ref = O.evaluate(M, db, p["kbin"], ph[i], 2.0)["lnl"]
        assert st[i] == 0 and abs(got[i] - ref) <= RTOL * max(1.0, abs(ref))


def test_lnl_multi_uneven_fp64(P):
    a = make_like(P, "C0")
    small = ("C1", (("nu", 5), ("nf", 6), ("n_t", 2), ("n_bl", 20), ("n_pix", 16), ("n_k", 3)))
    b = make_like_small(P, small)
    pa = phis("C0", 3, stream=31)
    pb = np.random.default_rng(3).uniform(-2, 2, (2, 3))
    outs, sts = P.lnl_multi([a, b], [pa, pb])
    for i in range(3):
        ref = oracle_eval("C0", pa[i])["lnl"]
        assert sts[0][i] == 0 and abs(outs[0][i] - ref) <= RTOL * abs(ref)
    inst = instrument_small(small)
    M = O.herm_structured(inst.A, inst.W, inst.noise_var)
    db = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
    for i in range(2):
        ref = O.evaluate(M, db, inst.kbin, pb[i], inst.spec.lssm_prior_var)["lnl"]
        assert sts[1][i] == 0 and abs(outs[1][i] - ref) <= RTOL * abs(ref)


def instrument_small(small):
    from synth import build_instrument
    from synth.instrument import get_spec
    return build_instrument(get_spec(small[0], **dict(small[1])))


def make_like_small(P, small):
    inst = instrument_small(small)
    lk = P.Likelihood("fp64")
    lk.set_instrument(inst.A, inst.W, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
    lk.set_data(inst.d, inst.noise_var)
    lk.precompute()
    return lk


def test_errors(P):
    lk = P.Likelihood("fp64")
    with pytest.raises(P.BeorError):
        lk.precompute()                      # out of order
    inst = instrument("C0")
    bad = inst.kbin.copy()
    bad[0] = 99
    with pytest.raises(P.BeorError):
        lk.set_instrument(inst.A, inst.W, bad, inst.spec.n_k, 100.0)
    lk.set_instrument(inst.A, inst.W, inst.kbin, inst.spec.n_k, 100.0)
    with pytest.raises(P.BeorError):
        lk.set_data(inst.d, -inst.noise_var)
