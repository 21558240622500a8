"""The benchmark's own launch configuration at full size: three sub-band
instruments (N_model 6048 / 7840 / 11424), B = 16 each, one batched
evaluation (one beor_lnl_multi call).

Checked against the oracle, which evaluates one point of the largest
sub-band in about half a minute on the host:
* two sampled points of every sub-band, the 11,424-mode one included:
  mixed-precision |dlnL| <= 1e-2 (absolute);
* the posterior mean of one 11,424-mode point: relative error <= 1e-6;
* one 11,424-mode point on the float64 GPU path: relative error <= 1e-10.
Also: every sampled point against its own single-problem evaluation (batch
invariance), all statuses 0, and dbar of the largest instrument."""

import gc

import numpy as np
import pytest

import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NAMES = ("C3_24", "C3_32", "C3_48")
SAMPLED = (0, 15)


def _instruments():
    from synth import build_instrument
    insts = {"C3_48": build_instrument("C3_48")}
    for n in ("C3_24", "C3_32"):
        insts[n] = build_instrument(n, A_from=insts["C3_48"])
    return insts


def _like(P, inst, precision):
    lk = P.Likelihood(precision)
    lk.set_instrument(inst.A, inst.W, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
    lk.set_data(inst.d, inst.noise_var)
    lk.precompute()
    return lk


def test_c3_batched_launch_oracle_parity():
    import paper_2501_12928_gb300 as P
    from synth import draw_phi

    insts = _instruments()
    likes = [_like(P, insts[n], "mixed") for n in NAMES]
    phis = [draw_phi(insts[n].spec, 16) for n in NAMES]
    outs, sts = P.lnl_multi(likes, phis)
    for s in sts:
        assert np.all(s == 0), s
    # batch invariance: the same point alone gives the same lnL (the float64
    # refinement residual sums with atomics, so only to within its rounding)
    for s, (lk, ph) in enumerate(zip(likes, phis)):
        for b in SAMPLED:
            single, st = lk.lnl(ph[b:b + 1])
            assert st[0] == 0
            assert abs(single[0] - outs[s][b]) <= 1e-3, (s, b, single[0], outs[s][b])

    # the oracle on sampled points of every sub-band, one sub-band at a time
    big = NAMES.index("C3_48")
    abar_gpu, st = likes[big].posterior_mean(phis[big][0])
    assert st == 0
    lf = _like(P, insts["C3_48"], "fp64")
    f64, fst = lf.lnl(phis[big][:1])
    assert fst[0] == 0
    lf.close()
    report = {}
    for s, n in enumerate(NAMES):
        inst = insts[n]
        M = O.herm_structured(inst.A, inst.W, inst.noise_var)
        db = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
        if n == "C3_48":
            dbg = likes[s].get_dbar()
            assert np.abs(dbg - db).max() <= 1e-12 * np.abs(db).max()
        for b in SAMPLED:
            ref = O.evaluate(M, db, inst.kbin, phis[s][b], inst.spec.lssm_prior_var)
            err = abs(outs[s][b] - ref["lnl"])
            report[(n, b)] = err
            print(f"{n} (N_model {inst.spec.n_model}) point {b}: |dlnL| = {err:.3e}")
            assert err <= 1e-2, (n, b, err)
            if n == "C3_48" and b == 0:
                a_ref = ref["abar"]
                rel = np.linalg.norm(abar_gpu - a_ref) / np.linalg.norm(a_ref)
                print(f"C3_48 posterior mean: relative error {rel:.3e}")
                assert rel <= 1e-6, rel
                rel64 = abs(f64[0] - ref["lnl"]) / abs(ref["lnl"])
                print(f"C3_48 float64 GPU: relative error {rel64:.3e}")
                assert rel64 <= 1e-10, rel64
        del M, db
        gc.collect()
    assert len(report) == 2 * len(NAMES)
