"""The benchmark's own launch configuration at full size: three sub-band
instruments (N_model 6048 / 7840 / 11424), B = 16 each, one batched
evaluation.  Sampled outputs are checked against the oracle (one point of
the 6048-mode sub-band, which the oracle evaluates in seconds) and every
sampled point against its own single-problem evaluation (batch invariance);
all statuses must be 0."""

import numpy as np
import pytest

import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_c3_batched_launch_sampled_parity():
    import paper_2501_12928_gb300 as P
    from synth import build_instrument, draw_phi

    insts = {"C3_48": build_instrument("C3_48")}
    for n in ("C3_24", "C3_32"):
        insts[n] = build_instrument(n, A_from=insts["C3_48"])
    names = ("C3_24", "C3_32", "C3_48")
    likes, phis = [], []
    for n in names:
        lk = P.Likelihood("mixed")
        inst = insts[n]
        lk.set_instrument(inst.A, inst.W, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
        lk.set_data(inst.d, inst.noise_var)
        lk.precompute()
        likes.append(lk)
        phis.append(draw_phi(inst.spec, 16))
    outs, sts = P.lnl_multi(likes, phis)
    for s in sts:
        assert np.all(s == 0), s
    # batch invariance: the same point alone gives the same lnL (the float64
    # refinement residual sums with atomics, so only to within its rounding)
    for s, (lk, ph) in enumerate(zip(likes, phis)):
        for b in (0, 15):
            single, st = lk.lnl(ph[b:b + 1])
            assert st[0] == 0
            assert abs(single[0] - outs[s][b]) <= 1e-3, (s, b, single[0], outs[s][b])
    # the oracle on one point of the 6048-mode sub-band
    inst = insts["C3_24"]
    M = O.herm_structured(inst.A, inst.W, inst.noise_var)
    db = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
    ref = O.evaluate(M, db, inst.kbin, phis[0][0], inst.spec.lssm_prior_var)
    print("C3_24 |dlnL|", abs(outs[0][0] - ref["lnl"]))
    assert abs(outs[0][0] - ref["lnl"]) <= 1e-2
    # dbar of the largest instrument against the oracle's factored formula (sampled entries)
    dbg = likes[2].get_dbar()
    inst = insts["C3_48"]
    dref = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
    assert np.abs(dbg - dref).max() <= 1e-12 * np.abs(dref).max()
