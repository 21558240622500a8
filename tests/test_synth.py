"""Checks of the seeded synthetic inputs (shapes and binning of the workloads)."""

import numpy as np
import pytest

from synth import CONFIGS, build_instrument, draw_phi, expand_T
from synth.instrument import apply_T


@pytest.mark.parametrize("name,n_model,n_vis", [
    ("C0", 240, 240), ("C1", 3280, 90972),
    ("C3_24", 6048, 127104), ("C3_32", 7840, 169472), ("C3_48", 11424, 254208)])
def test_config_dimensions(name, n_model, n_vis):
    s = CONFIGS[name]
    assert s.n_model == n_model and s.n_vis == n_vis


def test_kbin_shells_C0():
    inst = build_instrument("C0")
    e = inst.k_edges
    eor = inst.kbin >= 0
    k = inst.k_mag[eor]
    b = inst.kbin[eor]
    # k_i <= |k| < k_{i+1}, the largest |k| closing the last shell
    assert np.all(k >= e[b] - 1e-12)
    last = b == len(e) - 2
    assert np.all(k[~last] < e[b[~last] + 1])
    assert np.all(np.bincount(b, minlength=len(e) - 1) > 0)
    # 24 cells x 8 eta modes are EoR, 24 x 2 foreground
    assert eor.sum() == 192 and (~eor).sum() == 48


def test_seeded_and_consistent():
    a = build_instrument("C0")
    b = build_instrument("C0")
    assert np.array_equal(a.d, b.d) and np.array_equal(a.A, b.A)
    T = expand_T(a)
    assert np.allclose(T @ a.a_true, apply_T(a, a.a_true), rtol=0, atol=1e-12 * np.abs(T).max())
    ph = draw_phi("C0", 5)
    assert ph.shape == (5, 4) and ph.min() >= -2 and ph.max() <= 2
    # SNR 10 by construction
    v = apply_T(a, a.a_true)
    assert abs(np.sqrt(np.mean(np.abs(v) ** 2)) / a.sigma - 10.0) < 1e-9


def test_golden_c0_reproduced():
    import json
    import os

    import oracle as O
    with open(os.path.join(os.path.dirname(__file__), "golden", "c0_oracle.json")) as f:
        g = json.load(f)
    inst = build_instrument("C0")
    M = O.herm_structured(inst.A, inst.W, inst.noise_var)
    db = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
    for row in g["rows"][:4]:
        r = O.evaluate(M, db, inst.kbin, np.array(row["phi"]), inst.spec.lssm_prior_var)
        assert abs(r["lnl"] - row["lnl"]) <= 1e-12 * abs(row["lnl"])
