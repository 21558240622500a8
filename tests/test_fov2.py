"""The two-field-of-view instrument (separate EoR and foreground model FoVs,
`synth/fov2.py`), checked on the CPU:

* with the foreground FoV equal to the EoR one (s = 1, nu_fg = nu) its dense
  T is the single-FoV instrument's T with the columns reordered (EoR block
  first) and the same k-bin map: the new builder adds nothing else;
* with a wider foreground FoV the EoR block is unchanged and the foreground
  block is not;
* on data drawn from the wide-FoV model, the oracle's lnL prefers the model
  that has the wide foreground FoV over the single-FoV model by a large
  margin at every sampled phi (the model comparison the separate FoVs are
  for; the Bayes factor of the evidences follows on the GPU).
"""

import numpy as np

import oracle as O
from synth import build_instrument, draw_phi, expand_T
from synth.fov2 import build_fov2, single_fov_T


def test_equal_fovs_reduce_to_the_single_fov_instrument():
    i1 = build_fov2("C0", 1.0, with_data=False)
    inst = build_instrument("C0", with_data=False)
    T0 = expand_T(inst)
    sp = inst.spec
    perm = ([c * sp.n_x + x for c in range(sp.n_cells) for x in range(sp.nf)] +
            [c * sp.n_x + sp.nf + y for c in range(sp.n_cells) for y in range(sp.n_lssm)])
    np.testing.assert_array_equal(i1.T, T0[:, perm])
    np.testing.assert_array_equal(i1.kbin, inst.kbin[perm])
    assert i1.n_eor == sp.n_cells * sp.nf


def test_wide_foreground_fov_changes_only_the_foreground_block():
    i1 = build_fov2("C0", 1.0, with_data=False)
    i2 = build_fov2("C0", 2.0, with_data=False)
    ne = i1.n_eor
    np.testing.assert_array_equal(i2.T[:, :ne], i1.T[:, :ne])
    assert i2.T.shape == i1.T.shape
    assert np.abs(i2.T[:, ne:] - i1.T[:, ne:]).max() > 0.1 * np.abs(i1.T[:, ne:]).max()


def test_oracle_prefers_the_wide_foreground_fov_on_wide_field_data():
    inst = build_fov2("C0", 2.0)
    T1 = single_fov_T(inst)
    lv = inst.spec.lssm_prior_var
    pre = [(O.herm_dense(T, inst.noise_var), O.dbar_dense(T, inst.noise_var, inst.d)) for T in (inst.T, T1)]
    phis = np.concatenate([np.log10(inst.extra["pk_true"])[None], draw_phi(inst.spec, 4)])
    for p in phis:
        l2, l1 = (O.evaluate(M, db, inst.kbin, p, lv)["lnl"] for M, db in pre)
        assert l2 - l1 > 100.0, (p, l2 - l1)
