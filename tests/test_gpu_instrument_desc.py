"""The instrument built by the library from its geometry
(beor_set_instrument_desc) against the same instrument passed as arrays
(beor_set_instrument, arrays from the seeded input builder): the precompute
of both must agree (M and dbar to float64 rounding), and so must lnL on the
float64 path, which also requires identical k-bin maps."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [("C0", {}), ("C1", {}),
         # a sub-band on its band's grid (nf_grid > nf), kept small
         ("C3_24", {"nu": 5, "n_bl": 40, "n_t": 2, "n_pix": 16})]


@pytest.mark.parametrize("name,over", CASES)
def test_descriptor_matches_arrays(name, over):
    import paper_2501_12928_gb300 as P
    from synth import build_instrument, draw_phi, geometry, get_spec

    inst = build_instrument(get_spec(name, **over))
    a = P.Likelihood("fp64")
    a.set_instrument(inst.A, inst.W, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
    a.set_data(inst.d, inst.noise_var)
    a.precompute()
    b = P.Likelihood("fp64")
    b.set_instrument_desc(geometry(inst))
    b.set_data(inst.d, inst.noise_var)
    b.precompute()
    assert b.dims() == a.dims()
    Ma, Mb = a.get_M(), b.get_M()
    assert np.abs(Mb - Ma).max() <= 1e-11 * np.abs(Ma).max()
    da, db = a.get_dbar(), b.get_dbar()
    assert np.abs(db - da).max() <= 1e-11 * np.abs(da).max()
    ph = draw_phi(inst.spec, 4)
    la, sa = a.lnl(ph)
    lb, sb = b.lnl(ph)
    assert np.all(sa == 0) and np.all(sb == 0)
    assert np.abs(lb - la).max() <= 1e-9 * np.abs(la).max()
    a.close()
    b.close()


def test_descriptor_rejects_bad_geometry():
    import paper_2501_12928_gb300 as P
    from synth import build_instrument, geometry

    g = geometry(build_instrument("C0"))
    lk = P.Likelihood("fp64")
    for bad in ({"nu": 4}, {"n_pix": 1}, {"f0_hz": -1.0}, {"beam_fwhm_rad": 0.0}, {"n_k": 0},
                {"bl_enu_m": np.zeros((3, 3))}):
        with pytest.raises(P.BeorError):
            lk.set_instrument_desc({**g, **bad})
    lk.close()
