"""Emulator-assisted nested sampling on the 240-mode instrument (GPU): the
emulator is trained on exact GPU likelihoods, then seed-matched runs with and
without its screen must agree in ln Z (within 0.1) while the screened run
uses fewer exact evaluations."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_emulator_screen_saves_exact_evaluations():
    import paper_2501_12928_gb300 as P
    from paper_2501_12928_gb300.emulated_sampler import (ExactLikelihood, compare_runs, make_training_set,
                                                         train_emulator)
    from tests.gpu_common import make_like

    lk = make_like(P, "C0", precision="mixed")
    exact = ExactLikelihood(lk, max_batch=256)
    phi, lnl = make_training_set(exact, 4, 8192, seed=17)
    model, info = train_emulator(phi, lnl, width=128, depth=3, epochs=40, batch=512)
    print("emulator", info["rms_u_all"], info["rms_u_top"], info["train_s"])
    out = compare_runs(exact, model, 4, delta_u=5.0 * model.rms_u, n_live=100, k_remove=8, batch=64, seed=5)
    print(out)
    assert abs(out["dlogz"]) <= 0.1
    assert out["emulator"]["n_exact"] < out["exact"]["n_exact"]


def test_active_emulator_screen():
    """Refitting the emulator on the sampler's own exact evaluations extends
    the screen's support up the likelihood; ln Z still matches the exact run."""
    import paper_2501_12928_gb300 as P
    from paper_2501_12928_gb300.emulated_sampler import ExactLikelihood, compare_runs_active, make_training_set
    from tests.gpu_common import make_like

    lk = make_like(P, "C0", precision="mixed")
    exact = ExactLikelihood(lk, max_batch=256)
    phi, lnl = make_training_set(exact, 4, 8192, seed=17)
    out = compare_runs_active(exact, phi, lnl, 4, n_live=100, k_remove=8, batch=64, seed=5, every=10,
                              width=128, depth=3, epochs=30, train_batch=512)
    print(out)
    assert abs(out["dlogz"]) <= 0.1
    assert out["emulator"]["n_exact"] < out["exact"]["n_exact"]
