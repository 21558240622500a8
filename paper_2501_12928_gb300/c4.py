"""Emulator-assisted nested sampling on the 3280-mode instrument (9 k bins).

    python -m paper_2501_12928_gb300.c4 [--n-train 200000] [--n-live 500] ...

1. exact lnL at n_train prior points phi ~ U[-2, 2]^9 (the library's batched
   mixed-precision path), timed;
2. the emulator (9 -> 4 x 256 GELU -> 1) trained on them by the library's
   kernels, timed, with its validation error;
3. seed-matched nested-sampling runs: exact likelihood only, and with the
   emulator screen (static, or refit on the run's own exact evaluations);
   ln Z of both, the number of exact evaluations and wall times.
Prints one JSON object.
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-train", type=int, default=200_000)
    ap.add_argument("--n-live", type=int, default=500)
    ap.add_argument("--k-remove", type=int, default=32)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--active", action="store_true", help="refit the screen on the run's exact evaluations")
    ap.add_argument("--config", default="C1")
    args = ap.parse_args(argv)

    from synth import build_instrument
    from . import Likelihood
    from .emulated_sampler import ExactLikelihood, compare_runs, compare_runs_active, make_training_set, \
        train_emulator

    inst = build_instrument(args.config)
    lk = Likelihood("mixed")
    lk.set_instrument(inst.A, inst.W, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
    lk.set_data(inst.d, inst.noise_var)
    lk.precompute()
    # points the mixed path flags (status -1) are re-evaluated in float64
    fb = Likelihood("fp64")
    fb.set_instrument(inst.A, inst.W, inst.kbin, inst.spec.n_k, inst.spec.lssm_prior_var)
    fb.set_data(inst.d, inst.noise_var)
    fb.precompute()
    exact = ExactLikelihood(lk, max_batch=256, fallback=fb)
    out = {"config": args.config, "n_model": inst.spec.n_model, "n_k": inst.spec.n_k, "args": vars(args)}

    t0 = time.perf_counter()
    phi, lnl = make_training_set(exact, inst.spec.n_k, args.n_train, seed=17, batch=256)
    out["train_set_s"] = time.perf_counter() - t0
    out["exact_evals_per_s_B256"] = args.n_train / out["train_set_s"]

    if args.active:
        res = compare_runs_active(exact, phi, lnl, inst.spec.n_k, n_live=args.n_live, k_remove=args.k_remove,
                                  batch=args.batch, seed=args.seed, every=20, width=256, depth=4,
                                  epochs=args.epochs, train_batch=1024)
    else:
        model, info = train_emulator(phi, lnl, width=256, depth=4, epochs=args.epochs, batch=1024)
        out["emulator"] = {k: v for k, v in info.items() if k != "loss"}
        out["emulator"]["final_loss"] = info["loss"][-1]
        res = compare_runs(exact, model, inst.spec.n_k, delta_u=5.0 * model.rms_u, n_live=args.n_live,
                           k_remove=args.k_remove, batch=args.batch, seed=args.seed)
    out["runs"] = res
    out["n_flagged_total"] = exact.n_flagged
    print(json.dumps(out, default=float))


if __name__ == "__main__":
    main()
