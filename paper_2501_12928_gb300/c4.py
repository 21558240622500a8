"""Emulator-assisted nested sampling on the 3280-mode instrument (9 k bins).

    python -m paper_2501_12928_gb300.c4 [--n-train 200000] [--n-live 500] ...

1. exact lnL at n_train prior points phi ~ U[-2, 2]^9 (the library's batched
   mixed-precision path), timed;
2. the emulator (9 -> 4 x 256 GELU -> 1) trained on them by the library's
   kernels, timed, with its validation error;
3. seed-matched nested-sampling runs for each sampler seed: exact likelihood
   only, and with the emulator screen (static, or refit on the run's own
   exact evaluations); ln Z of both, the number of exact evaluations and wall
   times, and over the seeds the mean and spread of the ln Z difference and
   the exact-evaluation ratio.
Prints one JSON object (and writes it to --out when given).
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
    ap.add_argument("--seeds", type=int, default=1, help="seed pairs: sampler seeds seed, seed + 1, ...")
    ap.add_argument("--active", action="store_true", help="refit the screen on the run's exact evaluations")
    ap.add_argument("--every", type=int, default=50, help="active refit every this many screen calls")
    ap.add_argument("--refit-epochs", type=int, default=8)
    ap.add_argument("--max-train", type=int, default=60000, help="points per active refit")
    ap.add_argument("--config", default="C1")
    ap.add_argument("--out", default=None)
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

    t0 = time.perf_counter()
    model, info = train_emulator(phi, lnl, width=256, depth=4, epochs=args.epochs, batch=1024)
    out["emulator"] = {k: v for k, v in info.items() if k != "loss"}
    out["emulator"]["final_loss"] = info["loss"][-1]
    out["emulator_train_s"] = time.perf_counter() - t0
    res = []
    for sd in range(args.seed, args.seed + args.seeds):
        if args.active:
            r = compare_runs_active(exact, phi, lnl, inst.spec.n_k, n_live=args.n_live, k_remove=args.k_remove,
                                    batch=args.batch, seed=sd, every=args.every, max_train=args.max_train,
                                    initial=model, width=256, depth=4, epochs=args.refit_epochs,
                                    train_batch=1024)
        else:
            r = compare_runs(exact, model, inst.spec.n_k, delta_u=5.0 * model.rms_u, n_live=args.n_live,
                             k_remove=args.k_remove, batch=args.batch, seed=sd)
        r["seed"] = sd
        res.append(r)
        print(json.dumps({"seed": sd, "dlogz": r["dlogz"], "exact_eval_ratio": r["exact_eval_ratio"],
                          "n_exact": [r["exact"]["n_exact"], r["emulator"]["n_exact"]]}), flush=True)
        if args.out:   # the pairs so far, in case the run is cut short
            with open(args.out + ".partial", "w") as f:
                f.write(json.dumps({**out, "runs": res}, default=float) + "\n")
    d = np.array([r["dlogz"] for r in res])
    q = np.array([r["exact_eval_ratio"] for r in res])
    out["summary"] = {"pairs": len(res), "dlogz_mean": float(d.mean()), "dlogz_std": float(d.std()),
                      "dlogz_max_abs": float(np.abs(d).max()), "exact_eval_ratio_mean": float(q.mean()),
                      "exact_eval_ratio_max": float(q.max()), "fewer_in_every_pair": bool(np.all(q < 1.0)),
                      "logz_err_exact": [r["exact"]["logz_err"] for r in res]}
    out["runs"] = res
    out["n_flagged_total"] = exact.n_flagged
    text = json.dumps(out, default=float)
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")


if __name__ == "__main__":
    main()
