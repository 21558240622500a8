"""Emulator-assisted nested sampling of the power-spectrum posterior.

The exact likelihood (the library's batched GPU path) generates the training
set of the emulator and judges every point the sampler accepts; the emulator
(library kernels) only screens candidates.  `compare_runs` runs the sampler
twice with the same seed -- exact likelihood only, and with the emulator
screen -- so that both see the same candidate sequence; their evidences agree
unless the screen rejects a candidate the exact run would have accepted, and
the second run needs fewer exact evaluations.
"""

from __future__ import annotations

import math
import time

import numpy as np

from .beor import Emulator, Likelihood
from .ns import NestedSampler


def _pow2_pad(blk):
    """blk padded to the next power of two by repeating its last row."""
    b = 1
    while b < len(blk):
        b *= 2
    return np.concatenate([blk, np.repeat(blk[-1:], b - len(blk), axis=0)]) if b > len(blk) else blk


class ExactLikelihood:
    """Batched exact lnL(phi) through the C ABI.  Batches are padded to powers
    of two (one captured graph per size); padding rows are not counted.  With
    `record` set, every evaluated (phi, lnL) pair is kept (training data).

    Per-point status: a failed pivot (status > 0) or a non-finite phi
    (status -2) gives lnL = -inf.  A mixed-precision result flagged as
    possibly outside its tolerance (status -1) is not used as it stands:
    it is re-evaluated on `fallback` (a float64 Likelihood of the same
    instrument) when one is given, else rejected (-inf), so that no flagged
    value becomes an accepted point, a training label or an evidence term.
    `n_flagged` counts such points and `n_fallback` those re-evaluated."""

    def __init__(self, like: Likelihood, max_batch: int = 256, fallback: Likelihood | None = None):
        self.like = like
        self.fallback = fallback
        self.max_batch = max_batch
        self.n_calls = 0
        self.n_points = 0
        self.n_flagged = 0
        self.n_fallback = 0
        self.record = False
        self.rec_x, self.rec_l = [], []

    def _fallback(self, phi):
        out = np.full(len(phi), -np.inf)
        for i in range(0, len(phi), self.max_batch):
            blk = phi[i:i + self.max_batch]
            l, st = self.fallback.lnl(_pow2_pad(blk))
            out[i:i + len(blk)] = np.where(st[: len(blk)] != 0, -np.inf, l[: len(blk)])
        self.n_fallback += len(phi)
        return out

    def __call__(self, x):
        x = np.atleast_2d(np.asarray(x, np.float64))
        out = np.empty(len(x))
        for i in range(0, len(x), self.max_batch):
            blk = x[i:i + self.max_batch]
            l, st = self.like.lnl(_pow2_pad(blk))
            st = np.asarray(st[: len(blk)])
            l = np.where((st > 0) | (st == -2), -np.inf, l[: len(blk)])
            flagged = np.flatnonzero(st == -1)
            if len(flagged):
                self.n_flagged += len(flagged)
                l[flagged] = self._fallback(blk[flagged]) if self.fallback is not None else -np.inf
            out[i:i + len(blk)] = l
            self.n_calls += 1
            self.n_points += len(blk)
        if self.record:
            self.rec_x.append(x.copy())
            self.rec_l.append(out.copy())
        return out


def make_training_set(exact: ExactLikelihood, n_k: int, n: int, seed: int, lo=-2.0, hi=2.0, batch=256):
    g = np.random.Generator(np.random.PCG64(seed))
    phi = g.uniform(lo, hi, (n, n_k))
    lnl = np.concatenate([exact(phi[i:i + batch]) for i in range(0, n, batch)])
    return phi, lnl


class ScreenModel:
    """The emulator and its target transform.  The network learns
    u = log(1 + max(lnL_ref - lnL, 0)), the depth below the best training
    value on a log scale: bf16 activations carry about 3 significant digits,
    so the transform spends them near the peak, where the sampler's
    threshold lies, instead of across the whole prior range of lnL."""

    def __init__(self, em: Emulator, lnl_ref: float, rms_u: float, support_limit: float):
        self.em = em
        self.lnl_ref = lnl_ref
        self.rms_u = rms_u
        # thresholds above this (the 99th percentile of the training lnL) lie where
        # the training set has almost no points; the sampler stops screening there
        self.support_limit = support_limit

    def u_of(self, lnl):
        return np.log1p(np.maximum(self.lnl_ref - np.asarray(lnl, np.float64), 0.0))

    def predict_u(self, phi):
        return self.em.infer(np.asarray(phi, np.float32)).astype(np.float64)

    def screen(self, delta_u: float):
        """Callable for the sampler: a predicted lnL that is below the
        threshold exactly when the predicted depth exceeds the threshold's
        depth by more than delta_u.  Where the prediction (less the margin)
        reaches the best training value the network knows nothing more, so
        the point is never rejected (+inf)."""
        def f(phi):
            u = self.predict_u(phi) - delta_u
            return np.where(u > 0.0, self.lnl_ref - np.expm1(np.maximum(u, 0.0)), np.inf)
        return f


def train_emulator(phi, lnl, width=256, depth=4, seed=4, epochs=60, batch=1024, lr=1e-3, val_frac=0.1,
                   lo=-2.0, hi=2.0, device=0):
    """Fit the MLP to u(phi) (see ScreenModel); inputs mapped to [-1, 1];
    Adam with a cosine learning rate; 90/10 train/validation split.  Returns
    (ScreenModel, training log); rms_u is the validation RMS error of u over
    the best fifth of the validation points."""
    n, n_in = phi.shape
    g = np.random.Generator(np.random.PCG64(seed))
    perm = g.permutation(n)
    nv = max(1, int(val_frac * n))
    vi, ti = perm[:nv], perm[nv:]
    lnl_ref = float(np.max(lnl[ti]))
    u = np.log1p(np.maximum(lnl_ref - lnl, 0.0))
    em = Emulator(n_in, width, depth, seed=seed, device=device)
    mid = 0.5 * (lo + hi)
    em.set_norm(np.full(n_in, mid, np.float32), np.full(n_in, 2.0 / (hi - lo), np.float32),
                float(u[ti].mean()), float(u[ti].std() + 1e-12))
    xt, yt = phi[ti].astype(np.float32), u[ti].astype(np.float32)
    steps = epochs * max(1, len(ti) // batch)
    step = 0
    log = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = g.permutation(len(ti))
        for i in range(0, len(ti) - batch + 1, batch):
            sel = order[i:i + batch]
            lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * step / steps))
            loss = em.train_step(xt[sel], yt[sel], max(lr_t, 1e-6))
            step += 1
        log.append(loss)
    train_s = time.perf_counter() - t0
    pred = em.infer(phi[vi].astype(np.float32)).astype(np.float64)
    err = pred - u[vi]
    top = u[vi] <= np.quantile(u[vi], 0.2)
    rms_top = float(np.sqrt(np.mean(err[top] ** 2)))
    rms_all = float(np.sqrt(np.mean(err ** 2)))
    model = ScreenModel(em, lnl_ref, rms_top, float(np.quantile(lnl[ti], 0.99)))
    return model, {"loss": log, "train_s": train_s, "rms_u_all": rms_all, "rms_u_top": rms_top, "steps": step,
                   "n_train": len(ti), "n_val": nv, "lnl_ref": lnl_ref}


class ActiveScreen:
    """Emulator screen refit every `every` candidate blocks of the sampler
    (tick(), called for every block, screened or not, so that the support
    limit keeps up with L_min) on the exact evaluations so far, so that its
    support follows the run: the sampler's own evaluations
    (which concentrate in the shrinking constrained region; the most recent
    ones first) and a random part of the initial set, `max_train` points in
    all.  `initial` is a ScreenModel to start from (not closed here); the
    screen's own refits are."""

    def __init__(self, exact: ExactLikelihood, phi0, lnl0, every=20, n_sigma=5.0, max_train=None, initial=None,
                 seed=0, **train_kw):
        self.exact = exact
        self.phi0, self.lnl0 = phi0, lnl0
        self.run_phi, self.run_lnl = [], []
        self.every = every
        self.n_sigma = n_sigma
        self.max_train = max_train
        self.train_kw = train_kw
        self.rng = np.random.Generator(np.random.PCG64(seed))
        self.calls = 0
        self.refits = 0
        self.refit_s = 0.0
        self.model = initial
        self.own = False
        if initial is None:
            self._refit()

    def _training_set(self):
        if self.exact.rec_x:
            self.run_phi.append(np.concatenate(self.exact.rec_x))
            self.run_lnl.append(np.concatenate(self.exact.rec_l))
            self.exact.rec_x, self.exact.rec_l = [], []
        rp = np.concatenate(self.run_phi) if self.run_phi else np.zeros((0, self.phi0.shape[1]))
        rl = np.concatenate(self.run_lnl) if self.run_lnl else np.zeros(0)
        if self.max_train is None:
            return np.concatenate([self.phi0, rp]), np.concatenate([self.lnl0, rl])
        keep_run = min(len(rl), (2 * self.max_train) // 3)
        rp, rl = rp[len(rl) - keep_run:], rl[len(rl) - keep_run:]
        n0 = min(len(self.lnl0), self.max_train - keep_run)
        pick = self.rng.choice(len(self.lnl0), n0, replace=False)
        return np.concatenate([self.phi0[pick], rp]), np.concatenate([self.lnl0[pick], rl])

    def _refit(self):
        t0 = time.perf_counter()
        phi, lnl = self._training_set()
        ok = np.isfinite(lnl)
        model, _ = train_emulator(phi[ok], lnl[ok], seed=4 + self.refits, **self.train_kw)
        if self.model is not None and self.own:
            self.model.em.close()
        self.model, self.own = model, True
        self.refits += 1
        self.refit_s += time.perf_counter() - t0

    @property
    def support_limit(self):
        return self.model.support_limit

    def tick(self):
        self.calls += 1
        if self.calls % self.every == 0:
            self._refit()

    def __call__(self, cand):
        return self.model.screen(self.n_sigma * self.model.rms_u)(cand)


def compare_runs_active(exact: ExactLikelihood, phi0, lnl0, n_k: int, n_live=500, k_remove=16, batch=64, seed=5,
                        every=20, max_train=None, initial=None, **train_kw):
    """Seed-matched runs: exact likelihood only, and with an actively refit
    emulator screen (used while L_min lies below its current support limit).
    train_kw go to train_emulator (train_batch is its minibatch size)."""
    if "train_batch" in train_kw:
        train_kw["batch"] = train_kw.pop("train_batch")
    out = {}
    for name in ("exact", "emulator"):
        exact.n_points = 0
        flagged0, fallback0 = exact.n_flagged, exact.n_fallback
        exact.record = name == "emulator"
        exact.rec_x, exact.rec_l = [], []
        t0 = time.perf_counter()
        scr = (ActiveScreen(exact, phi0, lnl0, every=every, max_train=max_train, initial=initial, seed=seed,
                            **train_kw) if name == "emulator" else None)
        ns = NestedSampler(exact, n_k, n_live=n_live, k_remove=k_remove, batch=batch, seed=seed, screen=scr,
                           screen_delta=0.0)
        ns._screen_owner = scr        # the support limit follows the refit model
        r = ns.run()
        exact.record = False
        out[name] = {"logz": r.logz, "logz_err": r.logz_err, "h": r.h, "n_exact": r.n_exact,
                     "n_screened": r.n_screened, "n_iter": r.n_iter, "seconds": time.perf_counter() - t0,
                     "refits": scr.refits if scr else 0, "refit_s": scr.refit_s if scr else 0.0,
                     "n_flagged": exact.n_flagged - flagged0, "n_fallback": exact.n_fallback - fallback0}
        if scr is not None and scr.own:
            scr.model.em.close()
    out["dlogz"] = out["emulator"]["logz"] - out["exact"]["logz"]
    out["same_sequence"] = out["emulator"]["n_iter"] == out["exact"]["n_iter"] and abs(out["dlogz"]) < 1e-9
    out["exact_eval_ratio"] = out["emulator"]["n_exact"] / max(1, out["exact"]["n_exact"])
    return out


def compare_runs(exact: ExactLikelihood, model: ScreenModel, n_k: int, delta_u: float, n_live=500, k_remove=16,
                 batch=64, seed=5):
    """Seed-matched nested-sampling runs without and with the emulator screen
    (margin delta_u on the log-depth scale)."""
    out = {}
    for name, screen in (("exact", None), ("emulator", model.screen(delta_u))):
        exact.n_points = 0
        flagged0, fallback0 = exact.n_flagged, exact.n_fallback
        t0 = time.perf_counter()
        ns = NestedSampler(exact, n_k, n_live=n_live, k_remove=k_remove, batch=batch, seed=seed,
                           screen=screen, screen_delta=0.0, screen_limit=model.support_limit)
        r = ns.run()
        out[name] = {"logz": r.logz, "logz_err": r.logz_err, "h": r.h, "n_exact": r.n_exact,
                     "n_screened": r.n_screened, "n_iter": r.n_iter, "seconds": time.perf_counter() - t0,
                     "n_flagged": exact.n_flagged - flagged0, "n_fallback": exact.n_fallback - fallback0,
                     "posterior_mean": (r.posterior()[0] * r.posterior()[1][:, None]).sum(axis=0).tolist()}
    out["dlogz"] = out["emulator"]["logz"] - out["exact"]["logz"]
    # identical accepted sequences (no false negative of the screen) give identical runs
    out["same_sequence"] = out["emulator"]["n_iter"] == out["exact"]["n_iter"] and abs(out["dlogz"]) < 1e-9
    out["exact_eval_ratio"] = out["emulator"]["n_exact"] / max(1, out["exact"]["n_exact"])
    return out
