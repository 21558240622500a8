"""Nested sampling of the power-spectrum posterior with an optional emulator screen.

The paper samples the marginal posterior of the power-spectrum amplitudes and
computes the Bayesian evidence with a nested sampler (Sec. "Summary": the
evidence makes the package usable for model selection).  This is a
project-written sampler with the same outputs (evidence ln Z, its
uncertainty, weighted posterior samples):

* n_live live points drawn from a uniform prior box;
* each iteration removes the k lowest points (ln X shrinks by 1/(n_live - i)
  for the i-th of them) and replaces them by draws from the constrained
  prior L > L_min;
* replacements are drawn uniformly inside one bounding ellipsoid of the live
  points (their covariance, scaled to enclose all of them, enlarged by
  `enlarge` per dimension), intersected with the prior box;
* candidates are generated in blocks from one seeded generator and accepted
  in draw order, so that a run with an emulator screen sees exactly the same
  candidate sequence as a run without it;
* with an emulator, a candidate whose predicted lnL is below L_min - delta is
  skipped without an exact evaluation, but only while L_min is below
  `screen_limit` (the range where the emulator's training data give it
  support); an adaptive screen (`_screen_owner`, with `tick()` and
  `support_limit`) is told of every candidate block, so that it can refit
  and move its support limit while it is not consulted; every accepted
  point, and therefore the evidence, uses the exact likelihood;
* the run stops when the live points can add less than `stop_frac` of the
  current evidence, then the live points are added.

The likelihood callables take an (m, D) array and return m values; exact
calls are batched so that the GPU evaluates many candidates per launch.
"""

from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np


def _logaddexp(a, b):
    if a == -math.inf:
        return b
    if b == -math.inf:
        return a
    m = max(a, b)
    return m + math.log(math.exp(a - m) + math.exp(b - m))


@dataclass
class NSResult:
    logz: float
    logz_err: float
    h: float
    n_exact: int
    n_screened: int
    n_iter: int
    samples: np.ndarray
    logl: np.ndarray
    logw: np.ndarray
    extra: dict = field(default_factory=dict)

    def posterior(self):
        w = np.exp(self.logw - self.logw.max())
        return self.samples, w / w.sum()


class NestedSampler:
    def __init__(self, loglike, ndim, lo=-2.0, hi=2.0, n_live=500, k_remove=1, batch=64, enlarge=1.2,
                 stop_frac=0.01, seed=5, screen=None, screen_delta=0.0, screen_limit=math.inf,
                 max_iter=10_000_000, checkpoint=None, checkpoint_every=1000):
        self.loglike = loglike
        self.ndim = ndim
        self.lo = np.full(ndim, lo, float) if np.isscalar(lo) else np.asarray(lo, float)
        self.hi = np.full(ndim, hi, float) if np.isscalar(hi) else np.asarray(hi, float)
        self.n_live = n_live
        self.k = k_remove
        self.batch = batch
        self.enlarge = enlarge
        self.stop_frac = stop_frac
        self.rng = np.random.Generator(np.random.PCG64(seed))
        self.screen = screen
        self.delta = screen_delta
        self.screen_limit = screen_limit      # the screen is used only while L_min < screen_limit
        self.max_iter = max_iter
        self.checkpoint = checkpoint
        self.checkpoint_every = checkpoint_every
        self.max_empty_blocks = 200
        self.n_exact = 0
        self.n_screened = 0

    # ---- candidate generation -------------------------------------------------
    def _ellipsoid(self, pts):
        mu = pts.mean(axis=0)
        c = np.cov(pts.T) + 1e-12 * np.eye(self.ndim)
        ci = np.linalg.inv(c)
        d = pts - mu
        r2 = np.max(np.einsum("ij,jk,ik->i", d, ci, d))
        chol = np.linalg.cholesky(c * r2) * self.enlarge
        return mu, chol

    def _draw_block(self, mu, chol, m):
        """m uniform draws inside the ellipsoid and the prior box."""
        out = []
        while sum(len(o) for o in out) < m:
            z = self.rng.standard_normal((2 * m, self.ndim))
            z /= np.linalg.norm(z, axis=1, keepdims=True)
            rad = self.rng.random(2 * m) ** (1.0 / self.ndim)
            x = mu + (z * rad[:, None]) @ chol.T
            ok = np.all((x >= self.lo) & (x <= self.hi), axis=1)
            out.append(x[ok])
        return np.concatenate(out)[:m]

    def _exact(self, x):
        self.n_exact += len(x)
        return np.asarray(self.loglike(x), float)

    def _replace(self, lmin, mu, chol, need):
        """`need` accepted points with exact lnL > lmin, in draw order."""
        acc_x, acc_l = [], []
        empty = 0
        owner = getattr(self, "_screen_owner", None)
        while len(acc_x) < need:
            cand = self._draw_block(mu, chol, self.batch)
            if owner is not None:
                owner.tick()          # an adaptive screen updates itself on every block, screened or not
            limit = getattr(owner, "support_limit", self.screen_limit)
            if self.screen is not None and lmin < limit and empty < self.max_empty_blocks:
                pred = np.asarray(self.screen(cand), float)
                keep = pred >= lmin - self.delta
                self.n_screened += int((~keep).sum())
                cand = cand[keep]
                if len(cand) == 0:
                    empty += 1      # after max_empty_blocks in a row the screen is bypassed
                    continue
                empty = 0
            ll = self._exact(cand)
            for xi, li in zip(cand, ll):
                if li > lmin and len(acc_x) < need:
                    acc_x.append(xi)
                    acc_l.append(li)
        return np.array(acc_x), np.array(acc_l)

    # ---- checkpointing ------------------------------------------------------
    def _save(self, state):
        tmp = self.checkpoint + ".tmp.npz"
        np.savez(tmp, live=state["live"], live_l=state["live_l"], dead=np.array(state["dead"]),
                 dead_l=np.array(state["dead_l"]), dead_lw=np.array(state["dead_lw"]))
        meta = {k: state[k] for k in ("logz", "logx", "h", "it")}
        meta.update(n_exact=self.n_exact, n_screened=self.n_screened, rng=self.rng.bit_generator.state)
        with open(self.checkpoint + ".json.tmp", "w") as f:
            json.dump(meta, f)
        os.replace(tmp, self.checkpoint + ".npz")
        os.replace(self.checkpoint + ".json.tmp", self.checkpoint + ".json")

    def _load(self):
        z = np.load(self.checkpoint + ".npz")
        with open(self.checkpoint + ".json") as f:
            meta = json.load(f)
        self.n_exact = meta["n_exact"]
        self.n_screened = meta["n_screened"]
        self.rng.bit_generator.state = meta["rng"]
        dead = z["dead"]
        return {"live": z["live"], "live_l": z["live_l"],
                "dead": [row for row in dead] if len(dead) else [],
                "dead_l": list(z["dead_l"]), "dead_lw": list(z["dead_lw"]),
                "logz": meta["logz"], "logx": meta["logx"], "h": meta["h"], "it": meta["it"]}

    # ---- the run --------------------------------------------------------------
    def run(self, resume=False, stop_after=None) -> NSResult:
        if resume and self.checkpoint and os.path.exists(self.checkpoint + ".json"):
            st = self._load()
        else:
            live = self.lo + (self.hi - self.lo) * self.rng.random((self.n_live, self.ndim))
            live_l = np.concatenate([self._exact(live[i:i + self.batch]) for i in range(0, self.n_live, self.batch)])
            st = {"live": live, "live_l": live_l, "dead": [], "dead_l": [], "dead_lw": [],
                  "logz": -math.inf, "logx": 0.0, "h": 0.0, "it": 0}
        live, live_l = st["live"], st["live_l"]
        logz, logx, h = st["logz"], st["logx"], st["h"]
        n = self.n_live
        it = st["it"]
        while it < self.max_iter:
            order = np.argsort(live_l)
            worst = order[: self.k]
            lmin = float(live_l[worst[-1]])
            for i, w in enumerate(worst):
                # X shrinks by t ~ Beta(n - i, 1): E[ln t] = -1 / (n - i)
                logx_new = logx - 1.0 / (n - i)
                logw = logx + math.log(-math.expm1(logx_new - logx))    # X_prev - X_new
                lw = logw + live_l[w]
                logz_new = _logaddexp(logz, lw)
                if logz_new > -math.inf:
                    h = (math.exp(lw - logz_new) * live_l[w]
                         + math.exp(logz - logz_new) * (h + logz) - logz_new) if logz > -math.inf else live_l[w] - logz_new
                logz = logz_new
                st["dead"].append(live[w].copy())
                st["dead_l"].append(float(live_l[w]))
                st["dead_lw"].append(lw)
                logx = logx_new
            mu, chol = self._ellipsoid(np.delete(live, worst, axis=0))
            new_x, new_l = self._replace(lmin, mu, chol, len(worst))
            live[worst] = new_x
            live_l[worst] = new_l
            it += 1
            lmax = float(live_l.max())
            # remaining mass L_max X below stop_frac of Z (compared in logs: no overflow)
            if logz > -math.inf and lmax + logx - logz < math.log(self.stop_frac):
                break
            if self.checkpoint and it % self.checkpoint_every == 0:
                st.update(live=live, live_l=live_l, logz=logz, logx=logx, h=h, it=it)
                self._save(st)
            if stop_after is not None and it >= stop_after:
                st.update(live=live, live_l=live_l, logz=logz, logx=logx, h=h, it=it)
                if self.checkpoint:
                    self._save(st)
                return None
        # add the remaining live points, each with weight X / n_live
        logw_live = logx - math.log(n)
        for x, l in zip(live, live_l):
            lw = logw_live + l
            logz_new = _logaddexp(logz, lw)
            h = math.exp(lw - logz_new) * l + math.exp(logz - logz_new) * (h + logz) - logz_new
            logz = logz_new
            st["dead"].append(x.copy())
            st["dead_l"].append(float(l))
            st["dead_lw"].append(lw)
        h = max(h, 0.0)
        return NSResult(logz=logz, logz_err=math.sqrt(h / n), h=h, n_exact=self.n_exact,
                        n_screened=self.n_screened, n_iter=it, samples=np.array(st["dead"]),
                        logl=np.array(st["dead_l"]), logw=np.array(st["dead_lw"]) - logz)
