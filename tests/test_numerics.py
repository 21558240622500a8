"""Numerical facts the GPU path relies on, checked on the CPU.

* The residual-corrected quadratic form (used for lnL on the mixed path):
  for any approximate solution x~ of Sigma x = dbar and r = dbar - Sigma x~,
  q = dbar^H x~ + x~^H r + r^H Sigma^-1 r exactly.
* Exact round-to-nearest of a double-float value hi + lo with float32
  operations only (each part rounded, one correction from the two exact
  residuals), as the bf16 slicing does.
* Dot2 (Ogita, Rump and Oishi 2005) in float32 reaches about twice the
  working precision, as the solves and the residual rely on.
"""

import numpy as np

import oracle as O
from tests.gpu_common import instrument, oracle_pre


def test_corrected_quadratic_form_identity():
    inst = instrument("C0")
    M, db = oracle_pre("C0")
    phi = np.array([0.3, -0.7, 1.1, -1.5])
    phi_inv, _ = O.prior_diag(phi, inst.kbin, inst.spec.lssm_prior_var)
    S = M + np.diag(phi_inv)
    x = np.linalg.solve(S, db)
    q = float(np.real(np.vdot(db, x)))
    g = np.random.default_rng(0)
    for eta in (1e-7, 1e-4, 1e-2):
        xt = x * (1 + eta * (g.standard_normal(len(x)) + 1j * g.standard_normal(len(x))))
        r = db - S @ xt
        t = float(np.real(np.vdot(r, np.linalg.solve(S, r))))
        q1 = float(np.real(np.vdot(db, xt) + np.vdot(xt, r)))
        assert abs(q1 + t - q) <= 1e-9 * abs(q)           # exact up to rounding
        assert abs((q - q1) - t) <= 1e-9 * abs(q) + 1e-6 * t   # first order misses exactly t
        assert t > 0


def _round_df(a, b):
    a, b = np.float32(a), np.float32(b)
    ra, rb = np.rint(a), np.rint(b)
    x = np.int64(ra) + np.int64(rb)
    d = np.float32(np.float32(a - ra) + np.float32(b - rb))
    return x + (d > 0.5) - (d < -0.5)


def test_round_df_is_exact_round_to_nearest():
    g = np.random.default_rng(1)
    for e in (-3, 0, 10, 23, 24, 30, 38):
        v = g.uniform(-1, 1, 20000) * 2.0 ** e
        hi = v.astype(np.float32)
        lo = (v - hi.astype(np.float64)).astype(np.float32)
        exact = hi.astype(np.float64) + lo.astype(np.float64)   # the double-float value
        got = np.array([_round_df(a, b) for a, b in zip(hi[:2000], lo[:2000])])
        ref = np.rint(exact[:2000]).astype(np.int64)
        frac = np.abs(exact[:2000] - np.floor(exact[:2000]) - 0.5)
        assert np.all((got == ref) | (frac == 0)), e


def _dot2_f32(x, y):
    """Dot2 in float32: TwoProduct (FMA-exact here via float64) and TwoSum."""
    s = np.float32(0.0)
    c = np.float32(0.0)
    for a, b in zip(x.astype(np.float32), y.astype(np.float32)):
        p = np.float32(a * b)
        e = np.float32(np.float64(a) * np.float64(b) - np.float64(p))   # exact product error
        t = np.float32(s + p)
        bb = np.float32(t - s)
        err = np.float32(np.float32(s - np.float32(t - bb)) + np.float32(p - bb))
        s = t
        c = np.float32(c + np.float32(err + e))
    return np.float64(s) + np.float64(c)


def test_dot2_reaches_twice_the_working_precision():
    g = np.random.default_rng(2)
    n = 128
    x = g.standard_normal(n).astype(np.float32)
    y = g.standard_normal(n).astype(np.float32)
    exact = float(np.dot(x.astype(np.float64), y.astype(np.float64)))   # exact: 48-bit products, 128 terms
    plain = float(np.float32(np.sum(x * y, dtype=np.float32)))
    d2 = _dot2_f32(x, y)
    cond = float(np.dot(np.abs(x.astype(np.float64)), np.abs(y.astype(np.float64))))
    u = 2.0 ** -24
    assert abs(d2 - exact) <= u * abs(exact) + 2 * (n * u) ** 2 * cond
    assert abs(d2 - exact) < abs(plain - exact) * 1e-3 or abs(plain - exact) == 0
