"""Numerical facts the GPU path relies on, checked on the CPU.

* The residual-corrected quadratic form (used for lnL on the mixed path):
  for any approximate solution x~ of Sigma x = dbar and r = dbar - Sigma x~,
  q = dbar^H x~ + x~^H r + r^H Sigma^-1 r exactly.
* Exact round-to-nearest of a double-float value hi + lo with float32
  operations only (each part rounded, one correction from the two exact
  residuals), and the slicing kernels' conversion-free digit extraction,
  which gives the same digits.
* Dot2 (Ogita, Rump and Oishi 2005) in float32 reaches about twice the
  working precision, as the solves and the residual rely on.
* The bf16 slicing: five balanced base-256 digits reconstruct any
  fixed-point value |X| <= 2^39 exactly, each slice is exact in bf16, the
  float32 level accumulators of levels 0-2 are exact over a 128-complex
  block column, and the four levels give the product to about 2^-40 of the
  operand row scales.
* The accumulator drain's 13-operation level sum (exact integer and
  fraction parts, one fast two-sum) is exact up to one rounding of level 3
  and normalised, also where the low part exceeds the high part.
* The residual's exact split of M into three floats per component.
* The blocked recurrence of the diagonal blocks' inverse (four 32 x 32
  diagonal blocks, then block rows as block products).
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
    """round(a + b) for float32 a + b: each part rounded, one correction step
    decided by the sum of the two exact residuals (float32)."""
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


def _digits_bottom_up(X):
    """Balanced base-256 digits of int64 X: four from the bottom in
    [-128, 127], the rest on top."""
    d = [None] * 5
    for s in range(4, 0, -1):
        m = ((X + 128) & 255) - 128
        d[s] = m
        X = (X - m) >> 8
    d[0] = X
    return d


def _balanced_digits5_emulated(hi, lo, e):
    """The slicing kernels' digit extraction without conversion instructions:
    A = 2^17 Ah + Al with Ah = rint(A 2^-17), round(Al + B) as the parts'
    nearest integers plus one correction, then 32-bit digit arithmetic."""
    f = np.float32
    k = (39 - e).astype(np.int64)
    k1 = k >> 1
    A = (hi * np.exp2(k1).astype(f)) * np.exp2(k - k1).astype(f)
    B = (lo * np.exp2(k1).astype(f)) * np.exp2(k - k1).astype(f)
    ah = np.rint(A.astype(np.float64) * 2.0 ** -17)                 # magic-number rounding (RN-even)
    al = (A.astype(np.float64) - ah * 2.0 ** 17).astype(f)          # exact
    ra, rb = np.rint(al), np.rint(B)
    d = (al - ra) + (B - rb)
    xl = ra.astype(np.int64) + rb.astype(np.int64) + (d > 0.5) - (d < -0.5)
    ah = ah.astype(np.int64)
    d4 = ((xl + 128) & 255) - 128
    y = (xl - d4) >> 8
    d3 = ((y + 128) & 255) - 128
    x = 2 * ah + ((y - d3) >> 8)
    assert np.all(np.abs(x) < 2 ** 31)
    d2 = ((x + 128) & 255) - 128
    x = (x - d2) >> 8
    d1 = ((x + 128) & 255) - 128
    return [(x - d1) >> 8, d1, d2, d3, d4]


def test_conversion_free_digits_match_the_64_bit_rounding():
    """The slicing kernels' digits from fp32 and 32-bit integer operations
    equal those of the 64-bit route (round the scaled double-float to an
    int64 with _round_df, split it from the bottom), over exponents with
    headroom, tiny and large values, and ties; all digits within [-128, 128]."""
    g = np.random.default_rng(17)
    n = 100000
    f = np.float32
    x = g.standard_normal(n) * np.exp(g.uniform(-40, 40, n))
    x[:2000] = np.ldexp(np.round(g.uniform(-1, 1, 2000) * 2 ** 30), -30)   # on a coarse grid: ties
    hi = x.astype(f)
    lo = (x - hi.astype(np.float64)).astype(f)
    e = (np.floor(np.log2(np.abs(hi.astype(np.float64)))) + 1 + g.integers(0, 40, n) * (g.random(n) < 0.3)).astype(np.int64)
    got = _balanced_digits5_emulated(hi, lo, e)
    k = 39 - e
    A = (hi.astype(np.float64) * np.exp2(k)).astype(f)
    B = (lo.astype(np.float64) * np.exp2(k)).astype(f)
    X = np.array([_round_df(a, b) for a, b in zip(A, B)], dtype=np.int64)
    ref = _digits_bottom_up(X)
    for s in range(5):
        np.testing.assert_array_equal(got[s], ref[s])
    assert all(np.abs(di).max() <= 128 for di in got)


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


def _digits5(X):
    """Five balanced base-256 digits of integers |X| <= 2^39, as the bf16
    slicing forms them: X = sum_s d_s 256^(4 - s), |d_s| <= 128."""
    X = np.asarray(X, np.int64).copy()
    d = np.zeros((5,) + X.shape, np.int64)
    for s in range(4, 0, -1):
        m = ((X + 128) & 255) - 128
        d[s] = m
        X = (X - m) >> 8
    d[0] = X
    return d


def test_balanced_digits_reconstruct_and_are_exact_in_bf16():
    g = np.random.default_rng(3)
    edge = [2 ** 39, -2 ** 39, 2 ** 39 - 1, 0, 127, 128, -128, -129, 255 * 2 ** 31]
    X = np.concatenate([g.integers(-2 ** 39, 2 ** 39, 200_000), edge])
    d = _digits5(X)
    rec = sum(d[s] * 256 ** (4 - s) for s in range(5))
    assert np.array_equal(rec, X)
    assert np.abs(d).max() <= 128
    for s in range(5):
        v = (d[s] * 2.0 ** (-8 * s)).astype(np.float32)
        assert np.all((v.view(np.uint32) & 0xFFFF) == 0)   # bf16 keeps the top 16 bits of a float32


def test_slice_product_levels_exact_and_sum_accurate():
    """One 128-complex block column (K = 256 real terms per output) as the
    trailing update computes it: rows scaled by 2^(39 - e) and split into
    digits, the 15 slice pairs with s + t <= 4 accumulated in float32 in
    four level accumulators (pairs with s + t >= 3 share the last).  Levels
    0-2 are exact; the four levels scaled by 2^(e_a + e_b - 14) give A B^T to
    about 2^-40 of the row scales."""
    g = np.random.default_rng(4)
    K, m, n = 256, 48, 24
    A = g.standard_normal((m, K)) * np.exp(g.uniform(-3, 3, (m, 1)))
    B = g.standard_normal((n, K)) * np.exp(g.uniform(-3, 3, (n, 1)))

    def fixed(M):
        e = np.floor(np.log2(np.abs(M).max(axis=1))).astype(np.int64) + 1   # |row| < 2^e
        return np.rint(M * np.exp2(39 - e)[:, None]).astype(np.int64), e

    XA, eA = fixed(A)
    XB, eB = fixed(B)
    dA, dB = _digits5(XA), _digits5(XB)
    lev = np.zeros((4, m, n), np.float32)
    exact = np.zeros((3, m, n), np.int64)          # levels 0-2 in units of 2^(-8 l)
    for s in range(5):
        for t in range(5 - s):
            l = min(s + t, 3)
            a = (dA[s] * 2.0 ** (-8 * s)).astype(np.float32)
            b = (dB[t] * 2.0 ** (-8 * t)).astype(np.float32)
            for k in range(K):                      # sequential float32 accumulation
                lev[l] += np.outer(a[:, k], b[:, k])
            if l < 3:
                exact[l] += dA[s] @ dB[t].T
    for l in range(3):
        assert np.array_equal(lev[l].astype(np.float64) * 2.0 ** (8 * l), exact[l].astype(np.float64)), l
    P = lev.astype(np.float64).sum(axis=0) * np.exp2(eA[:, None] + eB[None, :] - 14)
    scale = K * np.exp2(eA[:, None] + eB[None, :])
    err = np.abs(P - A @ B.T) / scale
    assert err.max() <= 2.0 ** -40, err.max()          # measured: 2^-42.4


def _levels_sum_split(l0, l1, l2, l3):
    """The drain's level sum in float32 (RN at every step, as numpy float32
    arithmetic is): nearest integers of levels 1 and 2 by adding and
    subtracting 1.5 * 2^23, hi = l0 + int(l1) + int(l2), lo = frac(l1) +
    frac(l2) + l3, then one fast two-sum."""
    f = np.float32
    m = f(12582912.0)
    r1 = (l1 + m) - m
    r2 = (l2 + m) - m
    hi = (l0 + r1) + r2
    lo = ((l1 - r1) + (l2 - r2)) + l3
    s = hi + lo
    e = lo - (s - hi)
    return hi, lo, s, e


def test_cheap_level_sum_is_exact_and_normalised():
    """The accumulator drain adds the four levels in 13 float32 operations
    instead of two exact two-sums: the integer part is exact, the fast
    two-sum that normalises (hi, lo) loses nothing (also for |hi| <= 3 below
    |lo|), and the result is the exact level sum within one rounding of
    level 3 (2^-22 units, |lo| < 4)."""
    g = np.random.default_rng(11)
    n = 200000
    f = np.float32
    # levels in their units: l0 integer |l0| <= 2^22, l1 multiple of 2^-8
    # below 2^15, l2 multiple of 2^-16 below 192, l3 any float below 2
    l0 = g.integers(-2 ** 22, 2 ** 22 + 1, n).astype(f)
    l1 = (g.integers(-2 ** 23, 2 ** 23 + 1, n) * 2.0 ** -8).astype(f)
    l2 = (g.integers(-192 * 2 ** 16, 192 * 2 ** 16 + 1, n) * 2.0 ** -16).astype(f)
    l3 = g.uniform(-2, 2, n).astype(f)
    # small high parts too, where |lo| may exceed |hi|
    k = n // 4
    l0[:k] = g.integers(-3, 4, k)
    l1[:k] = (g.integers(-128, 129, k) * 2.0 ** -8).astype(f)
    l2[:k] = (g.integers(-2 ** 15, 2 ** 15 + 1, k) * 2.0 ** -16).astype(f)
    hi, lo, s, e = _levels_sum_split(l0, l1, l2, l3)
    assert np.array_equal(hi.astype(np.float64),
                          l0.astype(np.float64) + np.rint(l1.astype(np.float64)) + np.rint(l2.astype(np.float64)))
    assert np.all(np.abs(lo) < 4)
    # fast two-sum exact: s + e == hi + lo, and e within half an ulp of s
    assert np.array_equal(s.astype(np.float64) + e.astype(np.float64), hi.astype(np.float64) + lo.astype(np.float64))
    assert np.all(np.abs(e) <= np.spacing(np.abs(s)) / 2)
    exact = l0.astype(np.float64) + l1.astype(np.float64) + l2.astype(np.float64) + l3.astype(np.float64)
    err = np.abs(s.astype(np.float64) + e.astype(np.float64) - exact)
    assert err.max() <= 2.0 ** -22, err.max()
    # on accumulated levels of a real slice product it matches the two-sum version
    ta = _two_sum_levels(l0[k:k + 1000], l1[k:k + 1000], l2[k:k + 1000], l3[k:k + 1000])
    tb = s[k:k + 1000].astype(np.float64) + e[k:k + 1000].astype(np.float64)
    assert np.abs(ta - tb).max() <= 2.0 ** -21


def _two_sum_levels(l0, l1, l2, l3):
    """The reference level sum: two exact two-sums, the small terms into the
    low part, evaluated in float32 and returned as hi + lo in float64."""
    def two_sum(a, b):
        s = a + b
        bb = s - a
        return s, (a - (s - bb)) + (b - bb)
    ah, al = two_sum(l0, l1)
    bh, bl = two_sum(ah, l2)
    lo = bl + (al + l3)
    s = bh + lo
    e = lo - (s - bh)
    return s.astype(np.float64) + e.astype(np.float64)


def test_blocked_triangular_inverse_recurrence():
    """The diagonal-block kernel's inverse of L (128 x 128, lower): the four
    32 x 32 diagonal blocks inverted by the row recursion, then block row
    I = 1..3 as Linv_IJ = -Linv_II sum_{M=J}^{I-1} L_IM Linv_MJ; in float64
    it equals the inverse to rounding."""
    g = np.random.default_rng(5)
    n, b = 128, 32
    L = np.tril(g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) * 0.1
    L[np.diag_indices(n)] = np.abs(g.standard_normal(n)) + 1.0
    X = np.zeros_like(L)
    for I in range(4):   # diagonal blocks, row by row
        s = slice(b * I, b * I + b)
        Lb, Xb = L[s, s], np.zeros((b, b), complex)
        for i in range(b):
            Xb[i, i] = 1.0 / Lb[i, i]
            for j in range(i):
                Xb[i, j] = -(Lb[i, j:i] @ Xb[j:i, j]) / Lb[i, i]
        X[s, s] = Xb
    for I in range(1, 4):
        rI = slice(b * I, b * I + b)
        for J in range(I):
            rJ = slice(b * J, b * J + b)
            acc = sum(L[rI, b * M:b * M + b] @ X[b * M:b * M + b, rJ] for M in range(J, I))
            X[rI, rJ] = -X[rI, rI] @ acc
    ref = np.linalg.inv(L)
    assert np.abs(X - ref).max() <= 1e-12 * np.abs(ref).max()


def test_float_triple_split_of_m_is_exact():
    """The residual reads M as three floats per component: hi = fl(m),
    lo = fl(m - hi), t = fl(m - hi - lo).  Both remainders are exact in
    float64 and the last has at most 53 - 48 significant bits, so
    hi + lo + t == m exactly (for magnitudes far above float32's underflow,
    as M's entries are)."""
    g = np.random.default_rng(5)
    m = g.standard_normal(200_000) * np.exp(g.uniform(np.log(1e-6), np.log(1e7), 200_000))
    hi = m.astype(np.float32)
    rd = m - hi.astype(np.float64)
    lo = rd.astype(np.float32)
    t = (rd - lo.astype(np.float64)).astype(np.float32)
    assert np.array_equal((hi.astype(np.float64) + lo.astype(np.float64)) + t.astype(np.float64), m)
    assert np.all(np.abs(lo.astype(np.float64)) <= np.spacing(np.abs(hi)).astype(np.float64) / 2)
    assert np.all(np.abs(t.astype(np.float64)) <= np.spacing(np.abs(lo)).astype(np.float64) / 2)
