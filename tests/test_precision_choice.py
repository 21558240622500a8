"""Why the factorisation's off-diagonal products are exact bf16 slice
products and not split-TF32 products with fp32 accumulation.

CPU emulation on the 3280-mode instrument (the 9 x 9 uv grid, 38 channels,
126 baselines x 19 times).  A blocked right-looking Cholesky of
Sigma = M + diag(Phi^-1) (128-blocks, float64 diagonal blocks and working
matrix) is run with two forms of the products L_ik = A_ik Linv^H (panel)
and A_ij -= L_ik L_jk^H (trailing update), and log|Sigma| = 2 sum ln L_jj is
compared with the float64 factorisation of the same matrix:

* split TF32, fp32 accumulation: each complex operand split as hi + lo with
  hi, lo TF32 (10 explicit significand bits, rounded to nearest), products
  hi hi^H + hi lo^H + lo hi^H accumulated in fp32; the panel product is
  left in float64 (the most favourable reading);
* the library's slice products: every operand row scaled by 2^(7 - e_r) and
  rounded to five balanced base-256 digits, products of digit slices (s, t)
  with s + t <= 4 summed in float64 (the tensor cores' fp32 accumulators are
  exact for them, or round far below 2^-40 of the result), panel and
  trailing update alike;
* the library's trailing update as it runs: the reduced pair set (s + t <= 3
  and (2, 2)) on the off-diagonal tiles, the full set on the diagonal tiles
  (128 x 128 blocks of P P^H) and in the panel product; and, to show why
  the pair (2, 2) is kept, the pairs s + t <= 3 alone on every tile, which
  drops the biased |sigma_2|^2 terms from the diagonal of P P^H.

The likelihood's tolerance is |dlnL| <= 1e-2, i.e. 2e-2 in log|Sigma| (lnL
carries -1/2 log|Sigma|; the quadratic form is corrected by a float64
residual and is not what limits the precision).
"""

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.slow


def _tf32(x):
    """Round float32 values to TF32 (10 explicit significand bits), to nearest."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32)


def _ctf32(z):
    z = np.asarray(z, np.complex64)
    return (_tf32(z.real) + 1j * _tf32(z.imag)).astype(np.complex64)


def prod_tf32x3(X, Y):
    """X Y^H from TF32 hi / lo splits, three products, fp32 accumulation."""
    X = X.astype(np.complex64)
    Y = Y.astype(np.complex64)
    Xh, Yh = _ctf32(X), _ctf32(Y)
    Xl, Yl = _ctf32(X - Xh), _ctf32(Y - Yh)
    P = Xh @ Yh.conj().T
    P += Xh @ Yl.conj().T
    P += Xl @ Yh.conj().T
    return P.astype(np.complex128)


def _digits(X):
    """Row exponents e (largest |re|, |im| of the row below 2^e) and the five
    digit planes D_s (complex, integer valued, |re|, |im| <= 128) with
    X ~ 2^(e - 7) sum_s D_s 2^(-8 s)."""
    m = np.maximum(np.abs(X.real), np.abs(X.imag)).max(axis=1)
    e = np.zeros(len(m), np.int64)
    nz = m > 0
    e[nz] = np.floor(np.log2(m[nz])).astype(np.int64) + 1
    sc = np.ldexp(1.0, 39 - e)[:, None]
    planes = []
    for part in (X.real, X.imag):
        v = np.round(part * sc).astype(np.int64)
        dg = [None] * 5
        for s in range(4, 0, -1):
            d = ((v + 128) & 255) - 128
            dg[s] = d
            v = (v - d) >> 8
        dg[0] = v
        planes.append(dg)
    return e, [planes[0][s] + 1j * planes[1][s] for s in range(5)]


FULL = [(s, t) for s in range(5) for t in range(5) if s + t <= 4]
LE3 = [(s, t) for s in range(5) for t in range(5) if s + t <= 3]
REDUCED = LE3 + [(2, 2)]


def prod_slices(X, Y, pairs=FULL):
    """X Y^H as the library's slice products over the digit pairs (s, t) given."""
    ex, DX = _digits(X)
    ey, DY = _digits(Y)
    acc = np.zeros((X.shape[0], Y.shape[0]), np.complex128)
    for s in range(5):
        ts = [t for (a, t) in pairs if a == s]
        if not ts:
            continue
        # the slices t of Y for this s, summed exactly (40 bits); one product per s,
        # exact but for float64 rounding (2^-53, far below the dropped pairs' 2^-40)
        Yt = sum(DY[t] * 2.0 ** (-8 * t) for t in ts)
        acc += (DX[s] @ Yt.conj().T) * 2.0 ** (-8 * s)
    return acc * np.ldexp(1.0, ex - 7)[:, None] * np.ldexp(1.0, ey - 7)[None, :]


def trail_library(P, Q, nb=128):
    """The trailing update as the library runs it (P = Q = L_ik): reduced pair
    set off the diagonal tiles, full set on them."""
    U = prod_slices(P, Q, REDUCED)
    for i0 in range(0, P.shape[0], nb):
        i1 = min(i0 + nb, P.shape[0])
        U[i0:i1, i0:i1] = prod_slices(P[i0:i1], Q[i0:i1], FULL)
    return U


def logdet_blocked(S, trail, panel, nb=128):
    """log|S| from a blocked right-looking Cholesky whose panel and trailing
    products are `panel(A_ik, Linv)` and `trail(L_ik, L_ik)` (X Y^H)."""
    A = S.copy()
    n = A.shape[0]
    ld = 0.0
    for k in range(0, n, nb):
        e = min(k + nb, n)
        L = np.linalg.cholesky(A[k:e, k:e])
        ld += 2.0 * float(np.sum(np.log(L.diagonal().real)))
        if e < n:
            P = panel(A[e:, k:e], np.linalg.inv(L))
            A[e:, k:e] = P
            A[e:, e:] -= trail(P, P)
    return ld


def exact(X, Y):
    return X @ Y.conj().T


def test_digit_products_are_exact_to_40_bits():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((48, 128)) + 1j * rng.standard_normal((48, 128))
    Y = rng.standard_normal((40, 128)) + 1j * rng.standard_normal((40, 128))
    ref = X @ Y.conj().T
    err = np.abs(prod_slices(X, Y) - ref).max() / np.abs(ref).max()
    assert 0 < err < 2.0 ** -34
    err32 = np.abs(prod_tf32x3(X, Y) - ref).max() / np.abs(ref).max()
    assert err32 > 2.0 ** -24   # the split-TF32 product carries fp32-level error


def test_split_tf32_misses_the_lnl_tolerance_and_slices_do_not():
    from synth import build_instrument, draw_phi

    inst = build_instrument("C1")
    M = O.herm_structured(inst.A, inst.W, inst.noise_var)
    phis = draw_phi(inst.spec, 3)
    tf32_err, slice_err, lib_err, red_err = [], [], [], []
    for b, phi in enumerate(phis):
        pinv, _ = O.prior_diag(phi, inst.kbin, inst.spec.lssm_prior_var)
        S = M.copy()
        S[np.diag_indices_from(S)] += pinv
        ref = logdet_blocked(S, exact, exact)
        tf32_err.append(abs(logdet_blocked(S, prod_tf32x3, exact) - ref))
        if b == 0:
            slice_err.append(abs(logdet_blocked(S, prod_slices, prod_slices) - ref))
            lib_err.append(abs(logdet_blocked(S, trail_library, prod_slices) - ref))
            red_err.append(logdet_blocked(S, lambda P, Q: prod_slices(P, Q, LE3), prod_slices) - ref)
    print("log|Sigma| error, split TF32:", tf32_err, "slices:", slice_err, "library:", lib_err,
          "s + t <= 3 on every tile (signed):", red_err)
    # every sampled point: split TF32 moves lnL by more than its tolerance
    assert min(tf32_err) > 2e-2
    # the slice products stay at least ten times inside it, and far below split TF32
    assert max(slice_err) < 2e-3
    assert min(tf32_err) > 10 * max(slice_err)
    # the library's trailing pair sets stay at least four times inside the tolerance
    assert max(lib_err) < 5e-3
    # without (2, 2) each update subtracts too little from the diagonal
    # (the dropped |sigma_2|^2 terms are never negative), so log|Sigma| rises
    assert min(red_err) > 2e-2
