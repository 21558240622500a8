"""Pins of the CPU oracle against facts fixed by the mathematics.

Each test checks the oracle against something other than itself: a brute
force evaluation of the Gaussian marginal likelihood, a closed form, a
library routine, a limit, or finite differences.  The mutation tests at the
end plant plausible mistakes in the oracle and check that a pin catches them.
"""

import math

import numpy as np
import pytest

import oracle as O
import oracle.likelihood as OL
from synth import build_instrument, draw_phi, expand_T
from synth.instrument import get_spec, random_problem

LN_PI = math.log(math.pi)


def brute_force_lnl(T, noise_var, d, kbin, phi, lssm_var):
    """lnL from the definition through the data-space covariance C = T Phi T^H + N.

    For complex Gaussian data ln CN(d; 0, C) = -n ln(pi) - ln|C| - d^H C^-1 d.
    With |C| = |N||Phi||Sigma| (determinant lemma) and the Woodbury identity,
    -1/2 log|Phi| - 1/2 log|Sigma| + 1/2 dbar^H Sigma^-1 dbar
        = 1/2 ln CN(d; 0, C) + 1/2 (n ln(pi) + ln|N| + d^H N^-1 d).
    This side uses only C, numpy slogdet and solve.
    """
    n = T.shape[0]
    phi_diag = np.where(kbin >= 0, 10.0 ** np.asarray(phi)[np.maximum(kbin, 0)], lssm_var)
    C = (T * phi_diag[None, :]) @ T.conj().T + np.diag(noise_var)
    sign, logdet_c = np.linalg.slogdet(C)
    assert abs(sign - 1) < 1e-9
    quad = float(np.real(np.vdot(d, np.linalg.solve(C, d))))
    ln_cn = -n * LN_PI - logdet_c - quad
    const = n * LN_PI + float(np.sum(np.log(noise_var))) + float(np.sum(np.abs(d) ** 2 / noise_var))
    return 0.5 * ln_cn + 0.5 * const


def oracle_lnl(T, noise_var, d, kbin, phi, lssm_var):
    M = O.herm_dense(T, noise_var)
    db = O.dbar_dense(T, noise_var, d)
    return O.evaluate(M, db, kbin, phi, lssm_var)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_woodbury_bruteforce_tiny(seed):
    p = random_problem(12, 5, 2, seed)
    g = np.random.default_rng(seed)
    for _ in range(3):
        phi = g.uniform(-2, 2, 2)
        ref = brute_force_lnl(p["T"], p["noise_var"], p["d"], p["kbin"], phi, 3.0)
        got = oracle_lnl(p["T"], p["noise_var"], p["d"], p["kbin"], phi, 3.0)["lnl"]
        assert abs(got - ref) <= 1e-10 * abs(ref) + 1e-12


def test_woodbury_bruteforce_C0():
    inst = build_instrument("C0")
    T = expand_T(inst)
    for phi in draw_phi("C0", 4):
        ref = brute_force_lnl(T, inst.noise_var, inst.d, inst.kbin, phi, inst.spec.lssm_prior_var)
        got = oracle_lnl(T, inst.noise_var, inst.d, inst.kbin, phi, inst.spec.lssm_prior_var)["lnl"]
        assert abs(got - ref) <= 1e-10 * abs(ref)


def _unitary_closed_form(T, sigma2, d, kbin, phi, lssm_var):
    """T unitary, N = sigma^2 I: M = I / sigma^2, so Sigma is diagonal."""
    phi_diag = np.where(kbin >= 0, 10.0 ** np.asarray(phi)[np.maximum(kbin, 0)], lssm_var)
    s = 1.0 / sigma2 + 1.0 / phi_diag
    td = T.conj().T @ d
    logdet_sigma = float(np.sum(np.log(s)))
    q = float(np.sum(np.abs(td) ** 2 / sigma2 ** 2 / s))
    logdet_phi = float(np.sum(np.log(phi_diag)))
    return -0.5 * logdet_phi - 0.5 * logdet_sigma + 0.5 * q, logdet_sigma, q


@pytest.mark.parametrize("kind", ["qr", "dft"])
def test_unitary_closed_form(kind):
    g = np.random.default_rng(11)
    n = 16
    if kind == "qr":
        Z = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
        T, _ = np.linalg.qr(Z)
    else:
        k = np.arange(n)
        T = np.exp(-2j * np.pi * np.outer(k, k) / n) / math.sqrt(n)
    kbin = np.array([j % 4 - 1 for j in range(n)], dtype=np.int32)   # -1, 0, 1, 2
    sigma2 = 0.7
    d = g.standard_normal(n) + 1j * g.standard_normal(n)
    nv = np.full(n, sigma2)
    for phi in g.uniform(-2, 2, (3, 3)):
        ref, ref_ld, ref_q = _unitary_closed_form(T, sigma2, d, kbin, phi, 5.0)
        r = oracle_lnl(T, nv, d, kbin, phi, 5.0)
        assert abs(r["lnl"] - ref) <= 1e-12 * max(1.0, abs(ref))
        assert abs(r["logdet_sigma"] - ref_ld) <= 1e-12 * max(1.0, abs(ref_ld))
        assert abs(r["q"] - ref_q) <= 1e-12 * abs(ref_q)


def test_scalar_closed_form():
    # n_vis = n_model = 1: Sigma = |t|^2/s2 + 10^-phi, dbar = conj(t) d / s2.
    t, s2, d = 1.0 + 1.0j, 2.0, 3.0 - 1.0j
    for phi in (-1.5, 0.0, 0.7):
        sig = abs(t) ** 2 / s2 + 10.0 ** (-phi)
        dbar = np.conj(t) * d / s2
        ref = -0.5 * phi * math.log(10.0) - 0.5 * math.log(sig) + 0.5 * abs(dbar) ** 2 / sig
        got = oracle_lnl(np.array([[t]]), np.array([s2]), np.array([d]),
                         np.array([0], np.int32), [phi], 1.0)["lnl"]
        assert abs(got - ref) <= 1e-14 * max(1.0, abs(ref))
    # the phi = 0 case written out by hand: Sigma = 2, dbar = 1 - 2i, q = 5/2
    got = oracle_lnl(np.array([[t]]), np.array([s2]), np.array([d]),
                     np.array([0], np.int32), [0.0], 1.0)["lnl"]
    assert abs(got - (1.25 - 0.5 * math.log(2.0))) < 1e-15


def _small_hex():
    return build_instrument(get_spec("C1", nu=5, nf=6, n_t=2, n_bl=20, n_pix=16, n_k=3))


@pytest.mark.parametrize("which", ["C0", "hex"])
def test_dense_vs_structured_precompute(which):
    inst = build_instrument("C0") if which == "C0" else _small_hex()
    T = expand_T(inst)
    Md = O.herm_dense(T, inst.noise_var)
    Ms = O.herm_structured(inst.A, inst.W, inst.noise_var)
    scale = np.abs(Md).max()
    assert np.abs(Md - Ms).max() <= 1e-12 * scale
    db = O.dbar_dense(T, inst.noise_var, inst.d)
    db2 = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
    assert np.abs(db - db2).max() <= 1e-12 * np.abs(db).max()
    # exact Hermiticity and a real diagonal (lower triangle authoritative)
    assert np.array_equal(Md, Md.conj().T)
    assert np.all(Md.diagonal().imag == 0)
    # positive semi-definite up to rounding
    ev = np.linalg.eigvalsh(Md)
    assert ev.min() >= -1e-12 * scale * Md.shape[0]


def test_cholesky_against_library():
    inst = build_instrument("C0")
    M = O.herm_structured(inst.A, inst.W, inst.noise_var)
    for phi in draw_phi("C0", 3):
        phi_inv, _ = O.prior_diag(phi, inst.kbin, inst.spec.lssm_prior_var)
        S = M + np.diag(phi_inv)
        L, info = O.cholesky_lower(S)
        assert info == 0
        Lref = np.linalg.cholesky(S)
        assert np.abs(L - Lref).max() <= 1e-10 * np.abs(Lref).max()
        assert np.all(L.diagonal().real > 0) and np.all(L.diagonal().imag == 0)
        n = S.shape[0]
        assert np.linalg.norm(L @ L.conj().T - S) <= 10 * n * np.finfo(float).eps * np.linalg.norm(S)
        _, ld = np.linalg.slogdet(S)
        assert abs(2 * np.sum(np.log(L.diagonal().real)) - ld) <= 1e-12 * abs(ld)
        b = np.arange(n) + 1j
        y = O.forward_sub(L, b)
        assert np.abs(L @ y - b).max() <= 1e-9 * np.abs(b).max()
        x = O.back_sub(L, y)
        assert np.abs(L.conj().T @ x - y).max() <= 1e-9 * np.abs(y).max()


def test_posterior_mean_residual_C0():
    inst = build_instrument("C0")
    M = O.herm_structured(inst.A, inst.W, inst.noise_var)
    db = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
    for phi in draw_phi("C0", 3):
        r = O.evaluate(M, db, inst.kbin, phi, inst.spec.lssm_prior_var)
        phi_inv, _ = O.prior_diag(phi, inst.kbin, inst.spec.lssm_prior_var)
        S = M + np.diag(phi_inv)
        assert np.linalg.norm(S @ r["abar"] - db) <= 1e-12 * np.linalg.norm(db) * 1e3
        x = np.linalg.solve(S, db)
        assert np.linalg.norm(r["abar"] - x) <= 1e-8 * np.linalg.norm(x)


def test_posterior_mean_flat_prior_limit():
    # Phi -> infinity with T of full column rank: abar -> the weighted least-squares fit.
    p = random_problem(40, 10, 3, 5)
    kbin = (np.arange(10) % 3).astype(np.int32)
    sig = np.sqrt(p["noise_var"])
    ref, *_ = np.linalg.lstsq(p["T"] / sig[:, None], p["d"] / sig, rcond=None)
    r = oracle_lnl(p["T"], p["noise_var"], p["d"], kbin, [14.0, 14.0, 14.0], 1.0)
    assert np.linalg.norm(r["abar"] - ref) <= 1e-8 * np.linalg.norm(ref)


def test_lnl_gradient_finite_difference():
    inst = build_instrument("C0")
    M = O.herm_structured(inst.A, inst.W, inst.noise_var)
    db = O.dbar_structured(inst.A, inst.W, inst.noise_var, inst.d)
    lv = inst.spec.lssm_prior_var
    phi0 = draw_phi("C0", 1)[0]
    r = O.evaluate(M, db, inst.kbin, phi0, lv)
    phi_inv, _ = O.prior_diag(phi0, inst.kbin, lv)
    S_inv = np.linalg.inv(M + np.diag(phi_inv))
    # d lnL / d Phi^-1_jj = -1/2 (Sigma^-1)_jj - 1/2 |abar_j|^2 + 1/2 Phi_jj
    g_diag = -0.5 * S_inv.diagonal().real - 0.5 * np.abs(r["abar"]) ** 2 + 0.5 / phi_inv
    h = 1e-5
    for i in range(len(phi0)):
        sel = inst.kbin == i
        analytic = float(np.sum(g_diag[sel] * (-math.log(10.0)) * phi_inv[sel]))
        e = np.zeros_like(phi0)
        e[i] = h
        fd = (O.evaluate(M, db, inst.kbin, phi0 + e, lv)["lnl"]
              - O.evaluate(M, db, inst.kbin, phi0 - e, lv)["lnl"]) / (2 * h)
        assert abs(fd - analytic) <= 1e-6 * max(1.0, abs(analytic))


def test_not_positive_definite_status():
    M = np.diag([1.0, -5.0, 1.0]).astype(np.complex128)
    r = O.evaluate(M, np.ones(3, np.complex128), np.zeros(3, np.int32), [0.0], 1.0)
    assert r["status"] == 2 and r["lnl"] == -math.inf


def test_prior_diag_logdet():
    kbin = np.array([0, 1, -1, 1, 0], np.int32)
    phi = np.array([0.3, -1.2])
    inv, ld = O.prior_diag(phi, kbin, 7.0)
    expect = np.array([10 ** -0.3, 10 ** 1.2, 1 / 7.0, 10 ** 1.2, 10 ** -0.3])
    assert np.allclose(inv, expect, rtol=1e-15)
    assert abs(ld - (2 * 0.3 * math.log(10) + 2 * -1.2 * math.log(10) + math.log(7.0))) < 1e-14


# ---------------------------------------------------------------------------
# Planted mistakes: each mutation of the oracle must be caught by a pin above.
# ---------------------------------------------------------------------------

def _woodbury_ok():
    p = random_problem(12, 5, 2, 0)
    for phi in ([0.3, -0.8], [1.5, 1.9]):
        ref = brute_force_lnl(p["T"], p["noise_var"], p["d"], p["kbin"], phi, 3.0)
        try:
            got = oracle_lnl(p["T"], p["noise_var"], p["d"], p["kbin"], phi, 3.0)["lnl"]
        except (ValueError, ZeroDivisionError, FloatingPointError):
            return False                        # a crash also counts as caught
        if not abs(got - ref) <= 1e-10 * abs(ref):
            return False
    return True


def test_mutations_are_caught(monkeypatch):
    assert _woodbury_ok()

    def back_sub_no_conj(L, y):
        N = L.shape[0]
        x = np.zeros(N, dtype=np.complex128)
        for j in range(N - 1, -1, -1):
            x[j] = (y[j] - L[j + 1:, j] @ x[j + 1:]) / L[j, j].real
        return x

    def chol_no_conj(S):
        N = S.shape[0]
        L = np.zeros((N, N), dtype=np.complex128)
        for j in range(N):
            row = L[j, :j]
            L[j, j] = math.sqrt(S[j, j].real - float(np.sum(np.abs(row) ** 2)))
            L[j + 1:, j] = (S[j + 1:, j] - L[j + 1:, :j] @ row) / L[j, j].real
        return L, 0

    orig_prior = OL.prior_diag

    def prior_flipped(phi, kbin, lv):
        inv, ld = orig_prior(-np.asarray(phi), kbin, lv)
        return inv, -ld

    def herm_transposed(T, nv):
        M = (T.T * (1.0 / nv)[None, :]) @ T.conj()
        return OL._hermitian_from_lower(M)

    orig_eval = OL.evaluate

    def logdet_half(M, dbar, kbin, phi, lv):
        r = orig_eval(M, dbar, kbin, phi, lv)
        r["lnl"] += 0.25 * r["logdet_sigma"]       # as if log|Sigma| = sum ln L_jj
        return r

    for name, fn in [("back_sub", back_sub_no_conj), ("cholesky_lower", chol_no_conj),
                     ("prior_diag", prior_flipped), ("herm_dense", herm_transposed),
                     ("evaluate", logdet_half)]:
        with monkeypatch.context() as m:
            m.setattr(OL, name, fn)
            m.setattr(O, name, fn)
            assert not _woodbury_ok(), f"mutation of {name} not caught"
    assert _woodbury_ok()
