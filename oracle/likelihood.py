"""Oracle: the exact marginal likelihood of the joint EoR + foreground model.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

The method (Sec. "Statement of need": amplitudes are marginalised so that the
power-spectrum parameters phi can be sampled directly from their marginal
posterior) evaluates, for each sampler point phi,

    Phi      = diag prior variance of the model amplitudes set by phi
    Sigma    = T^H N^-1 T + Phi^-1
    dbar     = T^H N^-1 d
    abar     = Sigma^-1 dbar                  (maximum-a-posteriori amplitudes)
    lnL      = -1/2 log|Phi| - 1/2 log|Sigma| + 1/2 dbar^H Sigma^-1 dbar

with the prior built from the spherically-averaged power in k bins
(Eq. for P(k_i): shells k_i <= |k| < k_i + dk_i), one amplitude phi_i per bin
(phi_i in Fig. 1's caption).  Reading used here: phi_i is log10 of the prior
variance of every EoR amplitude in bin i; foreground (LSSM) amplitudes get a
fixed variance.  Everything is complex128 / float64, unblocked, in the order
the definitions state.  A library matrix product is used as one step where the
definition is a matrix product.
"""

from __future__ import annotations

import math

import numpy as np

LN10 = math.log(10.0)


# --------------------------------------------------------------------------
# Precompute: T^H N^-1 T and T^H N^-1 d
# --------------------------------------------------------------------------

def herm_dense(T: np.ndarray, noise_var: np.ndarray) -> np.ndarray:
    """M = T^H N^-1 T with N = diag(noise_var).

    One library matrix product, then the lower triangle is taken as
    authoritative and mirrored so that M is exactly Hermitian and its diagonal
    exactly real.
    """
    M = (T.conj().T * (1.0 / noise_var)[None, :]) @ T
    return _hermitian_from_lower(M)


def dbar_dense(T: np.ndarray, noise_var: np.ndarray, d: np.ndarray) -> np.ndarray:
    """dbar = T^H N^-1 d."""
    return T.conj().T @ (d / noise_var)


def herm_structured(A: np.ndarray, W: np.ndarray, noise_var: np.ndarray) -> np.ndarray:
    """M from the factored instrument T[(f,tb),(c,x)] = A_f[tb,c] W[f,x].

    M[(c,x),(c',x')] = sum_f conj(W[f,x]) W[f,x'] G_f[c,c'],
    G_f = A_f^H N_f^-1 A_f.  Independent of ``herm_dense``: it never forms T.
    """
    nf, ntb, nc = A.shape
    nx = W.shape[1]
    nv = noise_var.reshape(nf, ntb)
    M = np.zeros((nc * nx, nc * nx), dtype=np.complex128)
    for f in range(nf):
        G = (A[f].conj().T * (1.0 / nv[f])[None, :]) @ A[f]
        WW = np.outer(W[f].conj(), W[f])
        M += np.kron(G, WW)
    return _hermitian_from_lower(M)


def dbar_structured(A: np.ndarray, W: np.ndarray, noise_var: np.ndarray,
                    d: np.ndarray) -> np.ndarray:
    """dbar[(c,x)] = sum_f conj(W[f,x]) sum_tb conj(A_f[tb,c]) d[f,tb] / sigma^2."""
    nf, ntb, nc = A.shape
    nx = W.shape[1]
    dw = (d / noise_var).reshape(nf, ntb)
    out = np.zeros((nc, nx), dtype=np.complex128)
    for f in range(nf):
        ad = A[f].conj().T @ dw[f]               # (nc,)
        out += np.outer(ad, W[f].conj())
    return out.reshape(-1)


def _hermitian_from_lower(M: np.ndarray) -> np.ndarray:
    L = np.tril(M, -1)
    out = L + L.conj().T
    out[np.diag_indices_from(out)] = M.diagonal().real
    return out


# --------------------------------------------------------------------------
# Prior from phi
# --------------------------------------------------------------------------

def prior_diag(phi: np.ndarray, kbin: np.ndarray, lssm_prior_var: float):
    """Diagonal prior: Phi_jj = 10**phi[kbin[j]] for EoR modes, lssm_prior_var else.

    Returns (Phi^-1 diagonal, log|Phi|), log|Phi| = sum_j ln Phi_jj.
    """
    phi = np.asarray(phi, dtype=np.float64)
    N = kbin.shape[0]
    phi_inv = np.empty(N)
    logdet = 0.0
    for j in range(N):
        if kbin[j] >= 0:
            p = phi[kbin[j]]
            phi_inv[j] = 10.0 ** (-p)
            logdet += p * LN10
        else:
            phi_inv[j] = 1.0 / lssm_prior_var
            logdet += math.log(lssm_prior_var)
    return phi_inv, logdet


# --------------------------------------------------------------------------
# Cholesky and triangular solves (unblocked)
# --------------------------------------------------------------------------

def cholesky_lower(S: np.ndarray):
    """Sigma = L L^H, L lower with real positive diagonal; column by column.

    L[j,j] = sqrt(S[j,j] - sum_{k<j} |L[j,k]|^2)
    L[i,j] = (S[i,j] - sum_{k<j} L[i,k] conj(L[j,k])) / L[j,j],  i > j
    Only the lower triangle of S is read.  Returns (L, info) with info = 0 on
    success or the 1-based column at which the pivot was not positive.
    """
    N = S.shape[0]
    L = np.zeros((N, N), dtype=np.complex128)
    for j in range(N):
        row = L[j, :j]
        piv = S[j, j].real - float(np.sum(row.real ** 2 + row.imag ** 2))
        if not (piv > 0.0) or not math.isfinite(piv):
            return L, j + 1
        ljj = math.sqrt(piv)
        L[j, j] = ljj
        if j + 1 < N:
            col = S[j + 1:, j] - L[j + 1:, :j] @ row.conj()
            L[j + 1:, j] = col / ljj
    return L, 0


def forward_sub(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve L y = b, L lower triangular."""
    N = L.shape[0]
    y = np.zeros(N, dtype=np.complex128)
    for j in range(N):
        y[j] = (b[j] - L[j, :j] @ y[:j]) / L[j, j]
    return y


def back_sub(L: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Solve L^H x = y, L lower triangular: x_j = (y_j - sum_{k>j} conj(L[k,j]) x_k) / L[j,j]."""
    N = L.shape[0]
    x = np.zeros(N, dtype=np.complex128)
    for j in range(N - 1, -1, -1):
        x[j] = (y[j] - L[j + 1:, j].conj() @ x[j + 1:]) / L[j, j].real
    return x


# --------------------------------------------------------------------------
# The likelihood
# --------------------------------------------------------------------------

def evaluate(M: np.ndarray, dbar: np.ndarray, kbin: np.ndarray, phi: np.ndarray,
             lssm_prior_var: float) -> dict:
    """lnL(phi) and the posterior mean for one prior point.

    Sigma = M + diag(Phi^-1); L = chol(Sigma); log|Sigma| = 2 sum ln L_jj;
    abar = L^-H L^-1 dbar; q = Re(dbar^H abar);
    lnL = -1/2 log|Phi| - 1/2 log|Sigma| + 1/2 q.
    A non-positive pivot gives status = 1-based column and lnL = -inf.
    """
    phi_inv, logdet_phi = prior_diag(phi, kbin, lssm_prior_var)
    S = M.copy()
    S[np.diag_indices_from(S)] += phi_inv
    L, info = cholesky_lower(S)
    if info:
        return {"lnl": -math.inf, "status": info, "logdet_phi": logdet_phi,
                "logdet_sigma": math.nan, "q": math.nan, "abar": None}
    logdet_sigma = 2.0 * float(np.sum(np.log(L.diagonal().real)))
    y = forward_sub(L, dbar)
    abar = back_sub(L, y)
    q = float(np.real(np.vdot(dbar, abar)))
    lnl = -0.5 * logdet_phi - 0.5 * logdet_sigma + 0.5 * q
    return {"lnl": lnl, "status": 0, "logdet_phi": logdet_phi,
            "logdet_sigma": logdet_sigma, "q": q, "abar": abar}
