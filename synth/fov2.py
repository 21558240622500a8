"""An instrument whose EoR and foreground models have separate fields of view.

The paper lets the EoR and the foreground sky models cover different fields
of view, the foreground one as wide as the whole sky (Sec. "Running
BayesEoR": independent model FoVs; an all-sky foreground model for the
analysis of Burba et al. 2023).  This module fixes one seeded reading of
that, built from the same pieces as `instrument.build_instrument`:

* EoR model: the single-FoV instrument's uv cells (cell size du, FoV = 1/du,
  n_pix x n_pix sky pixels) with the eta basis E only; model index
  j = c * n_eta + x.
* Foreground model: its own uv grid with cell size du / s (s = fg_fov_scale
  >= 1, so FoV_fg = s FoV), nu_fg x nu_fg cells without (0, 0), n_pix x n_pix
  pixels over [-FoV_fg / 2, FoV_fg / 2), the same primary beam, and the
  power-law basis S; model index n_eor + c' * n_lssm + y.
* T = [A_f^eor (x) E | A_f^fg (x) S] as a dense matrix (small
  configurations), visibility index (f * n_t + t) * n_bl + b as before.
* Data: EoR amplitudes CN(0, P(k_i)) as before, foreground amplitudes of
  the wide model CN(0, lssm_var), noise at SNR 10 of the model visibilities.

With s = 1 and nu_fg = nu the columns are those of the single-FoV
instrument, reordered (EoR block first).  Seeds: the config's geometry,
signal (stream 11) and noise (stream 12) streams.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .instrument import (C_LIGHT, LATITUDE_DEG, LSSM_BETAS, SIDEREAL_DAY_S, CONFIGS, InstrumentSpec, _baselines,
                         _cells, _rng, _uv_at)


@dataclass
class Fov2Instrument:
    spec: InstrumentSpec
    fg_fov_scale: float
    nu_fg: int
    T: np.ndarray               # (n_vis, n_model) complex128, dense
    n_eor: int                  # EoR columns (first block)
    kbin: np.ndarray            # (n_model,) int32, -1 for foreground modes
    k_edges: np.ndarray
    a_true: np.ndarray
    sigma: float
    noise_var: np.ndarray
    d: np.ndarray
    extra: dict = field(default_factory=dict)

    @property
    def n_model(self) -> int:
        return self.T.shape[1]

    @property
    def n_vis(self) -> int:
        return self.T.shape[0]


def _response(spec: InstrumentSpec, uv_m: np.ndarray, freqs: np.ndarray, du: float, nu: int) -> np.ndarray:
    """A_f for f in freqs: NUDFT at the baselines' uv points . diag(beam) .
    unitary inverse 2-D DFT from the nu x nu grid of cell size du (no (0, 0)
    cell) to n_pix x n_pix sky pixels over a FoV of 1 / du."""
    fov = 1.0 / du
    npx = spec.n_pix
    lm = (np.arange(npx) - npx / 2.0) * (fov / npx)
    L, Mm = np.meshgrid(lm, lm, indexing="xy")
    l_flat, m_flat = L.ravel(), Mm.ravel()
    s = math.radians(spec.beam_fwhm_deg) / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    beam = np.exp(-(l_flat ** 2 + m_flat ** 2) / (2.0 * s * s))
    cells = _cells(nu)
    px = np.arange(npx) - npx / 2.0
    PX, PY = np.meshgrid(px, px, indexing="xy")
    phase = (np.outer(PX.ravel(), cells[:, 0]) + np.outer(PY.ravel(), cells[:, 1])) / npx
    BF = beam[:, None] * (np.exp(2j * np.pi * phase) / npx)
    A = np.empty((len(freqs), uv_m.shape[0], len(cells)), dtype=np.complex128)
    for f, nu_f in enumerate(freqs):
        uvw = uv_m * (nu_f / C_LIGHT)
        A[f] = np.exp(-2j * np.pi * (np.outer(uvw[:, 0], l_flat) + np.outer(uvw[:, 1], m_flat))) @ BF
    return A


def build_fov2(spec: InstrumentSpec | str, fg_fov_scale: float = 2.0, nu_fg: int | None = None,
               with_data: bool = True) -> Fov2Instrument:
    """The two-FoV instrument of a configuration (see the module docstring)."""
    if isinstance(spec, str):
        spec = CONFIGS[spec]
    if fg_fov_scale < 1.0:
        raise ValueError("the foreground FoV is at least the EoR one")
    nu_fg = spec.nu if nu_fg is None else nu_fg
    lat = math.radians(LATITUDE_DEG)
    bl = _baselines(spec)
    ha = (np.arange(spec.n_t) - (spec.n_t - 1) / 2.0) * spec.t_step_s * 2.0 * math.pi / SIDEREAL_DAY_S
    freqs = spec.f0_hz + spec.df_hz * np.arange(spec.nf)
    f_top = spec.f0_hz + spec.df_hz * ((spec.nf_grid or spec.nf) - 1)
    h = (spec.nu - 1) // 2
    du = np.max(np.hypot(bl[:, 0], bl[:, 1])) * f_top / C_LIGHT / h
    uv_m = _uv_at(bl, ha, lat).reshape(-1, 2)
    A_e = _response(spec, uv_m, freqs, du, spec.nu)
    A_g = _response(spec, uv_m, freqs, du / fg_fov_scale, nu_fg)
    fi = np.arange(spec.nf)
    eta = np.arange(spec.nf) - spec.nf // 2
    E = np.exp(2j * np.pi * np.outer(fi, eta) / spec.nf) / math.sqrt(spec.nf)
    S = np.stack([(freqs / spec.f0_hz) ** (-b) for b in LSSM_BETAS[: spec.n_lssm]], axis=1)
    S = (S / np.linalg.norm(S, axis=0, keepdims=True)).astype(np.complex128)
    n_tb = uv_m.shape[0]
    T_e = (A_e[:, :, :, None] * E[:, None, None, :]).reshape(spec.nf * n_tb, -1)
    T_g = (A_g[:, :, :, None] * S[:, None, None, :]).reshape(spec.nf * n_tb, -1)
    T = np.ascontiguousarray(np.concatenate([T_e, T_g], axis=1))
    n_eor = T_e.shape[1]
    # k bins of the EoR modes: |k| = sqrt(i_u^2 + i_v^2 + i_eta^2), N_k log-spaced shells
    cells = _cells(spec.nu)
    kmag = np.sqrt((cells[:, 0:1] ** 2 + cells[:, 1:2] ** 2 + eta[None, :] ** 2).astype(np.float64)).ravel()
    edges = kmag.min() * (kmag.max() / kmag.min()) ** (np.arange(spec.n_k + 1) / spec.n_k)
    kb = np.clip(np.searchsorted(edges, kmag, side="right") - 1, 0, spec.n_k - 1).astype(np.int32)
    if np.any(np.bincount(kb, minlength=spec.n_k) == 0):
        raise ValueError("empty k bin")
    kbin = np.concatenate([kb, np.full(T_g.shape[1], -1, np.int32)])
    inst = Fov2Instrument(spec=spec, fg_fov_scale=fg_fov_scale, nu_fg=nu_fg, T=T, n_eor=n_eor, kbin=kbin,
                          k_edges=edges, a_true=np.zeros(T.shape[1], np.complex128), sigma=0.0,
                          noise_var=np.zeros(T.shape[0]), d=np.zeros(T.shape[0], np.complex128))
    if with_data:
        kc = np.sqrt(edges[:-1] * edges[1:])
        pk = (kc / float(np.exp(np.mean(np.log(kc))))) ** -2.0
        g = _rng(spec, 11)
        z = (g.standard_normal(inst.n_model) + 1j * g.standard_normal(inst.n_model)) / math.sqrt(2.0)
        var = np.where(kbin >= 0, pk[np.maximum(kbin, 0)], spec.lssm_prior_var * 1e-2)
        a = z * np.sqrt(var)
        v = T @ a
        sigma = math.sqrt(float(np.mean(np.abs(v) ** 2))) / spec.snr
        g2 = _rng(spec, 12)
        n = sigma * (g2.standard_normal(inst.n_vis) + 1j * g2.standard_normal(inst.n_vis)) / math.sqrt(2.0)
        inst.a_true, inst.sigma = a, sigma
        inst.noise_var = np.full(inst.n_vis, sigma * sigma)
        inst.d = v + n
        inst.extra["pk_true"] = pk
    return inst


def single_fov_T(inst: Fov2Instrument) -> np.ndarray:
    """The single-FoV model of the same instrument (the foreground model on
    the EoR grid, s = 1, nu_fg = nu), in the same column order: the
    alternative model for a model comparison on inst's data."""
    return build_fov2(inst.spec, 1.0, inst.spec.nu, with_data=False).T
