"""Synthetic drift-scan interferometer shaped like the paper's workloads.

The paper forward-models an interferometer: visibilities per baseline, time
and frequency are a linear function of the EoR uv-eta Fourier amplitudes and
of a smooth-spectrum foreground model (Sec. "Running BayesEoR": instrument
model = primary beam + uv sampling; Sec. "Statement of need": joint EoR and
foreground model).  The paper does not print the model, so this module fixes
one concrete, seeded reading of it:

* uv grid: cells (i_u, i_v), |i_u|,|i_v| <= (nu-1)/2, the (0,0) cell removed.
* sky grid: n_pix x n_pix pixels over [-FoV/2, FoV/2), FoV = 1/du, with du
  set so that the longest baseline at the top channel reaches the grid edge.
* per frequency f:  A_f = NUDFT_f . diag(beam) . F_uv  (rows (t, b), cols c)
  - F_uv: unitary inverse 2-D DFT from uv cells to sky pixels,
  - beam: achromatic Gaussian, FWHM 10 deg,
  - NUDFT_f: exp(-2 pi i (u l + v m)) at the baseline's uv point at time t,
    frequency f (drift scan, 11 s per sample, latitude -30.72 deg).
* spectral basis W = [E | S]:  E = unitary inverse eta-DFT (n_eta = n_f,
  eta index in [-n_f/2, n_f/2-1]); S = power laws (nu/nu_0)^(-beta),
  beta = 2.63, 2.82, 3.0, each column scaled to unit 2-norm.
* T[(f, t, b), (c, x)] = A_f[(t, b), c] * W[f, x]; model index j = c*n_x + x,
  visibility index (f*n_t + t)*n_bl + b.
* k bins: |k| = sqrt(i_u^2 + i_v^2 + i_eta^2) in grid units for EoR modes;
  N_k log-spaced shells between min and max |k| (spherical shells
  k_i <= |k| < k_i + dk_i of the paper's P(k_i) average).  LSSM modes -> -1.
* signal a_true: EoR ~ CN(0, P(k_i)), P(k) = (k/k_piv)^-2; LSSM ~ CN(0, 1).
* noise: uniform sigma = rms(T a_true) / SNR, complex CN(0, sigma^2).

Random draws use NumPy PCG64 with per-config seeds: 0 geometry, 1 signal,
2 noise, 3 phi.  All arithmetic is float64 / complex128.
"""

from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299_792_458.0
SIDEREAL_DAY_S = 86_164.0905
LATITUDE_DEG = -30.72
LSSM_BETAS = (2.63, 2.82, 3.0)


@dataclass(frozen=True)
class InstrumentSpec:
    name: str
    nu: int                      # uv grid side (odd); cells exclude (0, 0)
    nf: int                      # frequency channels = eta modes
    f0_hz: float
    df_hz: float
    n_lssm: int
    n_pix: int
    n_t: int
    n_k: int
    n_bl: int
    layout: str                  # "random" (lengths U[bl_min, bl_max]) or "hex"
    bl_min_m: float = 14.0
    bl_max_m: float = 60.0
    hex_spacing_m: float = 14.6
    hex_rings: int = 8
    t_step_s: float = 11.0
    beam_fwhm_deg: float = 10.0
    lssm_prior_var: float = 100.0
    snr: float = 10.0
    nf_grid: int = 0             # channels used to set du (0 = nf): sub-bands share a grid
    seed: int = 0                # config id folded into every seed

    @property
    def n_cells(self) -> int:
        return self.nu * self.nu - 1

    @property
    def n_x(self) -> int:
        return self.nf + self.n_lssm

    @property
    def n_model(self) -> int:
        return self.n_cells * self.n_x

    @property
    def n_tb(self) -> int:
        return self.n_t * self.n_bl

    @property
    def n_vis(self) -> int:
        return self.nf * self.n_tb


# The five workload shapes.  C3 is three sub-band instruments on one uv grid.
CONFIGS: dict[str, InstrumentSpec] = {
    "C0": InstrumentSpec("C0", nu=5, nf=8, f0_hz=150e6, df_hz=1e6, n_lssm=2, n_pix=16,
                         n_t=1, n_k=4, n_bl=30, layout="random", seed=0),
    "C1": InstrumentSpec("C1", nu=9, nf=38, f0_hz=158.3e6, df_hz=97.65625e3, n_lssm=3,
                         n_pix=32, n_t=19, n_k=9, n_bl=126, layout="hex", seed=1),
    "C3_24": InstrumentSpec("C3_24", nu=15, nf=24, f0_hz=158.3e6, df_hz=97.65625e3, n_lssm=3,
                            n_pix=32, n_t=16, n_k=9, n_bl=331, layout="hex", nf_grid=48,
                            seed=324),
    "C3_32": InstrumentSpec("C3_32", nu=15, nf=32, f0_hz=158.3e6, df_hz=97.65625e3, n_lssm=3,
                            n_pix=32, n_t=16, n_k=9, n_bl=331, layout="hex", nf_grid=48,
                            seed=332),
    "C3_48": InstrumentSpec("C3_48", nu=15, nf=48, f0_hz=158.3e6, df_hz=97.65625e3, n_lssm=3,
                            n_pix=32, n_t=16, n_k=9, n_bl=331, layout="hex", nf_grid=48,
                            seed=348),
}


def get_spec(name: str, **overrides) -> InstrumentSpec:
    spec = CONFIGS[name]
    return dataclasses.replace(spec, **overrides) if overrides else spec


def _rng(spec: InstrumentSpec, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([stream, spec.seed])))


@dataclass
class Instrument:
    spec: InstrumentSpec
    bl_enu_m: np.ndarray          # (n_bl, 3)
    hour_angle_rad: np.ndarray    # (n_t,)
    freqs_hz: np.ndarray          # (nf,)
    du: float                     # uv cell size in wavelengths
    cells: np.ndarray             # (n_cells, 2) int (i_u, i_v)
    A: np.ndarray                 # (nf, n_tb, n_cells) complex128
    W: np.ndarray                 # (nf, n_x) complex128
    kbin: np.ndarray              # (n_model,) int32, -1 for LSSM modes
    k_edges: np.ndarray           # (n_k + 1,)
    k_mag: np.ndarray             # (n_model,) |k| in grid units (0 for LSSM)
    a_true: np.ndarray            # (n_model,) complex128
    sigma: float
    noise_var: np.ndarray         # (n_vis,) float64
    d: np.ndarray                 # (n_vis,) complex128
    extra: dict = field(default_factory=dict)

    @property
    def n_model(self) -> int:
        return self.spec.n_model

    @property
    def n_vis(self) -> int:
        return self.spec.n_vis


def _baselines(spec: InstrumentSpec) -> np.ndarray:
    if spec.layout == "random":
        g = _rng(spec, 0)
        length = g.uniform(spec.bl_min_m, spec.bl_max_m, spec.n_bl)
        angle = g.uniform(0.0, math.pi, spec.n_bl)
        return np.stack([length * np.cos(angle), length * np.sin(angle),
                         np.zeros(spec.n_bl)], axis=1)
    if spec.layout == "hex":
        R, s = spec.hex_rings, spec.hex_spacing_m
        ant = []
        for q in range(-R, R + 1):
            for r in range(-R, R + 1):
                if abs(q + r) <= R:
                    ant.append((s * (q + 0.5 * r), s * (math.sqrt(3.0) / 2.0) * r))
        ant = np.array(ant)
        diff = (ant[:, None, :] - ant[None, :, :]).reshape(-1, 2)
        key = np.round(diff * 1000.0).astype(np.int64)
        _, idx = np.unique(key, axis=0, return_index=True)
        vec = diff[np.sort(idx)]
        keep = (vec[:, 0] > 1e-6) | ((np.abs(vec[:, 0]) <= 1e-6) & (vec[:, 1] > 1e-6))
        vec = vec[keep]
        length = np.hypot(vec[:, 0], vec[:, 1])
        angle = np.arctan2(vec[:, 1], vec[:, 0])
        order = np.lexsort((np.round(angle, 9), np.round(length, 6)))
        vec = vec[order][: spec.n_bl]
        if len(vec) < spec.n_bl:
            raise ValueError("hex layout too small for n_bl")
        return np.concatenate([vec, np.zeros((spec.n_bl, 1))], axis=1)
    raise ValueError(spec.layout)


def _uv_at(bl_enu: np.ndarray, hour_angle: np.ndarray, lat_rad: float) -> np.ndarray:
    """(n_t, n_bl, 2) baseline uv in metres for a zenith-at-transit drift scan."""
    E, N, U = bl_enu[:, 0], bl_enu[:, 1], bl_enu[:, 2]
    X = -math.sin(lat_rad) * N + math.cos(lat_rad) * U
    Y = E
    Z = math.cos(lat_rad) * N + math.sin(lat_rad) * U
    H = hour_angle[:, None]
    dec = lat_rad
    u = np.sin(H) * X + np.cos(H) * Y
    v = -math.sin(dec) * np.cos(H) * X + math.sin(dec) * np.sin(H) * Y + math.cos(dec) * Z
    return np.stack([u, v], axis=-1)


def _cells(nu: int) -> np.ndarray:
    h = (nu - 1) // 2
    out = [(iu, iv) for iv in range(-h, h + 1) for iu in range(-h, h + 1) if (iu, iv) != (0, 0)]
    return np.array(out, dtype=np.int64)


def build_instrument(spec: InstrumentSpec | str, with_data: bool = True,
                     A_from: "Instrument | None" = None) -> Instrument:
    """Build the factored instrument (A_f, W), k-bin map, signal and data.

    A_from: an instrument with the same geometry, grid and channel plan but at
    least as many channels; its per-frequency response matrices are reused
    (sub-bands of one band share them)."""
    if isinstance(spec, str):
        spec = CONFIGS[spec]
    lat = math.radians(LATITUDE_DEG)
    bl = _baselines(spec)
    ha = (np.arange(spec.n_t) - (spec.n_t - 1) / 2.0) * spec.t_step_s * 2.0 * math.pi / SIDEREAL_DAY_S
    freqs = spec.f0_hz + spec.df_hz * np.arange(spec.nf)
    nf_grid = spec.nf_grid or spec.nf
    f_top = spec.f0_hz + spec.df_hz * (nf_grid - 1)
    h = (spec.nu - 1) // 2
    u_max = np.max(np.hypot(bl[:, 0], bl[:, 1])) * f_top / C_LIGHT
    du = u_max / h
    fov = 1.0 / du
    npx = spec.n_pix
    lm = (np.arange(npx) - npx / 2.0) * (fov / npx)
    L, Mm = np.meshgrid(lm, lm, indexing="xy")          # [py, px]
    l_flat, m_flat = L.ravel(), Mm.ravel()
    s = math.radians(spec.beam_fwhm_deg) / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    beam = np.exp(-(l_flat ** 2 + m_flat ** 2) / (2.0 * s * s))
    cells = _cells(spec.nu)
    px = (np.arange(npx) - npx / 2.0)
    PX, PY = np.meshgrid(px, px, indexing="xy")
    phase = (np.outer(PX.ravel(), cells[:, 0]) + np.outer(PY.ravel(), cells[:, 1])) / npx
    F_uv = np.exp(2j * np.pi * phase) / npx               # (n_pix^2, n_cells), orthonormal cols
    BF = beam[:, None] * F_uv
    uv_m = _uv_at(bl, ha, lat).reshape(-1, 2)             # (n_tb, 2) metres, row = t*n_bl + b
    A = np.empty((spec.nf, spec.n_tb, spec.n_cells), dtype=np.complex128)
    reuse = (A_from is not None and A_from.A.shape[0] >= spec.nf
             and A_from.A.shape[1:] == A.shape[1:]
             and np.allclose(A_from.freqs_hz[: spec.nf], freqs, rtol=0, atol=1e-6)
             and abs(A_from.du - du) <= 1e-12 * du)
    for f, nu_f in enumerate(freqs):
        if reuse:
            A[f] = A_from.A[f]
            continue
        uvw = uv_m * (nu_f / C_LIGHT)
        nudft = np.exp(-2j * np.pi * (np.outer(uvw[:, 0], l_flat) + np.outer(uvw[:, 1], m_flat)))
        A[f] = nudft @ BF
    # spectral basis
    fi = np.arange(spec.nf)
    eta = np.arange(spec.nf) - spec.nf // 2
    E = np.exp(2j * np.pi * np.outer(fi, eta) / spec.nf) / math.sqrt(spec.nf)
    S = np.stack([(freqs / spec.f0_hz) ** (-b) for b in LSSM_BETAS[: spec.n_lssm]], axis=1)
    S = S / np.linalg.norm(S, axis=0, keepdims=True)
    W = np.concatenate([E, S.astype(np.complex128)], axis=1)
    # k bins
    n_x = spec.n_x
    kmag = np.zeros(spec.n_model)
    is_eor = np.zeros(spec.n_model, dtype=bool)
    for c, (iu, iv) in enumerate(cells):
        for x in range(spec.nf):
            j = c * n_x + x
            kmag[j] = math.sqrt(iu * iu + iv * iv + eta[x] * eta[x])
            is_eor[j] = True
    kmin, kmax = kmag[is_eor].min(), kmag[is_eor].max()
    edges = kmin * (kmax / kmin) ** (np.arange(spec.n_k + 1) / spec.n_k)
    kbin = np.full(spec.n_model, -1, dtype=np.int32)
    b = np.searchsorted(edges, kmag[is_eor], side="right") - 1
    kbin[is_eor] = np.clip(b, 0, spec.n_k - 1).astype(np.int32)
    counts = np.bincount(kbin[is_eor], minlength=spec.n_k)
    if np.any(counts == 0):
        raise ValueError(f"empty k bin in {spec.name}: {counts}")
    inst = Instrument(spec=spec, bl_enu_m=bl, hour_angle_rad=ha, freqs_hz=freqs, du=du,
                      cells=cells, A=A, W=W, kbin=kbin, k_edges=edges, k_mag=kmag,
                      a_true=np.zeros(spec.n_model, np.complex128), sigma=0.0,
                      noise_var=np.zeros(spec.n_vis), d=np.zeros(spec.n_vis, np.complex128))
    if with_data:
        _draw_data(inst)
    return inst


def geometry(inst: Instrument) -> dict:
    """The instrument's geometry in the fields of the library's instrument
    descriptor (beor_instrument_desc): from these the library builds the
    same A_f, W and k-bin map as build_instrument."""
    spec = inst.spec
    return {"nu": spec.nu, "nf": spec.nf, "nf_grid": spec.nf_grid, "n_pix": spec.n_pix, "n_k": spec.n_k,
            "f0_hz": spec.f0_hz, "df_hz": spec.df_hz, "beam_fwhm_rad": math.radians(spec.beam_fwhm_deg),
            "latitude_rad": math.radians(LATITUDE_DEG), "lssm_prior_var": spec.lssm_prior_var,
            "bl_enu_m": inst.bl_enu_m, "hour_angle_rad": inst.hour_angle_rad,
            "lssm_beta": np.array(LSSM_BETAS[: spec.n_lssm], np.float64)}


def bin_centres(edges: np.ndarray) -> np.ndarray:
    return np.sqrt(edges[:-1] * edges[1:])


def _draw_data(inst: Instrument) -> None:
    spec = inst.spec
    kc = bin_centres(inst.k_edges)
    k_piv = float(np.exp(np.mean(np.log(kc))))
    pk = (kc / k_piv) ** -2.0
    g = _rng(spec, 1)
    z = (g.standard_normal(spec.n_model) + 1j * g.standard_normal(spec.n_model)) / math.sqrt(2.0)
    var = np.where(inst.kbin >= 0, pk[np.maximum(inst.kbin, 0)], spec.lssm_prior_var * 1e-2)
    a = z * np.sqrt(var)
    v = apply_T(inst, a)
    sigma = math.sqrt(float(np.mean(np.abs(v) ** 2))) / spec.snr
    g2 = _rng(spec, 2)
    n = sigma * (g2.standard_normal(spec.n_vis) + 1j * g2.standard_normal(spec.n_vis)) / math.sqrt(2.0)
    inst.a_true = a
    inst.sigma = sigma
    inst.noise_var = np.full(spec.n_vis, sigma * sigma)
    inst.d = v + n
    inst.extra["pk_true"] = pk


def apply_T(inst: Instrument, a: np.ndarray) -> np.ndarray:
    """Model visibilities T a using the factored form (no dense T)."""
    spec = inst.spec
    a2 = a.reshape(spec.n_cells, spec.n_x)
    aw = inst.W @ a2.T                                   # (nf, n_cells): sum_x W[f,x] a[c,x]
    v = np.einsum("ftc,fc->ft", inst.A, aw)
    return v.reshape(-1)


def expand_T(inst: Instrument) -> np.ndarray:
    """Dense T (n_vis x n_model, complex128) from the factors; small configs only."""
    spec = inst.spec
    T = inst.A[:, :, :, None] * inst.W[:, None, None, :]
    return np.ascontiguousarray(T.reshape(spec.n_vis, spec.n_model))


def draw_phi(spec: InstrumentSpec | str, n: int, lo: float = -2.0, hi: float = 2.0,
             stream: int = 3) -> np.ndarray:
    """n seeded prior draws of log10 power amplitudes, U[lo, hi]^{n_k}."""
    if isinstance(spec, str):
        spec = CONFIGS[spec]
    return _rng(spec, stream).uniform(lo, hi, size=(n, spec.n_k))


def random_problem(n_vis: int, n_model: int, n_k: int, seed: int,
                   noise: float = 0.3) -> dict:
    """Tiny unstructured problem (dense random T) for brute-force checks."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([7, seed])))
    T = (g.standard_normal((n_vis, n_model)) + 1j * g.standard_normal((n_vis, n_model))) / math.sqrt(2.0)
    a = (g.standard_normal(n_model) + 1j * g.standard_normal(n_model)) / math.sqrt(2.0)
    nv = noise * noise * (0.5 + g.random(n_vis))
    d = T @ a + np.sqrt(nv / 2.0) * (g.standard_normal(n_vis) + 1j * g.standard_normal(n_vis))
    kbin = (np.arange(n_model) % (n_k + 1)).astype(np.int32) - 1   # some LSSM-like -1 modes
    kbin[:n_k] = np.arange(n_k)
    return {"T": T, "d": d, "noise_var": nv, "kbin": kbin, "n_k": n_k}
