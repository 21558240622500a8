"""ctypes binding of the C ABI in include/beor.h (argument marshalling only).

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA); the
library detects device pointers itself.  Streams default to torch's current
CUDA stream when torch has initialised CUDA, else the legacy default stream.
There is no fallback: without the compiled library every call raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BEOR_LIBRARY selects another build of the library (e.g. the bounds-checked
# _build/libbeor_checked.so); default: the regular build
LIB_PATH = os.environ.get("BEOR_LIBRARY") or os.path.join(_HERE, "_build", "libbeor.so")

PREC_FP64 = 0
PREC_MIXED = 1

_c = ctypes
_P = ctypes.c_void_p
_I64 = ctypes.c_int64


class BeorError(RuntimeError):
    pass


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "or python -m paper_2501_12928_gb300._build")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "beor_create": [_c.POINTER(_P), _c.c_int, _c.c_int],
        "beor_destroy": [_P],
        "beor_set_T": [_P, _P, _I64, _I64, _I64, _P, _c.c_int, _c.c_double],
        "beor_set_instrument": [_P, _P, _P, _c.c_int, _I64, _c.c_int, _c.c_int, _P, _c.c_int, _c.c_double],
        "beor_set_data": [_P, _P, _P],
        "beor_precompute": [_P, _P],
        "beor_lnl": [_P, _P, _c.c_int, _P, _P, _P],
        "beor_lnl_multi": [_P, _c.c_int, _P, _P, _P, _P, _P],
        "beor_lnl_multi_async": [_P, _c.c_int, _P, _P, _P, _P, _c.c_int, _P],
        "beor_lnl_multi_wait": [_P, _c.c_int, _P, _c.c_int, _P],
        "beor_posterior_mean": [_P, _P, _P, _P, _P],
        "beor_get_model_dims": [_P, _c.POINTER(_I64), _c.POINTER(_I64), _c.POINTER(_c.c_int)],
        "beor_get_M": [_P, _P],
        "beor_get_dbar": [_P, _P],
        "beor_get_stats": [_P, _P],
        "beor_get_terms": [_P, _P, _P, _P, _c.c_int],
        "beor_get_factor": [_P, _c.c_int, _P],
        "beor_set_profiling": [_c.c_int],
        "beor_set_lookahead": [_c.c_int],
        "beor_set_wait_test": [_c.c_int, _c.c_double],
        "beor_set_instrument_desc": [_P, _P],
        "beor_set_schedule": [_P, _c.c_int, _P, _P],
        "beor_get_schedule": [_P, _c.c_int, _P, _P],
        "beor_autotune": [_P, _c.c_int, _P, _P, _c.c_int, _c.c_char_p, _P, _P, _P],
        "beor_dbar_factored_noalloc": [_P, _P, _c.c_int, _I64, _c.c_int, _c.c_int, _P, _P, _P, _P],
        "beor_mlp_create": [_c.POINTER(_P), _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_uint64],
        "beor_mlp_destroy": [_P],
        "beor_mlp_set_norm": [_P, _P, _P, _c.c_float, _c.c_float],
        "beor_mlp_train_step": [_P, _P, _P, _c.c_int, _c.c_float, _c.c_float, _c.c_float, _c.c_float, _P, _P],
        "beor_mlp_infer": [_P, _P, _c.c_int, _P, _P],
        "beor_mlp_get_params": [_P, _c.c_int, _P, _P],
        "beor_mlp_set_params": [_P, _c.c_int, _P, _P],
        "beor_mlp_grad": [_P, _P, _P, _c.c_int, _c.c_int, _P, _P, _P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _c.c_int
    L.beor_strerror.argtypes = [_c.c_int]
    L.beor_strerror.restype = _c.c_char_p
    L.beor_last_cuda_error.argtypes = []
    L.beor_last_cuda_error.restype = _c.c_char_p
    L.beor_build_info.argtypes = []
    L.beor_build_info.restype = _c.c_int
    return L


lib = None


def _lib():
    global lib
    if lib is None:
        lib = _load()
    return lib


def _check(code, what):
    if code != 0:
        msg = _lib().beor_strerror(code).decode()
        if code in (-2, -3):   # BEOR_ENOMEM, BEOR_ECUDA: name the CUDA error behind it
            msg += ", " + _lib().beor_last_cuda_error().decode()
        raise BeorError(f"{what}: {msg} ({code})")


class _Stats(ctypes.Structure):
    _fields_ = [("refine_iters_max", ctypes.c_int), ("resid_rel_max", ctypes.c_double),
                ("ms_last", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("ms_class", ctypes.c_double * 8), ("n_class", ctypes.c_int64 * 8),
                ("device_error", ctypes.c_int32), ("ms_busy_any", ctypes.c_double),
                ("ms_busy_main", ctypes.c_double), ("bounds_error", ctypes.c_int32)]


KERNEL_CLASSES = ("init", "diag", "slice", "panel", "trail", "solve", "refine", "lnl")


def set_profiling(on: bool):
    _check(_lib().beor_set_profiling(1 if on else 0), "beor_set_profiling")


def set_lookahead(on: bool):
    _check(_lib().beor_set_lookahead(1 if on else 0), "beor_set_lookahead")


def set_wait_test(skip_one_copy: bool, limit_ms: float = 0.0):
    """Failure-detection test hook (see beor_set_wait_test); (False, 0) is the default."""
    _check(_lib().beor_set_wait_test(1 if skip_one_copy else 0, float(limit_ms)), "beor_set_wait_test")


class InstrumentDesc(ctypes.Structure):
    """beor_instrument_desc: the instrument's geometry (see include/beor.h)."""
    _fields_ = [("nu", ctypes.c_int), ("nf", ctypes.c_int), ("nf_grid", ctypes.c_int), ("n_lssm", ctypes.c_int),
                ("n_pix", ctypes.c_int), ("n_bl", ctypes.c_int), ("n_t", ctypes.c_int), ("n_k", ctypes.c_int),
                ("f0_hz", ctypes.c_double), ("df_hz", ctypes.c_double), ("beam_fwhm_rad", ctypes.c_double),
                ("latitude_rad", ctypes.c_double), ("lssm_prior_var", ctypes.c_double),
                ("bl_enu_m", ctypes.c_void_p), ("hour_angle_rad", ctypes.c_void_p), ("lssm_beta", ctypes.c_void_p)]


class Schedule(ctypes.Structure):
    """beor_schedule: look-ahead, CTAs of the rest / next-column launches
    (0 = one per SM), aligned ends, SMs reserved for the diagonal blocks."""
    _fields_ = [("lookahead", ctypes.c_int), ("rest_ctas", ctypes.c_int), ("col_ctas", ctypes.c_int),
                ("align_ends", ctypes.c_int), ("reserve_diag", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _shape(likes, Bs):
    n = len(likes)
    ctxs = (ctypes.c_void_p * n)(*[lk._h.value for lk in likes])
    bb = (ctypes.c_int * n)(*[int(b) for b in Bs])
    return n, ctxs, bb


def set_schedule(likes: list, Bs: list, schedule: dict | None):
    """Schedule of lnL evaluations of this batch shape (None: the default)."""
    n, ctxs, bb = _shape(likes, Bs)
    sch = Schedule(**schedule) if schedule is not None else None
    _check(_lib().beor_set_schedule(ctypes.cast(ctxs, ctypes.c_void_p), n, ctypes.cast(bb, ctypes.c_void_p),
                                    ctypes.byref(sch) if sch is not None else None), "beor_set_schedule")


def get_schedule(likes: list, Bs: list) -> dict:
    n, ctxs, bb = _shape(likes, Bs)
    sch = Schedule()
    _check(_lib().beor_get_schedule(ctypes.cast(ctxs, ctypes.c_void_p), n, ctypes.cast(bb, ctypes.c_void_p),
                                    ctypes.byref(sch)), "beor_get_schedule")
    return sch.as_dict()


def autotune(likes: list, phis: list, reps: int = 2, cache_path: str | None = None) -> dict:
    """Time the schedule candidates of this batch shape (see beor_autotune);
    returns the chosen schedule and the times per evaluation."""
    keep = []
    phi_arr = [np.atleast_2d(np.asarray(p, np.float64)) for p in phis]
    n, ctxs, bb = _shape(likes, [p.shape[0] for p in phi_arr])
    pp = (ctypes.c_void_p * n)(*[_ptr(p, np.float64, keep).value for p in phi_arr])
    sch = Schedule()
    ms, ms0 = ctypes.c_double(-1.0), ctypes.c_double(-1.0)
    _check(_lib().beor_autotune(ctypes.cast(ctxs, ctypes.c_void_p), n, ctypes.cast(pp, ctypes.c_void_p),
                                ctypes.cast(bb, ctypes.c_void_p), int(reps),
                                cache_path.encode() if cache_path else None, ctypes.byref(sch), ctypes.byref(ms),
                                ctypes.byref(ms0)), "beor_autotune")
    return {"schedule": sch.as_dict(), "ms_per_eval": ms.value, "ms_default": ms0.value}


def _stream(stream):
    if stream is not None:
        if hasattr(stream, "cuda_stream"):     # a torch.cuda.Stream
            return ctypes.c_void_p(int(stream.cuda_stream))
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _ptr(a, dtype, keep):
    """Pointer to a contiguous array of `dtype` (numpy or torch); keeps it alive in `keep`."""
    if hasattr(a, "data_ptr"):       # torch tensor
        import torch
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32,
               np.complex128: torch.complex128}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            a = a.to(tdt).contiguous()
        keep.append(a)
        return ctypes.c_void_p(a.data_ptr())
    arr = np.ascontiguousarray(a, dtype=dtype)
    keep.append(arr)
    return ctypes.c_void_p(arr.ctypes.data)


class Likelihood:
    """One instrument: model, data, precompute and batched lnL evaluations."""

    def __init__(self, precision: str | int = "fp64", device: int = 0):
        prec = {"fp64": PREC_FP64, "mixed": PREC_MIXED}.get(precision, precision)
        h = ctypes.c_void_p()
        _check(_lib().beor_create(ctypes.byref(h), device, int(prec)), "beor_create")
        self._h = h
        self.precision = prec
        self.n_k = 0

    def close(self):
        if getattr(self, "_h", None):
            _lib().beor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_T(self, T, kbin, n_k: int, lssm_prior_var: float):
        keep = []
        n_vis, n = T.shape
        _check(_lib().beor_set_T(self._h, _ptr(T, np.complex128, keep), n_vis, n, n,
                                 _ptr(kbin, np.int32, keep), n_k, float(lssm_prior_var)), "beor_set_T")
        self.n_k = n_k

    def set_instrument(self, A, W, kbin, n_k: int, lssm_prior_var: float):
        keep = []
        nf, ntb, ncells = A.shape
        nx = W.shape[1]
        _check(_lib().beor_set_instrument(self._h, _ptr(A, np.complex128, keep), _ptr(W, np.complex128, keep),
                                          nf, ntb, ncells, nx, _ptr(kbin, np.int32, keep), n_k,
                                          float(lssm_prior_var)), "beor_set_instrument")
        self.n_k = n_k

    def set_instrument_desc(self, geometry: dict):
        """Instrument built by the library from its geometry: a dict with the
        beor_instrument_desc fields (arrays for bl_enu_m (n_bl x 3),
        hour_angle_rad (n_t) and lssm_beta (n_lssm))."""
        keep = []
        g = dict(geometry)
        bl = np.ascontiguousarray(g.pop("bl_enu_m"), np.float64)
        ha = np.ascontiguousarray(g.pop("hour_angle_rad"), np.float64)
        beta = np.ascontiguousarray(g.pop("lssm_beta", np.zeros(0)), np.float64)
        keep += [bl, ha, beta]
        desc = InstrumentDesc(n_bl=bl.shape[0], n_t=ha.shape[0], n_lssm=beta.shape[0],
                              bl_enu_m=bl.ctypes.data, hour_angle_rad=ha.ctypes.data,
                              lssm_beta=beta.ctypes.data if beta.size else None, **g)
        _check(_lib().beor_set_instrument_desc(self._h, ctypes.byref(desc)), "beor_set_instrument_desc")
        self.n_k = desc.n_k

    def set_data(self, d, noise_var):
        keep = []
        _check(_lib().beor_set_data(self._h, _ptr(d, np.complex128, keep), _ptr(noise_var, np.float64, keep)),
               "beor_set_data")

    def precompute(self, stream=None):
        _check(_lib().beor_precompute(self._h, _stream(stream)), "beor_precompute")

    def dims(self):
        nv, nm, nk = _I64(), _I64(), ctypes.c_int()
        _check(_lib().beor_get_model_dims(self._h, ctypes.byref(nv), ctypes.byref(nm), ctypes.byref(nk)), "dims")
        return nv.value, nm.value, nk.value

    def lnl(self, phi, stream=None, out=None, status=None):
        """lnL for a batch phi (B x n_k).  Returns (lnl[B], status[B]) as numpy
        arrays, or fills the given output arrays/tensors."""
        keep = []
        phi2 = phi if hasattr(phi, "data_ptr") else np.atleast_2d(np.asarray(phi, dtype=np.float64))
        B = phi2.shape[0]
        o = np.empty(B, np.float64) if out is None else out
        s = np.empty(B, np.int32) if status is None else status
        _check(_lib().beor_lnl(self._h, _ptr(phi2, np.float64, keep), B, _ptr(o, np.float64, keep),
                               _ptr(s, np.int32, keep), _stream(stream)), "beor_lnl")
        if out is None and isinstance(keep[1], np.ndarray):
            o = keep[1]
        if status is None and isinstance(keep[2], np.ndarray):
            s = keep[2]
        return o, s

    def posterior_mean(self, phi, stream=None):
        keep = []
        n = self.dims()[1]
        a = np.empty(n, np.complex128)
        st = np.zeros(1, np.int32)
        _check(_lib().beor_posterior_mean(self._h, _ptr(np.asarray(phi, np.float64), np.float64, keep),
                                          ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(st.ctypes.data),
                                          _stream(stream)), "beor_posterior_mean")
        return a, int(st[0])

    def get_M(self):
        n = self.dims()[1]
        M = np.empty((n, n), np.complex128)
        _check(_lib().beor_get_M(self._h, ctypes.c_void_p(M.ctypes.data)), "beor_get_M")
        return M

    def get_dbar(self):
        n = self.dims()[1]
        v = np.empty(n, np.complex128)
        _check(_lib().beor_get_dbar(self._h, ctypes.c_void_p(v.ctypes.data)), "beor_get_dbar")
        return v

    def stats(self) -> dict:
        st = _Stats()
        _check(_lib().beor_get_stats(self._h, ctypes.byref(st)), "beor_get_stats")
        out = {k: getattr(st, k) for k, _ in st._fields_[:4]}
        out["ms_class"] = dict(zip(KERNEL_CLASSES, list(st.ms_class)))
        out["n_class"] = dict(zip(KERNEL_CLASSES, list(st.n_class)))
        out["device_error"] = st.device_error
        out["ms_busy_any"] = st.ms_busy_any
        out["ms_busy_main"] = st.ms_busy_main
        out["bounds_error"] = st.bounds_error
        return out

    def factor(self, b: int = 0):
        """Cholesky factor of prior point b of the last lnl() call (host copy)."""
        n = self.dims()[1]
        L = np.empty((n, n), np.complex128)
        _check(_lib().beor_get_factor(self._h, b, ctypes.c_void_p(L.ctypes.data)), "beor_get_factor")
        return L

    def terms(self, B: int):
        a, b, c = (np.empty(B, np.float64) for _ in range(3))
        _check(_lib().beor_get_terms(self._h, ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(b.ctypes.data),
                                     ctypes.c_void_p(c.ctypes.data), B), "beor_get_terms")
        return {"logdet_phi": a, "logdet_sigma": b, "q": c}


def lnl_multi(likes: list, phis: list, stream=None):
    """One batched evaluation over several instruments (uneven sizes allowed)."""
    n = len(likes)
    keep = []
    ctxs = (ctypes.c_void_p * n)(*[lk._h.value for lk in likes])
    phi_arr = [np.atleast_2d(np.asarray(p, np.float64)) for p in phis]
    Bs = (ctypes.c_int * n)(*[p.shape[0] for p in phi_arr])
    pp = (ctypes.c_void_p * n)(*[_ptr(p, np.float64, keep).value for p in phi_arr])
    outs = [np.empty(p.shape[0], np.float64) for p in phi_arr]
    sts = [np.empty(p.shape[0], np.int32) for p in phi_arr]
    op = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
    sp = (ctypes.c_void_p * n)(*[s.ctypes.data for s in sts])
    _check(_lib().beor_lnl_multi(ctypes.cast(ctxs, ctypes.c_void_p), n, ctypes.cast(pp, ctypes.c_void_p),
                                 ctypes.cast(Bs, ctypes.c_void_p), ctypes.cast(op, ctypes.c_void_p),
                                 ctypes.cast(sp, ctypes.c_void_p), _stream(stream)), "beor_lnl_multi")
    return outs, sts


def _dev_ptr(x):
    """Address of a tensor-like object (data_ptr()), a numpy array, or an integer
    (the library rejects host memory where it needs device memory)."""
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    return int(x)


def lnl_multi_async(likes: list, phis: list, outs: list, sts: list, slot: int, stream):
    """Enqueue one batched evaluation without waiting (device buffers only:
    phis[s] (B_s, n_k) float64, outs[s] (B_s,) float64, sts[s] (B_s,) int32,
    e.g. torch CUDA tensors).  See beor_lnl_multi_async in include/beor.h."""
    n = len(likes)
    ctxs = (ctypes.c_void_p * n)(*[lk._h.value for lk in likes])
    Bs = (ctypes.c_int * n)(*[int(p.shape[0]) for p in phis])
    pp = (ctypes.c_void_p * n)(*[_dev_ptr(p) for p in phis])
    op = (ctypes.c_void_p * n)(*[_dev_ptr(o) for o in outs])
    sp = (ctypes.c_void_p * n)(*[_dev_ptr(x) for x in sts])
    _check(_lib().beor_lnl_multi_async(ctypes.cast(ctxs, ctypes.c_void_p), n, ctypes.cast(pp, ctypes.c_void_p),
                                       ctypes.cast(Bs, ctypes.c_void_p), ctypes.cast(op, ctypes.c_void_p),
                                       ctypes.cast(sp, ctypes.c_void_p), int(slot), _stream(stream)),
           "beor_lnl_multi_async")


def lnl_multi_wait(likes: list, Bs: list, slot: int, stream):
    """Wait for the slot's enqueued work on `stream`; raises on a device timeout."""
    n = len(likes)
    ctxs = (ctypes.c_void_p * n)(*[lk._h.value for lk in likes])
    bb = (ctypes.c_int * n)(*[int(b) for b in Bs])
    _check(_lib().beor_lnl_multi_wait(ctypes.cast(ctxs, ctypes.c_void_p), n, ctypes.cast(bb, ctypes.c_void_p),
                                      int(slot), _stream(stream)), "beor_lnl_multi_wait")


class Emulator:
    """MLP emulator of lnL(phi), trained and evaluated by the library's kernels."""

    def __init__(self, n_in: int, width: int = 256, depth: int = 4, seed: int = 4, device: int = 0):
        h = ctypes.c_void_p()
        _check(_lib().beor_mlp_create(ctypes.byref(h), device, n_in, width, depth, seed), "beor_mlp_create")
        self._h = h
        self.n_in, self.width, self.depth = n_in, width, depth

    def close(self):
        if getattr(self, "_h", None):
            _lib().beor_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_norm(self, x_shift, x_scale, y_shift: float, y_scale: float):
        keep = []
        _check(_lib().beor_mlp_set_norm(self._h, _ptr(x_shift, np.float32, keep), _ptr(x_scale, np.float32, keep),
                                        float(y_shift), float(y_scale)), "beor_mlp_set_norm")

    def train_step(self, x, y, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> float:
        keep = []
        loss = ctypes.c_float(0.0)
        n = x.shape[0]
        _check(_lib().beor_mlp_train_step(self._h, _ptr(x, np.float32, keep), _ptr(y, np.float32, keep), n,
                                          lr, beta1, beta2, eps, ctypes.byref(loss), _stream(stream)),
               "beor_mlp_train_step")
        return loss.value

    def infer(self, x, stream=None, out=None):
        keep = []
        n = x.shape[0]
        y = np.empty(n, np.float32) if out is None else out
        _check(_lib().beor_mlp_infer(self._h, _ptr(x, np.float32, keep), n, _ptr(y, np.float32, keep),
                                     _stream(stream)), "beor_mlp_infer")
        return keep[1] if out is None else out

    def layer_shape(self, layer: int):
        fan_in = self.n_in if layer == 0 else self.width
        fan_out = 1 if layer == self.depth else self.width
        return fan_out, fan_in

    def get_params(self, layer: int):
        o, i = self.layer_shape(layer)
        W = np.empty((o, i), np.float32)
        b = np.empty(o, np.float32)
        _check(_lib().beor_mlp_get_params(self._h, layer, ctypes.c_void_p(W.ctypes.data),
                                          ctypes.c_void_p(b.ctypes.data)), "beor_mlp_get_params")
        return W, b

    def set_params(self, layer: int, W, b):
        keep = []
        _check(_lib().beor_mlp_set_params(self._h, layer, _ptr(W, np.float32, keep), _ptr(b, np.float32, keep)),
               "beor_mlp_set_params")

    def grad(self, x, y, layer: int):
        keep = []
        o, i = self.layer_shape(layer)
        dW = np.empty((o, i), np.float32)
        db = np.empty(o, np.float32)
        loss = ctypes.c_float(0.0)
        _check(_lib().beor_mlp_grad(self._h, _ptr(x, np.float32, keep), _ptr(y, np.float32, keep), x.shape[0], layer,
                                    ctypes.c_void_p(dW.ctypes.data), ctypes.c_void_p(db.ctypes.data),
                                    ctypes.byref(loss)), "beor_mlp_grad")
        return dW, db, loss.value
