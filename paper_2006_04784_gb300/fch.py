"""Python binding of libfch (include/fch.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy
arrays and torch tensors into pointers and sizes, and status codes into
exceptions. It fails loudly when the library has not been built or cannot be
loaded; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfch.so")

FCH_IMEX, FCH_SAV, FCH_PSD, FCH_ETD = 0, 1, 2, 3
SCHEMES = {"imex": FCH_IMEX, "sav": FCH_SAV, "psd": FCH_PSD, "etd": FCH_ETD}
FCH_FP64, FCH_MIXED, FCH_FP32X2 = 0, 1, 2
STATUS = {0: "FCH_OK", 1: "FCH_EINVAL", 2: "FCH_ENOMEM", 3: "FCH_ECUDA", 4: "FCH_ENOCONV",
          5: "FCH_ENONFINITE", 6: "FCH_ETIMEOUT", 7: "FCH_ESTATE"}

# the symbols include/fch.h declares (checked by the CPU tests)
EXPORTS = ["fch_status_string", "fch_last_cuda_error", "fch_params_default", "fch_create",
           "fch_destroy", "fch_synchronize", "fch_set_state", "fch_set_state_device",
           "fch_set_history", "fch_get_state", "fch_get_state_device", "fch_step", "fch_energy",
           "fch_mass", "fch_rhs_device", "fch_get_sav_r", "fch_run_adaptive", "fch_get_stats",
           "fch_fft_plan_create", "fch_fft_plan_destroy", "fch_fft_r2c", "fch_fft_c2r",
           "fch_adaptive_begin", "fch_adaptive_enqueue", "fch_adaptive_end", "fch_pass_timing",
           "fch_pass_times", "fch_fft_r2c_noalloc", "fch_autotune", "fch_autotune_reset",
           "fch_ensemble_create", "fch_ensemble_destroy", "fch_ensemble_member",
           "fch_ensemble_run_adaptive", "fch_fno_create", "fch_fno_destroy", "fch_fno_num_params",
           "fch_fno_set_params", "fch_fno_get_params", "fch_fno_get_grads", "fch_fno_forward",
           "fch_fno_backward", "fch_fno_adam", "fch_step_psd_from", "fch_run_fixed",
           "fch_adaptive_trial_info", "fch_get_history_device", "fch_adaptive_enqueue_psd_from",
           "fch_ensemble_run_adaptive_each", "fch_autotune_step", "fch_step_from", "fch_fno_set_bf16",
           "fch_alu_peak", "fch_fno_learned_start", "fch_adaptive_enqueue_from", "fch_fft_plan_status"]
NCOL, NROW = 10, 8
NPASS = NCOL + NROW + 1
PASS_NAMES = (["col_fwd_store", "col_inv_load", "col_start", "col_imex_solve", "col_f_finish",
               "col_sav_pq", "col_sav_combine", "col_psd_iter", "col_etd_stage1", "col_etd_stage2"]
              + ["row_r2c_load", "row_c2r_store", "row_nimex", "row_f", "row_sav", "row_energy",
                 "row_nimex_direct", "row_sav_direct"]
              + ["ctrl"])


class FchError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class Grid(C.Structure):
    _fields_ = [("n", C.c_int), ("L", C.c_double), ("x0", C.c_double)]


class Params(C.Structure):
    _fields_ = [
        ("eps", C.c_double), ("q", C.c_double), ("gamma", C.c_double),
        ("b_minus", C.c_double), ("b_plus", C.c_double), ("eta1", C.c_double), ("eta2", C.c_double),
        ("beta1", C.c_double), ("beta2", C.c_double), ("zeta", C.c_double), ("D0", C.c_double),
        ("kappa0", C.c_double), ("kappa2", C.c_double),
        ("rho_s", C.c_double), ("k_min", C.c_double), ("k_max", C.c_double),
        ("zero_stab_cap", C.c_int),
        ("psd_nu", C.c_double), ("psd_itol", C.c_double), ("psd_lambda", C.c_double),
        ("psd_k_max", C.c_double),
        ("psd_max_iter", C.c_int), ("prec", C.c_int), ("sync_every", C.c_int),
        ("fft_path", C.c_int), ("autotune", C.c_int), ("tile_row", C.c_int), ("tile_col", C.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Tile(C.Structure):
    _fields_ = [("tile_row", C.c_int), ("tile_col", C.c_int), ("row_us", C.c_double),
                ("col_us", C.c_double), ("row_default_us", C.c_double), ("col_default_us", C.c_double),
                ("candidates", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("n_steps", C.c_longlong), ("n_rejects", C.c_longlong),
                ("n_attempts", C.c_longlong), ("n_psd_iter", C.c_longlong),
                ("n_fft", C.c_longlong), ("t", C.c_double), ("k_last", C.c_double),
                ("e_last", C.c_double), ("last_psd_iter", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load libfch.so (built by paper_2006_04784_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfch is not built ({LIB_PATH} missing): run "
                               "python -c 'import __graft_entry__ as g; g.build()'")
        L = C.CDLL(LIB_PATH)
        vp, dp, sz = C.c_void_p, C.POINTER(C.c_double), C.c_size_t
        L.fch_status_string.restype = C.c_char_p
        L.fch_status_string.argtypes = [C.c_int]
        L.fch_last_cuda_error.restype = C.c_char_p
        L.fch_last_cuda_error.argtypes = [vp]
        L.fch_params_default.argtypes = [C.POINTER(Params), C.c_double]
        L.fch_create.argtypes = [C.POINTER(Grid), C.POINTER(Params), vp, C.POINTER(vp)]
        L.fch_destroy.argtypes = [vp]
        L.fch_synchronize.argtypes = [vp]
        L.fch_set_state.argtypes = [vp, dp, sz]
        L.fch_set_state_device.argtypes = [vp, vp, C.c_int]
        L.fch_set_history.argtypes = [vp, dp, dp, sz, C.c_double]
        L.fch_get_state.argtypes = [vp, dp, sz]
        L.fch_get_state_device.argtypes = [vp, vp, C.c_int]
        L.fch_step.argtypes = [vp, C.c_int, C.c_double]
        L.fch_energy.argtypes = [vp, dp]
        L.fch_mass.argtypes = [vp, dp]
        L.fch_rhs_device.argtypes = [vp, vp, vp, C.c_int]
        L.fch_get_sav_r.argtypes = [vp, dp, dp]
        L.fch_run_adaptive.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_longlong,
                                       C.POINTER(Stats)]
        L.fch_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.fch_fft_plan_create.argtypes = [C.c_int, C.c_int, vp, C.POINTER(vp)]
        L.fch_autotune.argtypes = [C.c_int, C.c_int, vp, C.POINTER(Tile)]
        L.fch_autotune_step.argtypes = [C.c_int, C.c_int, vp, C.POINTER(Tile)]
        L.fch_ensemble_create.argtypes = [C.c_int, C.POINTER(Grid), C.POINTER(Params), vp, C.POINTER(vp)]
        L.fch_ensemble_destroy.argtypes = [vp]
        fp = C.POINTER(C.c_float)
        L.fch_fno_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, vp, C.POINTER(vp)]
        L.fch_fno_destroy.argtypes = [vp]
        L.fch_fno_num_params.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.fch_fno_set_params.argtypes = [vp, fp, C.c_size_t]
        L.fch_fno_get_params.argtypes = [vp, fp, C.c_size_t]
        L.fch_fno_get_grads.argtypes = [vp, fp, C.c_size_t]
        L.fch_fno_forward.argtypes = [vp, C.c_int, C.c_int, vp, vp]
        L.fch_fno_backward.argtypes = [vp, vp, C.POINTER(C.c_double)]
        L.fch_fno_adam.argtypes = [vp, C.c_float, C.c_float, C.c_float, C.c_float]
        L.fch_fno_set_bf16.argtypes = [vp, C.c_int]
        L.fch_step_psd_from.argtypes = [vp, C.c_double, vp, C.c_int]
        L.fch_step_from.argtypes = [vp, C.c_int, C.c_double, vp, C.c_int]
        L.fch_run_fixed.argtypes = [vp, C.c_int, C.c_double, C.c_longlong]
        L.fch_adaptive_trial_info.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                              C.POINTER(C.c_int)]
        L.fch_get_history_device.argtypes = [vp, vp, vp, C.c_int]
        L.fch_adaptive_enqueue_psd_from.argtypes = [vp, vp, C.c_int]
        L.fch_ensemble_member.argtypes = [vp, C.c_int, C.POINTER(vp)]
        L.fch_ensemble_run_adaptive.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_int, C.c_longlong,
                                                C.POINTER(Stats)]
        L.fch_ensemble_run_adaptive_each.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_double,
                                                     C.c_int, C.c_longlong, C.POINTER(Stats)]
        L.fch_autotune_reset.argtypes = []
        L.fch_alu_peak.argtypes = [C.c_int, vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]
        L.fch_fno_learned_start.argtypes = [vp, vp, C.c_double, vp]
        L.fch_adaptive_enqueue_from.argtypes = [vp, vp, C.c_int]
        L.fch_fft_plan_destroy.argtypes = [vp]
        L.fch_fft_r2c.argtypes = [vp, vp, vp, C.c_int]
        L.fch_fft_c2r.argtypes = [vp, vp, vp, C.c_int]
        L.fch_fft_plan_status.argtypes = [vp]
        L.fch_adaptive_begin.argtypes = [vp, C.c_int, C.c_double, C.c_double]
        L.fch_adaptive_enqueue.argtypes = [vp, C.c_int]
        L.fch_adaptive_end.argtypes = [vp, C.POINTER(Stats)]
        L.fch_pass_timing.argtypes = [vp, C.c_int]
        L.fch_pass_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int]
        L.fch_debug_geometry.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int)]
        L.fch_debug_graphs.argtypes = [vp, C.POINTER(C.c_int)]
        L.fch_debug_twiddles.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double)]
        L.fch_debug_twiddles.restype = C.c_int
        L.fch_debug_graphs.restype = C.c_int
        for name in EXPORTS:
            if name not in ("fch_status_string", "fch_last_cuda_error"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(st, where, ctx=None):
    if st != 0:
        detail = ""
        if st == 3:
            detail = lib().fch_last_cuda_error(ctx).decode()
        raise FchError(st, where, detail)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def autotune(n: int, prec: int, stream=None) -> dict:
    """fch_autotune: the pass tiles kept for (n, prec), timed on first use."""
    t = Tile()
    _check(lib().fch_autotune(n, prec, _stream_ptr(stream), C.byref(t)), "fch_autotune")
    return t.as_dict()


def autotune_step(n: int, prec: int, stream=None) -> dict:
    """fch_autotune_step: the pass tiles timed on adaptive IMEX trials, kept for (n, prec)."""
    t = Tile()
    _check(lib().fch_autotune_step(n, prec, _stream_ptr(stream), C.byref(t)), "fch_autotune_step")
    return t.as_dict()


def autotune_reset():
    _check(lib().fch_autotune_reset(), "fch_autotune_reset")


def alu_peak(prec: int, stream=None) -> tuple:
    """(measured FMA-pipe peak in flop/s, SM count) of the current device: FP32 pipe
    for FCH_MIXED, FP64 pipe for FCH_FP64 (fch_alu_peak)"""
    r, sms = C.c_double(), C.c_int()
    _check(lib().fch_alu_peak(int(prec), _stream_ptr(stream), C.byref(r), C.byref(sms)), "fch_alu_peak")
    return r.value, sms.value


def params_default(q: float = 0.0, **kw) -> Params:
    p = Params()
    _check(lib().fch_params_default(C.byref(p), float(q)), "fch_params_default")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def geometry(n: int, prec: int = 0):
    out = (C.c_int * 9)()
    if lib().fch_debug_geometry(n, prec, out):
        raise ValueError(n)
    keys = ["col_blocks", "col_threads", "col_smem", "row_blocks", "row_threads", "row_smem",
            "rpb", "P", "ctrl_bytes"]
    return dict(zip(keys, list(out)))


def stage_twiddles(n: int, lp: int):
    """the host's per-stage twiddle table for radix-2^lp shared-memory transforms
    (n complex entries; host-side query, no device work)"""
    out = (C.c_double * (2 * n))()
    if lib().fch_debug_twiddles(n, lp, out):
        raise ValueError((n, lp))
    a = np.frombuffer(out, dtype=np.float64)
    return a[0::2] + 1j * a[1::2]


def tile_geometry(n: int, prec: int, tile_row: int, tile_col: int):
    """(valid, geometry) of the pass tiles (host-side query; no device work)"""
    out = (C.c_int * 8)()
    r = lib().fch_debug_tile(n, prec, tile_row, tile_col, out)
    if r < 0:
        raise ValueError(n)
    keys = ["col_blocks", "col_threads", "col_smem", "row_blocks", "row_threads", "row_smem", "rpb", "P"]
    return bool(r), dict(zip(keys, list(out)))


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _tensor_ptr(t):
    return C.c_void_p(int(t.data_ptr()))


def _dtype_code(t):
    import torch

    if t.dtype == torch.float64:
        return 0
    if t.dtype == torch.float32:
        return 1
    raise TypeError(f"unsupported dtype {t.dtype}")


class Context:
    """One FCH stepper on the current CUDA device (fch_create ... fch_destroy)."""

    def __init__(self, n: int, params: Params | None = None, L: float = 4 * math.pi,
                 x0: float = -2 * math.pi, stream=None):
        self.n, self.L = n, L
        self.params = params if params is not None else params_default()
        g = Grid(n, L, x0)
        h = C.c_void_p()
        _check(lib().fch_create(C.byref(g), C.byref(self.params), _stream_ptr(stream), C.byref(h)),
               "fch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().fch_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, st, where):
        _check(st, where, self._h)

    def synchronize(self):
        self._ck(lib().fch_synchronize(self._h), "fch_synchronize")

    def set_state(self, u: np.ndarray):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == (self.n, self.n)
        self._ck(lib().fch_set_state(self._h, _dp(u), u.size), "fch_set_state")

    def set_state_device(self, t):
        assert t.is_cuda and t.is_contiguous() and tuple(t.shape) == (self.n, self.n)
        self._ck(lib().fch_set_state_device(self._h, _tensor_ptr(t), _dtype_code(t)),
                 "fch_set_state_device")

    def set_history(self, un, unm1, kn):
        un = np.ascontiguousarray(un, dtype=np.float64)
        unm1 = np.ascontiguousarray(unm1, dtype=np.float64)
        self._ck(lib().fch_set_history(self._h, _dp(un), _dp(unm1), un.size, float(kn)),
                 "fch_set_history")

    def get_state(self) -> np.ndarray:
        u = np.empty((self.n, self.n))
        self._ck(lib().fch_get_state(self._h, _dp(u), u.size), "fch_get_state")
        return u

    def get_state_device(self, t):
        assert t.is_cuda and t.is_contiguous() and tuple(t.shape) == (self.n, self.n)
        self._ck(lib().fch_get_state_device(self._h, _tensor_ptr(t), _dtype_code(t)),
                 "fch_get_state_device")

    def step(self, scheme, dt: float):
        s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        self._ck(lib().fch_step(self._h, s, float(dt)), "fch_step")

    def run_fixed(self, scheme, dt: float, nsteps: int):
        """nsteps fixed steps (a captured step replayed after the first)"""
        s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        self._ck(lib().fch_run_fixed(self._h, s, float(dt), int(nsteps)), "fch_run_fixed")

    def adaptive_trial_info(self):
        """(k, gamma, done) of the next trial of the open adaptive run"""
        k, g, d = C.c_double(), C.c_double(), C.c_int()
        self._ck(lib().fch_adaptive_trial_info(self._h, C.byref(k), C.byref(g), C.byref(d)),
                 "fch_adaptive_trial_info")
        return k.value, g.value, bool(d.value)

    def get_history_device(self, un, unm1):
        self._ck(lib().fch_get_history_device(self._h, _tensor_ptr(un), _tensor_ptr(unm1), _dtype_code(un)),
                 "fch_get_history_device")

    def adaptive_enqueue_psd_from(self, v0):
        self._ck(lib().fch_adaptive_enqueue_psd_from(self._h, _tensor_ptr(v0), _dtype_code(v0)),
                 "fch_adaptive_enqueue_psd_from")

    def adaptive_enqueue_from(self, ustar):
        """one IMEX or SAV trial of the open adaptive run whose u* is the device field ustar"""
        assert ustar.is_cuda and ustar.is_contiguous() and tuple(ustar.shape) == (self.n, self.n)
        self._ck(lib().fch_adaptive_enqueue_from(self._h, _tensor_ptr(ustar), _dtype_code(ustar)),
                 "fch_adaptive_enqueue_from")

    def step_from(self, scheme, dt: float, ustar):
        """one IMEX or SAV step whose extrapolation u* is the device field ustar"""
        assert ustar.is_cuda and ustar.is_contiguous() and tuple(ustar.shape) == (self.n, self.n)
        s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        self._ck(lib().fch_step_from(self._h, s, float(dt), _tensor_ptr(ustar), _dtype_code(ustar)),
                 "fch_step_from")

    def fno_learned_start(self, net, v0, dt: float = 0.0):
        """v_0 = u* + s (y - mean y) from the history and the network (fch_fno_learned_start):
        dt = 0 for the open adaptive run's next trial, dt > 0 for a fixed step"""
        assert v0.is_cuda and v0.is_contiguous() and v0.dtype.is_floating_point and v0.element_size() == 8
        assert tuple(v0.shape) == (self.n, self.n)
        self._ck(lib().fch_fno_learned_start(self._h, net._h, float(dt), _tensor_ptr(v0)),
                 "fch_fno_learned_start")

    def step_psd_from(self, dt: float, v0):
        """one PSD-BDF2 step whose iteration starts from the device field v0"""
        assert v0.is_cuda and v0.is_contiguous() and tuple(v0.shape) == (self.n, self.n)
        self._ck(lib().fch_step_psd_from(self._h, float(dt), _tensor_ptr(v0), _dtype_code(v0)),
                 "fch_step_psd_from")

    def energy(self) -> float:
        e = C.c_double()
        self._ck(lib().fch_energy(self._h, C.byref(e)), "fch_energy")
        return e.value

    def mass(self) -> float:
        m = C.c_double()
        self._ck(lib().fch_mass(self._h, C.byref(m)), "fch_mass")
        return m.value

    def rhs_device(self, u, F):
        assert u.dtype == F.dtype
        self._ck(lib().fch_rhs_device(self._h, _tensor_ptr(u), _tensor_ptr(F), _dtype_code(u)),
                 "fch_rhs_device")

    def sav_r(self):
        a, b = C.c_double(), C.c_double()
        self._ck(lib().fch_get_sav_r(self._h, C.byref(a), C.byref(b)), "fch_get_sav_r")
        return a.value, b.value

    def run_adaptive(self, scheme, sigma: float, t_final: float, max_attempts: int = 0,
                     raise_on_timeout: bool = True):
        s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        st = Stats()
        rc = lib().fch_run_adaptive(self._h, s, float(sigma), float(t_final), int(max_attempts),
                                    C.byref(st))
        if rc == 6 and not raise_on_timeout:
            return st.as_dict()
        self._ck(rc, "fch_run_adaptive")
        return st.as_dict()

    def adaptive_begin(self, scheme, sigma: float, t_final: float):
        s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        self._ck(lib().fch_adaptive_begin(self._h, s, float(sigma), float(t_final)),
                 "fch_adaptive_begin")

    def adaptive_enqueue(self, n: int):
        self._ck(lib().fch_adaptive_enqueue(self._h, int(n)), "fch_adaptive_enqueue")

    def adaptive_end(self):
        st = Stats()
        self._ck(lib().fch_adaptive_end(self._h, C.byref(st)), "fch_adaptive_end")
        return st.as_dict()

    def debug_graphs(self):
        """per scheme: (trial graph 1 captured / -1 failed / 0 not yet, fixed-step graph 1/0)"""
        out = (C.c_int * 8)()
        if lib().fch_debug_graphs(self._h, out):
            raise ValueError("fch_debug_graphs")
        return {name: (out[i], out[4 + i]) for name, i in SCHEMES.items()}

    def pass_timing(self, on: bool):
        self._ck(lib().fch_pass_timing(self._h, int(bool(on))), "fch_pass_timing")

    def pass_times(self):
        ms = (C.c_double * NPASS)()
        n = (C.c_longlong * NPASS)()
        self._ck(lib().fch_pass_times(self._h, ms, n, NPASS), "fch_pass_times")
        return {PASS_NAMES[i]: (ms[i], n[i]) for i in range(NPASS) if n[i]}

    def stats(self):
        st = Stats()
        self._ck(lib().fch_get_stats(self._h, C.byref(st)), "fch_get_stats")
        return st.as_dict()


class FFTPlan:
    """Standalone N x N real transforms (fch_fft_plan_*); tensors on the device."""

    def __init__(self, n: int, prec: int = FCH_FP64, stream=None):
        self.n, self.prec = n, prec
        h = C.c_void_p()
        _check(lib().fch_fft_plan_create(n, prec, _stream_ptr(stream), C.byref(h)),
               "fch_fft_plan_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().fch_fft_plan_destroy(self._h)
            self._h = None

    __del__ = close

    def r2c(self, x, X):
        """x: (B, N, N) real tensor; X: (B, N/2+1, N) complex tensor (kx-major)."""
        b = x.shape[0] if x.dim() == 3 else 1
        _check(lib().fch_fft_r2c(self._h, _tensor_ptr(x), _tensor_ptr(X), b), "fch_fft_r2c")

    def c2r(self, X, x):
        b = x.shape[0] if x.dim() == 3 else 1
        _check(lib().fch_fft_c2r(self._h, _tensor_ptr(X), _tensor_ptr(x), b), "fch_fft_c2r")

    def status(self):
        """fch_fft_plan_status: synchronizes the plan's stream; raises if a pass's
        bounded wait on a bulk copy ran out since the last call"""
        _check(lib().fch_fft_plan_status(self._h), "fch_fft_plan_status")


class _Member(Context):
    """A context owned by an Ensemble (the single-instance API; not destroyed here)."""

    def __init__(self, h, n, L, params):
        self._h, self.n, self.L, self.params = h, n, L, params

    def close(self):
        self._h = None

    __del__ = close


class Ensemble:
    """m independent contexts advanced together by one CUDA graph per launch
    (fch_ensemble_*); members are reached with member(i) or indexing."""

    def __init__(self, sizes, params, L: float = 4 * math.pi, x0: float = -2 * math.pi, stream=None):
        m = len(sizes)
        assert len(params) == m
        self.sizes, self.L = list(sizes), L
        self.params = list(params)
        grids = (Grid * m)(*[Grid(n, L, x0) for n in sizes])
        pars = (Params * m)(*self.params)
        h = C.c_void_p()
        _check(lib().fch_ensemble_create(m, grids, pars, _stream_ptr(stream), C.byref(h)),
               "fch_ensemble_create")
        self._h = h
        self._members = []
        for i in range(m):
            c = C.c_void_p()
            _check(lib().fch_ensemble_member(h, i, C.byref(c)), "fch_ensemble_member")
            self._members.append(_Member(c, self.sizes[i], L, self.params[i]))

    def __len__(self):
        return len(self._members)

    def member(self, i: int) -> Context:
        return self._members[i]

    __getitem__ = member

    def close(self):
        if getattr(self, "_h", None):
            for mb in self._members:
                mb.close()
            lib().fch_ensemble_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def run_adaptive(self, scheme, sigma: float, t_final: float, rounds: int = 8, max_launches: int = 0,
                     raise_on_timeout: bool = True):
        s = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        st = (Stats * len(self))()
        rc = lib().fch_ensemble_run_adaptive(self._h, s, float(sigma), float(t_final), int(rounds),
                                             int(max_launches), st)
        if not (rc == 6 and not raise_on_timeout):
            _check(rc, "fch_ensemble_run_adaptive")
        return [x.as_dict() for x in st]

    def run_adaptive_each(self, schemes, sigmas, t_final: float, rounds: int = 8, max_launches: int = 0,
                          raise_on_timeout: bool = True):
        """run_adaptive with a scheme and a sigma_tol per member (a sigma_tol sweep)."""
        m = len(self)
        assert len(schemes) == m and len(sigmas) == m
        sc = (C.c_int * m)(*[SCHEMES[x] if isinstance(x, str) else int(x) for x in schemes])
        sg = (C.c_double * m)(*[float(x) for x in sigmas])
        st = (Stats * m)()
        rc = lib().fch_ensemble_run_adaptive_each(self._h, sc, sg, float(t_final), int(rounds),
                                                  int(max_launches), st)
        if not (rc == 6 and not raise_on_timeout):
            _check(rc, "fch_ensemble_run_adaptive_each")
        return [x.as_dict() for x in st]


class FNO:
    """Fourier neural operator for the PSD initial iterate (fch_fno_*); tensors on
    the device, float32."""

    def __init__(self, width=32, layers=4, modes=16, proj=64, stream=None):
        self.width, self.layers, self.modes, self.proj = width, layers, modes, proj
        h = C.c_void_p()
        _check(lib().fch_fno_create(width, layers, modes, proj, _stream_ptr(stream), C.byref(h)),
               "fch_fno_create")
        self._h = h
        n = C.c_size_t()
        _check(lib().fch_fno_num_params(h, C.byref(n)), "fch_fno_num_params")
        self.num_params = n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().fch_fno_destroy(self._h)
            self._h = None

    __del__ = close

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.num_params
        _check(lib().fch_fno_set_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), p.size),
               "fch_fno_set_params")

    def params(self) -> np.ndarray:
        p = np.empty(self.num_params, dtype=np.float32)
        _check(lib().fch_fno_get_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), p.size),
               "fch_fno_get_params")
        return p

    def grads(self) -> np.ndarray:
        g = np.empty(self.num_params, dtype=np.float32)
        _check(lib().fch_fno_get_grads(self._h, g.ctypes.data_as(C.POINTER(C.c_float)), g.size),
               "fch_fno_get_grads")
        return g

    def forward(self, a, y):
        """a: (B, 2, n, n) float32 device tensor; y: (B, n, n) output"""
        assert a.dtype == y.dtype and a.is_contiguous() and y.is_contiguous()
        B, _, n, _ = a.shape
        _check(lib().fch_fno_forward(self._h, B, n, _tensor_ptr(a), _tensor_ptr(y)), "fch_fno_forward")

    def backward(self, target) -> float:
        loss = C.c_double()
        _check(lib().fch_fno_backward(self._h, _tensor_ptr(target), C.byref(loss)), "fch_fno_backward")
        return loss.value

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().fch_fno_adam(self._h, lr, beta1, beta2, eps), "fch_fno_adam")

    def set_bf16(self, on):
        """forward passes on a bfloat16 copy of the weights (FP32 sums), or back to FP32;
        on = 2: also the spectral convolutions as truncated DFTs, the one along x on the
        tensor cores with bfloat16 operands (fch_fno_set_bf16)"""
        mode = 2 if on == 2 else int(bool(on))
        _check(lib().fch_fno_set_bf16(self._h, mode), "fch_fno_set_bf16")
