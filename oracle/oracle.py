"""ctypes front end of the FP64 CPU oracle (fch_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
benchmark's CPU-baseline leg are the only users. The oracle shares no code with
the CUDA path; this file only marshals numpy arrays into the C routines, each of
which restates one passage of the paper (cited in fch_oracle.c).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fch_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

IMEX, SAV, PSD, ETD = 0, 1, 2, 3
SCHEMES = {"imex": IMEX, "sav": SAV, "psd": PSD, "etd": ETD}


class Params(C.Structure):
    """Mirror of orc_params in fch_oracle.c."""

    _fields_ = [
        ("eps", C.c_double), ("q", C.c_double), ("gamma", C.c_double),
        ("b_minus", C.c_double), ("b_plus", C.c_double),
        ("eta1", C.c_double), ("eta2", C.c_double),
        ("beta1", C.c_double), ("beta2", C.c_double), ("zeta", C.c_double), ("D0", C.c_double),
        ("kappa0", C.c_double), ("kappa2", C.c_double),
        ("rho_s", C.c_double), ("k_min", C.c_double), ("k_max", C.c_double),
        ("zero_stab_cap", C.c_int), ("well", C.c_int),
        ("psd_nu", C.c_double), ("psd_itol", C.c_double), ("psd_lambda", C.c_double),
        ("psd_max_iter", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile fch_oracle.c into oracle/_build/liboracle.so (plain gcc, -O2)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            pp = C.POINTER(Params)
            L.orc_fft2.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_dft2.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int]
            L.orc_well.argtypes = [pp, C.c_double, dp, dp, dp]
            L.orc_alpha_m.argtypes = [pp]
            L.orc_alpha_m.restype = C.c_double
            L.orc_energy.argtypes = [pp, C.c_int, C.c_double, dp]
            L.orc_energy.restype = C.c_double
            L.orc_mass.argtypes = [C.c_int, C.c_double, dp]
            L.orc_mass.restype = C.c_double
            L.orc_mu.argtypes = [pp, C.c_int, C.c_double, dp, dp]
            L.orc_rhs.argtypes = [pp, C.c_int, C.c_double, dp, dp]
            L.orc_n_imex.argtypes = [pp, C.c_int, C.c_double, dp, dp]
            L.orc_sav_e1.argtypes = [pp, C.c_int, C.c_double, dp, dp]
            L.orc_sav_e1.restype = C.c_double
            L.orc_bdf2_coef.argtypes = [C.c_double, C.c_double, dp, dp, dp]
            L.orc_am3_coef.argtypes = [C.c_double, C.c_double, dp, dp, dp]
            L.orc_psd_lambda.argtypes = [pp, C.c_double]
            L.orc_psd_lambda.restype = C.c_double
            L.orc_phi.argtypes = [C.c_double, dp, dp, dp]
            L.orc_create.argtypes = [C.c_int, C.c_double, pp]
            L.orc_create.restype = C.c_void_p
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_state.argtypes = [C.c_void_p, dp]
            L.orc_set_history.argtypes = [C.c_void_p, dp, dp, C.c_double]
            L.orc_get_state.argtypes = [C.c_void_p, dp]
            L.orc_get_prev.argtypes = [C.c_void_p, dp]
            L.orc_get_time.argtypes = [C.c_void_p]
            L.orc_get_time.restype = C.c_double
            L.orc_get_r.argtypes = [C.c_void_p, C.c_int]
            L.orc_get_r.restype = C.c_double
            L.orc_get_kn.argtypes = [C.c_void_p]
            L.orc_get_kn.restype = C.c_double
            L.orc_get_counts.argtypes = [C.c_void_p, C.POINTER(C.c_long)]
            L.orc_get_last_e.argtypes = [C.c_void_p]
            L.orc_get_last_e.restype = C.c_double
            L.orc_step.argtypes = [C.c_void_p, C.c_int, C.c_double]
            L.orc_step.restype = C.c_int
            L.orc_step_from.argtypes = [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double)]
            L.orc_step_from.restype = C.c_int
            L.orc_run_adaptive.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_long]
            L.orc_run_adaptive.restype = C.c_int
            L.orc_adaptive_begin.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
            L.orc_adaptive_begin.restype = C.c_int
            L.orc_adaptive_trial.argtypes = [C.c_void_p]
            L.orc_adaptive_trial.restype = C.c_int
            L.orc_adaptive_trial_from.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
            L.orc_adaptive_trial_from.restype = C.c_int
            L.orc_get_last_k.argtypes = [C.c_void_p]
            L.orc_get_last_k.restype = C.c_double
            L.orc_get_next_k.argtypes = [C.c_void_p]
            L.orc_get_next_k.restype = C.c_double
            L.orc_get_last_accepted.argtypes = [C.c_void_p]
            L.orc_get_last_accepted.restype = C.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params(**kw) -> Params:
    """Oracle parameter record; defaults follow Table t:Benchmark (sub-critical, q=0)
    and the scheme constants of Secs. 3.2-3.6. Keyword arguments override fields."""
    d = dict(eps=0.1, q=0.0, gamma=0.3, b_minus=-1.0, b_plus=1.0, eta1=0.145, eta2=0.3,
             beta1=2.0, beta2=1.0, zeta=1.1, D0=170.0, kappa0=1e-2, kappa2=15.0,
             rho_s=0.9, k_min=1e-9, k_max=float("inf"), zero_stab_cap=0, well=0,
             psd_nu=1e-3, psd_itol=1e-12, psd_lambda=0.0, psd_max_iter=1000)
    d.update(kw)
    return Params(**d)


def fft2(a: np.ndarray, sign: int) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=np.complex128).copy()
    lib().orc_fft2(out.ctypes.data, out.shape[0], sign)
    return out


def dft2(a: np.ndarray, sign: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    out = np.empty_like(a)
    lib().orc_dft2(a.ctypes.data, out.ctypes.data, a.shape[0], sign)
    return out


def well(p: Params, u: float):
    W, W1, W2 = C.c_double(), C.c_double(), C.c_double()
    lib().orc_well(C.byref(p), float(u), C.byref(W), C.byref(W1), C.byref(W2))
    return W.value, W1.value, W2.value


def alpha_m(p: Params) -> float:
    return lib().orc_alpha_m(C.byref(p))


def energy(p: Params, u: np.ndarray, L: float) -> float:
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_energy(C.byref(p), u.shape[0], L, _dp(u))


def mass(u: np.ndarray, L: float) -> float:
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_mass(u.shape[0], L, _dp(u))


def _field_op(name, p, u, L):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    getattr(lib(), name)(C.byref(p), u.shape[0], L, _dp(u), _dp(out))
    return out


def mu(p, u, L):
    return _field_op("orc_mu", p, u, L)


def rhs(p, u, L):
    return _field_op("orc_rhs", p, u, L)


def n_imex(p, u, L):
    return _field_op("orc_n_imex", p, u, L)


def sav_e1(p, u, L, want_v=False):
    u = np.ascontiguousarray(u, dtype=np.float64)
    V = np.empty_like(u) if want_v else None
    e1 = lib().orc_sav_e1(C.byref(p), u.shape[0], L, _dp(u), _dp(V) if want_v else None)
    return (e1, V) if want_v else e1


def bdf2_coef(k1, kn):
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    lib().orc_bdf2_coef(k1, kn, C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def am3_coef(k1, kn):
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    lib().orc_am3_coef(k1, kn, C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def psd_lambda(p, k):
    return lib().orc_psd_lambda(C.byref(p), k)


def phi(z):
    e, p1, p2 = C.c_double(), C.c_double(), C.c_double()
    lib().orc_phi(z, C.byref(e), C.byref(p1), C.byref(p2))
    return e.value, p1.value, p2.value


class Stepper:
    """The oracle's time stepper (state u^n, u^{n-1}, r^n, r^{n-1}, t, k_n)."""

    def __init__(self, N: int, L: float, p: Params):
        self.N, self.L, self.p = N, L, p
        self._h = lib().orc_create(N, L, C.byref(p))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def set_state(self, u0):
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        lib().orc_set_state(self._h, _dp(u0))

    def set_history(self, un, unm1, kn):
        un = np.ascontiguousarray(un, dtype=np.float64)
        unm1 = np.ascontiguousarray(unm1, dtype=np.float64)
        lib().orc_set_history(self._h, _dp(un), _dp(unm1), float(kn))

    def state(self):
        u = np.empty((self.N, self.N))
        lib().orc_get_state(self._h, _dp(u))
        return u

    def prev(self):
        u = np.empty((self.N, self.N))
        lib().orc_get_prev(self._h, _dp(u))
        return u

    @property
    def t(self):
        return lib().orc_get_time(self._h)

    @property
    def kn(self):
        return lib().orc_get_kn(self._h)

    def r(self, which=0):
        return lib().orc_get_r(self._h, which)

    def counts(self):
        a = (C.c_long * 5)()
        lib().orc_get_counts(self._h, a)
        return dict(steps=a[0], rejects=a[1], psd_iter=a[2], attempts=a[3], last_psd_iter=a[4])

    @property
    def last_e(self):
        return lib().orc_get_last_e(self._h)

    def step(self, scheme, dt):
        s = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        rc = lib().orc_step(self._h, s, float(dt))
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")

    def step_from(self, scheme, dt, ustar):
        """one IMEX or SAV step whose extrapolation u* is the given N x N field"""
        s = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        a = np.ascontiguousarray(ustar, dtype=np.float64)
        assert a.shape == (self.N, self.N)
        rc = lib().orc_step_from(self._h, s, float(dt), _dp(a))
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")

    def run_adaptive(self, scheme, sigma, t_final, max_attempts=10**9):
        s = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        return lib().orc_run_adaptive(self._h, s, float(sigma), float(t_final), int(max_attempts))

    def adaptive_begin(self, scheme, sigma, t_final):
        """open an adaptive run (start step and F history); 0 or -1 (PSD failure)"""
        s = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        return lib().orc_adaptive_begin(self._h, s, float(sigma), float(t_final))

    def adaptive_trial(self):
        """one trial of the open run: 0 after a trial, 2 at t_final, -1 PSD failure"""
        return lib().orc_adaptive_trial(self._h)

    def adaptive_trial_from(self, ustar):
        """one trial of the open run whose u* (IMEX, SAV) or v_0 (PSD) is the given field"""
        a = np.ascontiguousarray(ustar, dtype=np.float64)
        assert a.shape == (self.N, self.N)
        return lib().orc_adaptive_trial_from(self._h, _dp(a))

    @property
    def last_k(self):
        """size of the last trial step"""
        return lib().orc_get_last_k(self._h)

    @property
    def next_k(self):
        """size of the next trial step"""
        return lib().orc_get_next_k(self._h)

    @property
    def last_accepted(self):
        return bool(lib().orc_get_last_accepted(self._h))
