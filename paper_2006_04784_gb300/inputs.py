"""Seeded synthetic initial data for the FCH steppers.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle's tests. It builds input fields only and holds none of the method's
arithmetic (no well, no operator, no time stepping).

Every field is an N x N float64 array on the periodic square [x0, x0 + L)^2,
row index = y, column index = x, point (i, j) at (x0 + j h, x0 + i h), h = L/N.

Bilayer dressing of a level-set function phi (used by all recipes):
    u0 = -1 + tanh((phi + R)/eps) - tanh((phi - R)/eps) + eps d / 1.7^2 (+ noise)
with half-width R = 0.14725 (Sec. 2.3) and the background eps d / alpha_m(0)^2,
alpha_m(0) = 1.7 (Table t:Benchmark).

Noise is counter-based: splitmix64 (S. Vigna's published mixer) of
seed * 2^32 + linear index, mapped to a 53-bit uniform in [-1, 1).
"""
from __future__ import annotations

import functools

import numpy as np

R_BILAYER = 0.14725
ALPHA_M0 = 1.7
L_DEFAULT = 4.0 * np.pi
X0_DEFAULT = -2.0 * np.pi

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """One splitmix64 output per 64-bit counter value (wrapping uint64 arithmetic)."""
    with np.errstate(over="ignore"):
        z = counter.astype(np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n uniforms in [-1, 1) from splitmix64(seed * 2^32 + i), i = 0..n-1."""
    base = np.uint64(seed) << np.uint64(32)
    z = splitmix64(base + np.arange(n, dtype=np.uint64))
    u01 = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u01 - 1.0


def uniform01(seed: int, n: int) -> np.ndarray:
    return 0.5 * (uniform_pm1(seed, n) + 1.0)


def grid(N: int, L: float = L_DEFAULT, x0: float = X0_DEFAULT):
    h = L / N
    c = x0 + h * np.arange(N)
    X, Y = np.meshgrid(c, c, indexing="xy")
    return X, Y


def dress(phi: np.ndarray, eps: float, d: float, R: float = R_BILAYER) -> np.ndarray:
    return -1.0 + np.tanh((phi + R) / eps) - np.tanh((phi - R) / eps) + eps * d / ALPHA_M0 ** 2


def circle_bilayer(N: int, eps: float = 0.1, radius: float = 2.0, d: float = 0.2,
                   noise: float = 1e-3, seed: int = 1, L: float = L_DEFAULT,
                   x0: float = X0_DEFAULT) -> np.ndarray:
    """Circular bilayer of the given radius centred at the origin, plus seeded
    uniform noise of the given amplitude (the 128^2 fixed-step workload)."""
    X, Y = grid(N, L, x0)
    u = dress(np.hypot(X, Y) - radius, eps, d)
    if noise:
        u = u + noise * uniform_pm1(seed, N * N).reshape(N, N)
    return np.ascontiguousarray(u)


def multimode_bilayer(N: int, eps: float = 0.1, r0: float = 3.0, d: float = 0.2,
                      seed: int = 2, modes=range(2, 9), L: float = L_DEFAULT,
                      x0: float = X0_DEFAULT) -> np.ndarray:
    """Bilayer along rho(theta) = r0 + sum_m a_m cos(m (theta - phi_m)), with
    a_m = (eps/2) U[0,1) and phi_m = 2 pi U[0,1) drawn from the seed (the 512^2
    adaptive workload; the curve family follows the paper's Gamma, Sec. 2.3)."""
    modes = list(modes)
    r = uniform01(seed, 2 * len(modes))
    amp = 0.5 * eps * r[: len(modes)]
    ph = 2.0 * np.pi * r[len(modes):]
    X, Y = grid(N, L, x0)
    th = np.arctan2(Y, X)
    rho = r0 + sum(a * np.cos(m * (th - p)) for a, m, p in zip(amp, modes, ph))
    return np.ascontiguousarray(dress(np.hypot(X, Y) - rho, eps, d))


def random_network(N: int, eps: float = 0.1, d: float = 0.75, seed: int = 3,
                   mmin: int = 2, mmax: int = 6, L: float = L_DEFAULT,
                   x0: float = X0_DEFAULT) -> np.ndarray:
    """Random bilayer network: the zero set of a smooth random periodic field
    phi = sum_{mmin <= |m| <= mmax} c_m cos(2 pi m.x / L + theta_m), Gaussian c_m,
    normalised by its RMS gradient so the dressed interfaces have unit slope on
    average (the 1024^2 / 2048^2 mixed-precision workload)."""
    ms = [(mx, my) for mx in range(-mmax, mmax + 1) for my in range(0, mmax + 1)
          if mmin ** 2 <= mx * mx + my * my <= mmax ** 2 and (my > 0 or mx > 0)]
    nm = len(ms)
    u = uniform01(seed, 3 * nm)
    # Box-Muller for the Gaussian amplitudes, uniform phases
    c = np.sqrt(-2.0 * np.log(np.maximum(u[:nm], 1e-300))) * np.cos(2.0 * np.pi * u[nm:2 * nm])
    th = 2.0 * np.pi * u[2 * nm:]
    X, Y = grid(N, L, x0)
    kf = 2.0 * np.pi / L
    phi = np.zeros((N, N))
    gx = np.zeros((N, N))
    gy = np.zeros((N, N))
    for (mx, my), cm, tm in zip(ms, c, th):
        arg = kf * (mx * X + my * Y) + tm
        phi += cm * np.cos(arg)
        s = -cm * np.sin(arg)
        gx += s * kf * mx
        gy += s * kf * my
    phi /= np.sqrt(np.mean(gx * gx + gy * gy))
    return np.ascontiguousarray(dress(phi, eps, d))


def single_mode(N: int, mx: int, my: int, amp: float = 1.0, offset: float = 0.0,
                L: float = L_DEFAULT, x0: float = X0_DEFAULT) -> np.ndarray:
    """offset + amp cos(2 pi (mx x + my y)/L) on the grid (operator tests)."""
    X, Y = grid(N, L, x0)
    return np.ascontiguousarray(offset + amp * np.cos(2.0 * np.pi * (mx * X + my * Y) / L))


def smooth_random(N: int, seed: int, amp: float = 0.5, kmax: int = 4, offset: float = -0.5,
                  L: float = L_DEFAULT, x0: float = X0_DEFAULT) -> np.ndarray:
    """A smooth random field with modes |m| <= kmax (small-grid tests)."""
    ms = [(mx, my) for mx in range(-kmax, kmax + 1) for my in range(0, kmax + 1)
          if (my > 0 or mx > 0) and mx * mx + my * my <= kmax * kmax]
    r = uniform_pm1(seed, 2 * len(ms))
    X, Y = grid(N, L, x0)
    f = np.full((N, N), offset)
    kf = 2.0 * np.pi / L
    for (mx, my), a, t in zip(ms, r[: len(ms)], r[len(ms):]):
        f += amp / len(ms) ** 0.5 * a * np.cos(kf * (mx * X + my * Y) + np.pi * t)
    return np.ascontiguousarray(f)


# --------------------------------------------------------------------------- the paper's initial data
# Table t:Benchmark (Sec. 2.2-2.3): q, eta1/eps, eta2/eps, d, N for the five benchmarks
BENCHMARKS = {
    "subcritical": dict(q=0.0, eta1=1.45, eta2=3.0, d=0.2, N=256),
    "critical": dict(q=0.0, eta1=1.45, eta2=1.5, d=0.75, N=256),
    "supercritical": dict(q=0.0, eta1=1.45, eta2=3.0, d=0.5, N=256),
    "foot1": dict(q=0.2, eta1=1.45, eta2=3.0, d=0.2, N=256),
    "foot2": dict(q=0.5, eta1=1.45, eta2=3.0, d=0.2, N=512),
}
LAMBDA0 = 7.0269e-3


def paper_curve(theta, eps=0.1, L=L_DEFAULT):
    """Gamma of Sec. 2.3: radius rho(theta) = 3 - (eps/2) cos(6 (theta - pi/11))
    - eps^2 cos(theta - 3 pi/11) about the centre of the square."""
    return (3.0 - 0.5 * eps * np.cos(6.0 * (theta - np.pi / 11.0))
            - eps * eps * np.cos(theta - 3.0 * np.pi / 11.0))


def _curve_distance(px, py, eps=0.1, L=L_DEFAULT):
    """distance from points (px, py), relative to the centre of the square, to
    Gamma: minimised over curve points within +-0.15 rad of each point's polar
    angle (R is far below Gamma's radius of curvature), refined twice."""
    th0 = np.arctan2(py, px)
    best = np.full(px.shape, np.inf)
    bt = th0.copy()
    for width, ns in ((0.15, 61), (0.006, 31), (0.0003, 31)):
        centre = bt.copy()
        for dt in np.linspace(-width, width, ns):
            t = centre + dt
            r = paper_curve(t, eps, L)
            dist = np.hypot(px - r * np.cos(t), py - r * np.sin(t))
            m = dist < best
            best = np.where(m, dist, best)
            bt = np.where(m, t, bt)
    return best


@functools.lru_cache(maxsize=4)
def _paper_band_cached(No, eps, R, L, x0, sub):
    return _paper_band(No, eps, R, L, x0, sub)


def paper_band(No: int = 256, eps: float = 0.1, R: float = R_BILAYER, L: float = L_DEFAULT,
               x0: float = X0_DEFAULT, sub: int = 16) -> np.ndarray:
    """phi_Gamma (see _paper_band); cached, returns a copy."""
    return _paper_band_cached(No, eps, R, L, x0, sub).copy()


def _paper_band(No: int = 256, eps: float = 0.1, R: float = R_BILAYER, L: float = L_DEFAULT,
                x0: float = X0_DEFAULT, sub: int = 16) -> np.ndarray:
    """phi_Gamma on the No x No mesh: +1 inside the band Gamma_R (within normal
    distance R of Gamma, between Gamma_+ and Gamma_-), -1 outside, taken as the cell
    average of the indicator (the area fraction of each mesh cell inside the band,
    by sub x sub sampling of the cells the band boundary crosses), so that its mean
    is the band area 2 R |Gamma|."""
    h = L / No
    X, Y = grid(No, L, x0)
    c = x0 + 0.5 * L
    px, py = X.ravel() - c, Y.ravel() - c
    dist = _curve_distance(px, py, eps, L)
    frac = (dist <= R).astype(float)
    edge = np.nonzero(np.abs(dist - R) < 0.75 * h)[0]
    off = (np.arange(sub) + 0.5) / sub - 0.5
    ox, oy = np.meshgrid(off * h, off * h, indexing="xy")
    for chunk in np.array_split(edge, max(1, len(edge) // 512)):
        qx = (px[chunk][:, None] + ox.ravel()[None, :]).ravel()
        qy = (py[chunk][:, None] + oy.ravel()[None, :]).ravel()
        dq = _curve_distance(qx, qy, eps, L).reshape(len(chunk), -1)
        frac[chunk] = (dq <= R).mean(axis=1)
    return (2.0 * frac - 1.0).reshape(No, No)


def paper_initial_data(N: int, d: float, eps: float = 0.1, No: int = 256, lam0: float = LAMBDA0,
                       filter_k: str = "physical", L: float = L_DEFAULT,
                       x0: float = X0_DEFAULT) -> np.ndarray:
    """u0 of eq. (dcoef): the band indicator on the No x No mesh, smoothed by the
    Gaussian filter exp(-lam0 |k|^2), evaluated on the N x N grid by spectral
    interpolation, plus the background eps d / alpha_m(0)^2, alpha_m(0) = 1.7.
    filter_k = "physical": k = 2 pi m / L (the smoothed band keeps a bilayer-like
    peak, ~0.57); "integer": k = m, the literal index of the printed sum (peak
    ~-0.07). The mass does not depend on the choice (the k = 0 mode is kept)."""
    phi = paper_band(No, eps, R_BILAYER, L, x0)
    ph = np.fft.fft2(phi)
    m_ = np.fft.fftfreq(No, 1.0 / No)
    k = m_ if filter_k == "integer" else 2.0 * np.pi * m_ / L
    ph = ph * np.exp(-lam0 * (k[None, :] ** 2 + k[:, None] ** 2))
    m = min(N, No) // 2
    out = np.zeros((N, N), dtype=complex)
    out[:m, :m] = ph[:m, :m]
    out[:m, -m:] = ph[:m, -m:]
    out[-m:, :m] = ph[-m:, :m]
    out[-m:, -m:] = ph[-m:, -m:]
    phiN = np.real(np.fft.ifft2(out)) * (N * N) / (No * No)
    return np.ascontiguousarray(phiN + eps * d / ALPHA_M0 ** 2)
