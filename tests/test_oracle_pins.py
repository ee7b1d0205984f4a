"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: each check uses a printed value
(tests/golden, cited), a closed form, an invariant, brute force on a tiny grid,
or an independent library routine (numpy's FFT, dense linear algebra, mpmath).
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2006_04784_gb300 import inputs as I

L = 4.0 * np.pi
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line.split())
    return rows


def ksq(N):
    m = np.fft.fftfreq(N, 1.0 / N)
    k = 2 * np.pi * m / L
    return k[None, :] ** 2 + k[:, None] ** 2


def h2(N):
    return (L / N) ** 2


# ----------------------------------------------------------------------------- FFT
@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_fft_matches_bruteforce_dft(N):
    rng = np.random.default_rng(N)
    a = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    for sign in (-1, 1):
        ref = O.dft2(a, sign)
        got = O.fft2(a, sign)
        if sign > 0:
            ref = ref / N ** 2
        assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("N", [8, 32, 64])
def test_fft_parseval_roundtrip_single_mode(N):
    rng = np.random.default_rng(1)
    a = rng.standard_normal((N, N))
    A = O.fft2(a, -1)
    assert abs(np.sum(np.abs(A) ** 2) / N ** 2 - np.sum(a ** 2)) < 1e-11 * np.sum(a ** 2)
    assert np.abs(O.fft2(A, 1) - a).max() < 1e-14 * N
    # cos(2 pi (3x + 5y)/N) on the index grid: two spikes of height N^2/2
    y, x = np.mgrid[0:N, 0:N]
    f = np.cos(2 * np.pi * (3 * x + 5 * y) / N)
    F = O.fft2(f, -1)
    spikes = np.zeros((N, N))
    spikes[5, 3] = spikes[-5 % N, -3 % N] = N * N / 2
    assert np.abs(F - spikes).max() < 1e-10 * N * N


def test_fft_matches_numpy():
    a = np.random.default_rng(3).standard_normal((64, 64))
    assert np.abs(O.fft2(a, -1) - np.fft.fft2(a)).max() < 1e-11


# ----------------------------------------------------------------------------- well
def test_alpha_m_table_values():
    for q, am in _golden("alpha_m.txt"):
        p = O.params(q=float(q))
        assert abs(O.alpha_m(p) - float(am)) < 1e-12
        assert abs(O.well(p, -1.0)[2] - float(am)) < 1e-12


@pytest.mark.parametrize("q", [0.0, 0.05, 0.2, 0.5, 1.3])
def test_alpha_m_closed_form(q):
    # W_q''(b_-) = (1 + q/eps) * B(b_-), B(-1) = 2 - 0.3 = 1.7
    assert abs(O.alpha_m(O.params(q=q)) - 1.7 * (1 + q / 0.1)) < 1e-12


@pytest.mark.parametrize("q", [0.0, 0.2, 0.5])
def test_well_roots_and_derivatives(q):
    p = O.params(q=q)
    W, W1, W2 = O.well(p, -1.0)
    assert W == 0.0 and abs(W1) < 1e-15
    if q == 0.0:
        assert abs(O.well(p, 1.0)[1]) < 1e-14  # W'(b_+) = 0 for q = 0
    # derivatives against Richardson-extrapolated central differences
    for u in np.linspace(-1.6, 1.4, 23):
        def d(f, u, h):
            return (f(u + h) - f(u - h)) / (2 * h)

        def rich(f, u):
            h = 1e-3
            return (4 * d(f, u, h / 2) - d(f, u, h)) / 3

        w = O.well(p, u)
        fd1 = rich(lambda x: O.well(p, x)[0], u)
        fd2 = rich(lambda x: O.well(p, x)[1], u)
        assert abs(fd1 - w[1]) < 1e-7 * (1 + abs(w[1]))
        assert abs(fd2 - w[2]) < 1e-7 * (1 + abs(w[2]))


def test_well_q0_is_tilted_quartic():
    # q = 0: W = (u+1)^2/2 * ((u-1)^2/2 + 0.1 (u - 2)), a polynomial
    p = O.params(q=0.0)
    for u in np.linspace(-2, 2, 17):
        ref = 0.5 * (u + 1) ** 2 * (0.5 * (u - 1) ** 2 + 0.1 * (u - 2))
        assert abs(O.well(p, u)[0] - ref) < 1e-14


# ----------------------------------------------------------------------------- energy, mu
def test_energy_constant_state_closed_form():
    p = O.params(q=0.2)
    for c in (-1.0, -0.7, 0.3):
        u = np.full((16, 16), c)
        W, W1, _ = O.well(p, c)
        ref = L * L * (0.5 * W1 ** 2 - p.eta2 * W)
        assert abs(O.energy(p, u, L) - ref) < 1e-12 * (1 + abs(ref))


def test_energy_single_mode_quadratic_well():
    p = O.params(well=1)
    am = O.alpha_m(p)
    N, A, mx, my = 32, 0.3, 2, 1
    u = I.single_mode(N, mx, my, amp=A, offset=-1.0)
    k2 = (2 * np.pi / L) ** 2 * (mx * mx + my * my)
    ref = L * L * A * A / 4 * ((p.eps ** 2 * k2 + am) ** 2 - p.eps ** 2 * p.eta1 * k2 - p.eta2 * am)
    assert abs(O.energy(p, u, L) - ref) < 1e-11 * abs(ref)


def test_mu_is_variational_derivative_of_energy():
    # brute force: dE/du_j / h^2 by central differences on an 8x8 grid
    p = O.params(q=0.2)
    N = 8
    u = I.smooth_random(N, seed=11, amp=0.6, kmax=2)
    mu = O.mu(p, u, L)
    rng = np.random.default_rng(0)
    for j in rng.choice(N * N, 6, replace=False):
        e = np.zeros(N * N)
        e[j] = 1.0
        e = e.reshape(N, N)
        d = 1e-5
        fd = (O.energy(p, u + d * e, L) - O.energy(p, u - d * e, L)) / (2 * d * h2(N))
        assert abs(fd - mu.flat[j]) < 1e-5 * (1 + np.abs(mu).max())


def test_mu_single_mode_quadratic_well():
    # mu = eps^4 Lap^2 u - 2 a eps^2 Lap u + a^2 (u + 1) for W = a/2 (u+1)^2, eta = 0
    p = O.params(well=1, eta1=0.0, eta2=0.0)
    am = O.alpha_m(p)
    N, A = 32, 0.2
    u = I.single_mode(N, 3, 2, amp=A, offset=-0.9)
    k2 = (2 * np.pi / L) ** 2 * 13
    ref = (p.eps ** 4 * k2 ** 2 + 2 * am * p.eps ** 2 * k2 + am * am) * (u + 0.9) + am * am * 0.1
    assert np.abs(O.mu(p, u, L) - ref).max() < 1e-10 * np.abs(ref).max()
    F = O.rhs(p, u, L)
    assert np.abs(F - (-k2) * (ref - am * am * 0.1)).max() < 1e-9 * k2 * np.abs(ref).max()


def test_imex_split_identity():
    # L_IMEX u + N_IMEX(u) = dE/du (Sec. 3.4), L_IMEX applied with numpy's FFT
    p = O.params(q=0.5)
    am = O.alpha_m(p)
    N = 32
    u = I.smooth_random(N, seed=5)
    lim = (p.eps ** 2 * ksq(N) + am) ** 2
    Lu = np.real(np.fft.ifft2(lim * np.fft.fft2(u)))
    assert np.abs(Lu + O.n_imex(p, u, L) - O.mu(p, u, L)).max() < 1e-10 * np.abs(Lu).max()


def test_n_imex_has_zero_linearisation_at_bminus():
    p = O.params(q=0.2, eta1=0.0, eta2=0.0)
    N = 16
    v = I.smooth_random(N, seed=9, amp=1.0, offset=0.0)
    base = O.n_imex(p, np.full((N, N), -1.0), L)
    r1 = np.abs(O.n_imex(p, -1.0 + 1e-3 * v, L) - base).max()
    r2 = np.abs(O.n_imex(p, -1.0 + 5e-4 * v, L) - base).max()
    assert r1 / r2 > 3.5  # quadratic, not linear, in the perturbation


def test_sav_energy_split_and_variational_derivative():
    # E(u) = 1/2 (u, L_SAV u) + E1(u) (eq. 4.2); L_SAV u + V[u] = dE/du
    p = O.params(q=0.2)
    N = 16
    u = I.smooth_random(N, seed=21)
    k2 = ksq(N)
    lsav = p.eps ** 4 * k2 ** 2 - p.eps ** 2 * (p.eta1 + 2 * p.zeta) * k2
    Lu = np.real(np.fft.ifft2(lsav * np.fft.fft2(u)))
    e1, V = O.sav_e1(p, u, L, want_v=True)
    E = O.energy(p, u, L)
    assert abs(0.5 * h2(N) * np.sum(u * Lu) + e1 - E) < 1e-11 * (1 + abs(E))
    mu = O.mu(p, u, L)
    assert np.abs(Lu + V - mu).max() < 1e-10 * np.abs(mu).max()
    # V = dE1/du by brute force at a few points
    N = 8
    u = I.smooth_random(N, seed=4)
    _, V = O.sav_e1(p, u, L, want_v=True)
    for j in (0, 13, 40):
        e = np.zeros(N * N)
        e[j] = 1
        e = e.reshape(N, N)
        fd = (O.sav_e1(p, u + 1e-5 * e, L) - O.sav_e1(p, u - 1e-5 * e, L)) / (2e-5 * h2(N))
        assert abs(fd - V.flat[j]) < 1e-5 * (1 + np.abs(V).max())


def test_mass_definition():
    u = I.circle_bilayer(32)
    assert abs(O.mass(u, L) - 0.5 * h2(32) * np.sum(u + 1)) < 1e-12
    assert abs(O.mass(np.full((8, 8), -1.0), L)) == 0.0


# ----------------------------------------------------------------------------- coefficients
def test_uniform_coefficients_from_paper():
    g = {r[0]: [float(x) for x in r[1:]] for r in _golden("bdf2_am3_uniform.txt")}
    k = 0.37
    a, b, c = O.bdf2_coef(k, k)
    assert np.allclose([a * k, b * k, c * k], g["bdf2_k"], rtol=0, atol=1e-14)
    w = O.am3_coef(k, k)
    assert np.allclose(np.array(w) / k, g["am3_k"], rtol=0, atol=1e-14)


@pytest.mark.parametrize("k1,kn", [(0.3, 0.1), (0.05, 0.2), (1.0, 1.0), (2.4142, 1.0)])
def test_bdf2_exact_on_quadratics_am3_on_cubics(k1, kn):
    t0 = 1.3
    tm, tn, tp = t0 - kn, t0, t0 + k1
    a, b, c = O.bdf2_coef(k1, kn)
    for f, df in [(lambda t: 1.0, lambda t: 0.0), (lambda t: t, lambda t: 1.0),
                  (lambda t: t * t, lambda t: 2 * t)]:
        assert abs(a * f(tp) + b * f(tn) + c * f(tm) - df(tp)) < 1e-10
    w1, w2, w3 = O.am3_coef(k1, kn)
    for F, U in [(lambda t: 1.0, lambda t: t), (lambda t: t, lambda t: t * t / 2),
                 (lambda t: t * t, lambda t: t ** 3 / 3)]:
        assert abs(U(tp) - U(tn) - (w1 * F(tp) + w2 * F(tn) + w3 * F(tm))) < 1e-12


def test_bdf1_start_and_consistency():
    a, b, c = O.bdf2_coef(0.2, 0.0)
    assert (a, b, c) == (5.0, -5.0, 0.0)
    a, b, c = O.bdf2_coef(0.2, 0.7)
    assert abs(a + b + c) < 1e-14  # constants are preserved: mass conservation


def test_psd_lambda_table():
    rows = _golden("psd_lambda.txt")
    for r in rows:
        k = float(r[0])
        for q, v in zip((0.0, 0.2, 0.5), r[1:]):
            assert abs(O.psd_lambda(O.params(q=q), k) - float(v)) < 1e-14
    p = O.params(q=0.0)
    assert O.psd_lambda(p, 1e-8) == 1.0 and O.psd_lambda(p, 0.5) == 1.855
    assert abs(O.psd_lambda(p, 7.5e-3) - 0.5 * (1.60 + 1.738)) < 1e-14


def test_phi_functions_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for z in [-1e-12, -3e-7, -2e-3, -9.99e-3, -1.0001e-2, -0.5, -7.0, -300.0, 1e-4, 0.3]:
        e, p1, p2 = O.phi(z)
        Z = mp.mpf(z)
        r1 = (mp.e ** Z - 1) / Z
        r2 = (mp.e ** Z - 1 - Z) / Z ** 2
        assert abs(p1 - float(r1)) <= 2e-15 * abs(float(r1))
        assert abs(p2 - float(r2)) <= 5e-14 * abs(float(r2))


# ----------------------------------------------------------------------------- schemes
SCHEMES = ["imex", "sav", "psd", "etd"]


@pytest.mark.parametrize("scheme", SCHEMES)
def test_mass_conserved(scheme):
    p = O.params(q=0.2)
    N = 32
    u = I.circle_bilayer(N)
    s = O.Stepper(N, L, p)
    s.set_state(u)
    m0 = O.mass(u, L)
    for _ in range(4):
        s.step(scheme, 2e-4)
    assert abs(O.mass(s.state(), L) - m0) < 1e-11 * abs(m0)


def _per_mode_linear(N, p, u0, dt, nsteps):
    """Closed-form recurrence of the linear problem u_t = Lap L_IMEX u (quadratic
    well, eta = 0): (a + |k|^2 s) U^{n+1} = -b U^n - c U^{n-1}, BE start."""
    am = O.alpha_m(p)
    k2 = ksq(N)
    sym = k2 * (p.eps ** 2 * k2 + am) ** 2
    U = np.fft.fft2(u0)
    Um = None
    for n in range(nsteps):
        if Um is None:
            Un = U / (1 + dt * sym)
        else:
            a, b, c = 1.5 / dt, -2 / dt, 0.5 / dt
            Un = (-b * U - c * Um) / (a + sym)
        Um, U = U, Un
    return np.real(np.fft.ifft2(U)), sym


@pytest.mark.parametrize("scheme", ["imex", "psd"])
def test_linear_problem_closed_form_recurrence(scheme):
    p = O.params(well=1, eta1=0.0, eta2=0.0, psd_itol=1e-14, psd_lambda=1.0)
    N = 16
    u0 = I.smooth_random(N, seed=2, amp=0.3, offset=-0.8)
    s = O.Stepper(N, L, p)
    s.set_state(u0)
    for _ in range(5):
        s.step(scheme, 1e-3)
    ref, _ = _per_mode_linear(N, p, u0, 1e-3, 5)
    tol = 1e-12 if scheme == "imex" else 1e-10
    assert np.abs(s.state() - ref).max() < tol * np.abs(ref).max()


def test_etd_exact_on_linear_problem():
    p = O.params(well=1, eta1=0.0, eta2=0.0, kappa0=0.0, kappa2=0.0)
    N = 16
    u0 = I.smooth_random(N, seed=3, amp=0.3, offset=-0.8)
    s = O.Stepper(N, L, p)
    s.set_state(u0)
    for _ in range(3):
        s.step("etd", 2e-3)
    _, sym = _per_mode_linear(N, p, u0, 1, 0)
    ref = np.real(np.fft.ifft2(np.exp(-sym * 6e-3) * np.fft.fft2(u0)))
    assert np.abs(s.state() - ref).max() < 1e-12 * np.abs(ref).max()


def test_psd_matches_dense_newton_bdf2_solution():
    # N = 8: solve a u + b u^n + c u^{n-1} = F(u) by Newton with a dense
    # finite-difference Jacobian; PSD at a tight tolerance must land on it.
    p = O.params(q=0.2, psd_itol=1e-13, psd_max_iter=5000)
    N = 8
    u0 = I.smooth_random(N, seed=8, amp=0.5, kmax=2)
    s = O.Stepper(N, L, p)
    s.set_state(u0)
    dt = 1e-3
    s.step("psd", dt)  # backward-Euler start
    s.step("psd", dt)
    un, um = s.prev(), None
    s2 = O.Stepper(N, L, p)
    s2.set_state(u0)
    s2.step("imex", dt)
    # reference: Newton on the BE step from u0, then on the BDF2 step
    def newton(rhs_const, a, guess):
        v = guess.copy().ravel()
        for _ in range(30):
            def res(x):
                return a * x + rhs_const.ravel() - O.rhs(p, x.reshape(N, N), L).ravel()
            r = res(v)
            J = np.empty((N * N, N * N))
            for j in range(N * N):
                e = np.zeros(N * N)
                e[j] = 1e-6
                J[:, j] = (res(v + e) - res(v - e)) / 2e-6
            dv = np.linalg.lstsq(J, -r, rcond=None)[0]
            v += dv
            if np.abs(dv).max() < 1e-13:
                break
        return v.reshape(N, N)

    u1 = newton(-u0 / dt, 1 / dt, u0)
    assert np.abs(un - u1).max() < 1e-9
    a, b, c = 1.5 / dt, -2 / dt, 0.5 / dt
    u2 = newton(b * u1 + c * u0, a, u1)
    assert np.abs(s.state() - u2).max() < 1e-9


def test_sav_modified_energy_decays_fixed_step():
    # Theorem t:SAV: E_aux(u^{n+1}, u^n, r^{n+1}, r^n) <= E_aux(u^n, u^{n-1}, r^n, r^{n-1})
    p = O.params(q=0.0)
    N = 32
    u0 = I.circle_bilayer(N, noise=1e-2)
    am = O.alpha_m(p)
    k2 = ksq(N)
    e2 = p.eps ** 2
    lsav = e2 * e2 * k2 ** 2 - e2 * (p.eta1 + 2 * p.zeta) * k2
    l1 = -e2 * (p.eta1 + 2 * p.zeta) * k2 - p.beta1 * am * e2 * k2 - p.beta2 * am * am

    def quad(sym, f):
        return h2(N) * np.sum(f * np.real(np.fft.ifft2(sym * np.fft.fft2(f))))

    def eaux(u, um, r, rm):
        return (0.5 * quad(lsav, u) - quad(l1, u - um) + 0.5 * quad(lsav, 2 * u - um)
                + r * r + (2 * r - rm) ** 2)

    for dt in (1e-3, 5e-2):
        s = O.Stepper(N, L, p)
        s.set_state(u0)
        s.step("sav", dt)
        prev = None
        for _ in range(6):
            s.step("sav", dt)
            ea = eaux(s.state(), s.prev(), s.r(0), s.r(1))
            if prev is not None:
                assert ea <= prev + 1e-9 * abs(prev)
            prev = ea


@pytest.mark.parametrize("scheme", ["imex", "psd", "sav"])
def test_energy_decays_small_steps(scheme):
    p = O.params(q=0.0)
    N = 32
    s = O.Stepper(N, L, p)
    s.set_state(I.circle_bilayer(N, noise=1e-2))
    E = O.energy(p, s.state(), L)
    for _ in range(6):
        s.step(scheme, 5e-4)
        En = O.energy(p, s.state(), L)
        assert En <= E + 1e-10 * abs(E)
        E = En


@pytest.mark.parametrize("scheme", SCHEMES)
def test_temporal_order_two(scheme):
    # self-convergence at fixed k (Table tab:rates reports order ~2 for all four)
    p = O.params(q=0.0, psd_itol=1e-13)
    N = 16
    u0 = I.smooth_random(N, seed=7, amp=0.4, offset=-0.6, kmax=2)
    T = 0.04

    def run(n):
        s = O.Stepper(N, L, p)
        s.set_state(u0)
        for _ in range(n):
            s.step(scheme, T / n)
        return s.state()

    ref = run(640)
    e1 = np.linalg.norm(run(20) - ref)
    e2 = np.linalg.norm(run(40) - ref)
    e3 = np.linalg.norm(run(80) - ref)
    r1, r2 = math.log2(e1 / e2), math.log2(e2 / e3)
    assert 1.6 < r2 < 2.6, (r1, r2)


def test_lte_estimate_scales_as_k_cubed():
    # Linear problem (quadratic well, eta = 0) started from its exact solution
    # exp(-|k|^2 s t) at t0 - k and t0: BDF2 has local error O(k^3), AM3 O(k^4),
    # so e(k)/e(k/2) -> 8.
    p = O.params(well=1, eta1=0.0, eta2=0.0)
    N = 16
    u0 = I.smooth_random(N, seed=12, amp=0.4, offset=-0.6, kmax=2)
    _, sym = _per_mode_linear(N, p, u0, 1, 0)
    U0 = np.fft.fft2(u0)

    def exact(t):
        return np.real(np.fft.ifft2(np.exp(-sym * t) * U0))

    es = []
    t0 = 0.02
    for k in (4e-3, 2e-3, 1e-3):
        s = O.Stepper(N, L, p)
        s.set_history(exact(t0), exact(t0 - k), k)
        s.run_adaptive("imex", 1e9, s.t + k)
        es.append(s.last_e)
    assert 7.0 < es[0] / es[1] < 9.0 and 7.0 < es[1] / es[2] < 9.0, es


def test_adaptive_controller_invariants():
    p = O.params(q=0.0)
    N = 16
    s = O.Stepper(N, L, p)
    s.set_state(I.circle_bilayer(N))
    assert s.run_adaptive("imex", 1e-5, 0.05) == 0
    c = s.counts()
    assert abs(s.t - 0.05) < 1e-15 and c["steps"] > 3 and c["rejects"] >= 0
    # Without the zero-stability cap the first jump from k_min has step ratio ~1e4,
    # and variable-step BDF2 amplifies rounding in the mean mode by that ratio
    # (Sec. 3.2); with the cap A_dp <= (1 + sqrt 2) k the mean is kept to rounding.
    m0 = O.mass(I.circle_bilayer(N), L)
    assert O.mass(s.state(), L) == pytest.approx(m0, rel=1e-7)
    pc = O.params(q=0.0, zero_stab_cap=1)
    sc = O.Stepper(N, L, pc)
    sc.set_state(I.circle_bilayer(N))
    assert sc.run_adaptive("imex", 1e-5, 0.05) == 0
    assert O.mass(sc.state(), L) == pytest.approx(m0, rel=1e-11)
    # the attempt budget is honoured
    s.set_state(I.circle_bilayer(N))
    assert s.run_adaptive("imex", 1e-5, 10.0, max_attempts=5) == 1


def test_etd_stabiliser_splitting_is_consistent():
    # L u + N(u) = Lap L_IMEX u for any kappa0, kappa2 (eq. ETD-L): on the linear
    # problem ETDRK2 with the paper's kappas converges to exp(-|k|^2 s t) at order 2.
    p = O.params(well=1, eta1=0.0, eta2=0.0, kappa0=1e-2, kappa2=15.0)
    N = 16
    u0 = I.smooth_random(N, seed=3, amp=0.3, offset=-0.8, kmax=3)
    _, sym = _per_mode_linear(N, p, u0, 1, 0)
    T = 0.02
    ref = np.real(np.fft.ifft2(np.exp(-sym * T) * np.fft.fft2(u0)))
    errs = []
    for n in (10, 20, 40):
        s = O.Stepper(N, L, p)
        s.set_state(u0)
        for _ in range(n):
            s.step("etd", T / n)
        errs.append(np.linalg.norm(s.state() - ref))
    assert errs[2] < 1e-3 * np.linalg.norm(ref)
    assert 1.7 < math.log2(errs[1] / errs[2]) < 2.4, errs


def test_benchmark_initial_data_mass_matches_table():
    # Table t:Benchmark prints the mass of each benchmark's initial data; it pins
    # the mass functional (Sec. 2.3), the band width 2R, the curve Gamma and the
    # background eps d / alpha_m(0)^2 of eq. (dcoef) together.
    for case, d, n, mass in _golden("benchmark_mass.txt"):
        u0 = I.paper_initial_data(int(n), float(d))
        assert round(O.mass(u0, L), 2) == float(mass), case
    # the band itself: area 2 R |Gamma|, |Gamma| from rho(theta) by quadrature
    th = np.linspace(0, 2 * np.pi, 100001)[:-1]
    rho = I.paper_curve(th)
    drho = np.gradient(rho, th)
    length = np.sum(np.hypot(rho, drho)) * (2 * np.pi / len(th))
    band = I.paper_band()
    area = np.sum((band + 1) / 2) * (L / 256) ** 2
    assert abs(area - 2 * I.R_BILAYER * length) < 5e-4


# ----------------------------------------------------------------------------- given extrapolation
def _two_level_state(N, q=0.0):
    u1 = I.circle_bilayer(N, noise=1e-3)
    s = O.Stepper(N, L, O.params(q=q))
    s.set_state(u1)
    s.step("imex", 1e-4)
    return u1, s.state()


@pytest.mark.parametrize("scheme", ["imex", "sav"])
def test_step_from_with_the_extrapolation_is_the_plain_step(scheme):
    # eq. (Richardson) fed in from outside gives the plain step, bit for bit
    N, kn, dt = 32, 1e-4, 1.5e-4
    um, un = _two_level_state(N)
    ustar = un + (dt / kn) * (un - um)
    out = []
    for given in (False, True):
        s = O.Stepper(N, L, O.params())
        s.set_history(un, um, kn)
        if given:
            s.step_from(scheme, dt, ustar)
        else:
            s.step(scheme, dt)
        out.append(s.state())
    assert np.array_equal(out[0], out[1])


def test_step_from_takes_imex_and_sav_only():
    N = 16
    s = O.Stepper(N, L, O.params())
    s.set_state(I.circle_bilayer(N))
    for scheme in ("psd", "etd"):
        with pytest.raises(RuntimeError):
            s.step_from(scheme, 1e-4, s.state())


@pytest.mark.parametrize("q", [0.0, 0.2])
def test_imex_step_from_the_implicit_solution_returns_it(q):
    # a fixed point of the fully implicit BDF2, eq. (BDF2), is a fixed point of the
    # IMEX step, eq. (IMEX-eq), whose extrapolation is that fixed point: the IMEX
    # splitting only moves the nonlinear part to u*
    N, kn, dt = 32, 1e-4, 2e-4
    um, un = _two_level_state(N, q)
    s = O.Stepper(N, L, O.params(q=q, psd_itol=1e-14, psd_max_iter=5000))
    s.set_history(un, um, kn)
    s.step("psd", dt)
    u_bdf2 = s.state()
    t = O.Stepper(N, L, O.params(q=q))
    t.set_history(un, um, kn)
    t.step_from("imex", dt, u_bdf2)
    assert np.linalg.norm(t.state() - u_bdf2) / np.linalg.norm(u_bdf2) < 1e-11
    # while the plain extrapolation leaves the IMEX splitting error
    t2 = O.Stepper(N, L, O.params(q=q))
    t2.set_history(un, um, kn)
    t2.step("imex", dt)
    assert np.linalg.norm(t2.state() - u_bdf2) / np.linalg.norm(u_bdf2) > 1e-9


# ----------------------------------------------------------------------------- step-size controller
# Sec. 3.2, Steps 0-4 and A_dp, pinned on the linear problem (quadratic well,
# eta = 0), where a trial and its error estimate have closed forms per Fourier
# mode: the BDF2 trial (a + s(k)) U~ = -b U^n - c U^{n-1} of eq. (BDF2Coef), the
# right-hand side F(U) = -s(k) U, the AM3 predictor of eq. (Predictor) and
# e = ||U~ - U_p|| / ||U_p|| (Parseval: the ratio of the real-space norms). The
# decisions are then checked against the algorithm as printed, with the paper's
# safety factor rho_s = 0.9 and exponent 1/3.
RHO_S = 0.9  # Sec. 3.2


def _bdf2_abc(k1, kn):
    # eq. (BDF2Coef)
    return 1 / k1 + 1 / (k1 + kn), -1 / k1 - 1 / kn, 1 / kn - 1 / (k1 + kn)


def _am3_w(k1, kn):
    # eq. (Predictor) with gamma = k1 / kn
    g = k1 / kn
    return k1 / 6 * (3 + 2 * g) / (1 + g), k1 / 6 * (3 + g), -k1 / 6 * g * g / (1 + g)


class _Linear:
    """the linear problem on 16^2 started from its exact solution at t0 - kn, t0"""

    N, t0, kn = 16, 0.02, 2e-3

    def __init__(self):
        self.p0 = O.params(well=1, eta1=0.0, eta2=0.0)
        am = float(_golden("alpha_m.txt")[0][1])  # alpha_m(0) = 1.7, Table t:Benchmark
        k2 = ksq(self.N)
        self.sym = k2 * (self.p0.eps ** 2 * k2 + am) ** 2
        u0 = I.smooth_random(self.N, seed=12, amp=0.4, offset=-0.6, kmax=3)
        self.U0 = np.fft.fft2(u0)
        self.Un = np.exp(-self.sym * self.t0) * self.U0
        self.Um = np.exp(-self.sym * (self.t0 - self.kn)) * self.U0
        self.un = np.real(np.fft.ifft2(self.Un))
        self.um = np.real(np.fft.ifft2(self.Um))

    def trial(self, k1):
        """closed-form trial of size k1 from (U^n, U^{n-1}, k_n): (U~, e)"""
        a, b, c = _bdf2_abc(k1, self.kn)
        Ut = (-b * self.Un - c * self.Um) / (a + self.sym)
        w1, w2, w3 = _am3_w(k1, self.kn)
        F = lambda U: -self.sym * U
        Up = self.Un + w1 * F(Ut) + w2 * F(self.Un) + w3 * F(self.Um)
        e = np.linalg.norm(Ut - Up) / np.linalg.norm(Up)
        return np.real(np.fft.ifft2(Ut)), float(e)

    def stepper(self, **kw):
        s = O.Stepper(self.N, L, O.params(well=1, eta1=0.0, eta2=0.0, **kw))
        s.set_history(self.un, self.um, self.kn)
        return s


def _proposal(sigma, e, k, k_min=1e-9, k_max=np.inf, cap=False):
    kk = RHO_S * (sigma / e) ** (1.0 / 3.0) * k  # A_dp
    if cap:
        kk = min(kk, (1 + math.sqrt(2)) * k)
    return max(k_min, min(kk, k_max))


def test_controller_accepts_below_sigma_and_proposes_a_dp():
    lp = _Linear()
    ut, e = lp.trial(lp.kn)  # Step 0: the first trial repeats k_n
    assert 1e-9 < e < 1e-3
    sigma = 10 * e
    s = lp.stepper()
    t0 = s.t
    assert s.adaptive_begin("imex", sigma, 1.0) == 0
    assert s.adaptive_trial() == 0
    assert s.last_k == lp.kn
    assert s.last_e == pytest.approx(e, rel=1e-8)
    assert s.last_accepted and s.counts()["steps"] == 1 and s.counts()["rejects"] == 0
    assert s.t == t0 + lp.kn and s.kn == lp.kn
    assert np.abs(s.state() - ut).max() < 1e-12 * np.abs(ut).max()
    assert np.array_equal(s.prev(), lp.un)
    assert s.next_k == pytest.approx(_proposal(sigma, s.last_e, lp.kn), rel=1e-14)
    # 10^(1/3) * 0.9 * k: neither exponent 1/2 nor rho_s = 1 gives this
    assert s.next_k == pytest.approx(0.9 * 10 ** (1 / 3) * lp.kn, rel=1e-8)


def test_controller_rejects_above_sigma_and_retries_at_the_proposal():
    lp = _Linear()
    _, e = lp.trial(lp.kn)
    sigma = e / 10
    s = lp.stepper()
    assert s.adaptive_begin("imex", sigma, 1.0) == 0
    assert s.adaptive_trial() == 0
    assert not s.last_accepted and s.counts()["rejects"] == 1 and s.counts()["steps"] == 0
    assert s.t == 0.0 and s.kn == lp.kn  # time and history unchanged
    assert np.array_equal(s.state(), lp.un) and np.array_equal(s.prev(), lp.um)
    k2 = _proposal(sigma, s.last_e, lp.kn)
    assert k2 == pytest.approx(0.9 * 0.1 ** (1 / 3) * lp.kn, rel=1e-8)
    assert s.next_k == pytest.approx(k2, rel=1e-14)
    # Step 4 "Goto Step 1": the retry uses the proposal from the same history
    assert s.adaptive_trial() == 0
    assert s.last_k == pytest.approx(k2, rel=1e-14)
    ut2, e2 = lp.trial(s.last_k)
    assert s.last_e == pytest.approx(e2, rel=1e-8)
    assert s.last_accepted == (e2 <= sigma)
    if s.last_accepted:
        assert np.abs(s.state() - ut2).max() < 1e-12 * np.abs(ut2).max()
        assert s.t == s.last_k


def test_controller_accepts_any_error_at_k_min():
    lp = _Linear()
    _, e = lp.trial(lp.kn)
    s = lp.stepper(k_min=lp.kn)  # the trial size is k_min
    assert s.adaptive_begin("imex", e / 100, 1.0) == 0
    assert s.adaptive_trial() == 0
    assert s.last_accepted and s.counts()["rejects"] == 0
    assert s.t == lp.kn
    # the proposal 0.9 (1/100)^(1/3) k is below k_min: clamped
    assert s.next_k == lp.kn


def test_controller_clips_the_last_trial_to_t_final():
    lp = _Linear()
    tf = 0.4 * lp.kn
    ut, e = lp.trial(tf)
    s = lp.stepper()
    assert s.adaptive_begin("imex", 1e3 * e, tf) == 0
    assert s.adaptive_trial() == 0
    assert s.last_k == pytest.approx(tf, rel=1e-15) and s.last_accepted
    assert s.t == pytest.approx(tf, rel=1e-15)
    assert s.last_e == pytest.approx(e, rel=1e-8)
    assert np.abs(s.state() - ut).max() < 1e-12 * np.abs(ut).max()
    assert s.adaptive_trial() == 2  # t_final reached: no further trial


@pytest.mark.parametrize("cap", [0, 1])
def test_controller_zero_stability_cap_and_k_max(cap):
    lp = _Linear()
    _, e = lp.trial(lp.kn)
    sigma = 1e3 * e  # A_dp = 9 k without the cap
    s = lp.stepper(zero_stab_cap=cap)
    assert s.adaptive_begin("imex", sigma, 1.0) == 0
    assert s.adaptive_trial() == 0 and s.last_accepted
    want = (1 + math.sqrt(2)) * lp.kn if cap else 9.0 * lp.kn
    assert s.next_k == pytest.approx(want, rel=1e-8)
    assert s.next_k == pytest.approx(_proposal(sigma, s.last_e, lp.kn, cap=bool(cap)), rel=1e-14)
    s2 = lp.stepper(zero_stab_cap=cap, k_max=1.5 * lp.kn)
    assert s2.adaptive_begin("imex", sigma, 1.0) == 0
    assert s2.adaptive_trial() == 0
    assert s2.next_k == 1.5 * lp.kn


def test_controller_run_is_a_sequence_of_trials():
    # orc_run_adaptive is orc_adaptive_begin plus orc_adaptive_trial until t_final
    # (bit for bit), and a resumed run's first trial is the last proposal of the run
    # before it (reading: the run of Sec. 3.2 split over calls continues at Step 1)
    lp = _Linear()
    _, e = lp.trial(lp.kn)
    sigma, tf = 3 * e, 0.05
    a = lp.stepper()
    assert a.run_adaptive("imex", sigma, tf) == 0
    c = lp.stepper()
    assert c.adaptive_begin("imex", sigma, tf) == 0
    n = 0
    while n < 100000 and c.adaptive_trial() == 0:
        n += 1
    assert n == a.counts()["attempts"] and a.counts()["steps"] > 5
    assert np.array_equal(c.state(), a.state()) and c.t == a.t
    assert c.counts()["steps"] == a.counts()["steps"]
    b = lp.stepper()
    assert b.run_adaptive("imex", sigma, 0.01) == 0
    nk = b.next_k
    assert b.adaptive_begin("imex", sigma, tf) == 0 and b.adaptive_trial() == 0
    assert b.last_k == nk


@pytest.mark.parametrize("scheme", ["imex", "sav", "psd"])
def test_adaptive_trial_from_the_extrapolation_is_the_plain_trial(scheme):
    # a trial of an adaptive run given eq. (Richardson) from outside is the plain trial,
    # bit for bit (state, error estimate, decision, next size); ETD takes no u*
    N, kn = 32, 1e-4
    um, un = _two_level_state(N)
    out = []
    for given in (False, True):
        s = O.Stepper(N, L, O.params(k_max=0.05 if scheme == "psd" else np.inf))
        s.set_history(un, um, kn)
        assert s.adaptive_begin(scheme, 1e-5, 1.0) == 0
        for _ in range(3):
            k = s.next_k
            ustar = s.state() + (k / s.kn) * (s.state() - s.prev())
            rc = s.adaptive_trial_from(ustar) if given else s.adaptive_trial()
            assert rc == 0
        out.append((s.state(), s.last_e, s.next_k, s.counts()))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]
    s = O.Stepper(N, L, O.params())
    s.set_history(un, um, kn)
    s.adaptive_begin("etd", 1e-5, 1.0)
    assert s.adaptive_trial_from(un) == -2
