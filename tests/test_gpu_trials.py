"""GPU parity trial by trial, and on the kernels the large grids run.

Every adaptive trial of the CUDA path (through the C ABI) is compared with the
same trial of the FP64 oracle (Sec. 3.2, Steps 1-4): the trial size, the error
estimate e, the accept/reject decision and, after every trial, the state u^n at
1e-10 relative L2. The fixed-step cases run the compile-time kernels of the
512^2, 1024^2 and 2048^2 grids with the default tiles (at 1024^2 in FP64 and
FP32X2: two-block-cluster column passes, direct-start row passes, programmatic
dependent launch), which the 64^2 tests do not reach.

Tolerance of e: the states agree to 1e-10 relative, so ||u~ - u_p|| and ||u_p||
each move by at most ~2e-10 ||u||; |e_gpu - e_oracle| <= 5e-10 absolute. The
next trial size A_dp ~ e^(-1/3) then agrees to |de| / (3 e) relative. A decision
is compared when |e - sigma_tol| exceeds that bound (otherwise it is flagged as
decision-sensitive and skipped, as the two sides may round differently).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2006_04784_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2006_04784_gb300 import build as B  # noqa: E402

B.build()
from paper_2006_04784_gb300 import fch  # noqa: E402

L = 4 * math.pi
E_TOL = 5e-10


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oparams(fp, **kw):
    """oracle parameters equal to the library's effective fch_params"""
    d = dict(eps=fp.eps, q=fp.q, gamma=fp.gamma, b_minus=fp.b_minus, b_plus=fp.b_plus,
             eta1=fp.eta1, eta2=fp.eta2, beta1=fp.beta1, beta2=fp.beta2, zeta=fp.zeta, D0=fp.D0,
             kappa0=fp.kappa0, kappa2=fp.kappa2, rho_s=fp.rho_s, k_min=fp.k_min, k_max=fp.k_max,
             zero_stab_cap=fp.zero_stab_cap, well=0, psd_nu=fp.psd_nu, psd_itol=fp.psd_itol,
             psd_lambda=fp.psd_lambda, psd_max_iter=fp.psd_max_iter)
    d.update(kw)
    return O.params(**d)


def lib_params(q=0.0, **kw):
    """the library's parameters with explicit SAV constants zeta and D0 (the library
    computes them at fch_create when 0; the oracle gets the same explicit values)"""
    p = fch.params_default(q, **kw)
    p.zeta = 1.1 if q < 0.35 else 1.8
    p.D0 = 170.0
    return p


_CACHE = {}


def cached(key, make):
    """oracle results shared by the precisions of one case (computed once)"""
    if key not in _CACHE:
        _CACHE[key] = make()
    return _CACHE[key]


def oracle_trials(s, scheme, sigma, t_final, n_trials):
    """run the oracle's adaptive algorithm trial by trial; one record per trial"""
    assert s.adaptive_begin(scheme, sigma, t_final) == 0
    recs = [dict(state=s.state(), next_k=s.next_k)]
    for _ in range(n_trials):
        rc = s.adaptive_trial()
        if rc == 2:
            break
        assert rc == 0
        recs.append(dict(k=s.last_k, e=s.last_e, accepted=s.last_accepted, t=s.t,
                         state=s.state(), next_k=s.next_k))
    recs.append(dict(counts=s.counts()))
    return recs


def compare_trials(ctx, recs, scheme, sigma, t_final, state_tol=1e-10):
    """replay the oracle's trials on the GPU from the same state; compare each one.
    Returns the (accepted, rejected) counts seen."""
    ctx.adaptive_begin(scheme, sigma, t_final)
    assert rel(ctx.get_state(), recs[0]["state"]) < state_tol
    seen = [0, 0]
    trials = recs[1:-1]
    for i, r in enumerate(trials):
        k_gpu, _, done = ctx.adaptive_trial_info()
        assert not done, i
        assert k_gpu == pytest.approx(r["k"], rel=1e-9), i
        before = ctx.stats()
        ctx.adaptive_enqueue(1)
        st = ctx.stats()
        e_gpu, e_orc = st["e_last"], r["e"]
        assert abs(e_gpu - e_orc) <= E_TOL, (i, e_gpu, e_orc)
        acc_gpu = st["n_steps"] == before["n_steps"] + 1
        if abs(e_orc - sigma) > 2 * E_TOL:
            assert acc_gpu == r["accepted"], (i, e_gpu, e_orc, sigma)
        else:  # decision-sensitive: the GPU's decision is not compared
            assert acc_gpu or st["n_rejects"] == before["n_rejects"] + 1
        seen[0 if acc_gpu else 1] += 1
        assert st["t"] == pytest.approx(r["t"], rel=1e-9, abs=1e-15), i
        err = rel(ctx.get_state(), r["state"])
        assert err < state_tol, (i, err)
        k_next, _, done = ctx.adaptive_trial_info()
        if not done:  # at t_final the run ends: no next trial; the last one is clipped to it
            want = min(r["next_k"], t_final - r["t"])
            assert k_next == pytest.approx(want, rel=E_TOL / (3 * e_orc) + 1e-12), i
    ctx.adaptive_end()
    return seen


def network(n, seed=3):
    return cached(("network", n, seed), lambda: I.random_network(n, d=0.75, seed=seed))


# --------------------------------------------------------------------------- the benchmark's chain
@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("sigma", [1e-5, 3e-6])
def test_benchmark_chain_1024_trial_by_trial(prec, sigma):
    # the benchmark's workload at 1024^2 (critical parameters, random bilayer network,
    # seed 3; default tiles) from its backward-Euler start: the first trials, each
    # accepted, growing the step from k_min
    n = 1024
    p = lib_params(0.0, eta2=0.15, prec=prec)
    u0 = network(n)

    def run():
        s = O.Stepper(n, L, oparams(p))
        s.set_state(u0)
        return oracle_trials(s, "imex", sigma, 10.0, 4)

    recs = cached(("chain", sigma), run)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        acc, rej = compare_trials(ctx, recs, "imex", sigma, 10.0)
    assert acc == 4 and rej == 0


@pytest.mark.parametrize("prec", [0, 2])
def test_1024_trials_from_a_history(prec):
    # set_history from the network (u^{n-1}) and the oracle's backward-Euler step
    # (u^n): the first trial is a full variable-step BDF2 trial of size k_n; the
    # start's transient makes the first trials fail (e ~ 1e-3 > sigma_tol) and the
    # controller retry at the A_dp proposals
    n, kn = 1024, 1e-6
    p = lib_params(0.0, eta2=0.15, prec=prec)
    um = network(n)

    def run():
        s0 = O.Stepper(n, L, oparams(p))
        s0.set_state(um)
        s0.step("imex", kn)
        un = s0.state()
        s = O.Stepper(n, L, oparams(p))
        s.set_history(un, um, kn)
        return un, oracle_trials(s, "imex", 1e-5, 10.0, 4)

    un, recs = cached("history", run)
    with fch.Context(n, p) as ctx:
        ctx.set_history(un, um, kn)
        acc, rej = compare_trials(ctx, recs, "imex", 1e-5, 10.0)
    assert rej >= 3 and acc + rej == 4


# --------------------------------------------------------------------------- 64^2, every scheme
@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("scheme", ["imex", "sav", "etd", "psd"])
def test_adaptive_64_every_trial(scheme, prec):
    # the whole adaptive run of test_adaptive_vs_oracle, compared after every trial
    n = 64
    p = lib_params(0.0, zero_stab_cap=1, prec=prec)
    if scheme == "psd":
        p.k_max = 0.05
    u0 = I.circle_bilayer(n, noise=1e-3)

    def run():
        s = O.Stepper(n, L, oparams(p))
        s.set_state(u0)
        return oracle_trials(s, scheme, 1e-5, 0.01, 100000)

    recs = cached(("64", scheme), run)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        acc, rej = compare_trials(ctx, recs, scheme, 1e-5, 0.01)
        assert ctx.stats()["t"] == pytest.approx(0.01, rel=1e-14)
    c = recs[-1]["counts"]
    assert acc == c["steps"] - 1 and rej == c["rejects"]  # the start is not a trial


# --------------------------------------------------------------------------- default kernels, large grids
def _history(n):
    def make():
        un = network(n)
        return un, un - 2e-3 * I.smooth_random(n, seed=5, amp=0.5, kmax=3, offset=0.0)
    return cached(("history", n), make)


def _oracle_step(n, scheme, p, kn, dt):
    def make():
        un, um = _history(n)
        s = O.Stepper(n, L, oparams(p))
        s.set_history(un, um, kn)
        s.step(scheme, dt)
        return s.state(), s.counts()["last_psd_iter"], s.r(0)
    return cached((n, scheme, kn, dt), make)


@pytest.mark.parametrize("n", [512, 1024])
@pytest.mark.parametrize("scheme", ["sav", "psd", "etd", "imex"])
@pytest.mark.parametrize("prec", [0, 2])
def test_fixed_step_default_kernels_vs_oracle(n, scheme, prec):
    # one variable-step BDF2 (or ETDRK2) step of every scheme on the compile-time
    # kernels of the grid with the default tiles, from identical history: 1e-12
    kn, dt = 1e-5, 1.5e-5
    p = lib_params(0.0, eta2=0.15, prec=prec, psd_itol=1e-12)
    ref, iters, r = _oracle_step(n, scheme, p, kn, dt)
    un, um = _history(n)
    with fch.Context(n, p) as ctx:
        ctx.set_history(un, um, kn)
        ctx.step(scheme, dt)
        assert rel(ctx.get_state(), ref) < 1e-12
        if scheme == "psd":
            assert ctx.stats()["last_psd_iter"] == iters
        if scheme == "sav":
            assert ctx.sav_r()[0] == pytest.approx(r, rel=1e-12)


@pytest.mark.parametrize("prec", [0, 2])
def test_imex_2048_step_vs_oracle(prec):
    # the largest grid: the backward-Euler start and one BDF2 step of IMEX
    n = 2048
    p = lib_params(0.0, eta2=0.15, prec=prec)
    u0 = network(n)

    def make():
        s = O.Stepper(n, L, oparams(p))
        s.set_state(u0)
        s.step("imex", 1e-6)
        u1 = s.state()
        s.step("imex", 1.5e-6)
        return u1, s.state()

    u1, u2 = cached("2048", make)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        ctx.step("imex", 1e-6)
        assert rel(ctx.get_state(), u1) < 1e-10
        ctx.step("imex", 1.5e-6)
        assert rel(ctx.get_state(), u2) < 1e-10


# --------------------------------------------------------------------------- given extrapolation, adaptive
@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("scheme", ["imex", "sav"])
def test_adaptive_trials_from_a_given_extrapolation(scheme, prec):
    # fch_adaptive_enqueue_from: adaptive trials whose u* is the caller's field (the
    # learned extrapolation's entry point) against the oracle's trials with the same u*:
    # eq. (Richardson) plus a smooth perturbation, from a history of a circular bilayer
    # and the oracle's backward-Euler step; the first trial fails, the next ones pass
    n, kn, sigma = 64, 1e-4, 1e-3
    p = lib_params(0.2, prec=prec)
    u0 = I.circle_bilayer(n, noise=0.0)
    pert = 1e-3 * I.smooth_random(n, seed=9, offset=0.0)

    def hist():
        s0 = O.Stepper(n, L, oparams(p))
        s0.set_state(u0)
        s0.step("imex", kn)
        return s0.state()

    un, um = cached("from_hist", hist), u0

    def run():
        s = O.Stepper(n, L, oparams(p))
        s.set_history(un, um, kn)
        assert s.adaptive_begin(scheme, sigma, 1.0) == 0
        recs = []
        for _ in range(4):
            ustar = s.state() + (s.next_k / s.kn) * (s.state() - s.prev()) + pert
            assert s.adaptive_trial_from(ustar) == 0
            recs.append(dict(ustar=ustar, k=s.last_k, e=s.last_e, accepted=s.last_accepted,
                             t=s.t, state=s.state(), next_k=s.next_k))
        return recs

    recs = cached(("from", scheme), run)
    with fch.Context(n, p) as ctx:
        ctx.set_history(un, um, kn)
        ctx.adaptive_begin(scheme, sigma, 1.0)
        for i, r in enumerate(recs):
            k_gpu, _, done = ctx.adaptive_trial_info()
            assert not done and k_gpu == pytest.approx(r["k"], rel=1e-9)
            before = ctx.stats()
            ctx.adaptive_enqueue_from(torch.tensor(r["ustar"], device=torch.device("cuda:0")))
            st = ctx.stats()
            assert abs(st["e_last"] - r["e"]) <= E_TOL, (i, st["e_last"], r["e"])
            assert (st["n_steps"] == before["n_steps"] + 1) == r["accepted"]
            assert rel(ctx.get_state(), r["state"]) < 1e-10, i
        ctx.adaptive_end()
    assert not recs[0]["accepted"] and all(r["accepted"] for r in recs[1:])
