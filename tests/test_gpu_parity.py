"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 1e-10 relative L2 per step (1e-12 for one step from identical
history), mixed precision 3e-5 relative L2 per step (single-precision transforms
of fields with ~1e2 dynamic range in the symbols), transforms 1e-13 (FP64) and
2e-6 (FP32) relative to the field norm.
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
DEV = torch.device("cuda:0")


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
    p = fch.params_default(q, **kw)
    if p.zeta <= 0:
        p.zeta = 1.1 if q < 0.35 else 1.8
    if p.D0 <= 0:
        p.D0 = 170.0
    return p


# --------------------------------------------------------------------------- transforms
@pytest.mark.parametrize("n", [16, 32, 64, 128, 256])
@pytest.mark.parametrize("prec", [0, 1])
def test_fft_r2c_c2r_vs_oracle(n, prec):
    batch = 3  # odd: the last pair carries one field
    rng = np.random.default_rng(n + prec)
    x = rng.standard_normal((batch, n, n))
    dt = torch.float64 if prec == 0 else torch.float32
    cdt = torch.complex128 if prec == 0 else torch.complex64
    xt = torch.tensor(x, dtype=dt, device=DEV)
    X = torch.empty((batch, n // 2 + 1, n), dtype=cdt, device=DEV)
    plan = fch.FFTPlan(n, prec)
    plan.r2c(xt, X)
    back = torch.empty_like(xt)
    plan.c2r(X, back)
    torch.cuda.synchronize()
    Xh = X.cpu().numpy()
    tol = 1e-13 if prec == 0 else 2e-6
    for b in range(batch):
        ref = O.fft2(x[b], -1)[:, : n // 2 + 1].T  # kx-major half spectrum
        assert np.abs(Xh[b] - ref).max() <= tol * np.abs(ref).max() * math.log2(n)
    assert np.abs(back.cpu().numpy() - x).max() <= tol * 10 * np.abs(x).max()


@pytest.mark.parametrize("n,prec,batch", [(64, 1, 259), (128, 0, 131), (1024, 1, 19), (1024, 0, 11)])
def test_fft_batched_launches_match_single_fields(n, prec, batch):
    # a batch runs as launches of many field pairs (up to a 64 MiB work array each)
    # plus an odd last field: every pair must come out exactly as when transformed
    # alone (fields 2j, 2j+1 share one complex transform, so the pair is the unit),
    # and match the oracle
    rng = np.random.default_rng(n + batch)
    x = rng.standard_normal((batch, n, n))
    dt = torch.float64 if prec == 0 else torch.float32
    cdt = torch.complex128 if prec == 0 else torch.complex64
    xt = torch.tensor(x, dtype=dt, device=DEV)
    X = torch.empty((batch, n // 2 + 1, n), dtype=cdt, device=DEV)
    plan = fch.FFTPlan(n, prec)
    plan.r2c(xt, X)
    back = torch.empty_like(xt)
    plan.c2r(X, back)
    plan.status()
    for b in sorted({0, 2 * (batch // 4), batch - 3, batch - 1}):
        m = 1 if b == batch - 1 else 2
        X1 = torch.empty((m, n // 2 + 1, n), dtype=cdt, device=DEV)
        b1 = torch.empty((m, n, n), dtype=dt, device=DEV)
        plan.r2c(xt[b:b + m], X1)
        plan.c2r(X[b:b + m], b1)
        torch.cuda.synchronize()
        assert torch.equal(X1, X[b:b + m]), b
        assert torch.equal(b1, back[b:b + m]), b
        if n <= 128:
            for f in range(b, b + m):
                ref = O.fft2(x[f], -1)[:, : n // 2 + 1].T
                tol = 1e-13 if prec == 0 else 2e-6
                assert np.abs(X[f].cpu().numpy() - ref).max() <= tol * np.abs(ref).max() * math.log2(n)
    tol = 1e-12 if prec == 0 else 3e-5
    assert (back - xt).abs().max().item() <= tol * xt.abs().max().item()


@pytest.mark.parametrize("n,prec", [(1024, 0), (2048, 0), (1024, 1), (2048, 1)])
def test_fft_full_size_sampled_outputs(n, prec):
    # three fields: a pair (the Hermitian split into both half spectra) and an odd one
    rng = np.random.default_rng(7)
    x = rng.standard_normal((3, n, n))
    dt = torch.float64 if prec == 0 else torch.float32
    cdt = torch.complex128 if prec == 0 else torch.complex64
    xt = torch.tensor(x, dtype=dt, device=DEV)
    X = torch.empty((3, n // 2 + 1, n), dtype=cdt, device=DEV)
    plan = fch.FFTPlan(n, prec)
    plan.r2c(xt, X)
    plan.status()
    Xh = X.cpu().numpy()
    idx = np.arange(n)
    scale = math.sqrt(n * n)  # typical |X| of unit white noise
    tol = 1e-12 if prec == 0 else 3e-6
    for f in range(3):
        for kx, ky in [(0, 0), (1, 0), (0, 1), (n // 2, 0), (n // 2, n // 2), (3, n - 5),
                       (n // 2 - 1, 17), (200, 999 % n), (2, 3), (n // 2 - 2, n - 1)]:
            ex = np.exp(-2j * np.pi * kx * idx / n)
            ey = np.exp(-2j * np.pi * ky * idx / n)
            ref = ey @ x[f] @ ex  # direct DFT of one output
            assert abs(Xh[f, kx, ky] - ref) <= tol * scale * math.log2(n), (f, kx, ky)
    back = torch.empty_like(xt)
    plan.c2r(X, back)
    plan.status()
    assert np.abs(back.cpu().numpy() - x).max() <= (1e-12 if prec == 0 else 3e-5)


def test_fft_fp32_1024_staged_inverse_columns_match_the_plain_kernel():
    # At N = 1024 in single precision a plan's inverse column pass fetches the half
    # spectra by bulk copy when they are 16-byte aligned; spectra one complex64 off
    # that alignment take the plain shared-memory kernel. Both run the same
    # arithmetic: the fields agree bit for bit (the pairs of a multi-pair launch and
    # the odd last field), and the plan reports no device-side timeout.
    n, batch = 1024, 5
    rng = np.random.default_rng(11)
    x = torch.tensor(rng.standard_normal((batch, n, n)), dtype=torch.float32, device=DEV)
    plan = fch.FFTPlan(n, 1)
    X = torch.empty((batch, n // 2 + 1, n), dtype=torch.complex64, device=DEV)
    plan.r2c(x, X)
    store = torch.empty(batch * (n // 2 + 1) * n + 2, dtype=torch.complex64, device=DEV)
    Xu = store[1:1 + batch * (n // 2 + 1) * n].view(batch, n // 2 + 1, n)
    Xu.copy_(X)
    assert Xu.data_ptr() % 16 == 8
    ya, yu = torch.empty_like(x), torch.empty_like(x)
    plan.c2r(X, ya)
    plan.c2r(Xu, yu)
    plan.status()
    assert torch.equal(ya, yu)
    assert (ya - x).abs().max().item() <= 3e-5 * x.abs().max().item()
    plan.close()


# --------------------------------------------------------------------------- F(u)
@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("q", [0.0, 0.5])
def test_rhs_vs_oracle(q, prec):
    n = 64
    p = lib_params(q, prec=prec)
    u = I.circle_bilayer(n, noise=1e-2)
    with fch.Context(n, p) as ctx:
        ut = torch.tensor(u, device=DEV)
        F = torch.empty_like(ut)
        torch.cuda.synchronize()  # the context runs on its own stream
        ctx.rhs_device(ut, F)
        ctx.synchronize()
        ref = O.rhs(oparams(p), u, L)
        assert rel(F.cpu().numpy(), ref) < 1e-11


# --------------------------------------------------------------------------- state io, energy, mass
def test_state_roundtrip_energy_mass():
    n = 128
    p = lib_params(0.2)
    u = I.circle_bilayer(n)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u)
        assert np.abs(ctx.get_state() - u).max() < 1e-13
        op = oparams(p)
        assert ctx.energy() == pytest.approx(O.energy(op, u, L), rel=1e-11)
        assert ctx.mass() == pytest.approx(O.mass(u, L), rel=1e-13)
        t = torch.tensor(u, device=DEV, dtype=torch.float32)
        torch.cuda.synchronize()  # the context runs on its own stream
        ctx.set_state_device(t)
        out = torch.empty((n, n), device=DEV, dtype=torch.float64)
        ctx.get_state_device(out)
        ctx.synchronize()
        assert np.abs(out.cpu().numpy() - t.double().cpu().numpy()).max() < 1e-13


# --------------------------------------------------------------------------- fixed steps
@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("scheme", ["imex", "sav", "psd", "etd"])
def test_fixed_steps_fp64_vs_oracle(scheme, prec):
    # FP64 and double-float (FP32X2) modes, 1e-10 relative L2 per step
    n = 64
    p = lib_params(0.0, psd_itol=1e-12, prec=prec)
    u0 = I.circle_bilayer(n, noise=1e-3)
    s = O.Stepper(n, L, oparams(p))
    s.set_state(u0)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        for k in range(6):
            dt = 1e-3 if k < 4 else 2e-3
            s.step(scheme, dt)
            ctx.step(scheme, dt)
            got = ctx.get_state()
            assert rel(got, s.state()) < 1e-10, (k, rel(got, s.state()))
        if scheme == "sav":
            rn, rm = ctx.sav_r()
            assert rn == pytest.approx(s.r(0), rel=1e-11) and rm == pytest.approx(s.r(1), rel=1e-11)
        if scheme == "psd":
            assert ctx.stats()["last_psd_iter"] == s.counts()["last_psd_iter"]


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("scheme", ["imex", "sav", "psd", "etd"])
def test_one_step_from_identical_history(scheme, prec):
    n = 32
    p = lib_params(0.2, psd_itol=1e-13, prec=prec)
    un = I.smooth_random(n, seed=3)
    um = I.smooth_random(n, seed=4, amp=0.49)
    s = O.Stepper(n, L, oparams(p))
    s.set_history(un, um, 1e-3)
    s.step(scheme, 1.5e-3)
    with fch.Context(n, p) as ctx:
        ctx.set_history(un, um, 1e-3)
        ctx.step(scheme, 1.5e-3)
        assert rel(ctx.get_state(), s.state()) < 1e-12


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("scheme", ["imex", "sav", "etd", "psd"])
def test_run_fixed_equals_single_steps(scheme, prec):
    # graph-replayed fixed steps launch the same kernels as fch_step calls
    n = 64
    p = lib_params(0.0, prec=prec)
    u0 = I.circle_bilayer(n, noise=1e-3)
    with fch.Context(n, p) as a, fch.Context(n, p) as b:
        a.set_state(u0)
        b.set_state(u0)
        for _ in range(12):
            a.step(scheme, 2e-4)
        b.run_fixed(scheme, 2e-4, 12)
        assert np.array_equal(a.get_state(), b.get_state())
        assert a.stats()["n_steps"] == b.stats()["n_steps"] == 12
        b.run_fixed(scheme, 1e-4, 3)  # another step size: a new graph
        for _ in range(3):
            a.step(scheme, 1e-4)
        assert np.array_equal(a.get_state(), b.get_state())


def test_imex_128_fixed_dt_400_steps():
    # the 128^2 fixed-step workload: circle of radius 2, d = 0.2, noise 1e-3 (seed 1)
    n = 128
    p = lib_params(0.0)
    u0 = I.circle_bilayer(n)
    s = O.Stepper(n, L, oparams(p))
    s.set_state(u0)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        for k in range(400):
            s.step("imex", 1e-3)
            ctx.step("imex", 1e-3)
            if k % 50 == 0 or k == 399:
                assert rel(ctx.get_state(), s.state()) < 1e-10, k
        assert ctx.mass() == pytest.approx(O.mass(u0, L), rel=1e-12)


@pytest.mark.parametrize("scheme", ["imex", "etd"])
def test_fixed_steps_mixed_precision(scheme):
    n = 128
    p = lib_params(0.0, prec=1)
    u0 = I.circle_bilayer(n)
    s = O.Stepper(n, L, oparams(p))
    s.set_state(u0)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        for k in range(10):
            s.step(scheme, 1e-3)
            ctx.step(scheme, 1e-3)
        assert rel(ctx.get_state(), s.state()) < 3e-5


# --------------------------------------------------------------------------- adaptive
@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("scheme", ["imex", "sav", "etd", "psd"])
def test_adaptive_vs_oracle(scheme, prec):
    n = 64
    p = lib_params(0.0, zero_stab_cap=1, k_max=0.05 if scheme == "psd" else float("inf"), prec=prec)
    p.sync_every = 4
    u0 = I.circle_bilayer(n, noise=1e-3)
    tf = 0.01
    s = O.Stepper(n, L, oparams(p))
    s.set_state(u0)
    rc = s.run_adaptive(scheme, 1e-5, tf)
    assert rc == 0
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        st = ctx.run_adaptive(scheme, 1e-5, tf)
        c = s.counts()
        assert st["n_steps"] == c["steps"] and st["n_rejects"] == c["rejects"]
        assert st["t"] == pytest.approx(tf, rel=1e-14)
        assert rel(ctx.get_state(), s.state()) < 1e-9


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("scheme", ["imex", "sav"])
def test_long_adaptive_run_conserves_mass(scheme, prec):
    # thousands of adaptive steps: the mean mode (the mass) may only carry rounding
    # of no systematic sign; a per-step bias of 2^-48 would add up to ~1e-11
    n = 64
    p = lib_params(0.0, zero_stab_cap=1, prec=prec)
    u0 = I.paper_initial_data(n, 0.5)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        m0 = ctx.mass()
        st = ctx.run_adaptive(scheme, 1e-6, 2.0)
        assert st["n_steps"] > 1000
        assert abs(ctx.mass() - m0) / m0 < (1e-12 if prec == 0 else 3e-12)


def test_adaptive_attempt_budget_and_resume():
    n = 32
    p = lib_params(0.0)
    u0 = I.circle_bilayer(n)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        st = ctx.run_adaptive("imex", 1e-5, 1.0, max_attempts=7, raise_on_timeout=False)
        assert st["n_attempts"] == 7  # the backward-Euler start + 6 trials
        st2 = ctx.run_adaptive("imex", 1e-5, st["t"] + 1e-3)
        assert st2["t"] == pytest.approx(st["t"] + 1e-3, rel=1e-13)


def test_errors_are_reported():
    n = 32
    p = lib_params(0.0, psd_max_iter=2, psd_itol=1e-14)
    with fch.Context(n, p) as ctx:
        with pytest.raises(fch.FchError) as e:
            ctx.step("imex", 1e-3)
        assert e.value.status == 7  # no state yet
        ctx.set_state(I.circle_bilayer(n))
        with pytest.raises(fch.FchError) as e:
            ctx.step("psd", 1e-3)
        assert e.value.status == 4  # PSD did not converge in 2 iterations
        with pytest.raises(fch.FchError) as e:
            ctx.step("imex", 1e-3)
        assert e.value.status == 7  # failed context until a new state is set
        ctx.set_state(I.circle_bilayer(n))
        ctx.step("imex", 1e-3)
        bad = I.circle_bilayer(n)
        bad[3, 4] = np.nan
        with pytest.raises(fch.FchError) as e:
            ctx.set_state(bad)  # the SAV energy E1(u^0) is not finite
        assert e.value.status == 5
        with pytest.raises(fch.FchError) as e:
            ctx.run_adaptive("imex", 1e-5, 1e-3)
        assert e.value.status == 7



@pytest.mark.parametrize("prec", [0, 2])
def test_psd_device_loop_matches_host_loop(prec):
    # captured PSD trials and steps iterate in a conditional while node that reads
    # the stopping test on the device; with per-pass timing on, the same runs launch
    # pass by pass and the host reads the test: identical fields and counts
    n = 64
    p = lib_params(0.0, zero_stab_cap=1, prec=prec)
    u0 = I.circle_bilayer(n, noise=1e-3)
    out = []
    for timing in (True, False):
        with fch.Context(n, p) as ctx:
            ctx.pass_timing(timing)
            ctx.set_state(u0)
            st = ctx.run_adaptive("psd", 1e-5, 2e-3)
            ua = ctx.get_state()
            ctx.set_state(u0)
            ctx.run_fixed("psd", 2e-5, 6)
            out.append((st, ua, ctx.get_state(), ctx.stats()))
            assert ctx.debug_graphs()["psd"] == ((0, 0) if timing else (1, 1))
    (s0, a0, f0, c0), (s1, a1, f1, c1) = out
    for k in ("n_steps", "n_rejects", "n_psd_iter", "last_psd_iter"):
        assert s0[k] == s1[k], k
        assert c0[k] == c1[k], k
    assert s1["n_steps"] > 10 and s1["t"] == pytest.approx(2e-3, rel=1e-13)
    assert c1["n_steps"] == 6 and c1["n_psd_iter"] > 6
    assert np.array_equal(a0, a1) and np.array_equal(f0, f1)


def test_psd_nonconvergence_inside_captured_trials():
    # psd_max_iter = 4: the start and the first trials converge in one or two
    # iterations, a later (replayed) trial does not; the device loop stops there and
    # the run reports FCH_ENOCONV with the time reached
    n = 32
    p = lib_params(0.0, zero_stab_cap=1, psd_max_iter=4)
    p.eta1 = 0.1
    with fch.Context(n, p) as ctx:
        ctx.set_state(I.multimode_bilayer(n, seed=100))
        with pytest.raises(fch.FchError) as e:
            ctx.run_adaptive("psd", 1e-5, 2e-3)
        assert e.value.status == 4
        st = ctx.stats()
        assert st["n_steps"] >= 5 and st["t"] < 2e-3 and st["last_psd_iter"] == 4
        with pytest.raises(fch.FchError) as e:
            ctx.run_adaptive("psd", 1e-5, 2e-3)
        assert e.value.status == 7


# --------------------------------------------------------------------------- full size (1024^2, mixed)
def test_mixed_1024_fixed_steps_vs_oracle():
    # the benchmark grid in single precision (warp transforms at N = 1024): a state
    # round trip and fixed IMEX steps, whose implicit solve damps the single-
    # precision rounding of the transforms, against the FP64 oracle
    n = 1024
    p = lib_params(0.0, eta2=0.15, prec=1)
    u0 = I.random_network(n, d=0.75, seed=3)
    s = O.Stepper(n, L, oparams(p))
    s.set_state(u0)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        assert rel(ctx.get_state(), u0) < 2e-5
        for _ in range(2):
            s.step("imex", 1e-6)
            ctx.step("imex", 1e-6)
        assert rel(ctx.get_state(), s.state()) < 3e-5
        assert ctx.energy() == pytest.approx(O.energy(oparams(p), ctx.get_state(), L), rel=1e-4)


def test_mixed_1024_rhs_noise_floor():
    # F(u) = Lap mu(u) carries eps^4 Lap^3 u and eps^2 Lap^2 W'(u): single-precision
    # rounding of the transforms is amplified at the top of the spectrum. The warp
    # and Stockham single-precision paths agree with each other to that noise level
    # and both differ from the FP64 path by a few percent at 1024^2 (the reason the
    # adaptive estimator is not run in single precision).
    n = 1024
    u = I.random_network(n, d=0.75, seed=3)
    ut = torch.tensor(u, device=DEV)
    torch.cuda.synchronize()
    F = {}
    for name, prec, path in (("f64", 0, 0), ("warp", 1, 2), ("stockham", 1, 1)):
        with fch.Context(n, lib_params(0.0, eta2=0.15, prec=prec, fft_path=path)) as ctx:
            src = ut if prec == 0 else ut.float()
            out = torch.empty_like(src)
            torch.cuda.synchronize()
            ctx.rhs_device(src, out)
            ctx.synchronize()
            F[name] = out.double().cpu().numpy()
    # FP64 path against the oracle; F carries six derivatives, so rounding at 1e-16
    # is amplified about 1e6 at the top of a 1024^2 spectrum
    ref = O.rhs(oparams(lib_params(0.0, eta2=0.15)), u, L)
    assert rel(F["f64"], ref) < 1e-9
    assert rel(F["warp"], F["f64"]) < 0.2 and rel(F["stockham"], F["f64"]) < 0.2
    # the low modes, where the solution lives, agree to single precision
    lo = lambda f: np.fft.rfft2(f)[:64, :64]
    assert rel(lo(F["warp"]), lo(F["f64"])) < 1e-2
    assert rel(lo(F["stockham"]), lo(F["f64"])) < 1e-2


def test_mixed_1024_graph_replay_matches_eager():
    # trials replayed from the captured CUDA graph give the same trajectory as
    # trials launched kernel by kernel (per-pass timing forces eager launches)
    n = 1024
    p = lib_params(0.0, eta2=0.15, prec=1)
    u0 = I.random_network(n, d=0.75, seed=5)
    out = []
    for eager in (False, True):
        with fch.Context(n, p) as ctx:
            ctx.set_state(u0)
            ctx.pass_timing(eager)
            ctx.adaptive_begin("imex", 1e-5, 1.0)
            ctx.adaptive_enqueue(12)
            st = ctx.adaptive_end()
            out.append((st["n_steps"], st["t"], ctx.get_state()))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])


def test_fp32x2_1024_adaptive_trials_track_fp64():
    # the benchmark workload in double-float: 40 adaptive trials at 1024^2 take the
    # same accept/reject decisions and step sizes as the FP64 mode and end within
    # 1e-10 of it (the FP64 mode itself matches the oracle at smaller sizes)
    n = 1024
    u0 = I.random_network(n, d=0.75, seed=3)
    out = {}
    for prec in (0, 2):
        with fch.Context(n, lib_params(0.0, eta2=0.15, prec=prec)) as ctx:
            ctx.set_state(u0)
            st = ctx.run_adaptive("imex", 1e-5, 10.0, max_attempts=40, raise_on_timeout=False)
            out[prec] = (st, ctx.get_state())
    s0, s2 = out[0][0], out[2][0]
    assert (s0["n_steps"], s0["n_rejects"]) == (s2["n_steps"], s2["n_rejects"])
    assert s2["t"] == pytest.approx(s0["t"], rel=1e-9)
    assert rel(out[2][1], out[0][1]) < 1e-10


def test_fp32x2_1024_one_step_vs_oracle():
    n = 1024
    p = lib_params(0.0, eta2=0.15, prec=2)
    u0 = I.random_network(n, d=0.75, seed=3)
    s = O.Stepper(n, L, oparams(p))
    s.set_state(u0)
    s.step("imex", 1e-6)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        ctx.step("imex", 1e-6)
        assert rel(ctx.get_state(), s.state()) < 1e-10


@pytest.mark.parametrize("prec", [0, 2])
def test_512_fixed_steps_vs_oracle(prec):
    # the 512^2 grid of the all-schemes adaptive workload (multimode bilayer)
    n = 512
    p = lib_params(0.0, prec=prec)
    u0 = I.multimode_bilayer(n)
    s = O.Stepper(n, L, oparams(p))
    s.set_state(u0)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        for dt in (1e-4, 1e-4, 2e-4):
            s.step("imex", dt)
            ctx.step("imex", dt)
            assert rel(ctx.get_state(), s.state()) < 1e-10


def test_paper_initial_data_adaptive_vs_oracle():
    # the super-critical benchmark's own initial data (Sec. 2.3) at 64^2, adaptive IMEX
    n = 64
    p = lib_params(0.0, zero_stab_cap=1, prec=2)
    u0 = I.paper_initial_data(n, 0.5)
    s = O.Stepper(n, L, oparams(p))
    s.set_state(u0)
    assert s.run_adaptive("imex", 1e-5, 0.02) == 0
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        st = ctx.run_adaptive("imex", 1e-5, 0.02)
        assert st["n_steps"] == s.counts()["steps"]
        assert rel(ctx.get_state(), s.state()) < 1e-9
        # 95 steps; each rounds the mean mode a few dozen times at the double-float unit
        # 2^-48 = 3.6e-15 (the FP64 oracle drifts 9.5e-14 over the same run, 2^-53 units)
        assert ctx.mass() == pytest.approx(O.mass(u0, L), rel=1e-11)


def test_psd_iteration_graph_equals_eager_launches():
    # the PSD iterations replay a captured chunk after the first solve; with per-pass
    # timing on every pass launches eagerly: same iterations, same result
    n = 64
    u0 = I.circle_bilayer(n, noise=1e-3)
    out = []
    for timing in (False, True):
        with fch.Context(n, lib_params(0.0)) as ctx:
            ctx.set_state(u0)
            ctx.pass_timing(timing)
            st = ctx.run_adaptive("psd", 1e-5, 5e-3)
            for _ in range(3):
                ctx.step("psd", 1e-4)
            out.append((st, ctx.stats(), ctx.get_state()))
    (a, a2, ua), (b, b2, ub) = out
    assert a["n_psd_iter"] == b["n_psd_iter"] and a["n_steps"] == b["n_steps"] and a["n_fft"] == b["n_fft"]
    assert a2["n_psd_iter"] == b2["n_psd_iter"]
    assert np.array_equal(ua, ub)


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("scheme", ["imex", "sav"])
def test_step_from_a_given_extrapolation_matches_oracle(scheme, prec):
    # fch_step_from: the IMEX / SAV step with the caller's u*, against the oracle's
    # step with the same u*; with u* = eq. (Richardson) it is the plain step
    n = 64
    p = lib_params(0.2, prec=prec)
    un = I.smooth_random(n, seed=3)
    um = I.smooth_random(n, seed=4, amp=0.49)
    kn, dt = 1e-3, 1.5e-3
    extrap = un + (dt / kn) * (un - um)
    given = extrap + 0.05 * I.smooth_random(n, seed=9)
    for ustar in (extrap, given):
        s = O.Stepper(n, L, oparams(p))
        s.set_history(un, um, kn)
        s.step_from(scheme, dt, ustar)
        with fch.Context(n, p) as ctx:
            ctx.set_history(un, um, kn)
            ctx.step_from(scheme, dt, torch.tensor(ustar, device=DEV))
            assert rel(ctx.get_state(), s.state()) < 1e-12
    with fch.Context(n, p) as ctx:
        ctx.set_history(un, um, kn)
        ctx.step_from(scheme, dt, torch.tensor(extrap, device=DEV, dtype=torch.float32))
        s = O.Stepper(n, L, oparams(p))
        s.set_history(un, um, kn)
        s.step(scheme, dt)
        assert rel(ctx.get_state(), s.state()) < 1e-6  # u* rounded to float
        with pytest.raises(fch.FchError):
            ctx.step_from("psd", dt, torch.tensor(extrap, device=DEV))
