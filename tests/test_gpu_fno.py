"""GPU: the Fourier neural operator (forward, backward, Adam) against its FP64 CPU
oracle, and the PSD step started from a given iterate."""
import math

import numpy as np
import pytest

from oracle import fno_oracle as F
from paper_2006_04784_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2006_04784_gb300 import build as B  # noqa: E402

B.build()
from paper_2006_04784_gb300 import fch  # noqa: E402

DEV = torch.device("cuda:0")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("width,layers,modes,proj,n,batch", [(8, 2, 4, 16, 32, 2), (32, 4, 16, 64, 64, 2)])
def test_fno_forward_backward_vs_oracle(width, layers, modes, proj, n, batch):
    cfg = F.Config(width=width, layers=layers, modes=modes, proj=proj)
    rng = np.random.default_rng(width + n)
    params = (F.init_params(cfg, 0) + 0.05 * rng.standard_normal(cfg.size())).astype(np.float32)
    a = rng.standard_normal((batch, 2, n, n)).astype(np.float32)
    target = rng.standard_normal((batch, n, n)).astype(np.float32)
    net = fch.FNO(width, layers, modes, proj)
    assert net.num_params == cfg.size()
    net.set_params(params)
    at = torch.tensor(a, device=DEV)
    y = torch.empty((batch, n, n), device=DEV)
    net.forward(at, y)
    loss = net.backward(torch.tensor(target, device=DEV))
    p64, a64, t64 = params.astype(np.float64), a.astype(np.float64), target.astype(np.float64)
    y_ref = F.forward(p64, a64, cfg)
    assert rel(y.cpu().numpy(), y_ref) < 2e-5
    assert loss == pytest.approx(F.loss(p64, a64, t64, cfg), rel=1e-4)
    g, g_ref = net.grads(), F.backward(p64, a64, t64, cfg)
    o = 0
    for name, sh in cfg.shapes():
        k = int(np.prod(sh))
        assert rel(g[o:o + k], g_ref[o:o + k]) < 2e-4, name
        o += k


def test_fno_bf16_weights_forward_vs_oracle():
    # BF16 weights, FP32 sums: the forward pass equals the oracle's on the weights
    # rounded to bfloat16; training refuses the bfloat16 forward pass
    cfg = F.Config(width=32, layers=4, modes=16, proj=64)
    n, batch = 64, 2
    rng = np.random.default_rng(12)
    params = (F.init_params(cfg, 0) + 0.05 * rng.standard_normal(cfg.size())).astype(np.float32)
    a = rng.standard_normal((batch, 2, n, n)).astype(np.float32)
    net = fch.FNO(32, 4, 16, 64)
    net.set_params(params)
    net.set_bf16(True)
    at = torch.tensor(a, device=DEV)
    y = torch.empty((batch, n, n), device=DEV)
    net.forward(at, y)
    a64 = a.astype(np.float64)
    y_bf = F.forward(F.bf16_round(params).astype(np.float64), a64, cfg)
    y_32 = F.forward(params.astype(np.float64), a64, cfg)
    assert rel(y.cpu().numpy(), y_bf) < 2e-5
    assert rel(y_bf, y_32) > 1e-4  # the rounding is visible, so the copy was read
    with pytest.raises(fch.FchError):
        net.backward(torch.zeros((batch, n, n), device=DEV))
    net.set_bf16(False)
    net.forward(at, y)
    assert rel(y.cpu().numpy(), y_32) < 2e-5
    net.backward(torch.zeros((batch, n, n), device=DEV))


def test_fno_training_reduces_the_loss():
    # fit a fixed smooth map (a band-limited filter of the first channel plus a
    # quadratic term) on a fixed batch: Adam on the library's gradients
    n, batch = 32, 4
    rng = np.random.default_rng(3)
    x = np.arange(n) * 2 * np.pi / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    a = np.zeros((batch, 2, n, n), dtype=np.float32)
    for b in range(batch):
        for c in range(2):
            for k in range(1, 4):
                a[b, c] += rng.standard_normal() * np.cos(k * X + rng.uniform(0, 6)) + \
                    rng.standard_normal() * np.sin(k * Y + rng.uniform(0, 6))
    target = (0.5 * np.roll(a[:, 0], 1, axis=-1) + 0.2 * a[:, 1] ** 2).astype(np.float32)
    cfg = F.Config(width=16, layers=2, modes=6, proj=32)
    net = fch.FNO(16, 2, 6, 32)
    net.set_params(F.init_params(cfg, 1).astype(np.float32))
    at, tt = torch.tensor(a, device=DEV), torch.tensor(target, device=DEV)
    y = torch.empty((batch, n, n), device=DEV)
    losses = []
    for it in range(300):
        net.forward(at, y)
        losses.append(net.backward(tt))
        net.adam(3e-3)
    assert losses[-1] < 0.1 * losses[0]


def test_psd_step_from_a_given_iterate():
    n, L = 64, 4 * math.pi
    p = fch.params_default(0.0, psd_itol=1e-12)
    p.zeta, p.D0 = 1.1, 170.0
    u0 = I.circle_bilayer(n, noise=1e-3)
    dt = 2e-4
    with fch.Context(n, p) as a, fch.Context(n, p) as b:
        for c in (a, b):
            c.set_state(u0)
            c.step("psd", dt)
        u1 = a.get_state()
        a.step("psd", dt)
        plain = a.get_state()
        it_plain = a.stats()["last_psd_iter"]
        ustar = 2 * u1 - u0  # eq. (Richardson) with equal steps
        noise = 1e-3 * np.random.default_rng(0).standard_normal((n, n))
        noise -= noise.mean()
        snap = b.get_state()
        # from u* plus a zero-mean perturbation: the same fixed point, the same mass
        b.step_psd_from(dt, torch.tensor(ustar + noise, device=DEV))
        assert rel(b.get_state(), plain) < 1e-9
        assert b.mass() == pytest.approx(a.mass(), rel=1e-12)
        # from the converged answer itself: at most two iterations
        b.set_state(u0)
        b.step("psd", dt)
        assert np.array_equal(b.get_state(), snap)
        b.step_psd_from(dt, torch.tensor(plain, device=DEV))
        assert b.stats()["last_psd_iter"] <= 2 < it_plain
        assert rel(b.get_state(), plain) < 1e-10


@pytest.fixture(scope="module")
def small_trained_net():
    # a small FNO trained on PSD trajectories at 64^2 (the library's own steps)
    from paper_2006_04784_gb300 import fno_train as T

    n = 64
    p = fch.params_default(0.0, psd_itol=1e-10)
    rng = np.random.default_rng(5)
    data = []
    for r, s in ((1.6, 1), (2.0, 2), (2.4, 3), (2.8, 4)):
        dts = T.random_steps(rng, 50, 1e-3)
        data += T.samples_from(T.psd_trajectory(n, I.circle_bilayer(n, radius=r, noise=1e-3, seed=s), dts, p), dts)
    net = fch.FNO(16, 2, 8, 32)
    net.set_params(T.init_params(net, seed=0))
    hist = T.train(net, data, 800, 8, 2e-3, DEV)
    return net, hist


def test_trained_fno_start_beats_the_extrapolation(small_trained_net):
    # on a held-out trajectory the learned start must be closer to the PSD fixed point
    # than u*, reach the same fixed point, and need no more iterations on average
    from paper_2006_04784_gb300 import fno_train as T

    net, hist = small_trained_net
    assert np.mean(hist[-20:]) < 0.2 * np.mean(hist[:20])
    n = 64
    p = fch.params_default(0.0, psd_itol=1e-10)
    dts = T.random_steps(np.random.default_rng(9), 20, 1e-3)
    u = [I.circle_bilayer(n, radius=2.2, noise=1e-3, seed=7)]
    ratios, it_p, it_f = [], [], []
    v0 = torch.empty((n, n), dtype=torch.float64, device=DEV)
    with fch.Context(n, p) as a, fch.Context(n, p) as b:
        a.set_state(u[0])
        for i, dt in enumerate(dts):
            if i >= 2:
                ustar = u[-1] + dt / dts[i - 1] * (u[-1] - u[-2])
                b.set_history(u[-1], u[-2], dts[i - 1])
                T.learned_start(b, net, v0, dt)  # on the device, from b's history
            a.step("psd", dt)
            u.append(a.get_state())
            if i >= 2:
                it_p.append(a.stats()["last_psd_iter"])
                b.step_psd_from(dt, v0)
                it_f.append(b.stats()["last_psd_iter"])
                assert rel(b.get_state(), u[-1]) < 1e-8
                assert b.mass() == pytest.approx(a.mass(), rel=1e-12)
                ratios.append(np.linalg.norm(v0.cpu().numpy() - u[-1]) / np.linalg.norm(ustar - u[-1]))
    assert np.mean(ratios) < 0.8
    assert np.mean(it_f) <= np.mean(it_p)


def test_adaptive_psd_with_learned_start(small_trained_net):
    # the adaptive PSD run of Sec. 3.2 trial by trial: started from u* and from the
    # network's v_0 (on the step sizes it was trained on), both reach t_final, agree
    # to the PSD tolerance and keep the mass to the rounding the PSD iteration's
    # mean mode carries (that of the extrapolation u*, about 1e-11 over a run)
    from paper_2006_04784_gb300 import fno_train as T

    net, _ = small_trained_net
    n = 64
    p = fch.params_default(0.0, zero_stab_cap=1)
    u0 = I.circle_bilayer(n, radius=2.2, noise=1e-3, seed=7)
    out = {}
    for name, use in (("plain", None), ("learned", net)):
        with fch.Context(n, p) as ctx:
            ctx.set_state(u0)
            m0 = ctx.mass()
            st, trials, learned = T.run_adaptive_psd(ctx, 1e-5, 2e-2, DEV, net=use, k_range=(5e-4, 2e-3))
            assert st["t"] == pytest.approx(2e-2, rel=1e-12) and trials > 5
            assert abs(ctx.mass() - m0) < 1e-10 * abs(m0)
            out[name] = (st, ctx.get_state(), learned)
    assert out["plain"][2] == 0
    assert rel(out["learned"][1], out["plain"][1]) < 1e-6
    assert out["learned"][0]["n_psd_iter"] <= 1.05 * out["plain"][0]["n_psd_iter"]


def test_learned_extrapolation_brings_imex_to_the_implicit_step(small_trained_net):
    # the IMEX step's explicit part at the network's prediction of u^{n+1} instead of
    # eq. (Richardson): on a held-out trajectory the step lands closer to the fully
    # implicit BDF2 step (the PSD fixed point); the plain method stays the reference
    from paper_2006_04784_gb300 import fno_train as T

    net, _ = small_trained_net
    n = 64
    p = fch.params_default(0.0, psd_itol=1e-12)
    dts = T.random_steps(np.random.default_rng(11), 16, 1e-3)
    u = [I.circle_bilayer(n, radius=2.2, noise=1e-3, seed=7)]
    plain, learned = [], []
    v0 = torch.empty((n, n), dtype=torch.float64, device=DEV)
    with fch.Context(n, p) as a, fch.Context(n, p) as b:
        a.set_state(u[0])
        for i, dt in enumerate(dts):
            if i >= 2:
                b.set_history(u[-1], u[-2], dts[i - 1])
                T.learned_start(b, net, v0, dt)
            a.step("psd", dt)
            u.append(a.get_state())
            if i >= 2:
                b.set_history(u[-2], u[-3], dts[i - 1])
                b.step("imex", dt)
                plain.append(rel(b.get_state(), u[-1]))
                b.set_history(u[-2], u[-3], dts[i - 1])
                b.step_from("imex", dt, v0)
                learned.append(rel(b.get_state(), u[-1]))
                assert b.mass() == pytest.approx(a.mass(), rel=1e-12)
    assert np.mean(learned) < 0.9 * np.mean(plain)


@pytest.mark.parametrize("mode", ["fixed", "adaptive"])
def test_learned_start_on_the_device_vs_oracle(small_trained_net, mode):
    # fch_fno_learned_start forms u*, s, the network input, y and v_0 on the device
    # from the context's history; against the FNO oracle's construction
    # (oracle/fno_oracle.py learned_start, FP64) on the same history and gam: v_0
    # differs by s times the forward pass's float rounding (2e-5 of y), and keeps the
    # mass of u* to rounding
    net, _ = small_trained_net
    cfg = F.Config(width=16, layers=2, modes=8, proj=32)
    params = net.params().astype(np.float64)
    n, kn = 64, 1e-3
    un = I.circle_bilayer(n, radius=2.2, noise=1e-3, seed=7)
    um = un - 3e-3 * I.smooth_random(n, seed=4, amp=0.5, kmax=3, offset=0.0)
    v0 = torch.empty((n, n), dtype=torch.float64, device=DEV)
    with fch.Context(n, fch.params_default(0.0)) as ctx:
        ctx.set_history(un, um, kn)
        if mode == "fixed":
            dt = 1.4e-3
            gam = dt / kn
            ctx.fno_learned_start(net, v0, dt)
        else:
            ctx.adaptive_begin("psd", 1e-5, 1.0)
            k, gam, done = ctx.adaptive_trial_info()
            assert not done and k == pytest.approx(kn) and gam == pytest.approx(1.0)
            ctx.fno_learned_start(net, v0)
        ctx.synchronize()
        got = v0.cpu().numpy()
        if mode == "adaptive":
            ctx.adaptive_enqueue_psd_from(v0)  # the trial runs from it
            st = ctx.adaptive_end()
            assert st["n_attempts"] >= 1
    ref, y, s = F.learned_start(params, un, um, gam, cfg)
    ustar = un + gam * (un - um)
    assert s > 0
    assert np.linalg.norm(got - ref) <= 4e-5 * s * np.linalg.norm(y)
    assert np.linalg.norm(ref - ustar) > 1e-2 * s * np.linalg.norm(y)  # not just u*
    assert abs(np.mean(got) - np.mean(ustar)) < 1e-15


@pytest.mark.parametrize("scheme", ["imex", "sav"])
def test_adaptive_imex_sav_with_learned_extrapolation(small_trained_net, scheme):
    # the adaptive IMEX / SAV run of Sec. 3.2 with the network's v_0 as every trial's
    # u* after the start (fch_fno_learned_start + fch_adaptive_enqueue_from):
    # it reaches t_final, keeps the mass (u* does not enter the k = 0 mode of either
    # solve) and stays within the local-error tolerance's reach of the plain run
    from paper_2006_04784_gb300 import fno_train as T

    net, _ = small_trained_net
    n = 64
    p = fch.params_default(0.0, zero_stab_cap=1)
    u0 = I.circle_bilayer(n, radius=2.2, noise=1e-3, seed=7)
    out = {}
    for name, use in (("plain", None), ("learned", net)):
        with fch.Context(n, p) as ctx:
            ctx.set_state(u0)
            m0 = ctx.mass()
            st, trials, learned = T.run_adaptive_learned(ctx, scheme, 1e-5, 2e-2, DEV, net=use)
            assert st["t"] == pytest.approx(2e-2, rel=1e-12) and trials > 5
            assert abs(ctx.mass() - m0) < 1e-12 * abs(m0)
            out[name] = (st, ctx.get_state(), learned)
    assert out["plain"][2] == 0 and out["learned"][2] > 0
    # two runs at sigma_tol = 1e-5 through different trials: apart by the global error
    # that tolerance allows (~sigma_tol^(2/3), Sec. 5.2)
    assert rel(out["learned"][1], out["plain"][1]) < 1e-3


def test_inference_gelu_vs_erf_and_its_error_bound():
    # the tensor-core kernels' GELU (pairs of values, packed FP32) takes erf from
    # Abramowitz and Stegun 7.1.28 (|error| <= 3e-7); against the training path's GELU
    # (the library erff) and the exact value, over the range activations take, the
    # tails and the special values; an odd count leaves the last value alone
    import ctypes as C

    f = fch.lib().fch_debug_fno_gelu
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_long, C.c_int, C.c_void_p]
    f.restype = C.c_int
    xs = np.concatenate([np.linspace(-12, 12, 400001), [0.0, -0.0, 1e-30, -1e-30, 40.0, -40.0, 1e30, -1e30]])
    x = torch.tensor(xs, dtype=torch.float32, device=DEV)
    ya, ye = torch.empty_like(x), torch.empty_like(x)
    assert f(x.data_ptr(), ya.data_ptr(), x.numel(), 1, None) == 0
    assert f(x.data_ptr(), ye.data_ptr(), x.numel(), 0, None) == 0
    xd = x.double().cpu().numpy()
    exact = 0.5 * xd * (1 + np.vectorize(math.erf)(xd / math.sqrt(2)))
    a, e = ya.double().cpu().numpy(), ye.double().cpu().numpy()
    assert np.isfinite(a).all()
    # 1 - erf within 3e-7 (the approximation) plus the float rounding of p^-16 (about
    # 2e-6 of it), then the GELU's own rounding
    bound = 0.5 * np.abs(xd) * 3e-6 + 3e-7 * np.abs(exact) + 1e-37
    assert (np.abs(a - exact) <= bound).all()
    assert (np.abs(a - e) <= 1e-6 * np.maximum(1.0, np.abs(xd))).all()
    assert (a[xd == 0] == 0).all() and a[-2] == xd[-2] and abs(a[-1]) < 1e-20


def _rowdft_fn():
    import ctypes as C

    f = fch.lib().fch_debug_rowdft_tc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    f.restype = C.c_int
    return f


@pytest.mark.parametrize("R,n", [(256, 64), (1000, 128), (32768, 1024)])
def test_row_dft_on_tensor_cores_vs_bf16_products(R, n):
    # the tensor-core GEMM of the truncated DFT along x (tcgen05, bf16 operands, FP32
    # sums in tensor memory): X[r][kx] = sum_x bf16(h[r][x]) bf16(cos - i sin)(2 pi kx x / n)
    # for kx < 16, against the same products summed exactly; 1000 rows leave a ragged
    # last tile of 128
    rng = np.random.default_rng(R + n)
    h = rng.standard_normal((R, n)).astype(np.float32)
    ht = torch.tensor(h, device=DEV)
    X = torch.full((R, 16, 2), float("nan"), dtype=torch.float32, device=DEV)
    torch.cuda.synchronize()
    assert _rowdft_fn()(ht.data_ptr(), X.data_ptr(), R, n, None) == 0
    got = X[..., 0].double().cpu().numpy() + 1j * X[..., 1].double().cpu().numpy()
    xs, kx = np.arange(n), np.arange(16)
    ang = 2 * np.pi * ((kx[:, None] * xs[None, :]) % n) / n
    hb = F.bf16_round(h.astype(np.float64))
    ref = hb @ F.bf16_round(np.cos(ang)).T + 1j * (hb @ F.bf16_round(-np.sin(ang)).T)
    assert np.isfinite(got).all()
    # FP32 sums of n products: rounding ~ sqrt(n) 2^-24 of the terms' size
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("width,layers,proj,n,batch", [(16, 2, 16, 128, 2), (32, 1, 64, 128, 1),
                                                       (32, 4, 64, 128, 1)])
def test_fno_truncated_dft_forward_vs_oracle(width, layers, proj, n, batch):
    # the tensor-core forward pass (x DFTs, channel mixing with the inverse x DFT, and
    # the projection as tcgen05 GEMMs with bfloat16 operands) against the oracle's
    # forward pass on the same bfloat16 weights and operands (oracle/fno_oracle.py
    # forward with tc). The values the two sides round to bfloat16 differ by float
    # rounding (~1e-6 relative for the spectral operand V, after three FP32 sums), so
    # a few operands land on the other side of a rounding boundary and move by 2^-8
    # (each V operand then moves a whole row of one channel): the outputs agree to float
    # rounding at the bulk of the points (median) and differ at a few, by about the
    # operands' own rounding effect in a deep network. Bounds: 1.5e-3 relative L2; a
    # median point error below 1e-5 of the output's size up to two layers.
    cfg = F.Config(width=width, layers=layers, modes=16, proj=proj)
    rng = np.random.default_rng(width + n)
    params = (F.init_params(cfg, 0) + 0.05 * rng.standard_normal(cfg.size())).astype(np.float32)
    a = rng.standard_normal((batch, 2, n, n)).astype(np.float32)
    net = fch.FNO(width, layers, 16, proj)
    net.set_params(params)
    net.set_bf16(2)
    at = torch.tensor(a, device=DEV)
    y = torch.empty((batch, n, n), device=DEV)
    net.forward(at, y)
    got = y.cpu().numpy().astype(np.float64)
    pb = F.bf16_round(params).astype(np.float64)
    a64 = a.astype(np.float64)
    ref = F.forward(pb, a64, cfg, tc=True)
    exact = F.forward(pb, a64, cfg)
    assert rel(got, ref) < 1.5e-3, (rel(got, ref), rel(exact, ref))
    if layers <= 2:
        assert np.median(np.abs(got - ref)) < 1e-5 * np.abs(ref).max()
        assert rel(got, ref) < 0.25 * rel(exact, ref)  # the same roundings as the oracle
    with pytest.raises(fch.FchError):
        net.backward(torch.zeros((batch, n, n), device=DEV))
    net.set_bf16(1)  # back to the full transforms on the same bfloat16 weights
    net.forward(at, y)
    assert rel(y.cpu().numpy(), F.forward(pb, a64, cfg)) < 2e-5
