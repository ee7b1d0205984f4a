"""CPU pins of the FNO oracle (oracle/fno_oracle.py): its spectral convolution
against closed forms and its hand-derived gradient against finite differences."""
import numpy as np
import pytest

from oracle import fno_oracle as F


def small():
    return F.Config(width=3, layers=2, modes=3, proj=4)


def test_retained_modes_closed_under_negation():
    cfg, n = F.Config(width=2, layers=1, modes=5, proj=2), 32
    kx, ky = F.mode_index(cfg, n)
    assert len(kx) == cfg.K == 5 * 9
    s = set(zip(kx.tolist(), ky.tolist()))
    for a, b in s:
        assert 0 <= a < 5
        if a == 0:
            assert (0, (-b) % n) in s


def test_identity_weights_reproduce_band_limited_fields():
    # R = I on every retained mode: S(h) = h for a real field whose spectrum lies
    # inside the retained set (the kx = 0 column of a real field is Hermitian)
    cfg, n = F.Config(width=2, layers=1, modes=4, proj=2), 16
    rng = np.random.default_rng(1)
    x = np.arange(n) * 2 * np.pi / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    h = np.zeros((1, 2, n, n))
    for c in range(2):
        for kx in range(4):
            for ky in range(-3, 4):
                a, b = rng.standard_normal(2)
                h[0, c] += a * np.cos(kx * X + ky * Y) + b * np.sin(kx * X + ky * Y)
    Rc = np.zeros((cfg.K, 2, 2), dtype=complex)
    Rc[:, 0, 0] = Rc[:, 1, 1] = 1.0
    s, _ = F.spectral_conv(h, Rc, cfg)
    assert np.abs(s - h).max() < 1e-12 * np.abs(h).max()
    # and a single-mode weight acts as that mode's multiplier: i on mode (1, 2) only
    Rc[:] = 0
    kx, ky = F.mode_index(cfg, n)
    m = int(np.flatnonzero((kx == 1) & (ky == 2))[0])
    Rc[m, 0, 0] = 1j
    g = np.cos(X + 2 * Y)[None, None].repeat(2, axis=1)
    s, _ = F.spectral_conv(g, Rc, cfg)
    assert np.abs(s[0, 0] - (-np.sin(X + 2 * Y))).max() < 1e-12
    assert np.abs(s[0, 1]).max() < 1e-14


def test_gelu_derivative():
    x = np.linspace(-5, 5, 101)
    d = (F.gelu(x + 1e-6) - F.gelu(x - 1e-6)) / 2e-6
    assert np.abs(d - F.gelu_grad(x)).max() < 1e-8
    assert F.gelu(0.0) == 0.0 and abs(F.gelu(10.0) - 10.0) < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_finite_differences(seed):
    cfg, n, B = small(), 12, 2
    rng = np.random.default_rng(seed)
    params = F.init_params(cfg, seed) + 0.1 * rng.standard_normal(cfg.size())
    a = rng.standard_normal((B, 2, n, n))
    target = rng.standard_normal((B, n, n))
    g = F.backward(params, a, target, cfg)
    offs, o = {}, 0
    for name, sh in cfg.shapes():
        k = int(np.prod(sh))
        offs[name] = (o, k)
        o += k
    eps = 1e-6
    for name, (o, k) in offs.items():
        idx = o + rng.choice(k, size=min(k, 12), replace=False)
        for i in idx:
            e = np.zeros_like(params)
            e[i] = eps
            fd = (F.loss(params + e, a, target, cfg) - F.loss(params - e, a, target, cfg)) / (2 * eps)
            assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (name, i, fd, g[i])


def test_bf16_round_ties_to_even_and_matches_torch():
    # the bfloat16 grid near 1 has spacing 2^-7: ties go to the even pattern
    x = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20, -2.5, 3e-30, 65504.0],
                 dtype=np.float32)
    got = F.bf16_round(x)
    assert list(got[:4]) == [1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7]
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(4).standard_normal(10000).astype(np.float32) * 10.0 ** np.random.default_rng(5).uniform(-6, 6, 10000).astype(np.float32)
    for v in (x, r):
        ref = torch.tensor(v).to(torch.bfloat16).float().numpy()
        assert np.array_equal(F.bf16_round(v), ref)


def test_learned_start_keeps_the_mass_and_reduces_to_the_extrapolation():
    # v_0 = u* + s (y - mean y): the k = 0 mode (mass) of u* is kept for any network;
    # a network whose output is constant (Q2 = 0) gives v_0 = u*, and so does s = 0
    cfg = F.Config(width=8, layers=2, modes=4, proj=16)
    n = 16
    rng = np.random.default_rng(3)
    params = F.init_params(cfg, 1) + 0.05 * rng.standard_normal(cfg.size())
    un = rng.standard_normal((n, n))
    um = un + 0.01 * rng.standard_normal((n, n))
    gam = 1.7
    ustar = un + gam * (un - um)
    v0, y, s = F.learned_start(params, un, um, gam, cfg)
    assert s == pytest.approx(gam * np.sqrt(np.mean((un - um) ** 2)), rel=1e-14)
    assert np.mean(v0) == pytest.approx(np.mean(ustar), abs=1e-15)
    assert np.linalg.norm(v0 - ustar) > 1e-3 * s  # the network moved it
    # the prediction is the network's forward pass on (u^n, (u* - u^n)/s)
    a = np.stack([un, (ustar - un) / s])[None]
    assert np.array_equal(y, F.forward(params, a, cfg)[0])
    d = cfg.unpack(params)
    d["Q2"][:] = 0.0
    v0c, _, _ = F.learned_start(cfg.pack(d), un, um, gam, cfg)
    assert np.abs(v0c - ustar).max() < 1e-14
    v00, _, s0 = F.learned_start(params, un, um, 0.0, cfg)
    assert s0 == 0.0 and np.array_equal(v00, un)


@pytest.mark.parametrize("n,M", [(16, 4), (32, 16)])
def test_truncated_dft_spectral_conv_equals_the_fft_form(n, M):
    # the truncated-DFT form of S(h) (x, then y, mixing, back along y, real part of
    # the kx sum with weights 1, 2) is the C2R-through-H form of spectral_conv
    cfg = F.Config(width=4, layers=1, modes=M, proj=4)
    rng = np.random.default_rng(n + M)
    h = rng.standard_normal((2, 4, n, n))
    Rc = rng.standard_normal((cfg.K, 4, 4)) + 1j * rng.standard_normal((cfg.K, 4, 4))
    s_fft, _ = F.spectral_conv(h, Rc, cfg)
    s_dft = F.spectral_conv_dft(h, Rc, cfg)
    assert np.abs(s_dft - s_fft).max() < 1e-12 * np.abs(s_fft).max()
    # bfloat16 operands move it by the operands' rounding only
    s_b = F.spectral_conv_dft(h, Rc, cfg, bf16_operands=True)
    assert 1e-5 < np.linalg.norm(s_b - s_fft) / np.linalg.norm(s_fft) < 2e-2
