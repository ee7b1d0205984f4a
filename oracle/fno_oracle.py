"""FP64 CPU reference of the Fourier neural operator (FNO) predictor: forward pass,
hand-derived backward pass and the loss.

TEST INFRASTRUCTURE ONLY: the test-suite and the benchmark's CPU-baseline leg are
the only users. It shares no code with the CUDA path. Its gradients are pinned by
finite differences (tests/test_fno_oracle.py), its transforms by numpy's FFT.

The network (Li et al.'s Fourier neural operator, restated): two input channels
per grid point, a = (u^n, (u* - u^n)/s), where u* is the extrapolated state of
eq. (Richardson) and s the RMS of u* - u^n; output y, the predicted correction
(u^{n+1} - u*)/s, so that v_0 = u* + s y is the initial iterate of the PSD
iteration, eqs. (residual), (recurrence) (Sec. 3.3 leaves v_0 free).

  h_0 = P a + bP                                    (lifting, W channels)
  h_{l+1} = act_l(W_l h_l + b_l + S_l(h_l)),  l < L  (act = GELU, identity for l = L-1)
  S(h)[o] = C2R( H( sum_i R[m][o][i] R2C(h[i])(m) on the retained modes m ) )
  y = Q2 GELU(Q1 h_L + bQ1) + bQ2                   (projection, W2 hidden channels)

R2C / C2R are the unnormalised forward / 1/N^2 inverse real 2D transforms (numpy's
rfft2 / irfft2 on fields indexed [y][x]; spectra [ky][kx], kx the half axis).
Retained modes: kx in [0, M), ky in {0..M-1} and {N-M+1..N-1} (a set closed under
ky -> -ky); the weights of mode (kx, kyi) live at index kx * (2M - 1) + kyi with
ky = kyi for kyi < M and ky = -(kyi - M + 1) otherwise. H replaces the kx = 0
column of the retained modes by its Hermitian part (Y(ky) + conj Y(-ky))/2, the
part any real inverse transform reads there. GELU(x) = x Phi(x) (exact, with erf).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT1_2 = 0.7071067811865476
INV_SQRT_2PI = 0.3989422804014327


def gelu(x):
    return 0.5 * x * (1.0 + erf(x * SQRT1_2))


def bf16_round(x):
    """float32 values rounded to bfloat16 (1 sign, 8 exponent, 7 stored mantissa
    bits: the top half of the float32 pattern), to nearest with ties to even; finite
    inputs. Returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x * SQRT1_2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


class Config:
    def __init__(self, width=32, layers=4, modes=16, proj=64, cin=2):
        self.W, self.L, self.M, self.W2, self.cin = width, layers, modes, proj, cin
        self.K = modes * (2 * modes - 1)

    def shapes(self):
        """(name, shape) of every parameter in the order of the flat vector"""
        W, M, W2 = self.W, self.M, self.W2
        s = [("P", (W, self.cin)), ("bP", (W,))]
        for l in range(self.L):
            s += [(f"W{l}", (W, W)), (f"b{l}", (W,)), (f"R{l}", (self.K, W, W, 2))]
        s += [("Q1", (W2, W)), ("bQ1", (W2,)), ("Q2", (W2,)), ("bQ2", (1,))]
        return s

    def size(self):
        return sum(int(np.prod(sh)) for _, sh in self.shapes())

    def unpack(self, flat):
        out, o = {}, 0
        for name, sh in self.shapes():
            n = int(np.prod(sh))
            out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(sh)
            o += n
        return out

    def pack(self, d):
        return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in self.shapes()])


def mode_index(cfg: Config, n: int):
    """(kx, ky) of every retained mode, in weight order"""
    M = cfg.M
    kxs, kys = [], []
    for kx in range(M):
        for kyi in range(2 * M - 1):
            ky = kyi if kyi < M else n - (kyi - M + 1)
            kxs.append(kx)
            kys.append(ky)
    return np.array(kxs), np.array(kys)


def hermitian_kx0(Y, cfg: Config, n: int):
    """H: the kx = 0 column of the retained modes replaced by its Hermitian part
    (Y has shape [..., n, n//2+1], indexed [ky][kx])."""
    Y = Y.copy()
    col = Y[..., :, 0].copy()
    for ky in range(cfg.M):
        m = (-ky) % n
        h = 0.5 * (col[..., ky] + np.conj(col[..., m]))
        Y[..., ky, 0] = h
        Y[..., m, 0] = np.conj(h)
    return Y


def spectral_conv(h, Rc, cfg: Config):
    """S(h) for h [B, W, n, n], Rc complex [K, W, W]; returns (s, X) with X the
    retained-mode spectra of h [B, W, K]"""
    n = h.shape[-1]
    kx, ky = mode_index(cfg, n)
    F = np.fft.rfft2(h)                       # [B, W, n, n//2+1], unnormalised
    X = F[:, :, ky, kx]                       # [B, W, K]
    Ym = np.einsum("koi,bik->bok", Rc, X)     # sum_i R[m][o][i] X[i](m)
    Y = np.zeros(F.shape, dtype=np.complex128)
    Y[:, :, ky, kx] = Ym
    Y = hermitian_kx0(Y, cfg, n)
    return np.fft.irfft2(Y, s=(n, n)), X


def spectral_conv_dft(h, Rc, cfg: Config, bf16_operands=False):
    """S(h) of spectral_conv written as truncated DFTs over the retained modes, in the
    order the tensor-core forward pass takes them: along x for kx < M, along y for the
    2M - 1 retained ky, the mode mixing, back along y, and back along x as the real
    part of the sum over kx < M with weight 1 at kx = 0 and 2 elsewhere, over n^2 (the
    C2R of the retained half spectrum through H). With bf16_operands the operands of
    the two x DFTs are rounded to bfloat16 first, as the tensor cores take them: the
    input h and the cos / -sin table forward; the cos / sin table and w(kx)/n^2 V
    (real part, and minus the imaginary part) back. Every sum is exact here."""
    B, W, n, _ = h.shape
    M, K2 = cfg.M, 2 * cfg.M - 1
    rnd = bf16_round if bf16_operands else (lambda v: v)
    xs = np.arange(n)
    kxs = np.arange(M)
    ang = 2.0 * np.pi * ((kxs[:, None] * xs[None, :]) % n) / n
    cx, sx = np.cos(ang), np.sin(ang)
    hh = rnd(h)
    X = np.einsum("bwyt,kt->bwyk", hh, rnd(cx)) + 1j * np.einsum("bwyt,kt->bwyk", hh, rnd(-sx))
    kys = np.array([q if q < M else n - (q - M + 1) for q in range(K2)])
    ey = np.exp(-2j * np.pi * np.outer(kys, xs) / n)          # [K2, n(y)]
    Y = np.einsum("bwyk,qy->bwqk", X, ey)                     # [B, W, kyi, kx]
    R4 = Rc.reshape(M, K2, W, W)                              # m = kx (2M - 1) + kyi
    Z = np.einsum("kqoi,biqk->boqk", R4, Y)
    V = np.einsum("boqk,qy->boyk", Z, np.conj(ey))            # [B, W, y, kx]
    w = np.where(kxs == 0, 1.0, 2.0) / (n * n)
    return (np.einsum("boyk,kt->boyt", rnd(w * V.real), rnd(cx))
            + np.einsum("boyk,kt->boyt", rnd(-w * V.imag), rnd(sx)))


def forward(params, a, cfg: Config, keep=False, tc=False):
    """y [B, n, n] for inputs a [B, cin, n, n]; with keep, also the activations the
    backward pass needs. tc: the library's tensor-core forward pass, whose contractions
    take bfloat16 operands (the weights are rounded by the caller): the spectral
    convolutions by spectral_conv_dft with bf16_operands, and the layer input rounded to
    bfloat16 where the channel mixing W h and the projection Q1 h read it."""
    p = cfg.unpack(params)
    rnd = bf16_round if tc else (lambda v: v)
    h = np.einsum("ci,bixy->bcxy", p["P"], a) + p["bP"][None, :, None, None]
    hs, zs, Xs = [h], [], []
    for l in range(cfg.L):
        Rc = p[f"R{l}"][..., 0] + 1j * p[f"R{l}"][..., 1]
        if tc:
            s, X = spectral_conv_dft(h, Rc, cfg, bf16_operands=True), None
        else:
            s, X = spectral_conv(h, Rc, cfg)
        z = np.einsum("cj,bjxy->bcxy", p[f"W{l}"], rnd(h)) + p[f"b{l}"][None, :, None, None] + s
        h = gelu(z) if l < cfg.L - 1 else z
        hs.append(h)
        zs.append(z)
        Xs.append(X)
    zq = np.einsum("dc,bcxy->bdxy", p["Q1"], rnd(h)) + p["bQ1"][None, :, None, None]
    q = gelu(zq)
    y = np.einsum("d,bdxy->bxy", p["Q2"], q) + p["bQ2"][0]
    if keep:
        return y, dict(hs=hs, zs=zs, Xs=Xs, zq=zq, q=q)
    return y


def learned_start(params, un, um, gam, cfg: Config):
    """The learned first iterate of the PSD iteration (Sec. 3.3 leaves v_0 free; u* is
    eq. (Richardson)), for one state: u* = u^n + gam (u^n - u^{n-1}), s = RMS(u* - u^n),
    a = (u^n, (u* - u^n)/s), y = forward(a), v_0 = u* + s (y - mean y). With s = 0
    (gam = 0 or u^n = u^{n-1}) v_0 = u*. Returns (v_0, y, s)."""
    un = np.asarray(un, dtype=np.float64)
    um = np.asarray(um, dtype=np.float64)
    ustar = un + gam * (un - um)
    d = ustar - un
    s = float(np.sqrt(np.mean(d * d)))
    if not s > 0:
        return ustar, None, 0.0
    a = np.stack([un, d / s])[None]
    y = forward(params, a, cfg)[0]
    return ustar + s * (y - y.mean()), y, s


def loss(params, a, target, cfg: Config):
    """mean over samples and points of (y - target)^2"""
    y = forward(params, a, cfg)
    return float(np.mean((y - target) ** 2))


def backward(params, a, target, cfg: Config):
    """gradient of loss() with respect to the flat parameter vector"""
    p = cfg.unpack(params)
    y, act = forward(params, a, cfg, keep=True)
    B, n = y.shape[0], y.shape[-1]
    g = {name: np.zeros(sh) for name, sh in cfg.shapes()}
    dy = 2.0 * (y - target) / y.size
    q, zq, hL = act["q"], act["zq"], act["hs"][-1]
    g["bQ2"][0] = dy.sum()
    g["Q2"] = np.einsum("bxy,bdxy->d", dy, q)
    dzq = dy[:, None] * p["Q2"][None, :, None, None] * gelu_grad(zq)
    g["bQ1"] = dzq.sum(axis=(0, 2, 3))
    g["Q1"] = np.einsum("bdxy,bcxy->dc", dzq, hL)
    dh = np.einsum("dc,bdxy->bcxy", p["Q1"], dzq)
    kx, ky = mode_index(cfg, n)
    wgt = np.where(kx == 0, 1.0, 2.0) / (n * n)   # C2R adjoint weights
    vgt = np.where(kx == 0, 1.0, 0.5)              # R2C adjoint through C2R
    for l in reversed(range(cfg.L)):
        z, hin, X = act["zs"][l], act["hs"][l], act["Xs"][l]
        dz = dh * gelu_grad(z) if l < cfg.L - 1 else dh
        g[f"b{l}"] = dz.sum(axis=(0, 2, 3))
        g[f"W{l}"] = np.einsum("bcxy,bjxy->cj", dz, hin)
        dh = np.einsum("cj,bcxy->bjxy", p[f"W{l}"], dz)
        # spectral branch: dY' = C2R^T(dz); dY = H(dY'); dR, dX; dh += R2C^T(dX)
        Fd = np.fft.rfft2(dz)
        Yd = np.zeros(Fd.shape, dtype=np.complex128)
        Yd[:, :, ky, kx] = Fd[:, :, ky, kx] * wgt
        Yd = hermitian_kx0(Yd, cfg, n)
        dY = Yd[:, :, ky, kx]                      # [B, W, K]
        Rc = p[f"R{l}"][..., 0] + 1j * p[f"R{l}"][..., 1]
        dR = np.einsum("bok,bik->koi", dY, np.conj(X))
        g[f"R{l}"][..., 0] = dR.real
        g[f"R{l}"][..., 1] = dR.imag
        dX = np.einsum("koi,bok->bik", np.conj(Rc), dY)
        Z = np.zeros(Fd.shape, dtype=np.complex128)
        Z[:, :, ky, kx] = dX * vgt
        Z = hermitian_kx0(Z, cfg, n)
        dh = dh + (n * n) * np.fft.irfft2(Z, s=(n, n))
    g["bP"] = dh.sum(axis=(0, 2, 3))
    g["P"] = np.einsum("bcxy,bixy->ci", dh, a)
    return cfg.pack(g)


def init_params(cfg: Config, seed: int = 0):
    """deterministic initial weights (uniform, fan-in scaled; spectral weights
    scaled by 1/(W W) as in the FNO reference design)"""
    rng = np.random.default_rng(seed)
    d = {}
    for name, sh in cfg.shapes():
        if name.startswith("b"):
            d[name] = np.zeros(sh)
        elif name.startswith("R"):
            d[name] = rng.uniform(0.0, 1.0, sh) / (cfg.W * cfg.W)
        else:
            fan = sh[-1] if len(sh) > 1 else sh[0]
            d[name] = rng.uniform(-1.0, 1.0, sh) / np.sqrt(fan)
    return cfg.pack(d)
