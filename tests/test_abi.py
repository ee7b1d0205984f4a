"""CPU checks of the C ABI: the library builds, loads and exports every symbol
include/fch.h declares; launch geometry fits its buffers; argument checks that
return before any device work."""
import ctypes as C
import os
import re

import pytest

from paper_2006_04784_gb300 import build as B
from paper_2006_04784_gb300 import fch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fch_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    syms = declared_symbols()
    assert len(syms) >= 20
    L = C.CDLL(fch.LIB_PATH)
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(fch.EXPORTS) == syms


def test_status_strings():
    L = fch.lib()
    for s in range(8):
        assert L.fch_status_string(s)
    assert L.fch_status_string(99) == b"unknown status"


@pytest.mark.parametrize("n", [16, 32, 64, 128, 256, 512, 1024, 2048])
@pytest.mark.parametrize("prec", [0, 1])
def test_geometry_covers_grid(n, prec):
    g = fch.geometry(n, prec)
    csz = 8 if prec else 16
    sl = n + n // 8  # skewed sequence length
    if n == 1024 and csz == 16:
        # two-block clusters: one column of each pair per block of N/8 threads
        assert g["col_blocks"] == n and g["col_threads"] == n // 8 and g["col_smem"] == sl * csz
    else:
        # column pass: P pairs per block, 2P sequences of N/8 threads, all N/2 pairs covered
        assert g["col_blocks"] * g["P"] == n // 2
        assert g["col_threads"] == 2 * g["P"] * (n // 8) and g["col_threads"] <= 1024
        assert g["col_smem"] == (n + 2 * g["P"] * sl) * csz and g["col_smem"] <= 227 * 1024
    assert g["col_threads"] % 32 == 0
    # row pass: rpb rows of N/8 threads, all N rows covered
    assert g["row_blocks"] * g["rpb"] == n
    assert g["row_threads"] == g["rpb"] * (n // 8) and g["row_threads"] <= 256
    assert g["row_threads"] % 32 == 0
    assert g["row_smem"] == g["rpb"] * sl * csz and g["row_smem"] <= 227 * 1024  # twiddles in global
    # per-block partial sums fit their slots (FCH_MAXBLK = 4096)
    assert max(g["row_blocks"], g["col_blocks"]) <= 4096


@pytest.mark.parametrize("n", [16, 64, 256, 512, 1024, 2048])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_tiles_cover_grid(n, prec):
    # every tile the autotuner may pick launches whole blocks over the grid within a
    # block's thread and shared-memory limits; invalid ones are refused
    csz = 8 if prec == 1 else 16
    sl = n + n // 8
    nvalid = 0
    for t in (1, 2, 4, 8, 16, 32):
        ok_r, g = fch.tile_geometry(n, prec, t, 0)
        fits_r = t <= n and t * (n // 8) <= 256 and t * (n // 8) % 32 == 0 and t * sl * csz <= 226 * 1024
        assert ok_r == fits_r, (t, g)
        if ok_r:
            nvalid += 1
            assert g["rpb"] == t and g["row_blocks"] * t == n
            assert g["row_threads"] == t * (n // 8) and g["row_smem"] == t * sl * csz
        ok_c, g = fch.tile_geometry(n, prec, 0, t)
        fits_c = (t >= (2 if prec == 1 else 1) and t <= n // 2 and t * n // 4 <= 1024
                  and t * n // 4 % 32 == 0 and (n + 2 * t * sl) * csz <= 226 * 1024)
        assert ok_c == fits_c, (t, g)
        if ok_c:
            assert g["P"] == t and g["col_blocks"] * t == n // 2
            assert g["col_threads"] == 2 * t * (n // 8) and g["col_smem"] == (n + 2 * t * sl) * csz
    assert nvalid >= 1
    assert fch.tile_geometry(n, prec, 0, 0)[0] and fch.tile_geometry(n, prec, -1, -1)[0]
    assert not fch.tile_geometry(n, prec, 3, 0)[0] and not fch.tile_geometry(n, prec, -2, 0)[0]
    # the warp-level column passes exist for single precision at 1024^2 only
    ok, g = fch.tile_geometry(n, prec, 0, -2)
    assert ok == (prec == 1 and n == 1024)
    if ok:
        assert g["col_blocks"] == n // 4 and g["col_threads"] == 128
    # tile_col = -2 - P: the generic column kernel with P pairs a block at four points a
    # thread (twice the threads of tile P)
    for t in (1, 2, 4, 8, 16):
        ok_c, g = fch.tile_geometry(n, prec, 0, -2 - t)
        fits_c = (t >= (2 if prec == 1 else 1) and t <= n // 2 and t * n // 2 <= 1024
                  and t * n // 2 % 32 == 0 and (n + 2 * t * sl) * csz <= 226 * 1024)
        assert ok_c == fits_c, (t, g)
        if ok_c:
            assert g["P"] == t and g["col_blocks"] * t == n // 2
            assert g["col_threads"] == 2 * t * (n // 4) and g["col_smem"] == (n + 2 * t * sl) * csz
    assert not fch.tile_geometry(n, prec, 0, -5)[0]  # P = 3
    # tile_row = -2 - R: the generic row kernel with R rows a block at four points a thread
    for t in (1, 2, 4, 8):
        ok_r, g = fch.tile_geometry(n, prec, -2 - t, 0)
        fits_r = t <= n and t * (n // 4) <= 256 and t * (n // 4) % 32 == 0 and t * sl * csz <= 226 * 1024
        assert ok_r == fits_r, (t, g)
        if ok_r:
            assert g["rpb"] == t and g["row_blocks"] * t == n
            assert g["row_threads"] == t * (n // 4) and g["row_smem"] == t * sl * csz
    assert not fch.tile_geometry(n, prec, -5, 0)[0]  # R = 3


def test_stockham_index_map_is_a_permutation():
    # the store index of every Stockham stage (fft_smem) is a bijection on [0, N)
    for logn in range(4, 12):
        n = 1 << logn
        tps = n // 8
        ns, lns, rem = 1, 0, logn
        while rem > 0:
            lr = 3 if rem >= 3 else rem
            r_ = 1 << lr
            seen = set()
            for t in range(tps):
                for i in range(8):
                    b, r = i >> lr, i & (r_ - 1)
                    j = t + b * tps
                    assert j + r * (n >> lr) < n  # load index in range
                    idx = ((j >> lns) << (lns + lr)) + (j & (ns - 1)) + r * ns
                    assert 0 <= idx < n
                    assert idx + (idx >> 3) < n + n // 8  # skewed slot inside the sequence
                    seen.add(idx)
            assert len(seen) == n
            ns <<= lr
            lns += lr
            rem -= lr


def test_params_default_paper_constants():
    p = fch.params_default(0.2)
    assert p.eps == 0.1 and p.gamma == 0.3 and p.b_minus == -1 and p.b_plus == 1
    assert p.eta1 == pytest.approx(0.145) and p.eta2 == pytest.approx(0.3)
    assert (p.beta1, p.beta2, p.kappa0, p.kappa2, p.rho_s, p.k_min) == (2, 1, 1e-2, 15, 0.9, 1e-9)
    assert p.psd_nu == 2e-5 and p.psd_k_max == 0.02


def test_create_rejects_bad_arguments_before_device_work():
    L = fch.lib()
    p = fch.params_default(0.0)
    h = C.c_void_p()
    for n in (0, 8, 100, 4096, 3000):
        g = fch.Grid(n, 4.0, 0.0)
        assert L.fch_create(C.byref(g), C.byref(p), None, C.byref(h)) == 1
    g = fch.Grid(64, -1.0, 0.0)
    assert L.fch_create(C.byref(g), C.byref(p), None, C.byref(h)) == 1
    bad = fch.params_default(0.0, eps=0.0)
    g = fch.Grid(64, 4.0, 0.0)
    assert L.fch_create(C.byref(g), C.byref(bad), None, C.byref(h)) == 1
    assert L.fch_step(None, 0, 1e-3) == 1
    assert L.fch_fft_plan_create(100, 0, None, C.byref(h)) == 1


def test_compile_time_pair_rule_matches_geometry():
    # the specialised column kernels (N = 512, 1024, 2048) assume the pairs-per-block
    # rule of fch_geometry: max(pmin, 1024 / N), pmin = 2 (8-byte) or 1 (16-byte)
    for n in (512, 1024, 2048):
        for prec, pmin in ((0, 1), (1, 2)):
            assert fch.geometry(n, prec)["P"] == max(pmin, 1024 // n)


def _stockham(x, tw, ppt, sign):
    """The shared-memory transform's stage schedule and index arithmetic, read from
    the kernels (fft_smem / fft_stage): radix-ppt stages, then one of the remaining
    radix; stage Ns reads x[j + r N/R], multiplies by the table's entry
    Ns - ppt + (r-1) Ns + (j mod Ns) (conjugated for the inverse), takes the R-point
    DFT and writes output r at ((j >> log Ns) << log(Ns R)) + (j mod Ns) + r Ns."""
    import numpy as np
    n = len(x)
    lp = 3 if ppt == 8 else 2
    stages, rem = [], int(np.log2(n))
    while rem >= lp:
        stages.append(lp)
        rem -= lp
    if rem:
        stages.append(rem)
    s, ns, lns = np.array(x, dtype=complex), 1, 0
    for lr in stages:
        R = 1 << lr
        nb = n >> lr
        out = np.full(n, np.nan, dtype=complex)
        k = np.arange(R)
        dft = np.exp(sign * 2j * np.pi * np.outer(k, k) / R)
        for j in range(nb):
            v = np.array([s[j + r * nb] for r in range(R)])
            if ns > 1:
                for r in range(1, R):
                    t = tw[ns - ppt + (r - 1) * ns + (j & (ns - 1))]
                    v[r] *= t if sign < 0 else np.conj(t)
            dst = ((j >> lns) << (lns + lr)) + (j & (ns - 1)) + ns * k
            assert np.all(np.isnan(out[dst]))
            out[dst] = dft @ v
        s, ns, lns = out, ns << lr, lns + lr
    return s


@pytest.mark.parametrize("n", [16, 32, 128, 256, 512, 2048])
@pytest.mark.parametrize("ppt", [8, 4])
def test_stage_twiddle_tables_give_the_dft(n, ppt):
    # the host's twiddle tables for eight and four points a thread, applied with the
    # kernels' stage indexing, give the DFT and its inverse (numpy's FFT)
    import numpy as np
    tw = fch.stage_twiddles(n, 3 if ppt == 8 else 2)
    x = np.random.default_rng(n + ppt).standard_normal(n) + 1j * np.random.default_rng(1).standard_normal(n)
    assert np.abs(_stockham(x, tw, ppt, -1) - np.fft.fft(x)).max() < 1e-12 * n
    assert np.abs(_stockham(x, tw, ppt, +1) - n * np.fft.ifft(x)).max() < 1e-12 * n
