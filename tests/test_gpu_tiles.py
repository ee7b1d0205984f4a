"""GPU: the pass tiles (launch shapes) and their autotuner. Every tile computes the
same method, so each forced tile must match the oracle like the default one, and
the tuner must pick a tile that launches."""
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


def oparams(fp):
    return O.params(eps=fp.eps, q=fp.q, gamma=fp.gamma, b_minus=fp.b_minus, b_plus=fp.b_plus,
                    eta1=fp.eta1, eta2=fp.eta2, beta1=fp.beta1, beta2=fp.beta2, zeta=fp.zeta, D0=fp.D0,
                    kappa0=fp.kappa0, kappa2=fp.kappa2, rho_s=fp.rho_s, k_min=fp.k_min, k_max=fp.k_max,
                    zero_stab_cap=fp.zero_stab_cap, well=0, psd_nu=fp.psd_nu, psd_itol=fp.psd_itol,
                    psd_lambda=fp.psd_lambda, psd_max_iter=fp.psd_max_iter)


def lib_params(**kw):
    p = fch.params_default(0.0, **kw)
    p.zeta, p.D0 = 1.1, 170.0
    return p


@pytest.mark.parametrize("n,prec,tiles", [
    (256, 0, [(1, 1), (2, 4), (4, 2), (-1, -1), (1, -3), (1, -4), (-3, -3), (-4, 2)]),
    (256, 2, [(1, 1), (4, 4), (-1, -1), (1, -3), (1, -6), (-3, -3), (-6, -4)]),
    (128, 2, [(2, -3), (2, -4), (-4, -3)]),
    (64, 0, [(0, -3), (0, -4), (-4, -3)]),
    (512, 0, [(1, 2), (2, 1), (-1, -1), (0, -3), (-3, 0)]),
    (1024, 2, [(1, 1), (2, 2), (0, -3), (-3, 0)]),
])
def test_forced_tiles_match_oracle(n, prec, tiles):
    # fixed IMEX and SAV steps under generic-kernel tiles of several shapes
    u0 = I.circle_bilayer(n, noise=1e-3)
    ref = {}
    for scheme in ("imex", "sav"):
        s = O.Stepper(n, L, oparams(lib_params(prec=prec)))
        s.set_state(u0)
        for dt in (1e-4, 1e-4, 2e-4):
            s.step(scheme, dt)
        ref[scheme] = s.state()
    for tr, tc in tiles:
        for scheme in ("imex", "sav"):
            with fch.Context(n, lib_params(prec=prec, tile_row=tr, tile_col=tc)) as ctx:
                ctx.set_state(u0)
                for dt in (1e-4, 1e-4, 2e-4):
                    ctx.step(scheme, dt)
                assert rel(ctx.get_state(), ref[scheme]) < 1e-10, (tr, tc, scheme)


def test_four_point_column_tiles_single_precision():
    # tile_col = -2 - P in single precision (P >= 2): the steps of the default tiles and
    # of the oracle to single-precision rounding (the bound of the other single-precision
    # tile test)
    n = 256
    u0 = I.circle_bilayer(n, noise=1e-3)
    o = O.Stepper(n, L, oparams(lib_params(prec=1)))
    o.set_state(u0)
    for dt in (1e-4, 1e-4, 2e-4):
        o.step("imex", dt)
    out = []
    for tc in (0, -4, -6):
        with fch.Context(n, lib_params(prec=1, tile_col=tc)) as ctx:
            ctx.set_state(u0)
            for dt in (1e-4, 1e-4, 2e-4):
                ctx.step("imex", dt)
            out.append(ctx.get_state())
    for u in out:
        assert rel(u, o.state()) < 3e-5
    assert rel(out[1], out[0]) < 3e-5 and rel(out[2], out[0]) < 3e-5


def test_forced_tiles_mixed_1024_warp_and_shared_memory():
    # single precision at 1024^2: the default (warp-level rows), the shared-memory
    # kernels (-1), a generic tile and the warp-level columns (-2) agree with each
    # other to single-precision rounding
    n = 1024
    u0 = I.random_network(n, d=0.75, seed=3)
    out = {}
    for tiles in ((0, 0), (-1, -1), (2, 4), (0, -2)):
        with fch.Context(n, lib_params(eta2=0.15, prec=1, tile_row=tiles[0], tile_col=tiles[1])) as ctx:
            ctx.set_state(u0)
            for _ in range(3):
                ctx.step("imex", 1e-6)
            out[tiles] = ctx.get_state()
    assert rel(out[(-1, -1)], out[(0, 0)]) < 3e-5
    assert rel(out[(2, 4)], out[(-1, -1)]) < 3e-5
    assert rel(out[(0, -2)], out[(0, 0)]) < 3e-5


@pytest.mark.parametrize("n,prec", [(256, 0), (1024, 1), (1024, 2)])
def test_autotune_picks_valid_tiles_and_adaptive_run_matches(n, prec):
    fch.autotune_reset()
    t = fch.autotune(n, prec)
    assert t["candidates"] >= 3
    assert t["row_us"] > 0 and t["col_us"] > 0
    assert t["row_us"] <= t["row_default_us"] * (1 + 1e-9) and t["col_us"] <= t["col_default_us"] * (1 + 1e-9)
    assert fch.tile_geometry(n, prec, t["tile_row"], t["tile_col"])[0]
    assert fch.autotune(n, prec) == t  # kept for the process
    if prec == 1:
        return
    # a context that takes the tuned tiles runs the adaptive method like the oracle
    m = 128 if n > 256 else n
    if m != n:
        fch.autotune(m, prec)
    p = lib_params(prec=prec, zero_stab_cap=1, autotune=1)
    u0 = I.circle_bilayer(m, noise=1e-3)
    s = O.Stepper(m, L, oparams(p))
    s.set_state(u0)
    assert s.run_adaptive("imex", 1e-5, 2e-3) == 0
    with fch.Context(m, p) as ctx:
        ctx.set_state(u0)
        st = ctx.run_adaptive("imex", 1e-5, 2e-3)
        assert st["n_steps"] == s.counts()["steps"]
        assert rel(ctx.get_state(), s.state()) < 1e-9


def test_plan_created_after_autotune_uses_tuned_tiles():
    n = 128
    fch.autotune_reset()
    fch.autotune(n, 0)
    x = np.random.default_rng(5).standard_normal((5, n, n))
    xt = torch.tensor(x, device=DEV)
    X = torch.empty((5, n // 2 + 1, n), dtype=torch.complex128, device=DEV)
    plan = fch.FFTPlan(n, 0)
    plan.r2c(xt, X)
    torch.cuda.synchronize()
    for b in range(5):
        ref = O.fft2(x[b], -1)[:, : n // 2 + 1].T
        assert np.abs(X[b].cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max() * math.log2(n)
    fch.autotune_reset()


def test_tile_shared_memory_limits_survive_other_grids():
    # double-float at 512^2 runs the generic kernels at the default tiles too: a large
    # generic tile at 1024^2, then the default tiles at 512^2, then a large tile at
    # 512^2 must all launch (one shared-memory limit per kernel)
    u = {n: I.circle_bilayer(n, noise=1e-3) for n in (512, 1024)}
    out = []
    for n, tc in ((1024, 4), (512, 0), (512, 8), (1024, 4)):
        with fch.Context(n, lib_params(prec=2, tile_col=tc)) as ctx:
            ctx.set_state(u[n])
            ctx.step("imex", 1e-4)
            out.append(ctx.get_state())
    assert rel(out[2], out[1]) < 1e-12 and np.array_equal(out[3], out[0])


@pytest.mark.parametrize("n,prec", [(256, 0), (512, 2)])
def test_autotune_step_picks_valid_tiles_and_adaptive_run_matches(n, prec):
    # the tuner that times adaptive trials: valid, kept, never slower than the default
    # it measured, and a context that takes its tiles runs the method like the oracle
    fch.autotune_reset()
    t = fch.autotune_step(n, prec)
    assert t["candidates"] >= 3
    assert 0 < t["row_us"] <= t["row_default_us"] * (1 + 1e-9)
    assert 0 < t["col_us"] <= t["col_default_us"] * (1 + 1e-9)
    assert t["col_default_us"] == t["row_us"]  # the column search starts from the rows' winner
    assert fch.tile_geometry(n, prec, t["tile_row"], t["tile_col"])[0]
    assert fch.autotune_step(n, prec) == t
    m = 128
    fch.autotune_step(m, prec)
    p = lib_params(prec=prec, zero_stab_cap=1, autotune=2)
    u0 = I.circle_bilayer(m, noise=1e-3)
    s = O.Stepper(m, L, oparams(p))
    s.set_state(u0)
    assert s.run_adaptive("imex", 1e-5, 2e-3) == 0
    with fch.Context(m, p) as ctx:
        ctx.set_state(u0)
        st = ctx.run_adaptive("imex", 1e-5, 2e-3)
        assert st["n_steps"] == s.counts()["steps"]
        assert rel(ctx.get_state(), s.state()) < 1e-9
    fch.autotune_reset()
