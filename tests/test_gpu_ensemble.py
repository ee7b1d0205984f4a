"""GPU: ensembles of independent instances (uneven grids, parameter sweeps,
seeds) advanced by one CUDA graph per launch must give every member exactly the
trajectory it has when run alone, and the adaptive method's result."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def member_params(i, prec):
    eps = 0.1
    p = fch.params_default(0.0, eta1=eps * (1.0 + 0.5 * i), prec=prec, zero_stab_cap=1)
    p.zeta, p.D0 = 1.1, 170.0
    return p


def member_init(n, i):
    return I.multimode_bilayer(n, seed=100 + i)


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("scheme", ["imex", "sav", "etd", "psd"])
def test_ensemble_members_match_solo_runs(scheme, prec):
    sizes = [64, 128, 64, 32]
    tf = 2e-3
    params = [member_params(i, prec) for i in range(len(sizes))]
    with fch.Ensemble(sizes, params) as ens:
        for i, n in enumerate(sizes):
            ens[i].set_state(member_init(n, i))
        stats = ens.run_adaptive(scheme, 1e-5, tf, rounds=4)
        got = [ens[i].get_state() for i in range(len(sizes))]
        masses = [ens[i].mass() for i in range(len(sizes))]
    for i, n in enumerate(sizes):
        assert stats[i]["t"] == pytest.approx(tf, rel=1e-12)
        with fch.Context(n, member_params(i, prec)) as ctx:
            ctx.set_state(member_init(n, i))
            st = ctx.run_adaptive(scheme, 1e-5, tf)
            assert st["n_steps"] == stats[i]["n_steps"] and st["n_rejects"] == stats[i]["n_rejects"]
            assert np.array_equal(ctx.get_state(), got[i]), i
            assert masses[i] == ctx.mass()


def test_ensemble_member_matches_oracle():
    sizes = [32, 64]
    params = [member_params(i, 0) for i in range(2)]
    with fch.Ensemble(sizes, params) as ens:
        for i, n in enumerate(sizes):
            ens[i].set_state(member_init(n, i))
        ens.run_adaptive("imex", 1e-5, 2e-3, rounds=3)
        for i, n in enumerate(sizes):
            p = params[i]
            s = O.Stepper(n, L, O.params(eps=p.eps, q=p.q, gamma=p.gamma, eta1=p.eta1, eta2=p.eta2,
                                         zeta=p.zeta, D0=p.D0, rho_s=p.rho_s, k_min=p.k_min, k_max=p.k_max,
                                         zero_stab_cap=1))
            s.set_state(member_init(n, i))
            assert s.run_adaptive("imex", 1e-5, 2e-3) == 0
            assert rel(ens[i].get_state(), s.state()) < 1e-9


def test_ensemble_errors_and_budget():
    sizes = [32, 32]
    params = [member_params(i, 0) for i in range(2)]
    with fch.Ensemble(sizes, params) as ens:
        for i, n in enumerate(sizes):
            ens[i].set_state(member_init(n, i))
        st = ens.run_adaptive("imex", 1e-5, 10.0, rounds=2, max_launches=3, raise_on_timeout=False)
        # the backward-Euler start, one trial on the member's stream, then 3 launches
        # of 2 trials each
        assert [s["n_attempts"] for s in st] == [8, 8]
        assert all(s["t"] < 10.0 for s in st)
        # the members continue from where the budget stopped them
        st2 = ens.run_adaptive("imex", 1e-5, st[0]["t"] + 1e-4, rounds=2)
        assert st2[0]["t"] == pytest.approx(st[0]["t"] + 1e-4, rel=1e-12)
    with pytest.raises(fch.FchError):
        fch.Ensemble([], [])


@pytest.mark.parametrize("prec", [0, 2])
def test_ensemble_sweep_members_match_solo_runs(prec):
    # a scheme and a sigma_tol per member: every member equals its solo run, and
    # rerunning the same ensemble with the schemes permuted recaptures the graph
    sizes = [64, 64, 32, 64]
    schemes = ["imex", "sav", "etd", "psd"]
    sigmas = [1e-4, 1e-5, 3e-5, 1e-6]
    tf = 2e-3
    params = [member_params(i, prec) for i in range(len(sizes))]
    for order in (schemes, schemes[::-1]):
        with fch.Ensemble(sizes, params) as ens:
            for i, n in enumerate(sizes):
                ens[i].set_state(member_init(n, i))
            stats = ens.run_adaptive_each(order, sigmas, tf, rounds=3)
            got = [ens[i].get_state() for i in range(len(sizes))]
        for i, n in enumerate(sizes):
            assert stats[i]["t"] == pytest.approx(tf, rel=1e-12)
            with fch.Context(n, member_params(i, prec)) as ctx:
                ctx.set_state(member_init(n, i))
                st = ctx.run_adaptive(order[i], sigmas[i], tf)
                assert st["n_steps"] == stats[i]["n_steps"] and st["n_rejects"] == stats[i]["n_rejects"]
                assert np.array_equal(ctx.get_state(), got[i]), (order, i)


def test_ensemble_sweep_errors():
    sizes = [32, 32]
    params = [member_params(i, 0) for i in range(2)]
    with fch.Ensemble(sizes, params) as ens:
        for i, n in enumerate(sizes):
            ens[i].set_state(member_init(n, i))
        with pytest.raises(fch.FchError):
            ens.run_adaptive_each(["imex", "sav"], [1e-5, 0.0], 1e-3)
        st = ens.run_adaptive_each(["sav", "imex"], [1e-5, 1e-4], 1e-3, rounds=2)
        assert all(s["t"] == pytest.approx(1e-3, rel=1e-12) for s in st)


def test_ensemble_psd_nonconvergence_is_reported():
    # a PSD member whose iteration stops at psd_max_iter (4) in a replayed trial
    # ends the ensemble run with FCH_ENOCONV; the IMEX member is unaffected
    sizes = [32, 32]
    params = [member_params(i, 0) for i in range(2)]
    params[0].psd_max_iter = 4
    params[0].eta1 = 0.1
    with fch.Ensemble(sizes, params) as ens:
        ens[0].set_state(I.multimode_bilayer(32, seed=100))
        ens[1].set_state(member_init(32, 1))
        with pytest.raises(fch.FchError) as e:
            ens.run_adaptive_each(["psd", "imex"], [1e-5, 1e-5], 2e-3, rounds=2)
        assert e.value.status == 4
        st = ens[0].stats()
        assert st["n_steps"] >= 5 and st["t"] < 2e-3 and st["last_psd_iter"] == 4
