"""Training data, training loop and use of the FNO initial iterate for PSD-BDF2.

The network (fch_fno_*) predicts the PSD fixed point u^{n+1} from u^n and the
extrapolation u* = u^n + gamma (u^n - u^{n-1}), gamma = k_{n+1}/k_n (eq. Richardson):
inputs a = (u^n, (u* - u^n)/s), target (u^{n+1} - u*)/s, s = RMS(u* - u^n). Samples
come from PSD-BDF2 trajectories the library itself computes (Sec. 3.3) with
randomly varied step sizes; the learned start is v_0 = u* + s (y - mean y), which
keeps the mass of u* (the PSD iteration keeps the k = 0 mode of its start).

The learned start of a step (u*, s, the network's input, its forward pass and v_0)
runs in the library's kernels (fch_fno_learned_start), and the trials in its
steppers; this module calls them and moves tensors. The training samples are
assembled on the host from the states of trajectories the library computed
(samples_from: the input pairs and targets of the regression), once, before
training.
"""
from __future__ import annotations

import numpy as np

from . import fch


def param_shapes(width, layers, modes, proj, cin=2):
    """(name, shape) of the flat parameter vector of fch_fno, in order"""
    K = modes * (2 * modes - 1)
    s = [("P", (width, cin)), ("bP", (width,))]
    for l in range(layers):
        s += [(f"W{l}", (width, width)), (f"b{l}", (width,)), (f"R{l}", (K, width, width, 2))]
    return s + [("Q1", (proj, width)), ("bQ1", (proj,)), ("Q2", (proj,)), ("bQ2", (1,))]


def init_params(net, seed=0):
    """seeded initial weights: biases 0, dense weights U(-1, 1)/sqrt(fan-in),
    spectral weights U(0, 1)/width^2 (the FNO reference design's scaling)"""
    rng = np.random.default_rng(seed)
    parts = []
    for name, sh in param_shapes(net.width, net.layers, net.modes, net.proj):
        if name.startswith("b"):
            parts.append(np.zeros(sh))
        elif name.startswith("R"):
            parts.append(rng.uniform(0.0, 1.0, sh) / (net.width * net.width))
        else:
            fan = sh[-1] if len(sh) > 1 else sh[0]
            parts.append(rng.uniform(-1.0, 1.0, sh) / np.sqrt(fan))
    flat = np.concatenate([x.ravel() for x in parts]).astype(np.float32)
    assert flat.size == net.num_params
    return flat


def psd_trajectory(n, u0, dts, params):
    """states u_0 .. u_m of fixed PSD-BDF2 steps dts (the first a backward-Euler
    start), as host arrays"""
    states = [np.array(u0, dtype=np.float64)]
    with fch.Context(n, params) as ctx:
        ctx.set_state(u0)
        for dt in dts:
            ctx.step("psd", dt)
            states.append(ctx.get_state())
    return states


def samples_from(states, dts):
    """(inputs [2, n, n], target [n, n], s) for every step with two predecessors"""
    out = []
    for i in range(2, len(states)):
        g = dts[i - 1] / dts[i - 2]
        um, un, up = states[i - 2], states[i - 1], states[i]
        ustar = un + g * (un - um)
        d = ustar - un
        s = float(np.sqrt(np.mean(d * d)))
        if not s > 0:
            continue
        out.append((np.stack([un, d / s]).astype(np.float32), ((up - ustar) / s).astype(np.float32), s))
    return out


def random_steps(rng, m, base, spread=2.0):
    """m step sizes base * spread^U(-1, 1)"""
    return [base * spread ** rng.uniform(-1.0, 1.0) for _ in range(m)]


def train(net, data, iters, batch, lr, device, seed=0, log_every=0):
    """Adam on minibatches of the samples; returns the loss history"""
    import torch

    rng = np.random.default_rng(seed)
    A = torch.tensor(np.stack([d[0] for d in data]), device=device)
    T = torch.tensor(np.stack([d[1] for d in data]), device=device)
    n = A.shape[-1]
    y = torch.empty((batch, n, n), device=device)
    hist = []
    for it in range(iters):
        idx = torch.tensor(rng.choice(len(data), size=batch, replace=False), device=device)
        a, t = A[idx].contiguous(), T[idx].contiguous()
        net.forward(a, y)
        hist.append(net.backward(t))
        net.adam(lr)
        if log_every and it % log_every == 0:
            print(f"fno train {it}: loss {hist[-1]:.4e}")
    return hist


def learned_start(ctx, net, v0, dt: float = 0.0):
    """v_0 for the next step of ctx from its history and the network, written into the
    device float64 tensor v0 (fch_fno_learned_start: dt = 0 for the open adaptive
    run's next trial, dt > 0 for a fixed step of size dt)"""
    ctx.fno_learned_start(net, v0, dt)
    return v0


def run_adaptive_learned(ctx, scheme, sigma, t_final, device, net=None, k_range=None, max_trials=100000):
    """The adaptive run of Sec. 3.2 trial by trial, each trial from the network's v_0
    (net given, trial size in k_range when given) or the plain trial: for PSD v_0 is the
    first iterate of the iteration (fch_adaptive_enqueue_psd_from), for IMEX and SAV the
    extrapolation u* of the trial (fch_adaptive_enqueue_from). The network's inputs are
    normalised and carry no step size, so outside the step sizes it was trained on its
    correction does not scale with the step: k_range limits it to those. The host reads
    each trial's size (fch_adaptive_trial_info) to choose; v_0 is formed on the device.
    Returns (stats, trials, learned trials)."""
    import torch

    n = ctx.n
    ctx.adaptive_begin(scheme, sigma, t_final)
    v0 = torch.empty((n, n), dtype=torch.float64, device=device)
    trials = learned = 0
    while trials < max_trials:
        k, g, done = ctx.adaptive_trial_info()
        if done:
            break
        if net is None or g == 0.0 or (k_range is not None and not (k_range[0] <= k <= k_range[1])):
            ctx.adaptive_enqueue(1)
        else:
            ctx.fno_learned_start(net, v0)
            if scheme == "psd":
                ctx.adaptive_enqueue_psd_from(v0)
            else:
                ctx.adaptive_enqueue_from(v0)
            learned += 1
        trials += 1
    return ctx.adaptive_end(), trials, learned


def run_adaptive_psd(ctx, sigma, t_final, device, net=None, k_range=None, max_trials=100000):
    """run_adaptive_learned for PSD-BDF2 (the learned first iterate of Sec. 3.3)"""
    return run_adaptive_learned(ctx, "psd", sigma, t_final, device, net, k_range, max_trials)
