"""Learned early exit: train the run-outcome network on trajectories the simulator
generates, pick a retire threshold, and integrate with retire-and-reseed.

Orchestration only: every step of the simulation, the features, the network's
forward and backward passes and the Adam updates run in the CUDA library
(through ``chym``); this module moves device pointers, shuffles mini-batch
indices and keeps counts.  PyTorch provides device buffers and index shuffling.

Schedule of one run: K steps, decision at local step k_dec (a divisor of K), with
a state snapshot at k_dec / 2 for the slope features.  In continuous mode every
slot of a context is always busy: the integration advances in chunks of k_dec
steps; after each chunk, slots that reached their decision step are scored and
retired when the logit is below the threshold, slots that reached K are harvested
(their Ising energy decides a ground-state hit), and both kinds restart from fresh
seeds (chym_reseed_device), so their local step starts again at 0.
"""
import time
from dataclasses import dataclass

import numpy as np

from . import chym, inputs


@dataclass
class Outcome:
    hits: int = 0
    completed: int = 0
    retired: int = 0
    run_steps: int = 0      # integration steps spent over all slots
    seconds: float = 0.0
    integrate_seconds: float = 0.0   # of `seconds`, spent in the integration calls

    @property
    def hits_per_mstep(self):
        return 1e6 * self.hits / max(self.run_steps, 1)

    @property
    def hits_per_second(self):
        return self.hits / max(self.seconds, 1e-12)


def _torch():
    import torch
    return torch


class SeedStream:
    """Fresh 64-bit run seeds from a SplitMix64 stream of one key."""

    def __init__(self, key):
        self.key = int(key)
        self.next = 0

    def take(self, n):
        out = inputs.run_seeds(self.key, n, offset=self.next)
        self.next += n
        return out


def generate(ctx, prm, sched, h, seeds, K, k_dec, E_gs, stream=0):
    """Run every seed to its decision step, record its features, finish it, label it.

    Returns (features [R, 24] device float32, labels [R] device float32, energies
    [R] host float64)."""
    torch = _torch()
    R = len(seeds)
    ctx.run(prm, h, seeds, k_dec // 2, sched, stream)
    el = ctx.N * ctx.D * R
    snap = torch.empty(el, dtype=torch.float64 if prm.prec == chym.PREC_FP64 else torch.float32,
                       device="cuda")
    ctx.copy_state_device(snap.data_ptr(), stream)
    ctx.run(prm, None, None, k_dec - k_dec // 2, sched, stream, n_runs=R)
    F = torch.empty(R, chym.N_FEATURES, dtype=torch.float32, device="cuda")
    ctx.features_device(snap.data_ptr(), k_dec / K, F.data_ptr(), stream)
    ctx.run(prm, None, None, K - k_dec, sched, stream, n_runs=R)
    E = ctx.energy(stream=stream)
    y = torch.from_numpy((np.abs(E - E_gs) <= 1e-9 * max(1.0, abs(E_gs))).astype(np.float32)).cuda()
    return F, y, E


def standardisation(F):
    """Per-feature mean and inverse standard deviation of the training rows."""
    mean = F.mean(0)
    istd = 1.0 / F.std(0).clamp_min(1e-6)
    return mean.cpu().numpy(), istd.cpu().numpy()


def train(net, F, y, epochs=30, batch=512, lr=2e-3, seed=0, stream=0):
    """Mini-batch Adam on the GPU; returns the mean loss of the last epoch."""
    torch = _torch()
    mean, istd = standardisation(F)
    net.set_params(None, mean, istd)
    g = torch.Generator(device="cpu").manual_seed(seed)
    R = F.shape[0]
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for _ in range(epochs):
        perm = torch.randperm(R, generator=g).cuda()
        Fp, yp = F[perm].contiguous(), y[perm].contiguous()
        for b0 in range(0, R - batch + 1, batch):
            net.train_step_device(Fp[b0:].data_ptr(), yp[b0:].data_ptr(), batch, lr, loss.data_ptr(),
                                  stream)
        torch.cuda.synchronize()
    return float(loss.item())


def logits(net, F, stream=0):
    torch = _torch()
    out = torch.empty(F.shape[0], dtype=torch.float32, device="cuda")
    net.forward_device(F.data_ptr(), F.shape[0], out.data_ptr(), stream)
    return out


def expected_gain(fn, rho, k_frac):
    """Ground-state hits per integration step with the exit over those without it,
    when a fraction rho of the runs is retired at the fraction k_frac of the
    schedule and a fraction fn of the successful runs is among them."""
    return (1.0 - fn) / (1.0 - (1.0 - k_frac) * rho)


def threshold_for_fn(scores, labels, fn_target):
    """Largest threshold whose false-negative rate (successful runs scored below it)
    stays at or below fn_target."""
    pos = np.sort(scores[labels > 0.5])
    if len(pos) == 0:
        return -np.inf
    k = int(np.floor(fn_target * len(pos)))
    return float(pos[k]) if k < len(pos) else float(pos[-1])


def continuous(ctx, prm, sched, h, R, seed_stream, K, k_dec, E_gs, chunks, net=None,
               theta=-np.inf, stream=0):
    """Integrate R slots (R a multiple of len(h)), every slot always busy, for `chunks`
    chunks of k_dec steps.  With a network, slots at their decision step whose logit
    is below theta are retired.  Restarted slots take the next pump values of the
    grid in turn, so the time a retirement saves is spent on fresh runs of every
    pump, not only of the retired run's own pump.  Returns an Outcome."""
    return continuous_many([ctx], [prm], [sched], [h], [R], [seed_stream], K, k_dec, [E_gs],
                           chunks, net, theta, stream)


def continuous_many(ctxs, prms, scheds, hs, Rs, seed_streams, K, k_dec, E_gss, chunks,
                    net=None, theta=-np.inf, stream=0, batch=None, burn_in=0, trace=None):
    """`continuous` over several contexts at once (one network and threshold for all;
    the features carry N, D and h).  With `batch` (a chym.Batch over ctxs) every chunk
    of steps is one batched integration of all contexts.  The first `burn_in` chunks
    run uncounted and untimed, so that the counted window starts from slots already
    spread over their schedules (and after first-call costs).  `theta` is one
    threshold or one per context.  With a `trace` list, every chunk appends (chunk,
    context, decisions, retired, completed, hits).

    The bookkeeping of a chunk stays on the device (local steps, energies, features,
    logits, restart masks and their ordered indices) and meets the host once: one
    copy of all counts, after which the fresh seeds and pump indices of the restarted
    slots go up in one pinned copy and the reseeds are queued."""
    import contextlib
    torch = _torch()
    n = len(ctxs)
    thetas = list(theta) if np.ndim(theta) else [theta] * n
    gated = [net is not None and th > -np.inf for th in thetas]
    # the device-side bookkeeping runs on the library's stream
    cur = torch.cuda.current_stream()
    if stream == cur.cuda_stream:
        on = contextlib.nullcontext()
    elif not stream:
        on = torch.cuda.stream(torch.cuda.default_stream())
    else:
        on = torch.cuda.stream(torch.cuda.ExternalStream(stream))
    with on:
        torch.cuda.synchronize()
        per = []
        for ctx, prm, sched, h, R, ss in zip(ctxs, prms, scheds, hs, Rs, seed_streams):
            ctx.run(prm, h, ss.take(R), 0, sched, stream)
            dt = torch.float64 if prm.prec == chym.PREC_FP64 else torch.float32
            per.append(dict(
                next_h=0, order=torch.empty(R, dtype=torch.int32, device="cuda"),
                snap=torch.empty(ctx.N * ctx.D * R, dtype=dt, device="cuda"),
                F=torch.empty(R, chym.N_FEATURES, dtype=torch.float32, device="cuda"),
                L=torch.empty(R, dtype=torch.float32, device="cuda"),
                E=torch.empty(R, dtype=torch.float64, device="cuda")))
        counts_d = torch.zeros(n, 5, dtype=torch.int64, device="cuda")
        R_all = sum(Rs)
        up_seeds = torch.empty(R_all, dtype=torch.int64).pin_memory()
        up_pumps = torch.empty(R_all, dtype=torch.int32).pin_memory()
        d_seeds = torch.empty(R_all, dtype=torch.int64, device="cuda")
        d_pumps = torch.empty(R_all, dtype=torch.int32, device="cuda")
        spans = []

        def advance(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            if batch is not None:
                batch.run(prms, scheds, steps, stream)
            else:
                for ctx, prm, sched, R in zip(ctxs, prms, scheds, Rs):
                    ctx.run(prm, None, None, steps, sched, stream, n_runs=R)
            e1.record()
            spans.append((e0, e1))

        out = Outcome()
        t0 = time.perf_counter()
        for ci in range(burn_in + chunks):
            if ci == burn_in:   # start of the counted window
                torch.cuda.synchronize()
                out = Outcome()
                spans.clear()
                t0 = time.perf_counter()
            if any(gated):      # snapshot at half the decision step for the slope features
                advance(k_dec // 2)
                for ctx, st, g in zip(ctxs, per, gated):
                    if g:
                        ctx.copy_state_device(st["snap"].data_ptr(), stream)
                advance(k_dec - k_dec // 2)
            else:
                advance(k_dec)
            for i in range(n):
                ctx, R, st = ctxs[i], Rs[i], per[i]
                out.run_steps += R * k_dec
                ctx.energy_device(st["E"].data_ptr(), 0, stream)
                d_logits = 0
                if gated[i]:
                    ctx.features_device(st["snap"].data_ptr(), k_dec / K, st["F"].data_ptr(), stream)
                    net.forward_device(st["F"].data_ptr(), R, st["L"].data_ptr(), stream)
                    d_logits = st["L"].data_ptr()
                # the decision pass on the device: counts, and the restarted slots first in
                # increasing slot order
                ctx.exit_scan_device(st["E"].data_ptr(), E_gss[i], d_logits,
                                     thetas[i] if gated[i] else 0.0, K, k_dec,
                                     counts_d[i].data_ptr(), st["order"].data_ptr(), stream)
            orders = [st["order"] for st in per]
            c = counts_d.cpu().numpy()   # the chunk's one meeting with the host
            base, todo = 0, []
            for i in range(n):
                n_dec, n_ret, n_done, n_hit, m = (int(v) for v in c[i])
                out.hits += n_hit
                out.completed += n_done
                out.retired += n_ret
                if trace is not None:
                    trace.append((ci, i, n_dec, n_ret, n_done, n_hit))
                if m:
                    n_h, st = len(hs[i]), per[i]
                    up_seeds[base:base + m] = torch.from_numpy(seed_streams[i].take(m).view(np.int64))
                    up_pumps[base:base + m] = torch.from_numpy(
                        ((st["next_h"] + np.arange(m)) % n_h).astype(np.int32))
                    st["next_h"] = (st["next_h"] + m) % n_h
                    todo.append((i, base, m))
                    base += m
            if base:
                d_seeds[:base].copy_(up_seeds[:base], non_blocking=True)
                d_pumps[:base].copy_(up_pumps[:base], non_blocking=True)
                for i, b0, m in todo:
                    ctxs[i].reseed_device(orders[i].data_ptr(), m, d_seeds[b0:].data_ptr(),
                                          prms[i].init_std, d_pumps[b0:].data_ptr(), stream)
        torch.cuda.synchronize()
        out.seconds = time.perf_counter() - t0
        out.integrate_seconds = sum(e0.elapsed_time(e1) for e0, e1 in spans) / 1e3
    return out
