"""Learned warm start for steady flow through sphere-packed channels.

1. Training data: n^3 channels (periodic x and z, walls at -y/+y, one sphere
   packing and one body force each) solved by the batched sweep until each
   instance's velocity change per step, measured over the (even) check
   interval, is below tol (lbm_run_to_residual_each with interval residuals:
   bounce-back on the spheres excites an undamped period-2 mode on which the
   one-step residual stalls);
   the steady (rho, u) become normalised targets (unet_targets_from_fields).
2. Training: the tensor-core U-Net (include/unet.h) fitted with Adam.
3. Use: the network's prediction for a new geometry becomes the solver's
   initial equilibrium (unet_fields_from_prediction, lbm_init_equilibrium_device),
   and the solver iterates to the same residual; the solver from rest stays
   the reference for the final fields.

Orchestration only: the solver, the network, the loss, the optimiser and the
field maps run in liblbm.so; torch provides device memory and streams.
Normalisation: Stokes flow is linear in the force, so targets are the fields
divided by the force F_k and by a velocity scale s_u (and s_rho = s_u / 3 for
the density): the mean fluid velocity per unit force over the first solved
chunk, from the library's FP64 per-instance momentum sums, which makes the
targets of order one.  The network's force input is F_k / F_REF.  A
prediction is smoothed once (unet_smooth_fields) before it becomes the
initial equilibrium: its short-wavelength error slows the solver more than
its smooth error.  Measured on held-out 32^3 and 64^3 channels, one pass and
a plain equilibrium start need the fewest steps; more passes, or a consistent
start (lbm_init_consistent_device, whose relaxation steps count), need more.
"""
from __future__ import annotations

import time

import numpy as np

from . import lbm as L
from . import unet as U
from . import workloads as W

TAU = 0.8
RHO0 = 1.0
F_REF = 5e-6


SMOOTH_PASSES = 1


def mean_velocity_per_force(ctx, forces):
    """Mean fluid velocity along x per unit force of every instance (FP64 sums)."""
    _, _, _, per = L.lbm_invariants(ctx, per_instance=True)
    mass = per[:, 0]
    return per[:, 1] / np.maximum(mass, 1e-300) / np.asarray(forces, np.float64)


def solve(flags, forces, n: int, tol: float = 1e-6, check_every: int = 50, max_steps: int = 200_000,
          init=None, storage: int = L.LBM_F32, consistent: int = 0):
    """Solves len(flags) channels of n^3 cells (one batch context) until each
    instance's residual is below tol.  init: optional device (rho, u) in the
    batch layout, set as equilibrium or, with consistent > 0, relaxed for that
    many steps to the prescribed velocity (lbm_init_consistent_device; those
    steps are counted).  Returns (ctx, steps per instance, residuals, seconds)."""
    import torch

    ctx = batch_context(flags, forces, n, storage)
    t0 = time.perf_counter()
    if init is not None:
        torch.cuda.synchronize()
        if consistent > 0:
            L.lbm_init_consistent_device(ctx, init[0], init[1], consistent)
        else:
            L.lbm_init_equilibrium_device(ctx, init[0], init[1])
    L.lbm_synchronize(ctx)
    steps, res = L.lbm_run_to_residual_each(ctx, tol, check_every, max_steps, interval=True)
    L.lbm_synchronize(ctx)
    if init is not None and consistent > 0:
        steps = np.where(steps >= 0, steps + consistent, steps)
    return ctx, steps, res, time.perf_counter() - t0


def batch_context(flags, forces, n: int, storage: int = L.LBM_F32):
    """One batch context of len(flags) n^3 channels with per-instance forces."""
    K = len(flags)
    p = L.make_params(storage=storage, storage_scale=256.0 if storage == L.LBM_F16S else 1.0, **W.channel_bc())
    ctx = L.lbm_batch_create([(n, n, n)] * K, [TAU] * K, [np.asarray(f, np.uint8) for f in flags], p)
    L.lbm_set_forces(ctx, np.stack([np.asarray(forces, np.float64), np.zeros(K), np.zeros(K)], axis=1))
    return ctx


def solve_handover(flags, forces, n: int, tol: float = 1e-6, switch_tol: float = 1e-4, check_every: int = 50,
                   max_steps_16: int = 20_000, max_steps: int = 200_000, init=None):
    """Shifted-FP16 storage until each instance's residual is below
    switch_tol, then the exact state handed over to FP32 storage
    (lbm_get_pdfs_device / lbm_set_pdfs_device) and iterated to tol.  FP16
    storage follows the FP32 residual down to ~1e-5 and stalls near 2e-6 (its
    rounding noise), so the hand-over keeps FP16's bandwidth for part of the
    steps and FP32's accuracy for the result.  The later the switch, the more
    FP32 steps the handed-over state needs: on 48 sphere-packed 64^3 channels
    a switch at 1e-4 took 871 steps in all (FP32 alone: 869), at 1e-5 918.  init as in solve (equilibrium
    start).  Both contexts are created before the clock starts.  Returns
    (FP32 ctx, total steps per instance, 16-bit steps, residuals, seconds)."""
    import torch

    K, V = len(flags), n ** 3
    c16 = batch_context(flags, forces, n, L.LBM_F16S)
    c32 = batch_context(flags, forces, n, L.LBM_F32)
    f = torch.empty(19 * K * V, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if init is not None:
        L.lbm_init_equilibrium_device(c16, init[0], init[1])
    L.lbm_synchronize(c16)
    s16, _ = L.lbm_run_to_residual_each(c16, switch_tol, check_every, max_steps_16, interval=True)
    s16 = np.where(s16 >= 0, s16, max_steps_16)
    L.lbm_get_pdfs_device(c16, f)
    L.lbm_synchronize(c16)
    L.lbm_set_pdfs_device(c32, f)
    L.lbm_synchronize(c32)
    s32, res = L.lbm_run_to_residual_each(c32, tol, check_every, max_steps, interval=True)
    L.lbm_synchronize(c32)
    sec = time.perf_counter() - t0
    c16.destroy()
    del f
    steps = np.where(s32 >= 0, s16 + s32, -1)
    return c32, steps, s16, res, sec


def fields(ctx, K: int, n: int):
    """Device (rho [K V], u [K 3 V]) of a batch context."""
    import torch

    V = n ** 3
    rho = torch.empty(K * V, dtype=torch.float32, device="cuda")
    u = torch.empty(3 * K * V, dtype=torch.float32, device="cuda")
    L.lbm_macroscopic_device(ctx, rho, u)
    L.lbm_synchronize(ctx)
    return rho, u


class Dataset:
    """Solid flags [N V] (uint8), forces [N], normalised targets [N V 4] on the device."""

    def __init__(self, n: int, N: int):
        import torch

        self.n, self.N, self.V = n, N, n ** 3
        self.solid = torch.empty(N * self.V, dtype=torch.uint8, device="cuda")
        self.target = torch.empty(N * self.V * 4, dtype=torch.float32, device="cuda")
        self.force = torch.empty(N, dtype=torch.float32, device="cuda")
        self.steps = np.zeros(N, np.int64)
        self.solve_seconds = 0.0
        self.s_u = None  # velocity scale of the targets
        self.s_rho = None


def make_dataset(seeds, n: int, chunk: int = 256, tol: float = 1e-6, check_every: int = 50,
                 max_steps: int = 200_000, samples=None, processes: int | None = None) -> Dataset:
    """Generates and solves the channels of `seeds` (in chunks of batch contexts)."""
    import torch

    samples = samples if samples is not None else W.channel_samples(seeds, n, processes)
    ds = Dataset(n, len(samples))
    V = ds.V
    stream = torch.cuda.current_stream()
    for a in range(0, ds.N, chunk):
        part = samples[a:a + chunk]
        K = len(part)
        flags = [f for f, _ in part]
        forces = [F for _, F in part]
        ctx, steps, _, sec = solve(flags, forces, n, tol, check_every, max_steps)
        ds.steps[a:a + K] = steps
        ds.solve_seconds += sec
        if ds.s_u is None:
            ds.s_u = float(np.mean(mean_velocity_per_force(ctx, forces)))
            ds.s_rho = ds.s_u / 3.0
        rho, u = fields(ctx, K, n)
        ctx.destroy()
        sl = slice(a * V, (a + K) * V)
        ds.solid[sl].copy_(torch.from_numpy(np.concatenate([f.reshape(-1) for f in flags])))
        ds.force[a:a + K].copy_(torch.tensor(forces, dtype=torch.float32))
        U.targets_from_fields(rho, u, ds.solid[sl], ds.force[a:a + K], K, V, RHO0, ds.s_rho, ds.s_u,
                              ds.target[a * V * 4:(a + K) * V * 4], stream)
        torch.cuda.synchronize()
    return ds


def train(net: U.UNet, ds: Dataset, epochs: int, lr: float = 2e-3, lr_final: float = 1e-4, seed: int = 0,
          log=None):
    """Adam over random minibatches of net.nb samples; cosine learning-rate decay.
    Returns the per-step losses."""
    import torch

    rng = np.random.default_rng(seed)
    nb, V = net.nb, ds.V
    solid = ds.solid.view(ds.N, V)
    target = ds.target.view(ds.N, V * 4)
    force = (ds.force.cpu().numpy() / F_REF).astype(np.float32)
    per_epoch = ds.N // nb
    total = max(1, epochs * per_epoch)
    losses = []
    step = 0
    for ep in range(epochs):
        order = rng.permutation(ds.N)
        for b in range(per_epoch):
            idx = order[b * nb:(b + 1) * nb]
            it = torch.from_numpy(idx).cuda()
            sb = solid.index_select(0, it).reshape(-1)
            tb = target.index_select(0, it).reshape(-1)
            a = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * step / total))
            torch.cuda.synchronize()
            losses.append(net.train_step(sb, force[idx], tb, float(a)))
            step += 1
        if log:
            log(f"epoch {ep}: loss {np.mean(losses[-per_epoch:]):.4e}")
    return losses


def predict(net: U.UNet, solid, forces, n: int, s_rho: float, s_u: float, smooth: int = SMOOTH_PASSES):
    """Predicted device (rho, u) in the batch layout for K = len(forces)
    samples (K a multiple of net.nb); solid: device uint8 [K V]; the scales
    of the training targets; `smooth` filter passes over u."""
    import torch

    K, V, nb = len(forces), n ** 3, net.nb
    if K % nb:
        raise ValueError("the number of samples must be a multiple of the network's batch")
    out = torch.empty(K * V * 4, dtype=torch.float32, device="cuda")
    fin = (np.asarray(forces, np.float64) / F_REF).astype(np.float32)
    for a in range(0, K, nb):
        net.predict(solid[a * V:(a + nb) * V], fin[a:a + nb], out[a * V * 4:(a + nb) * V * 4])
    rho = torch.empty(K * V, dtype=torch.float32, device="cuda")
    u = torch.empty(3 * K * V, dtype=torch.float32, device="cuda")
    fdev = torch.tensor(np.asarray(forces, np.float32), device="cuda")
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    U.fields_from_prediction(out, solid, fdev, K, V, RHO0, s_rho, s_u, rho, u, stream)
    if smooth:
        U.smooth_fields(u, solid, K, 3, n, smooth, stream)
    torch.cuda.synchronize()
    return rho, u
