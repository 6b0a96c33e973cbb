"""Pressure boundaries (anti-bounce-back to rho_b) on the GPU, through the C ABI.

- one step from random states on random geometries with pressure cells and
  pressure faces next to resting and moving walls: <= 2e-8 from the oracle
  (a few FP32 roundings), 40 steps from rest: <= 1e-5;
- the TMA sweep and every register-sweep variant (one and two cells per
  thread, row tiles, runs, persistent grids, both near-wall strategies):
  bitwise equal, FP32 and shifted FP16;
- a velocity-inlet / pressure-outlet channel split into Blocks: bitwise equal
  to the single Block, and within 1e-5 of the oracle after 300 steps;
- a uniform flow through pressure faces and past pressure cells stays put
  (the velocity correction makes it a fixed point of the rule).
"""
import numpy as np
import pytest

import oracle
from paper_1007_1388_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1388_gb300 import build

    build.build()
    import paper_1007_1388_gb300 as L

    L.use_torch_allocator()
    oracle.build()
    return L


def _flags_with_pressure(rng, dims, frac):
    fl = W.random_flags(rng, dims, frac)
    fl[(fl != 0) & (rng.random(fl.shape) < 0.4)] = 3
    return fl


def _case(seed):
    rng = np.random.default_rng(2000 + seed)
    nb = rng.integers(1, 3, 3)
    bd = rng.integers(3, 33, 3)
    dims = tuple(int(v) for v in nb * bd)
    kw = dict(periodic=tuple(int(v) for v in rng.integers(0, 2, 3)),
              face_bc=tuple(int(v) for v in rng.integers(1, 4, 6)),
              collision=int(seed % 2), magic=float(rng.uniform(0.05, 0.3)),
              force=tuple(rng.uniform(-1e-3, 1e-3, 3)) if seed % 3 else (0.0, 0.0, 0.0),
              wall_u=tuple(rng.uniform(-0.05, 0.05, 3)), rho_b=float(rng.uniform(0.995, 1.005)))
    tau = float(rng.uniform(0.52, 1.8))
    return rng, dims, tuple(int(v) for v in bd), tau, _flags_with_pressure(rng, dims, 0.15), kw


def _problem(dims, tau, flags, kw):
    return oracle.Problem(dims=dims, tau=tau, flags=flags, periodic=kw["periodic"], face_bc=kw["face_bc"],
                          collision=kw.get("collision", 0), magic=kw.get("magic", 3 / 16),
                          force=kw.get("force", (0, 0, 0)), wall_u=kw.get("wall_u", (0, 0, 0)),
                          rho_b=kw.get("rho_b"))


def _state(L, ctx, dims):
    nx, ny, nz = dims
    return L.lbm_get_pdfs(ctx).reshape(19, nz, ny, nx)


@pytest.mark.parametrize("seed", range(6))
def test_one_step_with_pressure_boundaries(L, seed):
    rng, dims, bd, tau, flags, kw = _case(seed)
    assert (flags == 3).any()
    ctx = L.lbm_create(dims, bd, tau, flags, L.make_params(**kw))
    L.lbm_set_pdfs(ctx, W.random_pdfs(rng, dims, 1e-2, flags))
    f0 = _state(L, ctx, dims)
    L.lbm_step(ctx, 1)
    got = _state(L, ctx, dims)
    ref = oracle.step(_problem(dims, tau, flags, kw), f0)
    assert np.abs(got - ref).max() <= 2e-8
    ctx.destroy()


@pytest.mark.parametrize("seed", range(2))
def test_forty_steps_with_pressure_boundaries(L, seed):
    rng, dims, bd, tau, flags, kw = _case(40 + seed)
    ctx = L.lbm_create(dims, bd, tau, flags, L.make_params(**kw))
    L.lbm_step(ctx, 40)
    p = _problem(dims, tau, flags, kw)
    ref = oracle.run(p, oracle.zeros(p), 40)
    assert np.abs(_state(L, ctx, dims) - ref).max() <= 1e-5
    ctx.destroy()


@pytest.mark.parametrize("storage", [0, 1])
def test_sweep_variants_bitwise_with_pressure(L, storage):
    rng = np.random.default_rng(5 + storage)
    dims, bd = (128, 24, 20), (64, 12, 10)
    flags = _flags_with_pressure(rng, dims, 0.1)
    f0 = W.random_pdfs(rng, dims, 1e-2, flags)
    kw = dict(collision=1, force=(2e-5, 0, 1e-5), wall_u=(0.03, 0, 0.01), periodic=(1, 0, 0),
              face_bc=(1, 1, 2, 3, 3, 1), rho_b=1.003, storage=storage,
              storage_scale=(256.0 if storage == 1 else 1.0))
    R, U, R2, U2 = L.SWEEP_ROWS, L.SWEEP_RUNS, L.SWEEP_ROWS2, L.SWEEP_RUNS2
    configs = [(R, 32, 4, 1, 0, 4, 8, 0), (R, 32, 8, 2, 0, 3, 8, 1), (U, 256, 1, 1, 0, 4, 8, 0),
               (U, 128, 1, 1, 304, 3, 8, 1), (R2, 32, 4, 1, 0, 3, 8, 0), (R2, 32, 8, 2, 0, 4, 8, 1),
               (U2, 128, 1, 1, 0, 3, 8, 1), (U2, 256, 1, 1, 304, 4, 8, 0),
               # the 48-register budget falls back to the budget-4 kernels here
               (U, 128, 1, 1, 0, 5, 8, 1)]
    outs = []
    for cfg in configs:
        ctx = L.lbm_create(dims, bd, 0.7, flags, L.make_params(kernel=L.LBM_KERNEL_REGISTER, **kw))
        L.lbm_set_sweep_config(ctx, cfg)
        L.lbm_set_pdfs(ctx, f0)
        L.lbm_step(ctx, 20)
        outs.append(L.lbm_get_pdfs(ctx))
        ctx.destroy()
    ctx = L.lbm_create(dims, bd, 0.7, flags, L.make_params(kernel=L.LBM_KERNEL_TMA, **kw))
    assert L.lbm_get_info(ctx).kernel == L.LBM_KERNEL_TMA
    L.lbm_set_pdfs(ctx, f0)
    L.lbm_step(ctx, 20)
    outs.append(L.lbm_get_pdfs(ctx))
    ctx.destroy()
    for k, o in enumerate(outs[1:], 1):
        assert np.array_equal(o, outs[0]), (k, np.abs(o - outs[0]).max())


def test_inlet_outlet_channel_blocks_and_oracle(L):
    """Velocity inlet (moving-wall face at -x) and pressure outlet (+x) on a
    channel with walls at -y/+y, periodic z."""
    dims, tau, steps = (64, 16, 8), 0.8, 300
    kw = dict(periodic=(0, 0, 1), face_bc=(2, 3, 1, 1, 1, 1), wall_u=(0.02, 0, 0), rho_b=1.0,
              collision=1)
    out = []
    for bd in (dims, (16, 8, 4)):
        ctx = L.lbm_create(dims, bd, tau, None, L.make_params(**kw))
        L.lbm_step(ctx, steps)
        out.append(_state(L, ctx, dims))
        ctx.destroy()
    assert np.array_equal(out[0], out[1])
    p = _problem(dims, tau, None, kw)
    ref = oracle.run(p, oracle.zeros(p), steps)
    assert np.abs(out[0] - ref).max() <= 1e-5
    # the inlet drives the flow: mass enters and leaves through the x faces
    rho, u = oracle.macroscopic(p, ref)
    assert u[0].mean() > 1e-3


@pytest.mark.parametrize("coll", [0, 1])
def test_uniform_flow_through_pressure_boundaries_stays_put(L, coll):
    rng = np.random.default_rng(9)
    dims = (32, 12, 10)
    flags = np.zeros(dims[::-1], np.uint8)
    flags[rng.random(flags.shape) < 0.05] = 3
    rho_b, u = 1.003, np.array([0.03, -0.02, 0.01])
    e, w, _ = oracle.lattice()
    eu = e @ u
    feq = (w * ((rho_b - 1.0) + 3 * eu + 4.5 * eu**2 - 1.5 * u @ u)).astype(np.float32)
    f0 = np.broadcast_to(feq[:, None, None, None], (19,) + dims[::-1]) * (flags == 0)
    kw = dict(periodic=(0, 1, 1), face_bc=(3, 3, 1, 1, 1, 1), rho_b=rho_b, collision=coll)
    ctx = L.lbm_create(dims, (16, 6, 10), 0.7, flags, L.make_params(**kw))
    L.lbm_set_pdfs(ctx, f0)
    L.lbm_step(ctx, 30)
    got = _state(L, ctx, dims)
    ctx.destroy()
    # FP32 roundoff of the collision and the boundary term only
    assert np.abs(got - f0).max() <= 2e-7
