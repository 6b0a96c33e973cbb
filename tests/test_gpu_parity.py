"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 arithmetic and storage unless stated):
- multi-step runs: max |f~_gpu - f~_oracle| <= 1e-5 (the stated PDF bound);
- one step from a given state: 2e-8 absolute on PDFs of magnitude <= 1e-2,
  i.e. a few FP32 roundings of the 19-term sums;
- FP64 storage: 1e-13;
- multi-Block vs single-Block, graph vs direct launch, autotuned vs default
  tiles: bitwise equal.
"""
import numpy as np
import pytest

import oracle
from paper_1007_1388_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_MULTISTEP = 1e-5
TOL_ONESTEP = 2e-8


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


def _gpu_params(L, **kw):
    return L.make_params(**kw)


def _orc_problem(dims, tau, flags, kw):
    return oracle.Problem(dims=dims, tau=tau, flags=flags,
                          periodic=kw.get("periodic", (0, 0, 0)),
                          face_bc=kw.get("face_bc", (1,) * 6),
                          collision=kw.get("collision", 0), magic=kw.get("magic", 3 / 16),
                          rho0=kw.get("rho0", 1.0), force=kw.get("force", (0, 0, 0)),
                          wall_u=kw.get("wall_u", (0, 0, 0)))


def _state(L, ctx, dims):
    nx, ny, nz = dims
    return L.lbm_get_pdfs(ctx).reshape(19, nz, ny, nx)


# --------------------------------------------------------------- config 1
def test_cavity_32_bgk_200_steps(L):
    """32^3 lid-driven cavity, tau 0.6, lid 0.05 along x on +y, from rest."""
    n, tau, steps = 32, 0.6, 200
    kw = dict(wall_u=(0.05, 0, 0), **W.cavity_bc())
    ctx = L.lbm_create((n,) * 3, (n,) * 3, tau, None, _gpu_params(L, **kw))
    L.lbm_step(ctx, steps)
    f = _state(L, ctx, (n,) * 3)
    p = _orc_problem((n,) * 3, tau, None, kw)
    ref = oracle.run(p, oracle.zeros(p), steps)
    err = np.abs(f - ref).max()
    assert err <= TOL_MULTISTEP, err
    rho, u = L.lbm_macroscopic(ctx)
    rr, ur = oracle.macroscopic(p, ref)
    assert np.abs(u - ur.reshape(-1)).max() < 1e-5
    assert np.abs(rho - rr.reshape(-1)).max() < 1e-5
    ctx.destroy()


# ------------------------------------------------------ one-step parity
def _random_case(seed):
    rng = np.random.default_rng(1000 + seed)
    nb = rng.integers(1, 4, 3)
    bd = rng.integers(3, 41, 3)
    dims = tuple(int(v) for v in nb * bd)
    kw = dict(periodic=tuple(int(v) for v in rng.integers(0, 2, 3)),
              face_bc=tuple(int(v) for v in rng.integers(1, 3, 6)),
              collision=int(seed % 2), magic=float(rng.uniform(0.05, 0.3)),
              force=tuple(rng.uniform(-1e-3, 1e-3, 3)) if seed % 3 else (0.0, 0.0, 0.0),
              wall_u=tuple(rng.uniform(-0.05, 0.05, 3)))
    tau = float(rng.uniform(0.52, 1.8))
    flags = W.random_flags(rng, dims, 0.15)
    return rng, dims, tuple(int(v) for v in bd), tau, flags, kw


@pytest.mark.parametrize("seed", range(10))
def test_one_step_from_random_state(L, seed):
    rng, dims, bd, tau, flags, kw = _random_case(seed)
    ctx = L.lbm_create(dims, bd, tau, flags, _gpu_params(L, **kw))
    f0 = W.random_pdfs(rng, dims, 1e-2, flags)
    L.lbm_set_pdfs(ctx, f0)
    f0 = _state(L, ctx, dims)  # the FP32-rounded state the GPU holds
    L.lbm_step(ctx, 1)
    got = _state(L, ctx, dims)
    p = _orc_problem(dims, tau, flags, kw)
    ref = oracle.step(p, f0)
    assert np.abs(got - ref).max() <= TOL_ONESTEP
    # invariants and residual of the same pair of states, in FP64 on the GPU
    m, j, bad = L.lbm_invariants(ctx)
    mr, jr = oracle.invariants(p, got)
    assert bad == 0
    assert abs(m - mr) <= 1e-12 * abs(mr)
    # FP64 sums over ~1e5 cells in different orders: relative 1e-11
    assert np.abs(j - jr).max() <= 1e-11 * max(1.0, np.abs(jr).max())
    # the residual forms each cell's velocity and its change in FP32 (the
    # norms accumulate in FP64): a few FP32 roundings, relative 1e-5
    r = L.lbm_residual(ctx)
    assert abs(r - oracle.residual(p, f0, got)) <= 1e-5 * r
    # moments of the stored state
    rho, u = L.lbm_macroscopic(ctx)
    rr, ur = oracle.macroscopic(p, got)
    assert np.abs(rho - rr.reshape(-1)).max() <= 2e-7
    assert np.abs(u - ur.reshape(-1)).max() <= 1e-7
    ctx.destroy()


@pytest.mark.parametrize("seed", range(4))
def test_multi_step_random_geometry(L, seed):
    rng, dims, bd, tau, flags, kw = _random_case(50 + seed)
    ctx = L.lbm_create(dims, bd, tau, flags, _gpu_params(L, **kw))
    L.lbm_step(ctx, 40)
    p = _orc_problem(dims, tau, flags, kw)
    ref = oracle.run(p, oracle.zeros(p), 40)
    assert np.abs(_state(L, ctx, dims) - ref).max() <= TOL_MULTISTEP
    ctx.destroy()


# ------------------------------------------------- multi-block = single
def test_multiblock_equals_single_block_bitwise(L):
    rng = np.random.default_rng(77)
    dims = (48, 32, 40)
    flags = W.random_flags(rng, dims, 0.05)
    for coll in (0, 1):
        kw = dict(collision=coll, force=(1e-5, 2e-6, 0), wall_u=(0.02, 0, 0.01),
                  periodic=(1, 0, 1), face_bc=(1, 1, 1, 2, 1, 1))
        runs = []
        for bd in [(48, 32, 40), (16, 16, 8), (24, 8, 20), (12, 32, 5)]:
            ctx = L.lbm_create(dims, bd, 0.7, flags, _gpu_params(L, **kw))
            L.lbm_step(ctx, 60)
            runs.append(_state(L, ctx, dims))
            ctx.destroy()
        for r in runs[1:]:
            assert np.array_equal(r, runs[0])


def test_fully_periodic_multiblock_against_oracle(L):
    rng = np.random.default_rng(5)
    dims = (24, 18, 30)
    kw = dict(periodic=(1, 1, 1), collision=1, force=(1e-4, -5e-5, 2e-5))
    ctx = L.lbm_create(dims, (8, 6, 10), 0.9, None, _gpu_params(L, **kw))
    f0 = W.random_pdfs(rng, dims, 1e-2)
    L.lbm_set_pdfs(ctx, f0)
    f0 = _state(L, ctx, dims)
    L.lbm_step(ctx, 25)
    p = _orc_problem(dims, 0.9, None, kw)
    assert np.abs(_state(L, ctx, dims) - oracle.run(p, f0, 25)).max() <= TOL_MULTISTEP


# ------------------------------------------------ launch-path invariance
def test_graph_direct_profiled_and_autotuned_runs_are_identical(L):
    dims = (40, 24, 36)
    kw = dict(periodic=(1, 0, 1), force=(2e-5, 0, 0), collision=1)
    outs = []
    for mode in ("graph", "direct", "profile", "autotune"):
        p = _gpu_params(L, graph_steps=(-1 if mode == "direct" else 4), **kw)
        ctx = L.lbm_create(dims, (20, 12, 18), 0.8, None, p)
        if mode == "profile":
            L.lbm_profile_enable(ctx, True)
        L.lbm_step(ctx, 7)
        if mode == "autotune":
            L.lbm_autotune(ctx)
        L.lbm_step(ctx, 10)
        if mode == "profile":
            prof = L.lbm_profile_read(ctx)
            assert prof.sweep_launches == 17 and prof.exchange_launches == 17
            assert prof.sweep_ms > 0
        outs.append(_state(L, ctx, dims))
        ctx.destroy()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


# ------------------------------------------------------------- storage
def _bf16_round(x):
    """Round-to-nearest-even of float32 values to bfloat16, back to float64."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("storage", [0, 1, 2, 3])
def test_set_get_roundtrip_rounds_as_documented(L, storage):
    rng = np.random.default_rng(3)
    dims = (12, 10, 9)
    scale = 256.0 if storage in (1, 2) else 1.0
    ctx = L.lbm_create(dims, (6, 5, 9), 0.7, None,
                       _gpu_params(L, storage=storage, storage_scale=scale))
    f = W.random_pdfs(rng, dims, 1e-2)
    L.lbm_set_pdfs(ctx, f)
    got = _state(L, ctx, dims)
    if storage == 0:
        exp = f.astype(np.float32).astype(np.float64)
    elif storage == 1:
        # the kernel rounds to FP32 first, then to the storage format
        exp = (f * scale).astype(np.float32).astype(np.float16).astype(np.float64) / scale
    elif storage == 2:
        exp = _bf16_round((f * scale).astype(np.float32)) / scale
    else:
        exp = f
    assert np.array_equal(got, exp)
    ctx.destroy()


def test_f64_storage_matches_oracle_tightly(L):
    n, tau = 16, 0.6
    kw = dict(wall_u=(0.05, 0, 0), storage=3, **W.cavity_bc())
    ctx = L.lbm_create((n,) * 3, (8, 16, 4), tau, None, _gpu_params(L, **kw))
    L.lbm_step(ctx, 100)
    p = _orc_problem((n,) * 3, tau, None, kw)
    assert np.abs(_state(L, ctx, (n,) * 3) - oracle.run(p, oracle.zeros(p), 100)).max() <= 1e-13
    ctx.destroy()


@pytest.mark.parametrize("storage,scale,tol_u", [(1, 1.0, 2e-4), (1, 256.0, 2e-4), (2, 1.0, 2e-3)])
def test_shifted_half_storage_cavity_error(L, storage, scale, tol_u):
    """Shifted FP16 / BF16 storage with FP32 arithmetic: the velocity error of
    a 32^3 cavity after 200 steps stays within the bound derived from the
    storage mantissa (11 / 8 bits) relative to the lid speed 0.05."""
    n, tau, steps = 32, 0.6, 200
    kw = dict(wall_u=(0.05, 0, 0), **W.cavity_bc())
    ctx = L.lbm_create((n,) * 3, (n,) * 3, tau, None,
                       _gpu_params(L, storage=storage, storage_scale=scale, **kw))
    L.lbm_step(ctx, steps)
    _, u = L.lbm_macroscopic(ctx)
    p = _orc_problem((n,) * 3, tau, None, kw)
    _, ur = oracle.macroscopic(p, oracle.run(p, oracle.zeros(p), steps))
    err = np.abs(u - ur.reshape(-1)).max()
    print(f"storage {storage} scale {scale}: max |du| = {err:.3e}")
    assert err <= tol_u
    ctx.destroy()


# -------------------------------------------------------------- batches
def test_batch_of_uneven_instances_matches_oracle(L):
    rng = np.random.default_rng(9)
    inst = []
    for k in range(5):
        dims = tuple(int(v) for v in rng.integers(5, 40, 3))
        tau = float(rng.uniform(0.55, 1.2))
        inst.append((dims, tau, W.sphere_packing(rng, dims, 0.8, 1, 3)))
    kw = dict(force=(1e-4, 0, 0), collision=1, **W.channel_bc())
    ctx = L.lbm_batch_create([d for d, _, _ in inst], [t for _, t, _ in inst],
                             [f for _, _, f in inst], _gpu_params(L, **kw))
    L.lbm_step(ctx, 30)
    f = L.lbm_get_pdfs(ctx)
    _, _, _, per = L.lbm_invariants(ctx, per_instance=True)
    off = 0
    for k, (dims, tau, flags) in enumerate(inst):
        nx, ny, nz = dims
        n = nx * ny * nz
        fk = f[off:off + 19 * n].reshape(19, nz, ny, nx)
        off += 19 * n
        p = _orc_problem(dims, tau, flags, kw)
        ref = oracle.run(p, oracle.zeros(p), 30)
        assert np.abs(fk - ref).max() <= TOL_MULTISTEP, k
        m, j = oracle.invariants(p, fk)
        assert abs(per[k, 0] - m) <= 1e-12 * m
        assert np.abs(per[k, 1:4] - j).max() <= 1e-11 * max(1.0, np.abs(j).max())
    ctx.destroy()


# ------------------------------------------------------------ edge cases
def test_edge_cases(L):
    # all solid: nothing to update, fields at rest
    ctx = L.lbm_create((8, 8, 8), (4, 4, 4), 0.7, np.ones(512, np.uint8), _gpu_params(L))
    L.lbm_step(ctx, 3)
    rho, u = L.lbm_macroscopic(ctx)
    assert np.all(rho == 1.0) and np.all(u == 0.0)
    m, _, _ = L.lbm_invariants(ctx)
    assert m == 0.0
    ctx.destroy()
    # one-cell thick periodic axes and one-cell blocks
    for dims, bd in [((1, 16, 1), (1, 16, 1)), ((3, 3, 3), (1, 1, 1)), ((2, 6, 1), (1, 3, 1))]:
        kw = dict(periodic=(1, 0, 1), force=(1e-4, 0, 0), collision=1)
        ctx = L.lbm_create(dims, bd, 0.8, None, _gpu_params(L, **kw))
        L.lbm_step(ctx, 50)
        p = _orc_problem(dims, 0.8, None, kw)
        assert np.abs(_state(L, ctx, dims) - oracle.run(p, oracle.zeros(p), 50)).max() <= 1e-6
        ctx.destroy()
    # a NaN is detected by the FP64 reduction and stops run_to_residual
    ctx = L.lbm_create((8, 8, 8), (8, 8, 8), 0.7, None, _gpu_params(L, periodic=(1, 1, 1)))
    f = np.zeros(19 * 512)
    f[5 * 512 + 17] = np.nan
    L.lbm_set_pdfs(ctx, f)
    assert L.lbm_invariants(ctx)[2] == 1.0
    with pytest.raises(L.LBMError) as ei:
        L.lbm_run_to_residual(ctx, 1e-6, 5, 50)
    assert ei.value.code == L.LBM_ENUMERIC
    # residual needs a previous state
    L.lbm_set_pdfs(ctx, np.zeros(19 * 512))
    with pytest.raises(L.LBMError):
        L.lbm_residual(ctx)
    ctx.destroy()
    # a block too large for 32-bit plane offsets is rejected
    with pytest.raises(L.LBMError) as ei:
        L.lbm_create((1024, 1024, 1024), (1024, 1024, 1024), 0.7, None, _gpu_params(L))
    assert ei.value.code == L.LBM_EINVAL


def test_init_equilibrium_from_random_fields(L):
    rng = np.random.default_rng(12)
    dims = (8, 12, 6)
    kw = dict(force=(1e-5, 0, 0), collision=1, **W.channel_bc())
    ctx = L.lbm_create(dims, (8, 6, 6), 0.8, None, _gpu_params(L, **kw))
    rho = (1 + rng.uniform(-1e-3, 1e-3, 8 * 12 * 6)).astype(np.float32)
    u = rng.uniform(-1e-2, 1e-2, 3 * 8 * 12 * 6).astype(np.float32)
    L.lbm_init_equilibrium(ctx, rho, u)
    p = _orc_problem(dims, 0.8, None, kw)
    ref = oracle.init_equilibrium(p, rho.astype(np.float64), u.astype(np.float64))
    assert np.abs(_state(L, ctx, dims) - ref).max() <= 1e-9
    # random velocity noise on an even periodic grid excites a non-decaying
    # period-2 (staggered) mode of the discrete scheme: the oracle shows the
    # same one-step residual, which therefore never falls
    L.lbm_step(ctx, 500)
    f = oracle.run(p, ref, 499)
    r_ref = oracle.residual(p, f, oracle.step(p, f))
    assert abs(L.lbm_residual(ctx) - r_ref) <= 1e-4 * r_ref
    ctx.destroy()


def test_run_to_residual_from_smooth_start(L):
    dims = (8, 12, 6)
    kw = dict(force=(1e-5, 0, 0), collision=1, **W.channel_bc())
    ctx = L.lbm_create(dims, (8, 6, 6), 0.8, None, _gpu_params(L, **kw))
    steps, r = L.lbm_run_to_residual(ctx, 1e-6, 10, 20000)
    assert r < 1e-6 and steps % 10 == 0
    _, uu = L.lbm_macroscopic(ctx)
    H, nu = 12, 0.1
    y = np.arange(H) + 0.5
    prof = uu[:8 * 12 * 6].reshape(6, 12, 8)[:, :, :].mean(axis=(0, 2))
    ua = 1e-5 / (2 * nu) * y * (H - y)
    # converged to within the one-step residual criterion of the parabola
    assert np.abs(prof - ua).max() < 2e-3 * ua.max()
    ctx.destroy()
