"""The sweep's launch paths give identical results.

- the TMA-staged sweep and the register sweep are bitwise equal (Block
  widths 32, 64 and 128; FP32, F16S and BF16S storage; BGK and TRT; forced;
  obstacles and moving walls);
- a TMA sweep whose staged data never arrives reports LBM_ETIMEOUT through
  its bounded waits instead of hanging, and the library stays usable;
- the register sweep's variants (row tiles, runs of consecutive cells, one or
  two cells per thread, persistent grids, register budgets, near-wall cells by
  per-lane branch or by link masks under a warp vote) are bitwise equal on
  ragged, walled, porous and batched geometries.
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


def _run(L, dims, bd, tau, flags, steps, f0=None, **kw):
    ctx = L.lbm_create(dims, bd, tau, flags, L.make_params(**kw))
    info = L.lbm_get_info(ctx)
    if f0 is not None:
        L.lbm_set_pdfs(ctx, f0)
    L.lbm_step(ctx, steps)
    f = L.lbm_get_pdfs(ctx)
    ctx.destroy()
    return f, info


@pytest.mark.parametrize("bx,storage", [(64, 0), (32, 0), (128, 0), (64, 1), (64, 2), (32, 1)])
def test_tma_sweep_equals_register_sweep(L, bx, storage):
    rng = np.random.default_rng(bx + storage)
    by = 256 // bx * 3
    dims = (2 * bx, 2 * by, 20)
    flags = W.random_flags(rng, dims, 0.08)
    f0 = W.random_pdfs(rng, dims, 1e-2, flags)
    for coll in (0, 1):
        kw = dict(collision=coll, force=(2e-5, -1e-5, 0), wall_u=(0.03, 0, 0.01),
                  periodic=(1, 0, 1), face_bc=(1, 1, 2, 1, 1, 1), storage=storage,
                  storage_scale=(256.0 if storage == 1 else 1.0))
        a, ia = _run(L, dims, (bx, by, 10), 0.7, flags, 25, f0, kernel=L.LBM_KERNEL_TMA, **kw)
        b, ib = _run(L, dims, (bx, by, 10), 0.7, flags, 25, f0, kernel=L.LBM_KERNEL_REGISTER, **kw)
        assert ia.kernel == L.LBM_KERNEL_TMA and ib.kernel == L.LBM_KERNEL_REGISTER
        assert np.array_equal(a, b), (coll, np.abs(a - b).max())


def test_tma_sweep_matches_oracle_and_walls_in_x(L):
    """Non-periodic x (walls beyond the Patch's x faces) and periodic y."""
    rng = np.random.default_rng(4)
    dims = (128, 8, 12)
    flags = W.random_flags(rng, dims, 0.1)
    kw = dict(collision=1, force=(0, 1e-4, 0), periodic=(0, 1, 0),
              face_bc=(2, 1, 1, 1, 1, 2), wall_u=(0, 0.02, 0.01))
    f, info = _run(L, dims, (64, 4, 6), 0.8, flags, 30, kernel=L.LBM_KERNEL_TMA, **kw)
    assert info.kernel == L.LBM_KERNEL_TMA
    p = oracle.Problem(dims=dims, tau=0.8, flags=flags, **kw)
    ref = oracle.run(p, oracle.zeros(p), 30)
    assert np.abs(f.reshape(ref.shape) - ref).max() <= 1e-5


def test_tma_sweep_bounded_wait_reports_timeout(L):
    dims = (64, 8, 16)
    p = L.make_params(periodic=(1, 1, 1), kernel=L.LBM_KERNEL_TMA,
                      debug_flags=L.LBM_DEBUG_DROP_STAGE, graph_steps=-1)
    ctx = L.lbm_create(dims, dims, 0.8, None, p)
    L.lbm_step(ctx, 1)
    with pytest.raises(L.LBMError) as ei:
        L.lbm_synchronize(ctx)
    assert ei.value.code == L.LBM_ETIMEOUT
    ctx.destroy()
    # the device and the library remain usable
    f, info = _run(L, dims, dims, 0.8, None, 5, periodic=(1, 1, 1), kernel=L.LBM_KERNEL_TMA)
    assert info.kernel == L.LBM_KERNEL_TMA and np.all(f == 0.0)


# -------------------------------------------------- register sweep variants
def _configs(L, bx):
    """Row tiles, runs of consecutive cells, persistent grids, the register
    budgets (64, 80 and, one cell per thread, 48 registers) and both near-wall
    strategies."""
    R, U, R2, U2 = L.SWEEP_ROWS, L.SWEEP_RUNS, L.SWEEP_ROWS2, L.SWEEP_RUNS2
    out = [(R, 32, 4, 1, 0, 4, 8, 0), (R, 32, 8, 2, 0, 3, 8, 1), (U, 256, 1, 1, 0, 4, 8, 0),
           (U, 128, 1, 1, 0, 3, 8, 1), (U, 256, 1, 1, 304, 4, 8, 1), (R, 32, 4, 2, 152, 3, 8, 0),
           (R2, 32, 4, 1, 0, 3, 8, 0), (R2, 32, 8, 2, 0, 4, 8, 1), (U2, 128, 1, 1, 0, 3, 8, 1),
           (U2, 256, 1, 1, 304, 4, 8, 0), (U, 128, 1, 1, 0, 5, 8, 1), (R, 32, 4, 2, 0, 5, 8, 0)]
    if bx >= 64:
        out.append((R, 64, 4, 4, 0, 4, 8, 1))
    return out


def _run_cfg(L, ctx, f0, steps, cfg):
    if cfg is not None:
        L.lbm_set_sweep_config(ctx, cfg)
        assert tuple(L.lbm_get_sweep_config(ctx)) == tuple(cfg)
    L.lbm_set_pdfs(ctx, f0)
    L.lbm_step(ctx, steps)
    return L.lbm_get_pdfs(ctx)


@pytest.mark.parametrize("storage", [0, 1])
def test_sweep_variants_bitwise_single_patch(L, storage):
    """A ragged Patch (Block width 40) with obstacles, moving walls and force."""
    rng = np.random.default_rng(71 + storage)
    dims, bd = (80, 24, 20), (40, 12, 10)
    flags = W.random_flags(rng, dims, 0.15)
    f0 = W.random_pdfs(rng, dims, 1e-2, flags)
    for coll in (0, 1):
        p = L.make_params(collision=coll, force=(2e-5, 0, 1e-5), wall_u=(0.04, 0, 0.01),
                          periodic=(1, 0, 0), face_bc=(1, 1, 1, 2, 1, 1), storage=storage,
                          storage_scale=(256.0 if storage == 1 else 1.0))
        ctx = L.lbm_create(dims, bd, 0.62, flags, p)
        info = L.lbm_get_info(ctx)
        # the default for even Blocks that are not a multiple of 64 wide: runs, two cells per
        # thread; one cell per thread where near-wall cells are many (link masks)
        assert info.flat == 128 and info.pair == (0 if info.mask else 1)
        # FP32 one-cell runs take the 48-register budget, 16-bit storage 64 registers
        assert L.lbm_get_sweep_config(ctx)[5] == (5 if info.mask and storage == 0 else 4)
        ref = _run_cfg(L, ctx, f0, 17, None)
        for cfg in _configs(L, bd[0]):
            got = _run_cfg(L, ctx, f0, 17, cfg)
            assert np.array_equal(ref, got), (coll, cfg, np.abs(ref - got).max())
        ctx.destroy()


def test_sweep_variants_bitwise_batch(L):
    """Uneven sphere-packed channels in one batch."""
    rng = np.random.default_rng(5)
    inst = []
    for _ in range(4):
        dims = tuple(int(v) for v in rng.integers(10, 45, 3))
        inst.append((dims, float(rng.uniform(0.55, 1.2)), W.sphere_packing(rng, dims, 0.75, 2, 4)))
    p = L.make_params(force=(1e-4, 0, 0), **W.channel_bc())
    ctx = L.lbm_batch_create([d for d, _, _ in inst], [t for _, t, _ in inst],
                             [f for _, _, f in inst], p)
    assert L.lbm_get_info(ctx).mask == 1  # sphere packings: many near-wall cells
    f0 = np.concatenate([W.random_pdfs(rng, d, 1e-2, f).reshape(-1) for d, _, f in inst])
    ref = _run_cfg(L, ctx, f0, 13, None)
    even = all(d[0] % 2 == 0 for d, _, _ in inst)
    for cfg in _configs(L, 32):
        if cfg[0] >= L.SWEEP_ROWS2 and not even:
            with pytest.raises(L.LBMError):
                L.lbm_set_sweep_config(ctx, cfg)
            continue
        got = _run_cfg(L, ctx, f0, 13, cfg)
        assert np.array_equal(ref, got), (cfg, np.abs(ref - got).max())
    ctx.destroy()


def test_sweep_config_validation(L):
    # 40 cells wide: the TMA sweep does not apply, so kind 1 is invalid too
    ctx = L.lbm_create((40, 16, 8), (40, 16, 8), 0.7, None, L.make_params())
    before = L.lbm_get_sweep_config(ctx)
    for bad in [(5, 32, 4, 1, 0, 4, 8, 0), (0, 48, 4, 1, 0, 4, 8, 0), (0, 32, 16, 1, 0, 4, 8, 0),
                (2, 100, 1, 1, 0, 4, 8, 0), (0, 32, 4, 1, -1, 4, 8, 0), (0, 32, 4, 1, 0, 6, 8, 0),
                (3, 32, 4, 1, 0, 5, 8, 0),
                (0, 32, 4, 1, 0, 4, 8, 2), (1, 32, 4, 1, 0, 4, 8, 0)]:
        with pytest.raises(L.LBMError):
            L.lbm_set_sweep_config(ctx, bad)
        assert L.lbm_get_sweep_config(ctx) == before
    ctx.destroy()


def test_graph_direct_and_profiled_steps_agree(L):
    """Multi-Block steps through graph replay, direct launches and the
    profiled path (events around the exchange and the sweep) agree bitwise,
    and the profile counts one exchange and one sweep per step."""
    import numpy as np

    from paper_1007_1388_gb300 import workloads as W

    dims, bd = (64, 32, 32), (32, 16, 16)
    rng = np.random.default_rng(12)
    flags = W.random_flags(rng, dims, 0.1)
    f0 = W.random_pdfs(rng, dims, 1e-2, flags)
    kw = dict(periodic=(1, 1, 1), force=(1e-5, 0, 0), collision=1)
    outs = []
    for graph_steps, prof in ((0, False), (-1, False), (-1, True)):
        ctx = L.lbm_create(dims, bd, 0.8, flags, L.make_params(graph_steps=graph_steps, **kw))
        L.lbm_set_pdfs(ctx, f0)
        L.lbm_profile_enable(ctx, prof)
        L.lbm_step(ctx, 33)
        if prof:
            pr = L.lbm_profile_read(ctx)
            assert pr.sweep_launches == 33 and pr.exchange_launches == 33
            assert pr.sweep_ms > 0 and pr.exchange_ms > 0
        outs.append(L.lbm_get_pdfs(ctx))
        ctx.destroy()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("storage", [1, 2])
def test_two_cell_16bit_open_rows_bitwise(L, storage):
    """16-bit storage without obstacles, where whole warps take the two-cell
    sweep's vector path (one aligned pair load for the directions with
    e_x = 0, two 2-byte loads for the others): equal to the one-cell sweep bit
    for bit for row tiles narrower and wider than a warp, runs that wrap rows
    inside a warp, Blocks across x faces (periodic and a wall), moving walls."""
    R, U2, R2 = L.SWEEP_ROWS, L.SWEEP_RUNS2, L.SWEEP_ROWS2
    rng = np.random.default_rng(90 + storage)
    for dims, bd, periodic in [((128, 24, 20), (64, 12, 10), (1, 0, 1)), ((96, 16, 12), (48, 16, 6), (0, 0, 1)),
                               ((40, 18, 14), (20, 9, 14), (1, 1, 0))]:
        f0 = W.random_pdfs(rng, dims, 1e-2)
        kw = dict(force=(2e-5, -1e-5, 1e-5), wall_u=(0.03, 0, 0.01), periodic=periodic,
                  face_bc=(1, 1, 2, 1, 1, 1), storage=storage, storage_scale=(256.0 if storage == 1 else 1.0))
        ctx = L.lbm_create(dims, bd, 0.7, None, L.make_params(**kw))
        ref = _run_cfg(L, ctx, f0, 9, (R, 32, 4, 1, 0, 4, 8, 0))
        for cfg in [(R2, 32, 4, 1, 0, 4, 8, 0), (R2, 32, 8, 2, 0, 3, 8, 0), (U2, 128, 1, 1, 0, 4, 8, 0),
                    (U2, 256, 1, 1, 304, 3, 8, 0), (R2, 32, 2, 1, 0, 4, 8, 1), (U2, 64, 1, 1, 0, 4, 8, 1)]:
            got = _run_cfg(L, ctx, f0, 9, cfg)
            assert np.array_equal(got, ref), (dims, cfg, float(np.abs(got - ref).max()))
        ctx.destroy()
