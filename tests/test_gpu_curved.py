"""Curved resting walls (linear interpolated bounce-back) on the GPU, through
the C ABI.

- one step from random states on random geometries with random wall
  distances on every link into a resting wall (cells and faces, thin gaps),
  beside moving and pressure boundaries: <= 2e-8 from the oracle; 40 steps
  from rest: <= 1e-5;
- an off-grid Poiseuille channel: the oracle's steady state within 1e-5;
- every register-sweep variant and a Block split: bitwise equal;
- bad links are refused and leave no distances set.
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


def _kind(flags, periodic, face_bc, x, y, z):
    """What lies at (x, y, z): periodic wrap, face walls (edges rest)."""
    nz, ny, nx = flags.shape
    pos, n = [x, y, z], [nx, ny, nz]
    beyond, face = 0, 0
    for a in range(3):
        if 0 <= pos[a] < n[a]:
            continue
        if periodic[a]:
            pos[a] %= n[a]
        else:
            beyond += 1
            face = 2 * a + (0 if pos[a] < 0 else 1)
    if beyond >= 2:
        return 1
    if beyond == 1:
        return face_bc[face]
    return int(flags[pos[2], pos[1], pos[0]])


def _links(rng, flags, periodic, face_bc, lo=0.05, hi=1.0):
    """Random float32-exact distances on every pull from a resting wall."""
    e, _, _ = oracle.lattice()
    nz, ny, nx = flags.shape
    cells, dirs, qs = [], [], []
    qw = np.full((19,) + flags.shape, 0.5)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if flags[z, y, x] != 0:
                    continue
                for i in range(1, 19):
                    if _kind(flags, periodic, face_bc, x - e[i, 0], y - e[i, 1], z - e[i, 2]) != 1:
                        continue
                    q = float(np.float32(rng.uniform(lo, hi)))
                    cells.append(x + nx * (y + ny * z))
                    dirs.append(i)
                    qs.append(q)
                    qw[i, z, y, x] = q
    return np.array(cells), np.array(dirs), np.array(qs), qw


def _problem(dims, tau, flags, kw, qw):
    return oracle.Problem(dims=dims, tau=tau, flags=flags, periodic=kw["periodic"], face_bc=kw["face_bc"],
                          collision=kw.get("collision", 0), magic=kw.get("magic", 3 / 16),
                          force=kw.get("force", (0, 0, 0)), wall_u=kw.get("wall_u", (0, 0, 0)),
                          rho_b=kw.get("rho_b"), qw=qw)


def _case(seed):
    rng = np.random.default_rng(3000 + seed)
    nb = rng.integers(1, 3, 3)
    bd = rng.integers(3, 25, 3)
    dims = tuple(int(v) for v in nb * bd)
    kw = dict(periodic=tuple(int(v) for v in rng.integers(0, 2, 3)),
              face_bc=tuple(int(v) for v in rng.choice([1, 1, 2, 3], 6)),
              collision=int(seed % 2), magic=float(rng.uniform(0.05, 0.3)),
              force=tuple(rng.uniform(-1e-3, 1e-3, 3)) if seed % 3 else (0.0, 0.0, 0.0),
              wall_u=tuple(rng.uniform(-0.05, 0.05, 3)), rho_b=float(rng.uniform(0.995, 1.005)))
    fl = W.random_flags(rng, dims, 0.2)
    fl[(fl == 2) & (rng.random(fl.shape) < 0.3)] = 3
    tau = float(rng.uniform(0.52, 1.8))
    return rng, dims, tuple(int(v) for v in bd), tau, fl, kw


@pytest.mark.parametrize("seed", range(6))
def test_one_step_with_curved_walls(L, seed):
    rng, dims, bd, tau, flags, kw = _case(seed)
    cells, dirs, qs, qw = _links(rng, flags, kw["periodic"], kw["face_bc"])
    assert len(cells) > 0 and (qs < 0.5).any() and (qs > 0.5).any()
    ctx = L.lbm_create(dims, bd, tau, flags, L.make_params(**kw))
    L.lbm_set_wall_distances(ctx, cells, dirs, qs)
    L.lbm_set_pdfs(ctx, W.random_pdfs(rng, dims, 1e-2, flags))
    f0 = L.lbm_get_pdfs(ctx).reshape((19,) + dims[::-1])
    L.lbm_step(ctx, 1)
    got = L.lbm_get_pdfs(ctx).reshape(f0.shape)
    ref = oracle.step(_problem(dims, tau, flags, kw, qw), f0)
    assert np.abs(got - ref).max() <= 2e-8
    ctx.destroy()


@pytest.mark.parametrize("seed", range(2))
def test_forty_steps_with_curved_walls(L, seed):
    rng, dims, bd, tau, flags, kw = _case(40 + seed)
    cells, dirs, qs, qw = _links(rng, flags, kw["periodic"], kw["face_bc"], 0.2, 1.0)
    ctx = L.lbm_create(dims, bd, tau, flags, L.make_params(**kw))
    L.lbm_set_wall_distances(ctx, cells, dirs, qs)
    L.lbm_step(ctx, 40)
    p = _problem(dims, tau, flags, kw, qw)
    ref = oracle.run(p, oracle.zeros(p), 40)
    assert np.abs(L.lbm_get_pdfs(ctx).reshape(ref.shape) - ref).max() <= 1e-5
    ctx.destroy()


def test_off_grid_poiseuille_channel(L):
    """Walls 0.25 below the first and 0.7 above the last fluid row."""
    dims, tau, steps = (32, 12, 4), 0.8, 1500
    e, _, _ = oracle.lattice()
    nx, ny, nz = dims
    cells, dirs, qs = [], [], []
    qw = np.full((19, nz, ny, nx), 0.5)
    for z in range(nz):
        for x in range(nx):
            for i in range(1, 19):
                for y, want, q in ((0, 1, 0.25), (ny - 1, -1, 0.7)):
                    if e[i, 1] == want:
                        cells.append(x + nx * (y + ny * z))
                        dirs.append(i)
                        qs.append(q)
                        qw[i, z, y, x] = q
    kw = dict(periodic=(1, 0, 1), face_bc=(1,) * 6, collision=1, force=(1e-5, 0, 0))
    out = []
    for bd in (dims, (16, 6, 2)):
        ctx = L.lbm_create(dims, bd, tau, None, L.make_params(**kw))
        L.lbm_set_wall_distances(ctx, cells, dirs, qs)
        L.lbm_step(ctx, steps)
        out.append(L.lbm_get_pdfs(ctx))
        ctx.destroy()
    assert np.array_equal(out[0], out[1])
    p = _problem(dims, tau, None, kw, qw)
    ref = oracle.run(p, oracle.zeros(p), steps)
    assert np.abs(out[0].reshape(ref.shape) - ref).max() <= 1e-5


@pytest.mark.parametrize("storage", [0, 1])
def test_sweep_variants_bitwise_with_curved_walls(L, storage):
    rng = np.random.default_rng(50 + storage)
    dims, bd = (128, 24, 20), (64, 12, 10)
    flags = W.random_flags(rng, dims, 0.1)
    kw = dict(collision=1, force=(2e-5, 0, 1e-5), wall_u=(0.03, 0, 0.01), periodic=(1, 0, 1),
              face_bc=(1, 1, 1, 2, 1, 1), storage=storage, storage_scale=(256.0 if storage == 1 else 1.0))
    cells, dirs, qs, _ = _links(rng, flags, kw["periodic"], kw["face_bc"])
    f0 = W.random_pdfs(rng, dims, 1e-2, flags)
    R, U, R2, U2 = L.SWEEP_ROWS, L.SWEEP_RUNS, L.SWEEP_ROWS2, L.SWEEP_RUNS2
    configs = [(R, 32, 4, 1, 0, 4, 8, 0), (R, 32, 8, 2, 0, 3, 8, 1), (U, 256, 1, 1, 0, 4, 8, 0),
               (U, 128, 1, 1, 304, 3, 8, 1), (R2, 32, 4, 1, 0, 3, 8, 0), (R2, 32, 8, 2, 0, 4, 8, 1),
               (U2, 128, 1, 1, 0, 3, 8, 1), (U2, 256, 1, 1, 304, 4, 8, 0),
               # the 48-register budget falls back to the budget-4 kernels here
               (U, 128, 1, 1, 0, 5, 8, 1)]
    outs = []
    for cfg in configs:
        ctx = L.lbm_create(dims, bd, 0.7, flags, L.make_params(kernel=L.LBM_KERNEL_REGISTER, **kw))
        L.lbm_set_wall_distances(ctx, cells, dirs, qs)
        L.lbm_set_sweep_config(ctx, cfg)
        L.lbm_set_pdfs(ctx, f0)
        L.lbm_step(ctx, 20)
        outs.append(L.lbm_get_pdfs(ctx))
        ctx.destroy()
    for k, o in enumerate(outs[1:], 1):
        assert np.array_equal(o, outs[0]), (k, np.abs(o - outs[0]).max())


def test_bad_links_are_refused(L):
    dims = (16, 8, 4)
    flags = np.zeros(dims[::-1], np.uint8)
    kw = dict(periodic=(1, 0, 1))
    ctx = L.lbm_create(dims, dims, 0.8, flags, L.make_params(**kw))
    e, _, _ = oracle.lattice()
    up = int(np.flatnonzero((e[:, 1] == 1) & (e[:, 0] == 0) & (e[:, 2] == 0))[0])
    L.lbm_set_wall_distances(ctx, [3], [up], [0.3])  # row 0 pulls from the -y wall: fine
    for cells, dirs, q in (([3 + 16 * 4], [up], [0.3]),  # its source is fluid
                           ([3], [up], [1.5]), ([3], [0], [0.3]), ([10**6], [up], [0.3])):
        with pytest.raises(L.LBMError) as ei:
            L.lbm_set_wall_distances(ctx, cells, dirs, q)
        assert ei.value.code == L.LBM_EINVAL
    # nothing is left set after a refusal: the state follows half-way bounce-back
    L.lbm_set_pdfs(ctx, W.random_pdfs(np.random.default_rng(1), dims, 1e-2, flags))
    f0 = L.lbm_get_pdfs(ctx).reshape((19,) + dims[::-1])
    L.lbm_step(ctx, 1)
    p = oracle.Problem(dims=dims, tau=0.8, flags=flags, periodic=kw["periodic"])
    assert np.abs(L.lbm_get_pdfs(ctx).reshape(f0.shape) - oracle.step(p, f0)).max() <= 2e-8
    ctx.destroy()
    aa = L.lbm_create(dims, dims, 0.8, flags, L.make_params(streaming=L.LBM_STREAM_AA, **kw))
    with pytest.raises(L.LBMError):
        L.lbm_set_wall_distances(aa, [3], [up], [0.3])
    aa.destroy()
