"""In-place (AA-pattern) streaming on the GPU, through the C ABI.

The in-place scheme keeps one PDF array and alternates a pull-and-push step
with a local step; it computes the same update as the two-array sweep, so:

- FP32: bitwise equal to the two-array sweep after every number of steps, odd
  (the state read back from the streamed layout) and even (read through the
  swapped slots), on random geometries with resting, moving and pressure
  boundaries, forcing, BGK and TRT, split into Blocks along every axis,
  periodic or walled, Block widths that are and are not multiples of 32;
- macroscopic fields, invariants, the residual loop, writes at odd times
  (set, equilibrium, imposed velocity), CUDA-graph replay and the autotuner
  give the two-array results;
- 16-bit and FP64 storage: within the storage's rounding of the oracle;
- half the PDF memory.
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


def _flags(rng, dims, frac, pressure):
    fl = W.random_flags(rng, dims, frac)
    if pressure:
        fl[(fl != 0) & (rng.random(fl.shape) < 0.4)] = 3
    return fl


# (dims, block dims, periodic, face_bc): Blocks along every axis, widths
# that are multiples of 32 (row tiles) and not (runs of cells)
GEOMS = [
    ((64, 24, 20), (32, 12, 10), (1, 0, 1), (1, 1, 2, 3, 1, 1)),
    ((64, 24, 20), (32, 12, 10), (0, 1, 0), (2, 3, 1, 1, 3, 2)),
    ((40, 18, 12), (20, 9, 6), (1, 1, 1), (1, 1, 1, 1, 1, 1)),
    ((40, 18, 12), (40, 18, 12), (0, 0, 0), (3, 2, 1, 3, 2, 1)),
    ((96, 16, 8), (32, 16, 8), (0, 0, 1), (2, 3, 1, 1, 1, 1)),
    ((33, 10, 14), (33, 5, 7), (0, 1, 0), (1, 3, 2, 1, 1, 3)),
]


def _kw(rng, k, periodic, face_bc, **extra):
    kw = dict(periodic=periodic, face_bc=face_bc, collision=k % 2, magic=float(rng.uniform(0.05, 0.3)),
              force=tuple(rng.uniform(-1e-3, 1e-3, 3)) if k % 3 else (0.0, 0.0, 0.0),
              wall_u=tuple(rng.uniform(-0.05, 0.05, 3)), rho_b=float(rng.uniform(0.995, 1.005)),
              kernel=1)
    kw.update(extra)
    return kw


def _pair(L, dims, bd, tau, flags, kw):
    two = L.lbm_create(dims, bd, tau, flags, L.make_params(**kw))
    aa = L.lbm_create(dims, bd, tau, flags, L.make_params(streaming=L.LBM_STREAM_AA, **kw))
    return two, aa


@pytest.mark.parametrize("k", range(len(GEOMS)))
def test_fp32_bitwise_equal_to_two_arrays_every_step(L, k):
    dims, bd, periodic, face_bc = GEOMS[k]
    rng = np.random.default_rng(700 + k)
    flags = _flags(rng, dims, 0.12, pressure=k % 2 == 0)
    kw = _kw(rng, k, periodic, face_bc)
    tau = float(rng.uniform(0.52, 1.5))
    two, aa = _pair(L, dims, bd, tau, flags, kw)
    f0 = W.random_pdfs(rng, dims, 1e-2, flags)
    L.lbm_set_pdfs(two, f0)
    L.lbm_set_pdfs(aa, f0)
    assert np.array_equal(L.lbm_get_pdfs(two), L.lbm_get_pdfs(aa))
    done = 0
    for n in (1, 1, 2, 3, 6, 11):
        L.lbm_step(two, n)
        L.lbm_step(aa, n)
        done += n
        info = L.lbm_get_info(aa)
        assert info.streaming == L.LBM_STREAM_AA and info.aa_phase == done % 2
        a, b = L.lbm_get_pdfs(two), L.lbm_get_pdfs(aa)
        assert np.array_equal(a, b), (done, np.abs(a - b).max())
    # moments and invariants at an odd and an even time
    for n in (1, 1):
        L.lbm_step(two, n)
        L.lbm_step(aa, n)
        r1, u1 = L.lbm_macroscopic(two)
        r2, u2 = L.lbm_macroscopic(aa)
        assert np.array_equal(r1, r2) and np.array_equal(u1, u2)
        m1, j1, _ = L.lbm_invariants(two)
        m2, j2, _ = L.lbm_invariants(aa)
        assert m1 == m2 and np.array_equal(j1, j2)
    two.destroy()
    aa.destroy()


def test_matches_the_oracle_and_holds_half_the_memory(L):
    dims, bd = (64, 24, 20), (32, 12, 10)
    rng = np.random.default_rng(11)
    flags = _flags(rng, dims, 0.1, pressure=True)
    kw = _kw(rng, 1, (1, 0, 0), (2, 3, 1, 1, 1, 1))
    two, aa = _pair(L, dims, bd, 0.8, flags, kw)
    # one PDF array instead of two; its rows carry two more padding columns,
    # which weigh on Blocks this narrow, so the half shows on a wide one
    assert L.lbm_get_info(aa).device_bytes < 0.7 * L.lbm_get_info(two).device_bytes
    big = [L.lbm_create((256, 32, 32), (256, 32, 32), 0.8, None, L.make_params(streaming=s)) for s in (0, 1)]
    assert L.lbm_get_info(big[1]).device_bytes < 0.55 * L.lbm_get_info(big[0]).device_bytes
    for c in big:
        c.destroy()
    L.lbm_step(aa, 41)
    p = oracle.Problem(dims=dims, tau=0.8, flags=flags, periodic=kw["periodic"], face_bc=kw["face_bc"],
                       collision=kw["collision"], magic=kw["magic"], force=kw["force"], wall_u=kw["wall_u"],
                       rho_b=kw["rho_b"])
    ref = oracle.run(p, oracle.zeros(p), 41)
    got = L.lbm_get_pdfs(aa).reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-5
    two.destroy()
    aa.destroy()


@pytest.mark.parametrize("storage,tol", [(1, 4e-5), (2, 3e-4), (3, 1e-12)])
def test_other_storage_formats_against_the_oracle(L, storage, tol):
    dims, bd = (40, 18, 12), (20, 9, 6)
    rng = np.random.default_rng(20 + storage)
    flags = _flags(rng, dims, 0.1, pressure=True)
    kw = _kw(rng, storage, (0, 1, 0), (2, 3, 1, 1, 3, 1), storage=storage,
             storage_scale=(256.0 if storage in (1, 2) else 1.0))
    aa = L.lbm_create(dims, bd, 0.7, flags, L.make_params(streaming=L.LBM_STREAM_AA, **kw))
    p = oracle.Problem(dims=dims, tau=0.7, flags=flags, periodic=kw["periodic"], face_bc=kw["face_bc"],
                       collision=kw["collision"], magic=kw["magic"], force=kw["force"], wall_u=kw["wall_u"],
                       rho_b=kw["rho_b"])
    f = oracle.zeros(p)
    for n in (7, 8):  # an odd and an even time
        L.lbm_step(aa, n)
        f = oracle.run(p, f, n)
        got = L.lbm_get_pdfs(aa).reshape(f.shape)
        assert np.abs(got - f).max() <= tol, (n, np.abs(got - f).max())
    aa.destroy()


def test_graphs_writes_at_odd_times_residual_loop_and_autotune(L):
    dims, bd = (64, 24, 20), (32, 12, 10)
    rng = np.random.default_rng(31)
    flags = _flags(rng, dims, 0.1, pressure=True)
    kw = _kw(rng, 2, (1, 0, 1), (1, 1, 2, 3, 1, 1))
    kw.pop("kernel")
    two, aa = _pair(L, dims, bd, 0.9, flags, kw)
    nog = L.lbm_create(dims, bd, 0.9, flags, L.make_params(streaming=L.LBM_STREAM_AA, graph_steps=-1, **kw))
    f0 = W.random_pdfs(rng, dims, 1e-2, flags)
    for c in (two, aa, nog):
        L.lbm_set_pdfs(c, f0)
    # odd calls around graph replays (the default graph length is even)
    for n in (3, 30, 7):
        for c in (two, aa, nog):
            L.lbm_step(c, n)
    ref = L.lbm_get_pdfs(two)
    assert np.array_equal(ref, L.lbm_get_pdfs(aa)) and np.array_equal(ref, L.lbm_get_pdfs(nog))
    # at an odd time: equilibrium, then an imposed velocity
    rho = (1.0 + 1e-3 * rng.standard_normal(dims[::-1])).astype(np.float32)
    u = (1e-2 * rng.standard_normal((3,) + dims[::-1])).astype(np.float32)
    import torch

    ut = torch.from_numpy(u).cuda()
    for c in (two, aa):
        L.lbm_step(c, 1)  # 41 steps: aa at an odd time
        L.lbm_init_equilibrium(c, rho, u)
        L.lbm_step(c, 5)
        assert c is two or L.lbm_get_info(c).aa_phase == 1
        L.lbm_impose_velocity_device(c, ut)
        L.lbm_step(c, 4)
    assert np.array_equal(L.lbm_get_pdfs(two), L.lbm_get_pdfs(aa))
    # the residual loop: the same steps and (up to summation order) residual
    s2, r2 = L.lbm_run_to_residual(two, 0.0, 10, 40)
    sa, ra = L.lbm_run_to_residual(aa, 0.0, 10, 40)
    assert s2 == sa == 40 and abs(ra / r2 - 1) < 1e-3
    assert np.array_equal(L.lbm_get_pdfs(two), L.lbm_get_pdfs(aa))
    with pytest.raises(L.LBMError):
        L.lbm_residual(aa)
    # tuning leaves the state where it was, and the tuned sweep gives the same steps
    L.lbm_step(aa, 1)
    before = L.lbm_get_pdfs(aa)
    L.lbm_autotune(aa)
    assert np.array_equal(before, L.lbm_get_pdfs(aa))
    cfg = L.lbm_get_sweep_config(aa)
    assert cfg[0] in (0, 2) and cfg[7] == 0
    L.lbm_step(two, 1)
    L.lbm_step(two, 9)
    L.lbm_step(aa, 9)
    assert np.array_equal(L.lbm_get_pdfs(two), L.lbm_get_pdfs(aa))
    for c in (two, aa, nog):
        c.destroy()


@pytest.mark.parametrize("cfg", [(0, 64, 2, 2, 0, 4, 8, 0), (2, 256, 1, 1, 0, 3, 8, 0),
                                 (3, 32, 4, 1, 0, 3, 8, 0), (4, 128, 1, 1, 608, 4, 8, 0)])
def test_every_sweep_configuration_gives_the_same_steps(L, cfg):
    """One and two cells per thread, row tiles and runs, a persistent grid:
    the in-place steps stay bitwise equal to the two-array sweep."""
    dims, bd, periodic, face_bc = GEOMS[0]
    rng = np.random.default_rng(808)
    flags = _flags(rng, dims, 0.12, pressure=True)
    kw = _kw(rng, 1, periodic, face_bc)
    two, aa = _pair(L, dims, bd, 0.9, flags, kw)
    L.lbm_set_sweep_config(aa, cfg)
    assert tuple(L.lbm_get_sweep_config(aa)) == cfg
    f0 = W.random_pdfs(rng, dims, 1e-2, flags)
    L.lbm_set_pdfs(two, f0)
    L.lbm_set_pdfs(aa, f0)
    for n in (1, 4, 7):
        L.lbm_step(two, n)
        L.lbm_step(aa, n)
        assert np.array_equal(L.lbm_get_pdfs(two), L.lbm_get_pdfs(aa)), n
    two.destroy()
    aa.destroy()
