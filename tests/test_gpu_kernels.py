"""The sweep's launch paths give identical results.

- the TMA-staged sweep and the register sweep are bitwise equal (Block
  widths 32, 64 and 128; FP32, F16S and BF16S storage; BGK and TRT; forced;
  obstacles and moving walls);
- a TMA sweep whose staged data never arrives reports LBM_ETIMEOUT through
  its bounded waits instead of hanging, and the library stays usable.
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
