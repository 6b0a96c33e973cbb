"""The fluid-cell list layout (indirect addressing) on the GPU, through the C ABI.

The list sweep pulls the same operands and runs the same collision as the
Block sweeps, so, for every storage format:

- bitwise equal to the Block layout after 1, 2, 5, 13 and 30 steps on random
  geometries (Blocks along every axis, periodic and walled faces, solid,
  moving and pressure cells, forcing, BGK and TRT), with equal moments,
  invariants and residuals, graph replay and tuning included;
- less device memory than the Block layout in a porous medium.
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


GEOMS = [
    ((64, 24, 20), (32, 12, 10), (1, 0, 1), (1, 1, 2, 3, 1, 1)),
    ((64, 24, 20), (32, 12, 10), (0, 1, 0), (2, 3, 1, 1, 3, 2)),
    ((40, 18, 12), (20, 9, 6), (1, 1, 1), (1, 1, 1, 1, 1, 1)),
    ((33, 10, 14), (33, 5, 7), (0, 1, 0), (1, 3, 2, 1, 1, 3)),
]


def _flags(rng, dims):
    fl = W.random_flags(rng, dims, 0.3)
    fl[(fl != 0) & (rng.random(fl.shape) < 0.2)] = 3
    return fl


@pytest.mark.parametrize("storage", [0, 1, 2, 3])
@pytest.mark.parametrize("k", range(len(GEOMS)))
def test_bitwise_equal_to_blocks(L, k, storage):
    dims, bd, periodic, face_bc = GEOMS[k]
    rng = np.random.default_rng(900 + 10 * k + storage)
    flags = _flags(rng, dims)
    kw = dict(periodic=periodic, face_bc=face_bc, collision=k % 2, magic=float(rng.uniform(0.05, 0.3)),
              force=tuple(rng.uniform(-1e-3, 1e-3, 3)) if k % 3 else (0.0, 0.0, 0.0),
              wall_u=tuple(rng.uniform(-0.05, 0.05, 3)), rho_b=float(rng.uniform(0.995, 1.005)),
              storage=storage, storage_scale=256.0 if storage in (1, 2) else 1.0)
    tau = float(rng.uniform(0.52, 1.5))
    blk = L.lbm_create(dims, bd, tau, flags, L.make_params(**kw))
    lst = L.lbm_create(dims, bd, tau, flags, L.make_params(layout=L.LBM_LAYOUT_SPARSE, **kw))
    info = L.lbm_get_info(lst)
    assert info.layout == L.LBM_LAYOUT_SPARSE and info.list_cells == int((flags == 0).sum())
    assert info.exchange_pdfs == 0
    f0 = W.random_pdfs(rng, dims, 1e-2, flags)
    L.lbm_set_pdfs(blk, f0)
    L.lbm_set_pdfs(lst, f0)
    for n in (1, 1, 3, 8, 17):
        L.lbm_step(blk, n)
        L.lbm_step(lst, n)
        a, b = L.lbm_get_pdfs(blk), L.lbm_get_pdfs(lst)
        assert np.array_equal(a, b), (n, np.abs(a - b).max())
    r1, u1 = L.lbm_macroscopic(blk)
    r2, u2 = L.lbm_macroscopic(lst)
    assert np.array_equal(r1, r2) and np.array_equal(u1, u2)
    m1, j1, _ = L.lbm_invariants(blk)
    m2, j2, _ = L.lbm_invariants(lst)
    assert m1 == m2 and np.array_equal(j1, j2)
    assert L.lbm_residual(blk) == L.lbm_residual(lst)
    blk.destroy()
    lst.destroy()


def test_oracle_graphs_tuning_and_memory(L):
    dims, bd = (48, 40, 32), (24, 20, 16)
    rng = np.random.default_rng(77)
    flags = W.overlapping_spheres(rng, dims, 0.45)
    kw = dict(periodic=(1, 0, 1), force=(1e-5, 0, 0))
    p = oracle.Problem(dims=dims, tau=0.8, flags=flags, periodic=kw["periodic"], force=kw["force"])
    lst = L.lbm_create(dims, bd, 0.8, flags, L.make_params(layout=L.LBM_LAYOUT_SPARSE, **kw))
    nog = L.lbm_create(dims, bd, 0.8, flags, L.make_params(layout=L.LBM_LAYOUT_SPARSE, graph_steps=-1, **kw))
    blk = L.lbm_create(dims, bd, 0.8, flags, L.make_params(**kw))
    # fewer bytes than storing every cell, at this porosity
    assert L.lbm_get_info(lst).device_bytes < 0.95 * L.lbm_get_info(blk).device_bytes
    L.lbm_autotune(lst)
    for c in (lst, nog):
        L.lbm_step(c, 3)
        L.lbm_step(c, 60)
    got = L.lbm_get_pdfs(lst)
    assert np.array_equal(got, L.lbm_get_pdfs(nog))
    ref = oracle.run(p, oracle.zeros(p), 63)
    assert np.abs(got.reshape(ref.shape) - ref).max() <= 1e-5
    s, r = L.lbm_run_to_residual(lst, 0.0, 10, 20)
    assert s == 20 and np.isfinite(r)
    for c in (lst, nog, blk):
        c.destroy()
