"""Full-size body-force channel: 256^3 cells in 4x4x4 Blocks of 64^3 with the
on-device ghost exchange, periodic along x and z, resting walls at -y/+y,
tau 0.8, force 1e-6 along x, 2000 steps, FP32 (the launch configuration the
benchmark times).

Checked at full size by what holds at any size, and cell by cell where the
oracle can afford it:
- the 64-Block run equals the single-Block run bitwise (BGK and TRT);
- the velocity profile follows the analytic start-up series of plane
  Poiseuille flow within 1% of its maximum;
- 4096 sampled cells of one further step equal the oracle's update of the
  same cells from the GPU's own state (one-step FP32 tolerance).
"""
import numpy as np
import pytest

import oracle
from paper_1007_1388_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, B, TAU, FORCE, STEPS = 256, 64, 0.8, 1e-6, 2000


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


def _startup_profile(H, F, nu, t):
    y = np.arange(H) + 0.5
    u = F / (2 * nu) * y * (H - y)
    for n in range(1, 2001, 2):
        u -= 4 * F * H * H / (nu * np.pi**3 * n**3) * np.sin(n * np.pi * y / H) \
            * np.exp(-nu * n * n * np.pi**2 * t / H**2)
    return u


@pytest.mark.parametrize("coll", [0, 1])
def test_channel_256_blocks_vs_single_and_analytic(L, coll):
    kw = dict(collision=coll, force=(FORCE, 0, 0), **W.channel_bc())
    dims = (N, N, N)
    multi = L.lbm_create(dims, (B, B, B), TAU, None, L.make_params(**kw))
    single = L.lbm_create(dims, dims, TAU, None, L.make_params(**kw))
    info = L.lbm_get_info(multi)
    assert info.blocks == 64
    # faces carry 5 PDFs per cell, edges 1 (every block has all 6 faces in
    # x and z, and +-y faces inside the 4-block column)
    L.lbm_step(multi, STEPS)
    L.lbm_step(single, STEPS)
    fm = L.lbm_get_pdfs(multi)
    fs = L.lbm_get_pdfs(single)
    assert np.array_equal(fm, fs)
    del fs
    rho, u = L.lbm_macroscopic(multi)
    ux = u[:N**3].reshape(N, N, N)
    # the flow is translation invariant along x and z, cell for cell bitwise
    assert np.array_equal(ux, np.broadcast_to(ux[:1, :, :1], ux.shape))
    prof = ux[0, :, 0].astype(np.float64)
    ua = _startup_profile(N, FORCE, (TAU - 0.5) / 3, STEPS)
    assert np.abs(prof - ua).max() <= 0.01 * ua.max()
    # one more step: sampled cells against the oracle from the same state
    rng = np.random.default_rng(2000 + coll)
    cells = rng.choice(N**3, 4096, replace=False)
    # always include wall-adjacent rows and periodic seams
    seam = np.array([(z * N + y) * N + x for z, y, x in
                     [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N - 1, 5), (N - 1, 0, N - 1),
                      (63, 64, 64), (64, 63, 127), (128, 0, 191), (191, 255, 192)]])
    cells = np.unique(np.concatenate([cells, seam]))
    p = oracle.Problem(dims=dims, tau=TAU, periodic=(1, 0, 1), collision=coll,
                       force=(FORCE, 0, 0))
    ref = oracle.step_cells(p, fm, cells)
    L.lbm_step(multi, 1)
    fm1 = L.lbm_get_pdfs(multi).reshape(19, -1)[:, cells].T
    scale = np.abs(ref).max()
    assert np.abs(fm1 - ref).max() <= 2e-6 * scale + 1e-12
    multi.destroy()
    single.destroy()
