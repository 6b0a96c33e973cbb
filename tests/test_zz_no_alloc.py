"""The allocation-free invariant reduction (lbm_invariants_noalloc).

Some callers cannot allocate device memory: code called back from inside a
framework's allocator (a new allocation would re-enter it), or processes
whose device memory a caching allocator has reserved in full (cudaMalloc
fails).  This entry point gives them the FP64 invariants using a fixed
device array instead of scratch allocations.  Here its output is checked against lbm_invariants of the same
state on two calls in a row (the second on a different state, so stale
partial sums from the first call would show), with the tolerances of the
other reduction tests.  The file sorts last so that a stop at the first
failure has already run every other test.
"""
import numpy as np
import pytest

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
    return L


def test_noalloc_invariants_match_context_reduction(L):
    import torch

    rng = np.random.default_rng(31)
    dims = (40, 36, 28)
    n = int(np.prod(dims))
    flags = W.random_flags(rng, dims, 0.1)
    force = (3e-4, -1e-4, 2e-4)
    params = L.make_params(periodic=(1, 0, 1), force=force, collision=1, wall_u=(0.03, 0, 0),
                           face_bc=(1, 1, 1, 2, 1, 1))
    ctx = L.lbm_create(dims, (20, 18, 14), 0.75, flags, params)
    L.lbm_set_pdfs(ctx, W.random_pdfs(rng, dims, 1e-2, flags))
    flags_d = torch.from_numpy(flags.reshape(-1).copy()).cuda()
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        L.lbm_step(ctx, 3)
        m, j, bad = L.lbm_invariants(ctx)
        # the same state as a plain direction-major FP32 device array
        f_d = torch.from_numpy(L.lbm_get_pdfs(ctx).astype(np.float32)).cuda()
        L.lbm_invariants_noalloc(f_d, flags_d, n, 1.0, force, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - m) <= 1e-12 * abs(m), call
        assert np.abs(got[1:4] - j).max() <= 1e-11 * max(1.0, np.abs(j).max()), call
        assert got[4] == bad == 0.0, call
    ctx.destroy()


def test_noalloc_all_fluid_and_limit(L):
    import torch

    n = 5000
    f = torch.zeros(19 * n, dtype=torch.float32, device="cuda")
    f[3 * n:4 * n] = 1e-3   # +y direction everywhere
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    L.lbm_invariants_noalloc(f, None, n, 1.0, (0.0, 0.0, 0.0), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    v = float(np.float32(1e-3))  # the value the FP32 array holds
    assert abs(got[0] - n * (1.0 + v)) <= 1e-9
    assert abs(got[2] - n * v) <= 1e-9 and got[1] == 0.0 and got[3] == 0.0
    # beyond the scratch array's size the C entry point refuses before any
    # launch (called directly: the binding would refuse the small f first)
    import ctypes

    F = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    rc = L.lib().lbm_invariants_noalloc(f.data_ptr(), None, 67108864 + 1, 1.0, F, out.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == L.LBM_EINVAL
    assert "scratch limit" in L.lbm_last_error()
    # the binding checks sizes against the tensors
    with pytest.raises(ValueError):
        L.lbm_invariants_noalloc(f, None, n + 1, 1.0, (0.0, 0.0, 0.0), out)
