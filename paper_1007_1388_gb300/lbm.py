"""Thin ctypes binding of liblbm.so (include/lbm.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own; every step of the lattice Boltzmann path runs in the
library's CUDA kernels.  PyTorch supplies plumbing only: the device memory
(through ``use_torch_allocator``) and the CUDA stream each context runs on.

If liblbm.so has not been built, importing works but the first call raises
``RuntimeError``: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

Q = 19
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ETIMEOUT, LBM_ENUMERIC = 0, -1, -2, -3, -4, -5
LBM_FLUID, LBM_NOSLIP, LBM_MOVING, LBM_PRESSURE = 0, 1, 2, 3
LBM_BGK, LBM_TRT = 0, 1
LBM_F32, LBM_F16S, LBM_BF16S, LBM_F64 = 0, 1, 2, 3
LBM_KERNEL_AUTO, LBM_KERNEL_REGISTER, LBM_KERNEL_TMA = 0, 1, 2
LBM_STREAM_TWO_GRID, LBM_STREAM_AA = 0, 1
LBM_LAYOUT_BLOCKS, LBM_LAYOUT_SPARSE = 0, 1
LBM_DEBUG_DROP_STAGE = 1
STORAGE_NAMES = {LBM_F32: "f32", LBM_F16S: "f16s", LBM_BF16S: "bf16s", LBM_F64: "f64"}
BYTES_PER_PDF = {LBM_F32: 4, LBM_F16S: 2, LBM_BF16S: 2, LBM_F64: 8}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("collision", ctypes.c_int),
        ("magic", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("wall_u", ctypes.c_double * 3),
        ("periodic", ctypes.c_int * 3),
        ("face_bc", ctypes.c_int * 6),
        ("storage", ctypes.c_int),
        ("storage_scale", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("tile", ctypes.c_int * 3),
        ("graph_steps", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("debug_flags", ctypes.c_int),
        ("rho_b", ctypes.c_double),
        ("streaming", ctypes.c_int),
        ("layout", ctypes.c_int),
    ]


class lbm_info(ctypes.Structure):
    _fields_ = [
        ("cells", ctypes.c_longlong),
        ("fluid_cells", ctypes.c_longlong),
        ("stored_cells", ctypes.c_longlong),
        ("blocks", ctypes.c_int),
        ("instances", ctypes.c_int),
        ("storage", ctypes.c_int),
        ("bytes_per_pdf", ctypes.c_int),
        ("exchange_pdfs", ctypes.c_longlong),
        ("device_bytes", ctypes.c_longlong),
        ("tile", ctypes.c_int * 3),
        ("tiles", ctypes.c_longlong),
        ("kernel", ctypes.c_int),
        ("sweep_ctas", ctypes.c_int),
        ("stages", ctypes.c_int),
        ("flat", ctypes.c_int),
        ("mask", ctypes.c_int),
        ("pair", ctypes.c_int),
        ("streaming", ctypes.c_int),
        ("aa_phase", ctypes.c_int),
        ("layout", ctypes.c_int),
        ("list_cells", ctypes.c_longlong),
    ]


class lbm_profile(ctypes.Structure):
    _fields_ = [
        ("sweep_ms", ctypes.c_double),
        ("sweep_launches", ctypes.c_longlong),
        ("exchange_ms", ctypes.c_double),
        ("exchange_launches", ctypes.c_longlong),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

# every symbol include/lbm.h declares, with its ctypes signature
_P = ctypes.POINTER
_vp, _i, _d, _ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
SIGNATURES = {
    "lbm_default_params": ([_P(lbm_params)], None),
    "lbm_create": ([_P(ctypes.c_int), _P(ctypes.c_int), _d, _vp, _P(lbm_params), _P(_vp)], _i),
    "lbm_batch_create": ([_i, _P(ctypes.c_int), _P(_d), _P(_vp), _P(lbm_params), _P(_vp)], _i),
    "lbm_destroy": ([_vp], None),
    "lbm_step": ([_vp, _i], _i),
    "lbm_synchronize": ([_vp], _i),
    "lbm_macroscopic": ([_vp, _vp, _vp], _i),
    "lbm_macroscopic_device": ([_vp, _vp, _vp], _i),
    "lbm_get_pdfs": ([_vp, _vp], _i),
    "lbm_set_pdfs": ([_vp, _vp], _i),
    "lbm_get_pdfs_device": ([_vp, _vp], _i),
    "lbm_set_pdfs_device": ([_vp, _vp], _i),
    "lbm_init_equilibrium": ([_vp, _vp, _vp], _i),
    "lbm_init_equilibrium_device": ([_vp, _vp, _vp], _i),
    "lbm_invariants": ([_vp, _P(_d), _P(_d), _P(_d), _vp], _i),
    "lbm_residual": ([_vp, _P(_d), _vp], _i),
    "lbm_run_to_residual": ([_vp, _d, _i, _ll, _P(_ll), _P(_d)], _i),
    "lbm_run_to_residual_each": ([_vp, _d, _i, _i, _ll, _vp, _vp], _i),
    "lbm_snapshot_velocity": ([_vp], _i),
    "lbm_impose_velocity_device": ([_vp, _vp], _i),
    "lbm_init_consistent_device": ([_vp, _vp, _vp, _i], _i),
    "lbm_residual_vs_snapshot": ([_vp, _i, _P(_d), _vp], _i),
    "lbm_set_forces": ([_vp, _vp], _i),
    "lbm_get_info": ([_vp, _P(lbm_info)], _i),
    "lbm_profile_enable": ([_vp, _i], _i),
    "lbm_profile_read": ([_vp, _P(lbm_profile)], _i),
    "lbm_autotune": ([_vp, ctypes.c_char_p, _P(ctypes.c_int)], _i),
    "lbm_get_sweep_config": ([_vp, _P(ctypes.c_int)], _i),
    "lbm_set_sweep_config": ([_vp, _P(ctypes.c_int)], _i),
    "lbm_set_wall_distances": ([_vp, _ll, _vp, _vp, _vp], _i),
    "lbm_set_allocator": ([ALLOC_FN, FREE_FN, _vp], _i),
    "lbm_directions": ([_P(ctypes.c_int), _P(_d), _P(ctypes.c_int)], _i),
    "lbm_invariants_noalloc": ([_vp, _vp, _ll, _d, _P(_d), _vp, _vp], _i),
    "lbm_last_error": ([_vp], ctypes.c_char_p),
    "lbm_version": ([], ctypes.c_char_p),
    # include/unet.h (the learned warm start; wrapped in unet.py)
    "unet_param_count": ([], _ll),
    "unet_create": ([_i, _i, ctypes.c_ulonglong, _vp, _P(_vp)], _i),
    "unet_create_ex": ([_i, _i, ctypes.c_ulonglong, _i, _vp, _P(_vp)], _i),
    "unet_destroy": ([_vp], None),
    "unet_get_params": ([_vp, _vp], _i),
    "unet_set_params": ([_vp, _vp], _i),
    "unet_predict": ([_vp, _vp, _vp, _vp], _i),
    "unet_loss_grad": ([_vp, _vp, _vp, _vp, _P(_d), _vp], _i),
    "unet_adam_step": ([_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float], _i),
    "unet_last_error": ([_vp], ctypes.c_char_p),
    "unet_conv3": ([_vp, _i, _i, _vp, _i, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp], _i),
    "unet_conv3_wgrad": ([_vp, _i, _i, _vp, _i, _vp, _i, _vp, _i, _i, _i, _i, _vp], _i),
    "unet_targets_from_fields": ([_vp, _vp, _vp, _vp, _i, _ll, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  _vp, _vp], _i),
    "unet_fields_from_prediction": ([_vp, _vp, _vp, _i, _ll, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     _vp, _vp, _vp], _i),
    "unet_smooth_fields": ([_vp, _vp, _vp, _i, _i, _i, _i, _vp], _i),
    "unet_conv3_halo": ([_vp, _i, _vp, _i, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp], _i),
    "unet_conv3_halo_wgrad": ([_vp, _i, _vp, _i, _vp, _i, _vp, _i, _i, _i, _i, _vp], _i),
    "unet_planar_positions": ([_i, _i, _i, _i], _ll),
    "unet_conv3_planar": ([_vp, _i, _vp, _i, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp], _i),
    "unet_conv3_planar_wgrad": ([_vp, _i, _vp, _i, _vp, _i, _vp, _i, _i, _i, _i, _vp], _i),
}

_lib = None


def lib():
    """The loaded liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


def _check(rc, ctx=None):
    if rc != LBM_OK:
        msg = lib().lbm_last_error(ctx.ptr if ctx is not None else None)
        raise LBMError(rc, msg.decode() if msg else "")


def _host_buf(a, n, dtype):
    """Checks a caller-given host buffer (numpy array or CPU torch tensor)."""
    if isinstance(a, np.ndarray):
        ok = a.dtype == dtype and a.size == n and a.flags.c_contiguous
    else:
        import torch

        tdt = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
        ok = (a.dtype == tdt and a.numel() == n and a.is_contiguous() and a.device.type == "cpu")
    if not ok:
        raise ValueError(f"host buffer must be a contiguous {np.dtype(dtype).name} array of {n} values")
    return a


def _ptr(a):
    """Address of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch.Tensor


# ---------------------------------------------------------------- allocator
_torch_hooks = None


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _torch_hooks
    import torch

    if _torch_hooks is not None:
        return

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0)
        except Exception:  # out of memory -> NULL -> LBM_ENOMEM
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib().lbm_set_allocator(hooks[0], hooks[1], None))
    _torch_hooks = hooks


# ------------------------------------------------------------------ context
class Ctx:
    """Owner of one lbm_ctx*; destroyed by lbm_destroy or garbage collection."""

    def __init__(self, ptr, cells, ninst, stream, inst_cells):
        self.ptr = ptr
        self.cells = cells
        self.ninst = ninst
        self.stream = stream  # keeps the torch stream alive
        self.inst_cells = inst_cells
        self._fin = weakref.finalize(self, lib().lbm_destroy, ptr)

    def destroy(self):
        self._fin()


def lbm_default_params() -> lbm_params:
    p = lbm_params()
    lib().lbm_default_params(ctypes.byref(p))
    return p


def make_params(**kw) -> lbm_params:
    """lbm_default_params() with the given fields replaced (lists for arrays)."""
    p = lbm_default_params()
    for k, v in kw.items():
        if k in ("force", "wall_u", "periodic", "face_bc", "tile"):
            getattr(p, k)[:] = list(v)
        else:
            setattr(p, k, v)
    return p


def _stream_for(params):
    """A torch stream for the context unless the caller set one."""
    if params.stream:
        return None
    import torch

    if not torch.cuda.is_available():
        return None
    s = torch.cuda.Stream()
    params.stream = s.cuda_stream
    return s


def lbm_create(dims, block_dims, tau, flags=None, params=None) -> Ctx:
    p = params if params is not None else lbm_default_params()
    p = lbm_params.from_buffer_copy(p)
    stream = _stream_for(p)
    d = (ctypes.c_int * 3)(*[int(v) for v in dims])
    b = (ctypes.c_int * 3)(*[int(v) for v in block_dims])
    fl = None
    if flags is not None:
        fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
        if fl.size != int(np.prod(dims)):
            raise ValueError("flags must have nx*ny*nz entries")
    out = ctypes.c_void_p()
    _check(lib().lbm_create(d, b, float(tau), _ptr(fl), ctypes.byref(p), ctypes.byref(out)))
    n = int(np.prod(dims))
    return Ctx(out.value, n, 1, stream, [n])


def lbm_batch_create(dims, tau, flags=None, params=None) -> Ctx:
    dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 3)
    n = dims.shape[0]
    tau = np.ascontiguousarray(tau, dtype=np.float64).reshape(n)
    p = params if params is not None else lbm_default_params()
    p = lbm_params.from_buffer_copy(p)
    stream = _stream_for(p)
    keep = []
    fl_arr = None
    if flags is not None:
        fl_arr = (ctypes.c_void_p * n)()
        for k in range(n):
            if flags[k] is None:
                fl_arr[k] = None
                continue
            a = np.ascontiguousarray(flags[k], dtype=np.uint8).reshape(-1)
            if a.size != int(np.prod(dims[k])):
                raise ValueError(f"flags[{k}] must have nx*ny*nz entries")
            keep.append(a)
            fl_arr[k] = a.ctypes.data
    out = ctypes.c_void_p()
    _check(lib().lbm_batch_create(n, dims.ctypes.data_as(_P(ctypes.c_int)),
                                  tau.ctypes.data_as(_P(ctypes.c_double)), fl_arr,
                                  ctypes.byref(p), ctypes.byref(out)))
    inst_cells = [int(np.prod(d)) for d in dims]
    return Ctx(out.value, sum(inst_cells), n, stream, inst_cells)


def lbm_destroy(ctx: Ctx):
    ctx.destroy()


def lbm_step(ctx: Ctx, n: int = 1):
    _check(lib().lbm_step(ctx.ptr, int(n)), ctx)


def lbm_synchronize(ctx: Ctx):
    _check(lib().lbm_synchronize(ctx.ptr), ctx)


def lbm_macroscopic(ctx: Ctx, rho=None, u=None):
    """Host variant: fills (or allocates) numpy rho[N], u[3N] float32."""
    rho = _host_buf(np.empty(ctx.cells, np.float32) if rho is None else rho, ctx.cells, np.float32)
    u = _host_buf(np.empty(3 * ctx.cells, np.float32) if u is None else u, 3 * ctx.cells, np.float32)
    _check(lib().lbm_macroscopic(ctx.ptr, _ptr(rho), _ptr(u)), ctx)
    return rho, u


def lbm_macroscopic_device(ctx: Ctx, rho, u):
    """Device variant: rho, u are contiguous float32 CUDA tensors (N and 3N)."""
    _check(lib().lbm_macroscopic_device(ctx.ptr, _ptr(rho), _ptr(u)), ctx)


def lbm_get_pdfs(ctx: Ctx, f=None):
    f = _host_buf(np.empty(Q * ctx.cells, np.float64) if f is None else f, Q * ctx.cells, np.float64)
    _check(lib().lbm_get_pdfs(ctx.ptr, _ptr(f)), ctx)
    return f


def lbm_set_pdfs(ctx: Ctx, f):
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    assert f.size == Q * ctx.cells
    _check(lib().lbm_set_pdfs(ctx.ptr, _ptr(f)), ctx)


def _device_pdfs(ctx: Ctx, f):
    """Checks a device PDF buffer: a contiguous CUDA float64 tensor of 19 N."""
    import torch

    if not (isinstance(f, torch.Tensor) and f.dtype == torch.float64 and f.is_cuda and f.is_contiguous()
            and f.numel() == Q * ctx.cells):
        raise ValueError(f"f must be a contiguous CUDA float64 tensor of {Q * ctx.cells} values")
    return f


def lbm_get_pdfs_device(ctx: Ctx, f):
    """Enqueues the state's shifted PDFs into the CUDA float64 tensor f (19 N)."""
    _check(lib().lbm_get_pdfs_device(ctx.ptr, _ptr(_device_pdfs(ctx, f))), ctx)


def lbm_set_pdfs_device(ctx: Ctx, f):
    """Enqueues setting the state from the CUDA float64 tensor f (19 N)."""
    _check(lib().lbm_set_pdfs_device(ctx.ptr, _ptr(_device_pdfs(ctx, f))), ctx)


def lbm_init_equilibrium(ctx: Ctx, rho, u):
    if isinstance(rho, np.ndarray) or not hasattr(rho, "data_ptr"):
        rho = np.ascontiguousarray(rho, dtype=np.float32).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float32).reshape(-1)
    _host_buf(rho, ctx.cells, np.float32)
    _host_buf(u, 3 * ctx.cells, np.float32)
    _check(lib().lbm_init_equilibrium(ctx.ptr, _ptr(rho), _ptr(u)), ctx)


def lbm_init_equilibrium_device(ctx: Ctx, rho, u):
    _check(lib().lbm_init_equilibrium_device(ctx.ptr, _ptr(rho), _ptr(u)), ctx)


def lbm_invariants(ctx: Ctx, per_instance: bool = False):
    """(mass, momentum[3], nonfinite) or, with per_instance, also a (ninst, 5) array."""
    m, nf = ctypes.c_double(), ctypes.c_double()
    mom = (ctypes.c_double * 3)()
    per = np.zeros((ctx.ninst, 5)) if per_instance else None
    _check(lib().lbm_invariants(ctx.ptr, ctypes.byref(m), mom, ctypes.byref(nf), _ptr(per)), ctx)
    res = (m.value, np.array(mom[:]), nf.value)
    return res + (per,) if per_instance else res


def lbm_residual(ctx: Ctx, per_instance: bool = False):
    r = ctypes.c_double()
    per = np.zeros(ctx.ninst) if per_instance else None
    _check(lib().lbm_residual(ctx.ptr, ctypes.byref(r), _ptr(per)), ctx)
    return (r.value, per) if per_instance else r.value


def lbm_run_to_residual(ctx: Ctx, tol: float, check_every: int = 10, max_steps: int = 10**6):
    steps, r = ctypes.c_longlong(), ctypes.c_double()
    _check(lib().lbm_run_to_residual(ctx.ptr, float(tol), int(check_every), int(max_steps),
                                     ctypes.byref(steps), ctypes.byref(r)), ctx)
    return steps.value, r.value


def lbm_set_forces(ctx: Ctx, force):
    """force: (instances, 3) array of per-instance body forces."""
    f = np.ascontiguousarray(np.asarray(force, np.float64).reshape(-1))
    if f.size != 3 * lbm_get_info(ctx).instances:
        raise ValueError("need 3 force components per instance")
    _check(lib().lbm_set_forces(ctx.ptr, f.ctypes.data_as(ctypes.c_void_p)), ctx)


def lbm_run_to_residual_each(ctx: Ctx, tol: float, check_every: int = 50, max_steps: int = 10**6,
                             interval: bool = False):
    """Per-instance steps to residual tol (-1 where not reached) and residuals;
    interval: the change per step over each chunk instead of the one-step residual."""
    k = lbm_get_info(ctx).instances
    steps = np.empty(k, np.int64)
    res = np.empty(k, np.float64)
    _check(lib().lbm_run_to_residual_each(ctx.ptr, float(tol), int(check_every), int(bool(interval)),
                                          int(max_steps), steps.ctypes.data_as(ctypes.c_void_p),
                                          res.ctypes.data_as(ctypes.c_void_p)), ctx)
    return steps, res


def lbm_impose_velocity_device(ctx: Ctx, u):
    _check(lib().lbm_impose_velocity_device(ctx.ptr, _ptr(u)), ctx)


def lbm_init_consistent_device(ctx: Ctx, rho, u, iterations: int):
    _check(lib().lbm_init_consistent_device(ctx.ptr, _ptr(rho), _ptr(u), int(iterations)), ctx)


def lbm_snapshot_velocity(ctx: Ctx):
    _check(lib().lbm_snapshot_velocity(ctx.ptr), ctx)


def lbm_residual_vs_snapshot(ctx: Ctx, steps_since: int, per_instance: bool = False):
    r = ctypes.c_double()
    per = np.zeros(ctx.ninst) if per_instance else None
    _check(lib().lbm_residual_vs_snapshot(ctx.ptr, int(steps_since), ctypes.byref(r), _ptr(per)), ctx)
    return (r.value, per) if per_instance else r.value


def lbm_get_info(ctx: Ctx) -> lbm_info:
    info = lbm_info()
    _check(lib().lbm_get_info(ctx.ptr, ctypes.byref(info)), ctx)
    return info


def lbm_profile_enable(ctx: Ctx, on: bool = True):
    _check(lib().lbm_profile_enable(ctx.ptr, 1 if on else 0), ctx)


def lbm_profile_read(ctx: Ctx) -> lbm_profile:
    prof = lbm_profile()
    _check(lib().lbm_profile_read(ctx.ptr, ctypes.byref(prof)), ctx)
    return prof


def lbm_autotune(ctx: Ctx, cache_path: str | None = None):
    best = (ctypes.c_int * 3)()
    _check(lib().lbm_autotune(ctx.ptr, cache_path.encode() if cache_path else None, best), ctx)
    return tuple(best)


SWEEP_ROWS, SWEEP_TMA, SWEEP_RUNS, SWEEP_ROWS2, SWEEP_RUNS2 = 0, 1, 2, 3, 4


def lbm_get_sweep_config(ctx: Ctx):
    """{kind, tx, ty, tz, grid, minb, zchunk, mask} of the sweep in use."""
    cfg = (ctypes.c_int * 8)()
    _check(lib().lbm_get_sweep_config(ctx.ptr, cfg), ctx)
    return tuple(cfg)


def lbm_set_sweep_config(ctx: Ctx, cfg):
    c = (ctypes.c_int * 8)(*[int(v) for v in cfg])
    _check(lib().lbm_set_sweep_config(ctx.ptr, c), ctx)


def lbm_set_wall_distances(ctx: Ctx, cells, dirs, q):
    """Curved resting walls on the listed links (cell index, pull direction
    1..18 whose source is a resting wall, wall distance in (0, 1])."""
    cells = np.ascontiguousarray(cells, dtype=np.int64).reshape(-1)
    dirs = np.ascontiguousarray(dirs, dtype=np.int32).reshape(-1)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    if not (cells.size == dirs.size == q.size):
        raise ValueError("cells, dirs and q must have the same length")
    _check(lib().lbm_set_wall_distances(ctx.ptr, cells.size, _ptr(cells), _ptr(dirs), _ptr(q)), ctx)


def lbm_directions():
    e = (ctypes.c_int * (3 * Q))()
    w = (ctypes.c_double * Q)()
    o = (ctypes.c_int * Q)()
    _check(lib().lbm_directions(e, w, o))
    return np.array(e[:]).reshape(Q, 3), np.array(w[:]), np.array(o[:])


def _noalloc_tensor(name, t, dtype, numel):
    """Checks one tensor argument of lbm_invariants_noalloc before its address
    reaches the kernels: dtype, element count and contiguity."""
    import torch

    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def lbm_invariants_noalloc(f, flags, n_cells: int, rho0: float, force, out, stream=None):
    """Allocation-free FP64 invariants of a caller-owned device PDF array.

    f: CUDA float32 tensor of 19*n_cells (direction-major); flags: CUDA uint8
    tensor of n_cells or None; out: CUDA float64 tensor of 5; all on one
    device.  stream: a torch.cuda.Stream on that device (default: its current
    stream).  Enqueues only; the call is made with that device current.
    Raises ValueError before any device work for a wrong dtype, size,
    layout or device.
    """
    import torch

    n_cells = int(n_cells)
    if n_cells <= 0:
        raise ValueError("n_cells must be positive")
    ts = [_noalloc_tensor("f", f, torch.float32, Q * n_cells), _noalloc_tensor("out", out, torch.float64, 5)]
    if flags is not None:
        ts.append(_noalloc_tensor("flags", flags, torch.uint8, n_cells))
    for t in ts:
        if t.device.type != "cuda":
            raise ValueError("f, flags and out must be CUDA tensors")
    dev = f.device
    if any(t.device != dev for t in ts):
        raise ValueError("f, flags and out must be on the same device")
    if stream is not None and stream.device != dev:
        raise ValueError("stream must belong to the device of f")
    if len(force) != 3:
        raise ValueError("force must have 3 components")
    F = (ctypes.c_double * 3)(*[float(v) for v in force])
    with torch.cuda.device(dev):
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        _check(lib().lbm_invariants_noalloc(_ptr(f), _ptr(flags), n_cells, float(rho0), F,
                                            _ptr(out), s.cuda_stream))


def lbm_last_error(ctx: Ctx | None = None) -> str:
    return lib().lbm_last_error(ctx.ptr if ctx is not None else None).decode()


def lbm_version() -> str:
    return lib().lbm_version().decode()
