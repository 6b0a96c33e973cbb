"""ctypes binding of include/unet.h: the learned warm start's 3-D U-Net.

Argument marshalling only; every step of the forward pass, the backward
pass, the loss and the optimiser runs in liblbm.so (tensor-core
convolutions, CUDA element-wise kernels).  Device buffers are torch CUDA
tensors (plumbing: memory and streams); nothing here computes.
"""
from __future__ import annotations

import ctypes
import weakref

import numpy as np

from .lbm import LBMError, lib

C_IN, C_OUT = 2, 4  # input channels (solid flag, force), output (delta rho, u)


def _check(rc, ptr=None):
    if rc != 0:
        msg = lib().unet_last_error(ptr)
        raise LBMError(rc, msg.decode() if msg else "")


def _dev(t, dtype, numel):
    import torch

    if t.device.type != "cuda" or t.dtype != dtype or t.numel() != numel or not t.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor of {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


def param_count() -> int:
    return int(lib().unet_param_count())


BF16, F32 = 0, 1  # UNET_BF16 (tensor cores), UNET_F32 (debug mode, CUDA cores)


class UNet:
    """A network for batches of nb samples of n^3 voxels (n a power of two).
    precision: BF16 (the training path) or F32 (debug mode for gradient checks)."""

    def __init__(self, n: int, nb: int, seed: int = 0, stream=None, precision: int = BF16):
        import torch

        self.n, self.nb, self.precision = n, nb, precision
        self.stream = stream if stream is not None else torch.cuda.Stream()
        p = ctypes.c_void_p()
        _check(lib().unet_create_ex(n, nb, ctypes.c_ulonglong(seed), precision,
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(p)))
        self.ptr = p
        self._fin = weakref.finalize(self, lib().unet_destroy, p)

    def destroy(self):
        self._fin()

    @property
    def voxels(self) -> int:
        return self.nb * self.n ** 3

    def get_params(self) -> np.ndarray:
        out = np.empty(param_count(), np.float32)
        _check(lib().unet_get_params(self.ptr, out.ctypes.data_as(ctypes.c_void_p)), self.ptr)
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != param_count():
            raise ValueError("wrong parameter count")
        _check(lib().unet_set_params(self.ptr, p.ctypes.data_as(ctypes.c_void_p)), self.ptr)

    def _force(self, force):
        f = np.ascontiguousarray(np.broadcast_to(np.asarray(force, np.float32), (self.nb,)))
        return f, f.ctypes.data_as(ctypes.c_void_p)

    def predict(self, solid, force, out):
        """solid: CUDA uint8 [nb*n^3]; force: nb floats; out: CUDA float32 [nb*n^3*4]."""
        import torch

        f, fp = self._force(force)
        _check(lib().unet_predict(self.ptr, _dev(solid, torch.uint8, self.voxels), fp,
                                  _dev(out, torch.float32, self.voxels * C_OUT)), self.ptr)
        return out

    def loss_grad(self, solid, force, target, grads: bool = False):
        """Forward + backward; returns the loss (and the FP32 gradient if asked)."""
        import torch

        f, fp = self._force(force)
        loss = ctypes.c_double()
        g = np.empty(param_count(), np.float32) if grads else None
        _check(lib().unet_loss_grad(self.ptr, _dev(solid, torch.uint8, self.voxels), fp,
                                    _dev(target, torch.float32, self.voxels * C_OUT), ctypes.byref(loss),
                                    g.ctypes.data_as(ctypes.c_void_p) if grads else None), self.ptr)
        return (loss.value, g) if grads else loss.value

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        _check(lib().unet_adam_step(self.ptr, lr, beta1, beta2, eps), self.ptr)

    def train_step(self, solid, force, target, lr: float) -> float:
        loss = self.loss_grad(solid, force, target)
        self.adam_step(lr)
        return loss


def conv3(src0, c0, w, out, cout, grid, *, up0=False, src1=None, c1=0, bias=None, relu=False, stream=None):
    """One tensor-core 3x3x3 convolution on device tensors (bf16 activations
    and weights; out bf16 or float32).  grid = (nb, lz, ly, lx)."""
    import torch

    nb, lz, ly, lx = grid
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().unet_conv3(
        ctypes.c_void_p(src0.data_ptr()), c0, int(up0),
        ctypes.c_void_p(src1.data_ptr()) if src1 is not None else None, c1,
        ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(bias.data_ptr()) if bias is not None else None,
        ctypes.c_void_p(out.data_ptr()), int(out.dtype == torch.float32), int(relu), cout, nb, lz, ly, lx,
        ctypes.c_void_p(s.cuda_stream)))
    return out


def conv3_wgrad(src0, c0, dy, cout, dw, grid, *, up0=False, src1=None, c1=0, stream=None):
    """Weight gradient of conv3 into the float32 tensor dw [cout][27][c0+c1]."""
    import torch

    nb, lz, ly, lx = grid
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().unet_conv3_wgrad(
        ctypes.c_void_p(src0.data_ptr()), c0, int(up0),
        ctypes.c_void_p(src1.data_ptr()) if src1 is not None else None, c1,
        ctypes.c_void_p(dy.data_ptr()), cout, ctypes.c_void_p(dw.data_ptr()), nb, lz, ly, lx,
        ctypes.c_void_p(s.cuda_stream)))
    return dw


def targets_from_fields(rho, u, solid, force, nb, V, rho0, s_rho, s_u, target, stream):
    """Normalised targets [nb][V][4] from batch fields (all CUDA tensors)."""
    _check(lib().unet_targets_from_fields(
        ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(solid.data_ptr()),
        ctypes.c_void_p(force.data_ptr()), nb, V, rho0, s_rho, s_u, ctypes.c_void_p(target.data_ptr()),
        ctypes.c_void_p(stream.cuda_stream)))
    return target


def fields_from_prediction(pred, solid, force, nb, V, rho0, s_rho, s_u, rho, u, stream):
    """Batch fields rho [nb][V], u [nb][3][V] from a prediction (all CUDA tensors)."""
    _check(lib().unet_fields_from_prediction(
        ctypes.c_void_p(pred.data_ptr()), ctypes.c_void_p(solid.data_ptr()), ctypes.c_void_p(force.data_ptr()),
        nb, V, rho0, s_rho, s_u, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(u.data_ptr()),
        ctypes.c_void_p(stream.cuda_stream)))
    return rho, u


def smooth_fields(f, solid, K, comps, n, passes, stream):
    """In-place binomial smoothing of device fields [K][comps][n^3] (float32)."""
    import torch

    scratch = torch.empty_like(f)
    _check(lib().unet_smooth_fields(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(scratch.data_ptr()),
                                    ctypes.c_void_p(solid.data_ptr()), K, comps, n, passes,
                                    ctypes.c_void_p(stream.cuda_stream)))
    return f


def conv3_halo(src0, c0, w, out, cout, grid, *, src1=None, c1=0, bias=None, relu=False, stream=None):
    """conv3 on halo-layout tensors (TMA-fed tiles)."""
    import torch

    nb, lz, ly, lx = grid
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().unet_conv3_halo(
        ctypes.c_void_p(src0.data_ptr()), c0, ctypes.c_void_p(src1.data_ptr()) if src1 is not None else None, c1,
        ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(bias.data_ptr()) if bias is not None else None,
        ctypes.c_void_p(out.data_ptr()), int(out.dtype == torch.float32), int(relu), cout, nb, lz, ly, lx,
        ctypes.c_void_p(s.cuda_stream)))
    return out


def conv3_halo_wgrad(src0, c0, dy, cout, dw, grid, *, src1=None, c1=0, stream=None):
    """Weight gradient on halo-layout tensors (TMA-fed tiles)."""
    import torch

    nb, lz, ly, lx = grid
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().unet_conv3_halo_wgrad(
        ctypes.c_void_p(src0.data_ptr()), c0, ctypes.c_void_p(src1.data_ptr()) if src1 is not None else None, c1,
        ctypes.c_void_p(dy.data_ptr()), cout, ctypes.c_void_p(dw.data_ptr()), nb, lz, ly, lx,
        ctypes.c_void_p(s.cuda_stream)))
    return dw


def planar_positions(grid) -> int:
    """Positions per 8-channel group of a planar tensor over grid (nb, lz, ly, lx)."""
    nb, lz, ly, lx = grid
    p = lib().unet_planar_positions(nb, lz, ly, lx)
    if p < 0:
        raise ValueError("bad grid")
    return int(p)


def conv3_planar(src0, c0, wpk, out, cout, grid, *, src1=None, c1=0, bias=None, relu=False, stream=None):
    """conv3 on planar bf16 tensors (bulk-copied operands); wpk: weights packed
    per 16 input channels, [cin / 16][27][2][cout][8]."""
    import torch

    nb, lz, ly, lx = grid
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().unet_conv3_planar(
        ctypes.c_void_p(src0.data_ptr()), c0, ctypes.c_void_p(src1.data_ptr()) if src1 is not None else None, c1,
        ctypes.c_void_p(wpk.data_ptr()), ctypes.c_void_p(bias.data_ptr()) if bias is not None else None,
        ctypes.c_void_p(out.data_ptr()), int(out.dtype == torch.float32), int(relu), cout, nb, lz, ly, lx,
        ctypes.c_void_p(s.cuda_stream)))
    return out


def conv3_planar_wgrad(src0, c0, dy, cout, dw, grid, *, src1=None, c1=0, stream=None):
    """Weight gradient on planar bf16 tensors (bulk-copied operands)."""
    import torch

    nb, lz, ly, lx = grid
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().unet_conv3_planar_wgrad(
        ctypes.c_void_p(src0.data_ptr()), c0, ctypes.c_void_p(src1.data_ptr()) if src1 is not None else None, c1,
        ctypes.c_void_p(dy.data_ptr()), cout, ctypes.c_void_p(dw.data_ptr()), nb, lz, ly, lx,
        ctypes.c_void_p(s.cuda_stream)))
    return dw
