"""FP64 CPU oracle of the D3Q19 lattice Boltzmann sweep (Sec. 2.1, Eq. (1)-(2)).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA product path never imports it and shares no code with it.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, one straight loop per
cell).  This module only marshals numpy arrays into it through ctypes and
builds the shared library with gcc on first use.

Every function is pinned by ``tests/test_oracle.py`` against closed forms,
invariants and an independently written push-form step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass, field

import numpy as np

Q = 19
FLUID, NOSLIP, MOVING, PRESSURE = 0, 1, 2, 3
BGK, TRT = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, portable flags).  OpenMP
    is used when the compiler has it (orc_set_threads); otherwise the library
    is built serial."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True)
        if r.returncode != 0:
            subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("periodic", ctypes.c_int * 3),
        ("face_bc", ctypes.c_int * 6),
        ("collision", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("magic", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("wall_u", ctypes.c_double * 3),
        ("rho_b", ctypes.c_double),
        ("qw", ctypes.POINTER(ctypes.c_double)),
    ]


@dataclass
class Problem:
    """Domain and physics of one oracle run.

    dims: interior cells (nx, ny, nz); flags: uint8 array of shape (nz, ny, nx)
    or None (all fluid); face_bc: wall kind beyond -x,+x,-y,+y,-z,+z.
    """

    dims: tuple
    tau: float
    flags: np.ndarray | None = None
    periodic: tuple = (0, 0, 0)
    face_bc: tuple = (NOSLIP,) * 6
    collision: int = BGK
    magic: float = 3.0 / 16.0
    rho0: float = 1.0
    force: tuple = (0.0, 0.0, 0.0)
    wall_u: tuple = (0.0, 0.0, 0.0)
    rho_b: float | None = None  # density of PRESSURE boundaries; None = rho0
    # curved walls: wall distances (19, nz, ny, nx) of the pulls whose source is a
    # NOSLIP node (the wall at x - q e_i); None = half-way everywhere
    qw: np.ndarray | None = None
    _c: _Problem = field(default=None, repr=False)

    def __post_init__(self):
        c = _Problem()
        c.n[:] = [int(v) for v in self.dims]
        c.periodic[:] = [int(v) for v in self.periodic]
        c.face_bc[:] = [int(v) for v in self.face_bc]
        c.collision = int(self.collision)
        c.tau = float(self.tau)
        c.magic = float(self.magic)
        c.rho0 = float(self.rho0)
        c.force[:] = [float(v) for v in self.force]
        c.wall_u[:] = [float(v) for v in self.wall_u]
        c.rho_b = float(self.rho0 if self.rho_b is None else self.rho_b)
        if self.qw is not None:
            nx, ny, nz = self.dims
            self.qw = np.ascontiguousarray(self.qw, dtype=np.float64).reshape(19, nz, ny, nx)
            c.qw = self.qw.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._c = c
        if self.flags is not None:
            nx, ny, nz = self.dims
            self.flags = np.ascontiguousarray(self.flags, dtype=np.uint8).reshape(nz, ny, nx)

    @property
    def ncells(self) -> int:
        nx, ny, nz = self.dims
        return nx * ny * nz


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i32, u8, i64 = P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_uint8), P(ctypes.c_long)
        pp = P(_Problem)
        sig = {
            "orc_lattice": ([i32, d, i32], None),
            "orc_equilibrium": ([ctypes.c_double, d, ctypes.c_double, d], None),
            "orc_collide": ([pp, d, d, d], None),
            "orc_step": ([pp, u8, d, d, d], None),
            "orc_run": ([pp, u8, d, ctypes.c_int], ctypes.c_int),
            "orc_set_threads": ([ctypes.c_int], None),
            "orc_step_cells": ([pp, u8, d, i64, ctypes.c_long, d], None),
            "orc_macroscopic": ([pp, u8, d, d, d], None),
            "orc_init_equilibrium": ([pp, u8, d, d, d], None),
            "orc_invariants": ([pp, u8, d, d, d], None),
            "orc_residual": ([pp, u8, d, d], ctypes.c_double),
            "orc_interval_residual": ([pp, u8, d, d, ctypes.c_int], ctypes.c_double),
            "orc_push_step": ([pp, u8, d, d], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = res
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _fp(p: Problem):
    if p.flags is None:
        return None
    return p.flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def lattice():
    """(e[19,3] int, w[19] float64, opp[19] int) as the oracle defines them."""
    e = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    lib().orc_lattice(e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                      opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return e, w, opp


def equilibrium(drho: float, u, rho0: float = 1.0) -> np.ndarray:
    """Shifted equilibrium f~^eq(drho, u) of Eq. (2)."""
    u = _f64(u, (3,))
    out = np.zeros(Q)
    lib().orc_equilibrium(float(drho), _dp(u), float(rho0), _dp(out))
    return out


def collide(p: Problem, f):
    """Collision of one cell; returns (f_out[19], u[3])."""
    f = _f64(f, (Q,))
    out, u = np.zeros(Q), np.zeros(3)
    lib().orc_collide(ctypes.byref(p._c), _dp(f), _dp(out), _dp(u))
    return out, u


def zeros(p: Problem) -> np.ndarray:
    nx, ny, nz = p.dims
    return np.zeros((Q, nz, ny, nx))


def set_threads(n: int) -> None:
    """Threads for the step loop (1 = serial).  Results do not depend on it."""
    lib().orc_set_threads(int(n))


def step(p: Problem, f, return_u: bool = False):
    """One pull step; f has shape (19, nz, ny, nx).  Returns the new state."""
    f = _f64(f)
    out = np.empty_like(f)
    u = np.empty((3,) + f.shape[1:]) if return_u else None
    lib().orc_step(ctypes.byref(p._c), _fp(p), _dp(f), _dp(out), _dp(u))
    return (out, u) if return_u else out


def run(p: Problem, f, nsteps: int) -> np.ndarray:
    f = _f64(f).copy()
    if lib().orc_run(ctypes.byref(p._c), _fp(p), _dp(f), int(nsteps)) != 0:
        raise MemoryError("oracle run: allocation failed")
    return f


def step_cells(p: Problem, f, cells) -> np.ndarray:
    """Post-collision PDFs of one step at the given flat interior cells."""
    f = _f64(f)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros((len(cells), Q))
    lib().orc_step_cells(ctypes.byref(p._c), _fp(p), _dp(f),
                         cells.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), len(cells), _dp(out))
    return out


def push_step(p: Problem, f) -> np.ndarray:
    f = _f64(f)
    out = np.empty_like(f)
    lib().orc_push_step(ctypes.byref(p._c), _fp(p), _dp(f), _dp(out))
    return out


def macroscopic(p: Problem, f):
    """(rho[nz,ny,nx], u[3,nz,ny,nx]) of a stored post-collision state."""
    f = _f64(f)
    rho = np.empty(f.shape[1:])
    u = np.empty((3,) + f.shape[1:])
    lib().orc_macroscopic(ctypes.byref(p._c), _fp(p), _dp(f), _dp(rho), _dp(u))
    return rho, u


def init_equilibrium(p: Problem, rho, u) -> np.ndarray:
    nx, ny, nz = p.dims
    rho = _f64(rho, (nz, ny, nx))
    u = _f64(u, (3, nz, ny, nx))
    f = zeros(p)
    lib().orc_init_equilibrium(ctypes.byref(p._c), _fp(p), _dp(rho), _dp(u), _dp(f))
    return f


def invariants(p: Problem, f):
    """(mass, momentum[3]) summed over fluid cells in FP64."""
    f = _f64(f)
    m = np.zeros(1)
    mom = np.zeros(3)
    lib().orc_invariants(ctypes.byref(p._c), _fp(p), _dp(f), _dp(m), _dp(mom))
    return float(m[0]), mom


def residual(p: Problem, prev, cur) -> float:
    """One-step velocity residual ||u_n - u_{n-1}|| / ||u_n|| (fluid cells)."""
    return float(lib().orc_residual(ctypes.byref(p._c), _fp(p), _dp(_f64(prev)), _dp(_f64(cur))))


def interval_residual(p: Problem, prev, cur, k: int) -> float:
    """Change per step over k steps, ||u_n - u_{n-k}|| / (k ||u_n||), from the
    stored states k steps apart (the criterion for sphere-packed channels)."""
    return float(lib().orc_interval_residual(ctypes.byref(p._c), _fp(p), _dp(_f64(prev)),
                                             _dp(_f64(cur)), int(k)))


def run_to_interval_residual(p: Problem, f, tol: float, k: int, max_steps: int):
    """Steps f in chunks of k until the interval residual over the last chunk
    is below tol.  Returns (steps, residual of the last chunk, state); steps
    is -1 when max_steps passed first.  The stopping rule: the first multiple
    of k at which r < tol."""
    f = _f64(f).copy()
    done, r = 0, float("inf")
    while done < max_steps:
        g = run(p, f, k)
        done += k
        r = interval_residual(p, f, g, k)
        f = g
        if r < tol:
            return done, r, f
    return -1, r, f


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
