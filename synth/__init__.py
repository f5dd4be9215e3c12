"""Seeded synthetic inputs (gauge links, sources) for the Wilson-Dirac operator.

Shared input source of the FP64 oracle and the GPU path.  It contains no
arithmetic of the operator itself; see ``synth.c`` for the generator
definitions (counter-based SplitMix64, Box-Muller, exp(i eps H) links).

Array conventions (numpy, complex128, lexicographic site order
``site = x + Lx*(y + Ly*(z + Lz*t))``):

* spinor field: shape ``(V, 4, 3)`` -- site, spin, colour
* gauge field:  shape ``(V, 4, 3, 3)`` -- site, direction mu (x,y,z,t), row, column
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None

LINK_SEED_BASE = 1000     # links: seed = 1000 + volume id
SOURCE_SEED_BASE = 2000   # sources: seed = 2000 + k
EPS_SMOOTH = 0.2          # exp(i * 0.2 * H) links


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.synth_splitmix64_at.restype = ctypes.c_uint64
            lib.synth_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_gaussian.restype = None
            lib.synth_gaussian.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p]
            lib.synth_su3.restype = None
            lib.synth_su3.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p]
            _lib = lib
    return _lib


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def splitmix64_at(seed: int, n: int) -> int:
    return int(_load().synth_splitmix64_at(seed & (2**64 - 1), n))


def gaussian(n: int, seed: int) -> np.ndarray:
    out = np.empty(int(n), dtype=np.float64)
    _load().synth_gaussian(int(n), seed & (2**64 - 1), out.ctypes.data)
    return out


def su3(n: int, eps: float, seed: int) -> np.ndarray:
    """``n`` matrices exp(i eps H), re-unitarised; shape (n, 3, 3) complex128."""
    out = np.empty((int(n), 3, 3), dtype=np.complex128)
    _load().synth_su3(int(n), float(eps), seed & (2**64 - 1), out.ctypes.data)
    return out


def gauge(dims, seed: int, eps: float = EPS_SMOOTH) -> np.ndarray:
    """Smoothed SU(3) gauge field, shape (V, 4, 3, 3); matrix (site, mu) is number 4*site+mu."""
    v = volume(dims)
    return su3(4 * v, eps, seed).reshape(v, 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    v = volume(dims)
    u = np.zeros((v, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def spinor(dims, seed: int) -> np.ndarray:
    """Gaussian source: each of the 24 reals per site is N(0,1); shape (V, 4, 3)."""
    v = volume(dims)
    return gaussian(24 * v, seed).view(np.complex128).reshape(v, 4, 3)


def parity_mask(dims) -> np.ndarray:
    """Boolean array (V,), True on odd sites ((x+y+z+t) odd)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return (((x + y + z + t) & 1) == 1).reshape(-1)


def even_spinor(dims, seed: int) -> np.ndarray:
    """Gaussian source on even sites, zero on odd sites."""
    s = spinor(dims, seed)
    s[parity_mask(dims)] = 0.0
    return s
