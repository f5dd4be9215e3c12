"""FP64 CPU oracle for the Wilson-Dirac operator (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does, and shares
no code with it.  The arithmetic lives in ``wilson_oracle.c`` (plain C99,
complex.h, full 4x4 Dirac matrices, no FMA contraction); this module only
compiles it and passes numpy arrays.

Passages followed (arXiv:1901.07294): Sec. II-A, Eq. (1) (hopping term, field
and link definitions) and the CG solve named in Sec. II-A.  Readings where the
paper is silent are listed in the header of ``wilson_oracle.c``.

Arrays are numpy complex128 in lexicographic site order
``site = x + Lx*(y + Ly*(z + Lz*t))``: spinors ``(V, 4, 3)``, links
``(V, 4, 3, 3)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_DIMS = ctypes.c_int * 4


def build(force: bool = False) -> str:
    """Compile ``liboracle.so``: -O3, OpenMP, IEEE arithmetic, no FMA contraction."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
               "-fcx-fortran-rules", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            vp, ip = ctypes.c_void_p, ctypes.c_int
            lib.oracle_gamma.argtypes = [ip, vp]
            lib.oracle_gamma.restype = None
            lib.oracle_set_threads.argtypes = [ip]
            lib.oracle_set_threads.restype = None
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = ip
            lib.oracle_hop.argtypes = [_DIMS, vp, vp, vp, ip, ip]
            lib.oracle_hop.restype = None
            lib.oracle_gamma_apply.argtypes = [ctypes.c_int64, ip, vp, vp]
            lib.oracle_gamma_apply.restype = None
            lib.oracle_dirac.argtypes = [_DIMS, vp, vp, ctypes.c_double, vp]
            lib.oracle_dirac.restype = None
            lib.oracle_mhat.argtypes = [_DIMS, vp, ctypes.c_double, ip, vp, vp]
            lib.oracle_mhat.restype = None
            lib.oracle_mdagm.argtypes = [_DIMS, vp, ctypes.c_double, vp, vp]
            lib.oracle_mdagm.restype = None
            lib.oracle_cg.argtypes = [_DIMS, vp, ctypes.c_double, vp, vp, ctypes.c_double, ip,
                                      ctypes.POINTER(ctypes.c_double)]
            lib.oracle_cg.restype = ip
            for fn in (lib.oracle_bicgstab, lib.oracle_solve_full):
                fn.argtypes = [_DIMS, vp, ctypes.c_double, vp, vp, ctypes.c_double, ip,
                               ctypes.POINTER(ctypes.c_double)]
                fn.restype = ip
            _lib = lib
    return _lib


def _dims(dims):
    return _DIMS(*[int(d) for d in dims])


def _cf(a, shape):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    assert a.shape == shape, (a.shape, shape)
    return a


def _vol(dims):
    return int(np.prod([int(d) for d in dims]))


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def gamma(mu: int) -> np.ndarray:
    """Dirac matrix gamma_mu (mu=0..3 = x,y,z,t) or gamma5 (mu=4), shape (4,4)."""
    out = np.empty((4, 4), dtype=np.complex128)
    _load().oracle_gamma(int(mu), out.ctypes.data)
    return out


def hop(dims, links, psi, out_parity: int = -1, convention: int = 0) -> np.ndarray:
    """Hopping sum.  convention 0: library H (1-gamma forward, 1+gamma backward);
    convention 1: Eq. (1) literally.  out_parity p >= 0 gives H_{p,1-p}, zero elsewhere."""
    v = _vol(dims)
    links = _cf(links, (v, 4, 3, 3))
    psi = _cf(psi, (v, 4, 3))
    out = np.empty((v, 4, 3), dtype=np.complex128)
    _load().oracle_hop(_dims(dims), links.ctypes.data, psi.ctypes.data, out.ctypes.data,
                       int(out_parity), int(convention))
    return out


def gamma_apply(mu: int, psi) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    v = psi.shape[0]
    out = np.empty_like(psi)
    _load().oracle_gamma_apply(v, int(mu), psi.ctypes.data, out.ctypes.data)
    return out


def dirac(dims, links, psi, mass: float) -> np.ndarray:
    """D psi = (m+4) psi - H psi / 2 on the full lattice."""
    v = _vol(dims)
    links = _cf(links, (v, 4, 3, 3))
    psi = _cf(psi, (v, 4, 3))
    out = np.empty((v, 4, 3), dtype=np.complex128)
    _load().oracle_dirac(_dims(dims), links.ctypes.data, psi.ctypes.data, float(mass), out.ctypes.data)
    return out


def mhat(dims, links, mass: float, x, dagger: bool = False) -> np.ndarray:
    """Even-odd Schur operator on even sites (odd sites ignored / zero)."""
    v = _vol(dims)
    links = _cf(links, (v, 4, 3, 3))
    x = _cf(x, (v, 4, 3))
    out = np.empty((v, 4, 3), dtype=np.complex128)
    _load().oracle_mhat(_dims(dims), links.ctypes.data, float(mass), int(bool(dagger)),
                        x.ctypes.data, out.ctypes.data)
    return out


def mdagm(dims, links, mass: float, x) -> np.ndarray:
    v = _vol(dims)
    links = _cf(links, (v, 4, 3, 3))
    x = _cf(x, (v, 4, 3))
    out = np.empty((v, 4, 3), dtype=np.complex128)
    _load().oracle_mdagm(_dims(dims), links.ctypes.data, float(mass), x.ctypes.data, out.ctypes.data)
    return out


def cg(dims, links, mass: float, b, tol: float = 1e-10, maxiter: int = 20000):
    """Textbook FP64 CG on Mhat^dagger Mhat x = b (even sites).

    Returns (x, iterations, true relative residual); iterations < 0 means not converged."""
    v = _vol(dims)
    links = _cf(links, (v, 4, 3, 3))
    b = _cf(b, (v, 4, 3))
    x = np.empty((v, 4, 3), dtype=np.complex128)
    rel = ctypes.c_double(0.0)
    it = _load().oracle_cg(_dims(dims), links.ctypes.data, float(mass), b.ctypes.data, x.ctypes.data,
                           float(tol), int(maxiter), ctypes.byref(rel))
    return x, int(it), float(rel.value)


def bicgstab(dims, links, mass: float, b, tol: float = 1e-10, maxiter: int = 20000):
    """Textbook FP64 BiCGStab (van der Vorst 1992) on Mhat x = b (even sites, x_0 = 0).

    Returns (x, iterations, true relative residual |b - Mhat x| / |b|); iterations < 0
    means not converged."""
    v = _vol(dims)
    links = _cf(links, (v, 4, 3, 3))
    b = _cf(b, (v, 4, 3))
    x = np.empty((v, 4, 3), dtype=np.complex128)
    rel = ctypes.c_double(0.0)
    it = _load().oracle_bicgstab(_dims(dims), links.ctypes.data, float(mass), b.ctypes.data, x.ctypes.data,
                                 float(tol), int(maxiter), ctypes.byref(rel))
    return x, int(it), float(rel.value)


def solve_full(dims, links, mass: float, b, tol: float = 1e-10, maxiter: int = 20000):
    """D x = b on the full lattice by even-odd reduction: b^_e = b_e + H_eo b_o / (2(m+4)),
    BiCGStab on Mhat x_e = b^_e, x_o = (b_o + H_oe x_e / 2) / (m+4).

    Returns (x, iterations, true relative residual |b - D x| / |b|)."""
    v = _vol(dims)
    links = _cf(links, (v, 4, 3, 3))
    b = _cf(b, (v, 4, 3))
    x = np.empty((v, 4, 3), dtype=np.complex128)
    rel = ctypes.c_double(0.0)
    it = _load().oracle_solve_full(_dims(dims), links.ctypes.data, float(mass), b.ctypes.data, x.ctypes.data,
                                   float(tol), int(maxiter), ctypes.byref(rel))
    return x, int(it), float(rel.value)


def antiperiodic_links(dims, links) -> np.ndarray:
    """Links for antiperiodic boundary conditions in t: the operator with these
    links (and periodic wrap-around) is the antiperiodic one, because every hop
    across the t boundary goes through a link U_t on the slice t = Lt-1
    (forward from t = Lt-1 by U_t(x), backward from t = 0 by U_t(x - t)^dagger).
    Pinned by the free-field plane waves with half-integer t momenta."""
    v = _vol(dims)
    out = _cf(links, (v, 4, 3, 3)).copy()
    lt = int(dims[3])
    slab = v // lt
    out[(lt - 1) * slab:, 3] *= -1.0
    return out


# Element-wise products of Sec. IV (and the complex multiply-add forms of
# Sec. III-D), written out on interleaved (re, im) float64 arrays.
STREAM_REAL_MUL, STREAM_CPLX_MUL, STREAM_CPLX_CONJ_MUL, STREAM_CPLX_MADD, STREAM_CPLX_CONJ_MADD = range(5)


def stream_mul(kind: int, x, y, z=None) -> np.ndarray:
    """kind 0: z_i = x_i y_i on real float64 arrays;
    kind 1: z = x y, 2: z = conj(x) y, 3: z = z + x y, 4: z = z + conj(x) y on complex
    numbers stored as interleaved (re, im) float64 pairs.  Returns the new z."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if kind == STREAM_REAL_MUL:
        return x * y
    xr, xi = x[0::2], x[1::2]
    yr, yi = y[0::2], y[1::2]
    if kind in (STREAM_CPLX_CONJ_MUL, STREAM_CPLX_CONJ_MADD):
        xi = -xi
    re = xr * yr - xi * yi
    im = xr * yi + xi * yr
    out = np.empty_like(x)
    if kind in (STREAM_CPLX_MADD, STREAM_CPLX_CONJ_MADD):
        z = np.asarray(z, dtype=np.float64)
        out[0::2] = z[0::2] + re
        out[1::2] = z[1::2] + im
    else:
        out[0::2] = re
        out[1::2] = im
    return out
