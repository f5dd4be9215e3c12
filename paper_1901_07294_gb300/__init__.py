"""wdirac: Wilson-Dirac operator and solvers on one NVIDIA GB300 (sm_103a).

Thin Python binding of the C ABI declared in ``include/wdirac.h``.  Every
function here only marshals arguments (tensor pointers, sizes, the current
CUDA stream) into one call of the native library ``_build/libwdirac.so``;
all computation runs in its CUDA kernels.  There is no CPU path: if the
library cannot be built or loaded, every call raises.

Arrays: device fields are opaque byte buffers (torch.uint8 CUDA tensors of
``field_bytes(...)`` bytes); canonical spinors and links are FP64 complex
arrays (torch.complex128 / float64 CUDA tensors, or numpy arrays on the host
where stated) in lexicographic order ``site = x + Lx*(y + Ly*(z + Lz*t))``.
"""
from __future__ import annotations

import ctypes
import threading

from . import _build

F64, F32, F16, BF16, DF = 0, 1, 2, 3, 4   # DF: double-word FP32 (hi + lo)
PREC_NAMES = {F64: "f64", F32: "f32", F16: "f16", BF16: "bf16", DF: "df"}
SITES_FULL, SITES_EVEN, SITES_ODD = 0, 1, 2
EVEN, ODD = 0, 1

WD_OK, WD_EINVAL, WD_ENOMEM, WD_ECUDA, WD_ENOCONV, WD_ETIMEOUT, WD_ECANCELLED, WD_EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
_STATUS = {WD_EINVAL: "EINVAL", WD_ENOMEM: "ENOMEM", WD_ECUDA: "ECUDA", WD_ENOCONV: "ENOCONV",
           WD_ETIMEOUT: "ETIMEOUT", WD_ECANCELLED: "ECANCELLED", WD_EBUSY: "EBUSY"}

_lock = threading.Lock()
_lib = None
_vp, _ip, _dp, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_DIMS = ctypes.c_int * 4


class WdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"wdirac {_STATUS.get(status, status)}: {msg}")
        self.status = status


_SIGS = {
    "wd_version": (_ip, []),
    "wd_last_error": (ctypes.c_char_p, []),
    "wd_ctx_create": (_ip, [_ip, ctypes.POINTER(_vp)]),
    "wd_ctx_destroy": (_ip, [_vp]),
    "wd_field_bytes": (_ip, [_DIMS, _ip, _ip, _ip, ctypes.POINTER(_sz)]),
    "wd_pack": (_ip, [_vp, _DIMS, _ip, _ip, _vp, _vp, _vp]),
    "wd_pack_f32": (_ip, [_vp, _DIMS, _ip, _ip, _vp, _vp, _vp]),
    "wd_unpack": (_ip, [_vp, _DIMS, _ip, _ip, _vp, _vp, _vp]),
    "wd_unpack_f32": (_ip, [_vp, _DIMS, _ip, _ip, _vp, _vp, _vp]),
    "wd_gauge_create": (_ip, [_vp, _DIMS, _vp, _ip, ctypes.POINTER(_vp)]),
    "wd_gauge_prepare": (_ip, [_vp, _ip, _ip]),
    "wd_stream_mul": (_ip, [_vp, _ip, _sz, _vp, _vp, _vp, _vp]),
    "wd_device_info": (_ip, [_vp, _vp]),
    "wd_device_status": (_ip, [_vp, _vp]),
    "wd_dd_create": (_ip, [_vp, _DIMS, _ip, _vp, _ip, ctypes.POINTER(_vp)]),
    "wd_dd_local_dims": (_ip, [_vp, _DIMS]),
    "wd_dd_set_boundary": (_ip, [_vp, _ip]),
    "wd_dd_halo_bytes": (_ip, [_vp, _ip, ctypes.POINTER(_sz)]),
    "wd_dd_dslash": (_ip, [_vp, _vp, _vp, _dp, _ip, _ip, _ip, _vp]),
    "wd_dd_destroy": (_ip, [_vp]),
    "wd_slab_create": (_ip, [_vp, _DIMS, _ip, _ip, _vp, _ip, ctypes.POINTER(_vp)]),
    "wd_slab_local_dims": (_ip, [_vp, _DIMS]),
    "wd_slab_set_boundary": (_ip, [_vp, _ip]),
    "wd_slab_face_bytes": (_ip, [_vp, _ip, ctypes.POINTER(_sz)]),
    "wd_slab_gather": (_ip, [_vp, _vp, _ip, _ip, _ip, _vp, _vp, _vp]),
    "wd_slab_interior": (_ip, [_vp, _vp, _vp, _dp, _ip, _ip, _vp]),
    "wd_slab_boundary": (_ip, [_vp, _vp, _vp, _vp, _ip, _ip, _ip, _vp]),
    "wd_slab_destroy": (_ip, [_vp]),
    "wd_gauge_set_boundary": (_ip, [_vp, _ip]),
    "wd_gauge_bytes": (_ip, [_vp, _ip, _ip, ctypes.POINTER(_sz)]),
    "wd_gauge_destroy": (_ip, [_vp]),
    "dslash_apply": (_ip, [_vp, _vp, _vp, _vp, _dp, _ip, _ip, _ip, _vp]),
"dslash_apply_dagger": (_ip, [_vp, _vp, _vp, _vp, _dp, _ip, _ip, _ip, _vp]),
    "dslash_eo_apply": (_ip, [_vp, _vp, _vp, _vp, _vp, _ip, _dp, _dp, _ip, _ip, _ip, _ip, _vp]),
    "wd_norm2": (_ip, [_vp, _DIMS, _ip, _ip, _vp, _vp, _vp]),
    "wd_dot": (_ip, [_vp, _DIMS, _ip, _ip, _vp, _vp, _vp, _vp]),
    "wd_axpby": (_ip, [_vp, _DIMS, _ip, _ip, _dp, _vp, _dp, _vp, _vp]),
    "wd_convert": (_ip, [_vp, _DIMS, _ip, _ip, _vp, _ip, _vp, _vp]),
    "cg_solve": (_ip, [_vp, _vp, _dp, _vp, _vp, _dp, _vp, _vp, _vp]),
    "bicgstab_solve": (_ip, [_vp, _vp, _dp, _vp, _vp, _dp, _vp, _vp, _vp]),
    "wilson_solve": (_ip, [_vp, _vp, _dp, _vp, _vp, _dp, _ip, _vp, _vp, _vp]),
    "wd_norm2_noalloc": (_ip, [_DIMS, _ip, _ip, _vp, _vp, _vp]),
    "wd_tune_dslash": (_ip, [_vp, _vp, _ip, _ip, _ip, _ip, _ip, _vp, _ip, ctypes.POINTER(_ip)]),
    "wd_tune_set_dslash": (_ip, [_vp, _vp, _ip, _ip, _ip, _ip, _ip, _ip, _ip]),
    "wd_tune_clear": (_ip, [_vp]),
    "cg_solve_batch": (_ip, [_vp, _ip, _vp, _ip, _vp, _vp]),
    "rq_create": (_ip, [_vp, _sz, _ip, ctypes.POINTER(_vp)]),
    "rq_submit": (_ip, [_vp, _vp, ctypes.POINTER(ctypes.c_uint64)]),
    "rq_poll": (_ip, [_vp, ctypes.c_uint64, _vp]),
    "rq_wait": (_ip, [_vp, ctypes.c_uint64, _ip, _vp]),
    "rq_cancel": (_ip, [_vp, ctypes.c_uint64]),
    "rq_stats": (_ip, [_vp, _vp]),
    "rq_destroy": (_ip, [_vp]),
    "wd_solve_workspace_bytes": (_ip, [_DIMS, _ip, ctypes.POINTER(_sz)]),
    "wd_probe_fma": (_ip, [_vp, _ip, ctypes.POINTER(_dp)]),
}


class TuneEntry(ctypes.Structure):
    """wd_tune_entry"""
    _fields_ = [("threads", _ip), ("variant", _ip), ("ms", _dp)]


class CgOpts(ctypes.Structure):
    """wd_cg_opts"""
    _fields_ = [("inner_prec", _ip), ("inner_recon", _ip), ("outer_recon", _ip), ("reliable", _ip),
                ("delta", _dp), ("maxiter", _ip), ("autotune", _ip), ("use_graph", _ip), ("outer_prec", _ip)]


class CgStats(ctypes.Structure):
    """wd_cg_stats"""
    _fields_ = [("iters", _ip), ("reliable_updates", _ip), ("status", _ip), ("true_rel_resid", _dp),
                ("seconds", _dp)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def exported_symbols() -> list[str]:
    return list(_SIGS)


def library_path() -> str:
    return _build.LIB_PATH


def load(build: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) the native library; raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB_PATH
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int) -> None:
    if status != WD_OK:
        msg = load().wd_last_error().decode(errors="replace")
        raise WdError(status, msg)


def _dims(dims):
    return _DIMS(*[int(d) for d in dims])


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


class Context:
    """A wd_ctx bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self._h = _vp()
        _check(load().wd_ctx_create(int(device), ctypes.byref(self._h)))
        self.device = int(device)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().wd_ctx_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def field_bytes(dims, sites: int, prec: int, nrhs: int = 1) -> int:
    out = _sz()
    _check(load().wd_field_bytes(_dims(dims), int(sites), int(prec), int(nrhs), ctypes.byref(out)))
    return int(out.value)


def alloc_field(dims, sites: int, prec: int, nrhs: int = 1, device="cuda"):
    """Uninitialised device field (torch.uint8 tensor) of the right size."""
    import torch
    return torch.empty(field_bytes(dims, sites, prec, nrhs), dtype=torch.uint8, device=device)


def _is_f32(t) -> bool:
    return getattr(t, "dtype", None) is not None and str(t.dtype) in ("torch.float32", "float32")


def pack(ctx: Context, dims, sites: int, prec: int, aos, field, stream=None) -> None:
    """Canonical full-lattice spinor (FP64, or FP32 for a float32 tensor; device, or pinned
    host memory the kernel reads directly) -> device field holding `sites`."""
    fn = load().wd_pack_f32 if _is_f32(aos) else load().wd_pack
    _check(fn(ctx.handle, _dims(dims), int(sites), int(prec), _ptr(aos), _ptr(field), _stream(stream)))


def unpack(ctx: Context, dims, sites: int, prec: int, field, aos, stream=None) -> None:
    """Device field -> the sites it holds inside a canonical full-lattice array (FP64, or FP32
    for a float32 tensor; device, or pinned host memory the kernel writes directly)."""
    fn = load().wd_unpack_f32 if _is_f32(aos) else load().wd_unpack
    _check(fn(ctx.handle, _dims(dims), int(sites), int(prec), _ptr(field), _ptr(aos), _stream(stream)))


class Gauge:
    """Library-owned gauge field built from canonical FP64 links (V,4,3,3).

    `links` is a CUDA tensor (complex128 or float64) or a host numpy array."""

    def __init__(self, ctx: Context, dims, links):
        self._h = _vp()
        self.ctx = ctx
        self.dims = tuple(int(d) for d in dims)
        on_host = 0
        if hasattr(links, "data_ptr"):
            if not links.is_cuda:
                raise ValueError("torch links must be a CUDA tensor (or pass a numpy array)")
            if not links.is_contiguous():
                raise ValueError("links must be contiguous")
            ptr = links.data_ptr()
        else:
            import numpy as np
            arr = np.ascontiguousarray(links, dtype=np.complex128)
            self._host_keepalive = arr
            ptr = arr.ctypes.data
            on_host = 1
        _check(load().wd_gauge_create(ctx.handle, _dims(dims), ptr, on_host, ctypes.byref(self._h)))
        self._host_keepalive = None

    @property
    def handle(self):
        return self._h

    def prepare(self, prec: int, recon: int) -> None:
        _check(load().wd_gauge_prepare(self._h, int(prec), int(recon)))

    def set_boundary(self, t_sign: int) -> None:
        """+1: periodic in t (default); -1: antiperiodic in t."""
        _check(load().wd_gauge_set_boundary(self._h, int(t_sign)))

    def nbytes(self, prec: int, recon: int) -> int:
        out = _sz()
        _check(load().wd_gauge_bytes(self._h, int(prec), int(recon), ctypes.byref(out)))
        return int(out.value)

    def close(self):
        if self._h:
            load().wd_gauge_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dslash_apply(ctx: Context, gauge: Gauge, out, inp, mass: float, nrhs: int = 1, prec: int = F32,
                 recon: int = 18, stream=None) -> None:
    """out = D in = (m+4) in - H in / 2 on full fields (asynchronous)."""
    _check(load().dslash_apply(ctx.handle, gauge.handle, _ptr(out), _ptr(inp), float(mass), int(nrhs),
                               int(prec), int(recon), _stream(stream)))


def dslash_apply_dagger(ctx: Context, gauge: Gauge, out, inp, mass: float, nrhs: int = 1, prec: int = F32,
                        recon: int = 18, stream=None) -> None:
    """out = D^dagger in = gamma5 D gamma5 in (the paper's Eq. (1) sign convention); asynchronous."""
    _check(load().dslash_apply_dagger(ctx.handle, gauge.handle, _ptr(out), _ptr(inp), float(mass), int(nrhs),
                                      int(prec), int(recon), _stream(stream)))


def dslash_eo_apply(ctx: Context, gauge: Gauge, out, inp, x, out_parity: int, a: float, b: float,
                    dagger: bool = False, nrhs: int = 1, prec: int = F32, recon: int = 18, stream=None) -> None:
    """out_p = a x_p + b H^(dagger)_{p,1-p} in_{1-p} on half fields (asynchronous)."""
    _check(load().dslash_eo_apply(ctx.handle, gauge.handle, _ptr(out), _ptr(inp), _ptr(x), int(out_parity),
                                  float(a), float(b), int(bool(dagger)), int(nrhs), int(prec), int(recon),
                                  _stream(stream)))


def norm2(ctx: Context, dims, sites: int, prec: int, x, result, stream=None) -> None:
    """result[0] = |x|^2 (FP64, device tensor of >= 1 float64)."""
    _check(load().wd_norm2(ctx.handle, _dims(dims), int(sites), int(prec), _ptr(x), _ptr(result), _stream(stream)))


def dot(ctx: Context, dims, sites: int, prec: int, a, b, result, stream=None) -> None:
    """result[0:2] = <a, b> = sum conj(a) b (FP64 re, im; device tensor)."""
    _check(load().wd_dot(ctx.handle, _dims(dims), int(sites), int(prec), _ptr(a), _ptr(b), _ptr(result),
                         _stream(stream)))


def axpby(ctx: Context, dims, sites: int, prec: int, a: float, x, b: float, y, stream=None) -> None:
    """y = a x + b y."""
    _check(load().wd_axpby(ctx.handle, _dims(dims), int(sites), int(prec), float(a), _ptr(x), float(b), _ptr(y),
                           _stream(stream)))


def convert(ctx: Context, dims, sites: int, prec_out: int, out, prec_in: int, inp, stream=None) -> None:
    """out = in with a change of storage precision."""
    _check(load().wd_convert(ctx.handle, _dims(dims), int(sites), int(prec_out), _ptr(out), int(prec_in), _ptr(inp),
                             _stream(stream)))


def cg_solve(ctx: Context, gauge: Gauge, mass: float, x, b, tol: float = 1e-10, inner_prec: int = F64,
             inner_recon: int = 18, outer_recon: int = 18, reliable: bool = True, delta: float = 0.01,
             maxiter: int = 20000, autotune: bool = False, use_graph: bool = False, stream=None,
             check: bool = True, outer_prec: int = F64) -> dict:
    """Solve Mhat^dagger Mhat x = b on even half fields (FP64).  outer_prec (F64 or DF) is the
    arithmetic of the reliable updates' operator.  Returns the solve statistics; raises WdError
    on failure unless check=False (then 'status' carries the code)."""
    opts = _solve_opts(inner_prec, inner_recon, outer_recon, reliable, delta, maxiter, autotune, use_graph,
                       outer_prec)
    st = CgStats()
    rc = load().cg_solve(ctx.handle, gauge.handle, float(mass), _ptr(x), _ptr(b), float(tol), ctypes.byref(opts),
                         ctypes.byref(st), _stream(stream))
    if check:
        _check(rc)
    out = st.as_dict()
    out["status"] = rc
    return out


SOLVER_CGNE, SOLVER_BICGSTAB = 0, 1


def _solve_opts(inner_prec, inner_recon, outer_recon, reliable, delta, maxiter, autotune, use_graph,
                outer_prec=F64):
    return CgOpts(int(inner_prec), int(inner_recon), int(outer_recon), int(bool(reliable)), float(delta),
                  int(maxiter), int(bool(autotune)), int(bool(use_graph)), int(outer_prec))


def bicgstab_solve(ctx: Context, gauge: Gauge, mass: float, x, b, tol: float = 1e-10, inner_prec: int = F64,
                   inner_recon: int = 18, outer_recon: int = 18, reliable: bool = True, delta: float = 0.01,
                   maxiter: int = 20000, autotune: bool = False, stream=None, check: bool = True,
                   outer_prec: int = F64) -> dict:
    """Solve Mhat x = b on even half fields (FP64) by BiCGStab.  Returns the solve statistics;
    raises WdError on failure unless check=False (then 'status' carries the code)."""
    opts = _solve_opts(inner_prec, inner_recon, outer_recon, reliable, delta, maxiter, autotune, False, outer_prec)
    st = CgStats()
    rc = load().bicgstab_solve(ctx.handle, gauge.handle, float(mass), _ptr(x), _ptr(b), float(tol),
                               ctypes.byref(opts), ctypes.byref(st), _stream(stream))
    if check:
        _check(rc)
    out = st.as_dict()
    out["status"] = rc
    return out


def wilson_solve(ctx: Context, gauge: Gauge, mass: float, x, b, tol: float = 1e-10, solver: int = SOLVER_BICGSTAB,
                 inner_prec: int = F64, inner_recon: int = 18, outer_recon: int = 18, reliable: bool = True,
                 delta: float = 0.01, maxiter: int = 20000, autotune: bool = False, use_graph: bool = False,
                 stream=None, check: bool = True, outer_prec: int = F64) -> dict:
    """Solve D x = b on full fields (FP64) by even-odd reduction; solver SOLVER_BICGSTAB
    (BiCGStab on Mhat) or SOLVER_CGNE (CG on the normal equations).  Returns the solve
    statistics (true_rel_resid = |b - D x| / |b|)."""
    opts = _solve_opts(inner_prec, inner_recon, outer_recon, reliable, delta, maxiter, autotune, use_graph,
                       outer_prec)
    st = CgStats()
    rc = load().wilson_solve(ctx.handle, gauge.handle, float(mass), _ptr(x), _ptr(b), float(tol), int(solver),
                             ctypes.byref(opts), ctypes.byref(st), _stream(stream))
    if check:
        _check(rc)
    out = st.as_dict()
    out["status"] = rc
    return out


class DomainDecomposition:
    """The lattice `dims` split along t into `nsub` slabs, each with its own gauge and fields,
    and the Wilson-Dirac operator applied with a halo exchange between slabs."""

    def __init__(self, ctx: Context, dims, nsub: int, links):
        import numpy as np
        self.ctx = ctx
        self.dims = tuple(int(d) for d in dims)
        self.nsub = int(nsub)
        self._h = _vp()
        if hasattr(links, "data_ptr"):
            if not links.is_cuda or not links.is_contiguous():
                raise ValueError("torch links must be a contiguous CUDA tensor (or pass a numpy array)")
            ptr, on_host = links.data_ptr(), 0
        else:
            arr = np.ascontiguousarray(links, dtype=np.complex128)
            ptr, on_host = arr.ctypes.data, 1
        _check(load().wd_dd_create(ctx.handle, _dims(self.dims), self.nsub, ptr, on_host, ctypes.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def local_dims(self) -> tuple:
        d = _DIMS()
        _check(load().wd_dd_local_dims(self._h, d))
        return tuple(d)

    def set_boundary(self, t_sign: int) -> None:
        _check(load().wd_dd_set_boundary(self._h, int(t_sign)))

    def halo_bytes(self, halo_prec: int) -> int:
        out = _sz()
        _check(load().wd_dd_halo_bytes(self._h, int(halo_prec), ctypes.byref(out)))
        return int(out.value)

    def dslash(self, outs, ins, mass: float, prec: int = F32, recon: int = 18, halo_prec: int = F32,
               stream=None) -> None:
        n = self.nsub
        po = (_vp * n)(*[_ptr(t) for t in outs])
        pi = (_vp * n)(*[_ptr(t) for t in ins])
        _check(load().wd_dd_dslash(self._h, po, pi, float(mass), int(prec), int(recon), int(halo_prec),
                                   _stream(stream)))

    def close(self):
        if self._h:
            load().wd_dd_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Slab:
    """One process's slab k of the lattice `dims` split along t into `nsub` slabs (wd_slab):
    the face gather, interior pass and boundary pass of one operator application, with the
    faces exchanged by the caller (see ddrank.SlabOperator)."""

    def __init__(self, ctx: Context, dims, nsub: int, k: int, links):
        import numpy as np
        self.ctx = ctx
        self.dims = tuple(int(d) for d in dims)
        self.nsub, self.k = int(nsub), int(k)
        self._h = _vp()
        if hasattr(links, "data_ptr"):
            if not links.is_cuda or not links.is_contiguous():
                raise ValueError("torch links must be a contiguous CUDA tensor (or pass a numpy array)")
            ptr, on_host = links.data_ptr(), 0
        else:
            arr = np.ascontiguousarray(links, dtype=np.complex128)
            ptr, on_host = arr.ctypes.data, 1
        _check(load().wd_slab_create(ctx.handle, _dims(self.dims), self.nsub, self.k, ptr, on_host,
                                     ctypes.byref(self._h)))

    def local_dims(self) -> tuple:
        d = _DIMS()
        _check(load().wd_slab_local_dims(self._h, d))
        return tuple(d)

    def set_boundary(self, t_sign: int) -> None:
        _check(load().wd_slab_set_boundary(self._h, int(t_sign)))

    def face_bytes(self, halo_prec: int) -> int:
        out = _sz()
        _check(load().wd_slab_face_bytes(self._h, int(halo_prec), ctypes.byref(out)))
        return int(out.value)

    def gather(self, inp, send_fwd, send_bwd, prec: int, recon: int, halo_prec: int, stream=None) -> None:
        _check(load().wd_slab_gather(self._h, _ptr(inp), int(prec), int(recon), int(halo_prec), _ptr(send_fwd),
                                     _ptr(send_bwd), _stream(stream)))

    def interior(self, out, inp, mass: float, prec: int, recon: int, stream=None) -> None:
        _check(load().wd_slab_interior(self._h, _ptr(out), _ptr(inp), float(mass), int(prec), int(recon),
                                       _stream(stream)))

    def boundary(self, out, recv_fwd, recv_bwd, prec: int, recon: int, halo_prec: int, stream=None) -> None:
        _check(load().wd_slab_boundary(self._h, _ptr(out), _ptr(recv_fwd), _ptr(recv_bwd), int(prec), int(recon),
                                       int(halo_prec), _stream(stream)))

    def close(self):
        if self._h:
            load().wd_slab_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


STREAM_REAL_MUL, STREAM_CPLX_MUL, STREAM_CPLX_CONJ_MUL, STREAM_CPLX_MADD, STREAM_CPLX_CONJ_MADD = range(5)


def stream_mul(ctx: Context, kind: int, n: int, x, y, z, stream=None) -> None:
    """z = x y (real, n doubles) or z = x y, conj(x) y, z + x y, z + conj(x) y (n complex numbers as
    interleaved float64 pairs), element-wise on device arrays (asynchronous)."""
    _check(load().wd_stream_mul(ctx.handle, int(kind), int(n), _ptr(x), _ptr(y), _ptr(z), _stream(stream)))


def norm2_noalloc(dims, sites: int, prec: int, x, result, stream=None) -> None:
    """result[0] = |x|^2 without any device allocation and without a context.

    For callers that must not allocate (under a host framework that owns all device
    memory, or in latency-critical loops).  Uses a fixed scratch array in the library;
    fields larger than 2,097,152 sites are rejected; concurrent calls race.  The first
    call on a device does a one-time host-side address lookup."""
    _check(load().wd_norm2_noalloc(_dims(dims), int(sites), int(prec), _ptr(x), _ptr(result), _stream(stream)))


def tune_dslash(ctx: Context, gauge: Gauge, prec: int, recon: int, full: bool, with_x: bool = False,
                nrhs: int = 1) -> list[dict]:
    """Time every launch candidate of one operator shape; the fastest is kept in ctx."""
    table = (TuneEntry * 64)()
    n = _ip(0)
    _check(load().wd_tune_dslash(ctx.handle, gauge.handle, int(prec), int(recon), int(bool(full)),
                                 int(bool(with_x)), int(nrhs), table, 64, ctypes.byref(n)))
    return [{"threads": table[k].threads, "variant": table[k].variant, "ms": table[k].ms} for k in range(n.value)]


def tune_set_dslash(ctx: Context, gauge: Gauge, prec: int, recon: int, full: bool, with_x: bool, nrhs: int,
                    threads: int, variant: int) -> None:
    _check(load().wd_tune_set_dslash(ctx.handle, gauge.handle, int(prec), int(recon), int(bool(full)),
                                     int(bool(with_x)), int(nrhs), int(threads), int(variant)))


def tune_clear(ctx: Context) -> None:
    _check(load().wd_tune_clear(ctx.handle))


BATCH_SEQUENTIAL, BATCH_GRAPH, BATCH_PERSISTENT = 0, 1, 2


def _problem_opts(p: dict, inner_default: int) -> CgOpts:
    return _solve_opts(p.get("inner_prec", inner_default), p.get("inner_recon", 18), p.get("outer_recon", 18),
                       p.get("reliable", True), p.get("delta", 0.01), p.get("maxiter", 20000),
                       p.get("autotune", False), p.get("use_graph", False), p.get("outer_prec", F64))


class SolveDesc(ctypes.Structure):
    """wd_solve_desc"""
    _fields_ = [("gauge", _vp), ("mass", _dp), ("tol", _dp), ("x_e", _vp), ("b_e", _vp), ("opts", CgOpts)]


def cg_solve_batch(ctx: Context, problems: list[dict], mode: int = BATCH_SEQUENTIAL, stream=None,
                   check: bool = True) -> list[dict]:
    """Run many solves.  Each problem: dict(gauge, mass, tol, x, b, and optional cg_solve options
    inner_prec, inner_recon, outer_recon, reliable, delta, maxiter, autotune, outer_prec)."""
    n = len(problems)
    descs = (SolveDesc * max(n, 1))()
    for k, p in enumerate(problems):
        o = _problem_opts(p, F32)
        descs[k] = SolveDesc(p["gauge"].handle, float(p["mass"]), float(p["tol"]), _ptr(p["x"]), _ptr(p["b"]), o)
    stats = (CgStats * max(n, 1))()
    rc = load().cg_solve_batch(ctx.handle, n, descs, int(mode), stats, _stream(stream))
    if check:
        _check(rc)
    out = [stats[k].as_dict() for k in range(n)]
    for d in out:
        d["batch_status"] = rc
    return out


class SolveResult(ctypes.Structure):
    """wd_solve_result"""
    _fields_ = [("status", _ip), ("stats", CgStats), ("t_submit", _dp), ("t_admit", _dp), ("t_start", _dp),
                ("t_finish", _dp)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "stats"}
        d.update({f"cg_{k}": v for k, v in self.stats.as_dict().items()})
        return d


class RqCounters(ctypes.Structure):
    """rq_counters"""
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("admission_stalls", ctypes.c_uint64),
                ("steps", ctypes.c_uint64), ("mean_running", _dp), ("waiting", _ip), ("running", _ip),
                ("hbm_in_use", _sz), ("group_launches", ctypes.c_uint64), ("mean_group_size", _dp)]


def _desc(p: dict) -> SolveDesc:
    o = _problem_opts(p, F16)
    return SolveDesc(p["gauge"].handle, float(p["mass"]), float(p["tol"]), _ptr(p["x"]), _ptr(p["b"]), o)


_live_queues = None


def _close_live_queues():
    for q in list(_live_queues or ()):
        try:
            q.close()
        except Exception:
            pass


class Queue:
    """Solve-request queue with continuous batching (rq_* of the C ABI).

    Queues still open when the interpreter exits are closed by an exit handler, which
    runs before the CUDA runtime and torch are torn down: closing waits for the requests
    in flight, whose fields must stay alive until then."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int, max_slots: int):
        global _live_queues
        self._h = _vp()
        self.ctx = ctx
        _check(load().rq_create(ctx.handle, _sz(int(hbm_budget_bytes)), int(max_slots), ctypes.byref(self._h)))
        if _live_queues is None:
            import atexit
            import weakref
            _live_queues = weakref.WeakSet()
            atexit.register(_close_live_queues)   # registered after torch and the CUDA runtime: runs first
        _live_queues.add(self)

    def submit(self, problem: dict) -> int:
        t = ctypes.c_uint64(0)
        d = _desc(problem)
        _check(load().rq_submit(self._h, ctypes.byref(d), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int):
        r = SolveResult()
        rc = load().rq_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(r))
        if rc == WD_EBUSY:
            return None
        _check(rc)
        return r.as_dict()

    def wait(self, ticket: int, timeout_ms: int = -1):
        r = SolveResult()
        _check(load().rq_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(r)))
        return r.as_dict()

    def cancel(self, ticket: int) -> None:
        _check(load().rq_cancel(self._h, ctypes.c_uint64(ticket)))

    def stats(self) -> dict:
        c = RqCounters()
        _check(load().rq_stats(self._h, ctypes.byref(c)))
        return {k: getattr(c, k) for k, _ in c._fields_}

    def close(self) -> None:
        if self._h:
            load().rq_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_workspace_bytes(dims, inner_prec: int) -> int:
    """Device workspace one queued (or graph-batched) solve allocates while it runs."""
    out = _sz()
    _check(load().wd_solve_workspace_bytes(_dims(dims), int(inner_prec), ctypes.byref(out)))
    return int(out.value)


class DeviceProps(ctypes.Structure):
    """wd_device_props"""
    _fields_ = [("sm_count", _ip), ("mem_clock_khz", _ip), ("mem_bus_bits", _ip), ("l2_bytes", _ip),
                ("cc_major", _ip), ("cc_minor", _ip), ("nominal_hbm_gbs", _dp), ("pageable_memory_access", _ip)]


def device_info(ctx: Context) -> dict:
    """SM count, memory clock and bus width, L2 size, compute capability, the nominal HBM GB/s
    and whether kernels can access pageable host memory."""
    p = DeviceProps()
    _check(load().wd_device_info(ctx.handle, ctypes.byref(p)))
    return {f: getattr(p, f) for f, _ in DeviceProps._fields_}


def device_status(ctx: Context) -> int:
    """Waits for the device, then returns and clears the context's asynchronous status
    word (0, or a WD_E* code a kernel's bounded wait recorded)."""
    out = _ip(0)
    _check(load().wd_device_status(ctx.handle, ctypes.byref(out)))
    return int(out.value)


def probe_fma_tflops(ctx: Context, prec: int) -> float:
    """Measured FMA throughput (TFLOP/s) of the device in FP64 or FP32."""
    out = _dp(0.0)
    _check(load().wd_probe_fma(ctx.handle, int(prec), ctypes.byref(out)))
    return float(out.value)
