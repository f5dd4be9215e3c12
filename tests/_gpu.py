"""GPU test helpers: move canonical numpy arrays through the library's pack/unpack."""
import numpy as np

import paper_1901_07294_gb300 as wd

TOL = {wd.F64: 1e-13, wd.F32: 1e-5, wd.F16: 3e-3, wd.BF16: 3e-3}   # relative max error vs the FP64 oracle


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128).view(np.float64).copy()).cuda()


def to_host(t, shape):
    return t.cpu().numpy().view(np.complex128).reshape(shape)


def pack_field(ctx, dims, sites, prec, psi):
    """numpy (V,4,3) canonical spinor -> device field of `sites`."""
    f = wd.alloc_field(dims, sites, prec)
    wd.pack(ctx, dims, sites, prec, to_dev(psi), f)
    return f


def unpack_field(ctx, dims, sites, prec, field):
    """device field -> numpy (V,4,3); sites not held by the field are zero."""
    import torch
    v = int(np.prod(dims))
    out = torch.zeros(v * 24, dtype=torch.float64, device="cuda")
    wd.unpack(ctx, dims, sites, prec, field, out)
    torch.cuda.synchronize()
    return to_host(out, (v, 4, 3))


# ---- storage rounding emulated in numpy (test side, independent of the library) ----
# Used where a result is compared with the oracle applied to the same rounded
# inputs, which separates the kernel's arithmetic and output rounding from the
# rounding of its inputs.

def _bf16_rne(x32):
    """float32 array -> nearest bfloat16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def round_spinor(psi, prec):
    """The values a field of precision `prec` holds after wd.pack (per-site scaled for 16-bit types)."""
    if prec == wd.F64:
        return psi.copy()
    v = psi.view(np.float64).reshape(-1, 24).astype(np.float32)
    if prec == wd.F32:
        return v.astype(np.float64).view(np.complex128).reshape(psi.shape)
    m = np.max(np.abs(v), axis=1, keepdims=True).astype(np.float32)
    inv = np.where(m > 0, np.float32(1) / np.where(m > 0, m, 1), 0).astype(np.float32)
    t = (v * inv).astype(np.float32)
    q = t.astype(np.float16).astype(np.float32) if prec == wd.F16 else _bf16_rne(t)
    back = (q * m).astype(np.float32)
    return back.astype(np.float64).view(np.complex128).reshape(psi.shape)


def round_links(U, prec, recon):
    """Links as the kernel sees them: storage rounding (BF16 fields use FP16 links) and, for
    12-real storage, row 3 rebuilt as conj(row0 x row1) from the stored rows."""
    if prec == wd.F64:
        r = U.copy()
    else:
        re = U.real.astype(np.float32)
        im = U.imag.astype(np.float32)
        if prec in (wd.F16, wd.BF16):
            re = re.astype(np.float16).astype(np.float32)
            im = im.astype(np.float16).astype(np.float32)
        r = re.astype(np.float64) + 1j * im.astype(np.float64)
    if recon == 12:
        r[..., 2, :] = np.conj(np.cross(r[..., 0, :], r[..., 1, :]))
    return r


def check_dslash(got, ref, prec, dims, U, psi_src, recon, fn, out_roundings=1):
    """Parity check.  FP64/FP32/FP16: against the oracle on the exact inputs with the stated
    bar.  BF16 (unit roundoff 2^-8, so the output rounding alone may reach 2^-9 of a site's
    largest component): against the oracle applied to the same BF16/FP16-rounded inputs,
    within 2^-9 per rounding of the stored output (out_roundings: 2 where a second pass
    reads, updates and stores the output again) plus FP32 arithmetic."""
    from tests._lattice import rel_max_err
    if prec != wd.BF16:
        err = rel_max_err(got, ref)
        assert err < TOL[prec], err
        return err
    ref_r = fn(round_links(U, prec, recon), round_spinor(psi_src, prec))
    err = float(np.max(np.abs((got - ref_r).view(np.float64))) / np.max(np.abs(ref.view(np.float64))))
    assert err < out_roundings * 2.0 ** -9 * 1.05, err
    return err
