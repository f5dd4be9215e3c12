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
