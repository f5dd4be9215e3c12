"""BLAS-1 kernels (norm, dot, axpby, convert) against numpy on the unpacked fields."""
import numpy as np
import pytest

import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import pack_field, unpack_field
from tests._lattice import parity

pytestmark = pytest.mark.gpu

DIMS = (4, 6, 8, 10)
RTOL = {wd.F64: 1e-14, wd.F32: 1e-6, wd.F16: 1e-5, wd.BF16: 1e-5}


@pytest.fixture(scope="module")
def ctx():
    return wd.Context(0)


def _res():
    import torch
    return torch.zeros(4, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec", [wd.F64, wd.F32, wd.F16, wd.BF16])
@pytest.mark.parametrize("sites", [wd.SITES_FULL, wd.SITES_EVEN, wd.SITES_ODD])
def test_norm_and_dot(ctx, prec, sites):
    import torch
    a = synth.spinor(DIMS, seed=5)
    b = synth.spinor(DIMS, seed=6)
    fa = pack_field(ctx, DIMS, sites, prec, a)
    fb = pack_field(ctx, DIMS, sites, prec, b)
    # reference on the stored (rounded) values, so only the summation is tested
    ra = unpack_field(ctx, DIMS, sites, prec, fa)
    rb = unpack_field(ctx, DIMS, sites, prec, fb)
    res = _res()
    wd.norm2(ctx, DIMS, sites, prec, fa, res)
    torch.cuda.synchronize()
    n2 = float(np.sum(np.abs(ra) ** 2))
    assert abs(res[0].item() - n2) / n2 < RTOL[prec]
    wd.dot(ctx, DIMS, sites, prec, fa, fb, res)
    torch.cuda.synchronize()
    d = np.vdot(ra, rb)
    assert abs(complex(res[0].item(), res[1].item()) - d) / abs(d) < 10 * RTOL[prec] * n2 / abs(d)
    # deterministic: a second call gives the same bits
    wd.dot(ctx, DIMS, sites, prec, fa, fb, res[2:])
    torch.cuda.synchronize()
    assert res[0].item() == res[2].item() and res[1].item() == res[3].item()


@pytest.mark.parametrize("prec", [wd.F64, wd.F32, wd.F16, wd.BF16])
def test_axpby_and_convert(ctx, prec):
    a = synth.spinor(DIMS, seed=7)
    b = synth.spinor(DIMS, seed=8)
    sites = wd.SITES_EVEN
    par = parity(DIMS)
    fa = pack_field(ctx, DIMS, sites, prec, a)
    fb = pack_field(ctx, DIMS, sites, prec, b)
    ra = unpack_field(ctx, DIMS, sites, prec, fa)
    rb = unpack_field(ctx, DIMS, sites, prec, fb)
    wd.axpby(ctx, DIMS, sites, prec, 0.75, fa, -1.25, fb)
    got = unpack_field(ctx, DIMS, sites, prec, fb)
    ref = 0.75 * ra - 1.25 * rb
    tol = {wd.F64: 1e-15, wd.F32: 1e-6, wd.F16: 2e-3, wd.BF16: 1e-2}[prec]
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < tol
    f64 = wd.alloc_field(DIMS, sites, wd.F64)
    wd.convert(ctx, DIMS, sites, wd.F64, f64, prec, fa)
    back = unpack_field(ctx, DIMS, sites, wd.F64, f64)
    assert np.array_equal(back[par == 0], ra[par == 0])


def test_fma_probe_reports_plausible_rates(ctx):
    f64 = wd.probe_fma_tflops(ctx, wd.F64)
    f32 = wd.probe_fma_tflops(ctx, wd.F32)
    assert 0.1 < f64 < 200.0 and 1.0 < f32 < 500.0
    assert f32 > f64
    with pytest.raises(wd.WdError):
        wd.probe_fma_tflops(ctx, wd.F16)
