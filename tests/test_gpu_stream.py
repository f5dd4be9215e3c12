"""Element-wise products (Sec. IV, Sec. III-D forms) on the GPU against the oracle.

The real product is one rounding on both sides: bit-exact.  The complex forms
use FMA on the GPU and multiply-then-add in the oracle; both are within two
roundings of the exact value per component, so they agree within
6 u (|xr yr| + |xi yi| + |z|) with u = 2^-53.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1901_07294_gb300 as wd

pytestmark = pytest.mark.gpu

U53 = 2.0 ** -53


@pytest.fixture(scope="module")
def ctx():
    return wd.Context(0)


def _arrays(n_reals, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(n_reals) for _ in range(3)]


@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000, 1 << 20 | 3])
def test_real_product_bit_exact(ctx, n):
    x, y, _ = _arrays(max(n, 1), 61)
    x, y = x[:n], y[:n]
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    dz = torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device="cuda")
    wd.stream_mul(ctx, wd.STREAM_REAL_MUL, n, dx, dy, dz)
    got = dz.cpu().numpy()[:n]
    assert np.array_equal(got, oracle.stream_mul(oracle.STREAM_REAL_MUL, x, y))


@pytest.mark.parametrize("kind", [wd.STREAM_CPLX_MUL, wd.STREAM_CPLX_CONJ_MUL, wd.STREAM_CPLX_MADD,
                                  wd.STREAM_CPLX_CONJ_MADD])
@pytest.mark.parametrize("n", [1, 5, 1023, 1 << 19 | 1])
def test_complex_products(ctx, kind, n):
    x, y, z = _arrays(2 * n, 62 + kind)
    ref = oracle.stream_mul(kind, x, y, z)
    dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
    wd.stream_mul(ctx, kind, n, dx, dy, dz)
    got = dz.cpu().numpy()
    madd = kind in (wd.STREAM_CPLX_MADD, wd.STREAM_CPLX_CONJ_MADD)
    mag = np.abs(x[0::2] * y[0::2]) + np.abs(x[1::2] * y[1::2])
    mag_i = np.abs(x[0::2] * y[1::2]) + np.abs(x[1::2] * y[0::2])
    bound_r = 6 * U53 * (mag + (np.abs(z[0::2]) if madd else 0))
    bound_i = 6 * U53 * (mag_i + (np.abs(z[1::2]) if madd else 0))
    assert np.all(np.abs(got[0::2] - ref[0::2]) <= bound_r)
    assert np.all(np.abs(got[1::2] - ref[1::2]) <= bound_i)


def test_in_place_and_arguments(ctx):
    n = 4096
    x, y, _ = _arrays(2 * n, 70)
    ref = oracle.stream_mul(wd.STREAM_CPLX_MUL, x, y)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    wd.stream_mul(ctx, wd.STREAM_CPLX_MUL, n, dx, dy, dx)       # z = x in place
    got = dx.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-15 * np.max(np.abs(ref))
    with pytest.raises(wd.WdError):
        wd.stream_mul(ctx, 9, n, dx, dy, dy)
    raw = torch.empty(2 * n + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(wd.WdError):
        wd.stream_mul(ctx, wd.STREAM_CPLX_MUL, n, raw[1:], dy, dy)   # 8-byte offset: not 16-byte aligned
