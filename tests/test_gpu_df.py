"""GPU parity of the double-word FP32 format (WD_DF: each real is hi + lo, two FP32
numbers) against the FP64 oracle, through the C ABI.

Representation: hi is d rounded to 24 significant bits and lo the remainder d - hi rounded
to 24 bits, so |lo| <= ulp(hi)/2 <= 2^-24 |hi| and |d - (hi + lo)| <= 2^-24 |lo| <= 2^-48 |hi|.
Reading a stored value back as FP64 adds one FP64 rounding of hi + lo (2^-53 |d|), and
|hi| <= (1 + 2^-24) |d|: REPR = 1.04 x 2^-48 bounds the relative error of every real.

Operator bar.  The FP64 kernels are held to 1e-13 relative max error, about 900
unit roundoffs (2^-53).  The double-word unit roundoff is 2^-48, 32 times larger,
and its operations carry larger constants than one FP64 rounding (Joldes, Muller
and Popescu 2017: 3u^2 for the sloppy double-word sum of same-sign terms, 5u^2 for
the double-word product, u = 2^-24; the compensated dot product of Ogita, Rump and
Oishi 2005 adds gamma_n^2 times the sum of the term magnitudes).  TOL_DF = 32 x 3 x
1e-13 ~ 1e-11.
"""
import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import pack_field, unpack_field
from tests._lattice import parity, rel_max_err, volume

pytestmark = pytest.mark.gpu

TOL_DF = 1e-11
REPR = 1.04 * 2.0 ** -48
DIMS = [(8, 8, 8, 8), (4, 6, 8, 10), (16, 16, 16, 32)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    return wd.Context(0)


_cache = {}


def _inputs(dims):
    if dims not in _cache:
        U = synth.gauge(dims, seed=synth.LINK_SEED_BASE + volume(dims) % 997)
        psi = synth.spinor(dims, seed=synth.SOURCE_SEED_BASE + 1)
        _cache[dims] = (U, psi)
    return _cache[dims]


@pytest.mark.parametrize("sites", [wd.SITES_FULL, wd.SITES_EVEN])
def test_df_pack_round_trip(ctx, sites):
    dims = (4, 6, 8, 10)
    psi = synth.spinor(dims, seed=2011)
    back = unpack_field(ctx, dims, sites, wd.DF, pack_field(ctx, dims, sites, wd.DF, psi))
    held = np.ones(volume(dims), dtype=bool) if sites == wd.SITES_FULL else parity(dims) == 0
    d = psi[held].view(np.float64).ravel()
    e = np.abs(back[held].view(np.float64).ravel() - d)
    assert np.all(e <= REPR * np.abs(d)), float(np.max(e / np.abs(d)))
    assert np.all(back[~held] == 0)


def test_df_field_bytes_equal_f64(ctx):
    for sites in (wd.SITES_FULL, wd.SITES_EVEN):
        assert wd.field_bytes((4, 6, 8, 10), sites, wd.DF) == wd.field_bytes((4, 6, 8, 10), sites, wd.F64)


def test_df_convert_and_norm(ctx):
    """wd_convert F64 -> DF -> F64 keeps each real to REPR; DF -> F32 gives the bytes of
    F64 -> F32 (hi is the FP32 rounding of the real); |x|^2 of the DF field matches the
    FP64 one to 1e-14."""
    import torch
    dims = (4, 6, 8, 10)
    psi = synth.spinor(dims, seed=2021)
    f64 = pack_field(ctx, dims, wd.SITES_FULL, wd.F64, psi)
    fdf = wd.alloc_field(dims, wd.SITES_FULL, wd.DF)
    back = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
    a32 = wd.alloc_field(dims, wd.SITES_FULL, wd.F32)
    b32 = wd.alloc_field(dims, wd.SITES_FULL, wd.F32)
    wd.convert(ctx, dims, wd.SITES_FULL, wd.DF, fdf, wd.F64, f64)
    wd.convert(ctx, dims, wd.SITES_FULL, wd.F64, back, wd.DF, fdf)
    wd.convert(ctx, dims, wd.SITES_FULL, wd.F32, a32, wd.DF, fdf)
    wd.convert(ctx, dims, wd.SITES_FULL, wd.F32, b32, wd.F64, f64)
    r = torch.zeros(2, dtype=torch.float64, device="cuda")
    wd.norm2(ctx, dims, wd.SITES_FULL, wd.DF, fdf, r[0:1])
    wd.norm2(ctx, dims, wd.SITES_FULL, wd.F64, f64, r[1:2])
    torch.cuda.synchronize()
    got = unpack_field(ctx, dims, wd.SITES_FULL, wd.F64, back).view(np.float64).ravel()
    d = psi.view(np.float64).ravel()
    assert np.all(np.abs(got - d) <= REPR * np.abs(d))
    assert torch.equal(a32, b32)
    n_df, n_64 = r.cpu().numpy()
    assert abs(n_df - n_64) <= 1e-14 * n_64


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("recon", [18, 12])
def test_dslash_full_df_matches_oracle(ctx, dims, recon):
    U, psi = _inputs(dims)
    g = wd.Gauge(ctx, dims, U)
    fin = pack_field(ctx, dims, wd.SITES_FULL, wd.DF, psi)
    fout = wd.alloc_field(dims, wd.SITES_FULL, wd.DF)
    wd.dslash_apply(ctx, g, fout, fin, 0.1, prec=wd.DF, recon=recon)
    got = unpack_field(ctx, dims, wd.SITES_FULL, wd.DF, fout)
    err = rel_max_err(got, oracle.dirac(dims, U, psi, 0.1))
    assert err < TOL_DF, f"err {err:.3e}"


@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("out_parity", [0, 1])
@pytest.mark.parametrize("with_x", [False, True])
@pytest.mark.parametrize("variant,recon", [(0, 18), (1, 18), (15, 18), (0, 12), (15, 12)])
def test_dslash_eo_df_matches_oracle(ctx, dagger, out_parity, with_x, variant, recon):
    """Variant 15 is the three-threads-per-site kernel; with 12-real links each of its
    warps rebuilds one entry of the third row and the block shares them."""
    dims = (4, 6, 8, 10)
    U, psi = _inputs(dims)
    xs = synth.spinor(dims, seed=2099)
    a, b = 1.7, -0.35
    g = wd.Gauge(ctx, dims, U)
    wd.tune_set_dslash(ctx, g, wd.DF, recon, False, with_x, 1, 128, variant)
    p = out_parity
    in_sites = wd.SITES_ODD if p == 0 else wd.SITES_EVEN
    out_sites = wd.SITES_EVEN if p == 0 else wd.SITES_ODD
    fin = pack_field(ctx, dims, in_sites, wd.DF, psi)
    fx = pack_field(ctx, dims, out_sites, wd.DF, xs) if with_x else None
    fout = wd.alloc_field(dims, out_sites, wd.DF)
    wd.dslash_eo_apply(ctx, g, fout, fin, fx, p, a, b, dagger=dagger, prec=wd.DF, recon=recon)
    got = unpack_field(ctx, dims, out_sites, wd.DF, fout)
    par = parity(dims)
    src = psi.copy()
    src[par == p] = 0
    if dagger:
        h = oracle.gamma_apply(4, oracle.hop(dims, U, oracle.gamma_apply(4, src), out_parity=p))
    else:
        h = oracle.hop(dims, U, src, out_parity=p)
    ref = b * h + (a * xs if with_x else 0)
    err = rel_max_err(got[par == p], ref[par == p])
    assert err < TOL_DF, f"err {err:.3e}"


def test_df_tuner_candidates(ctx):
    """The tuner times only the double-word kernels: schedules 0 and 1 (one block per SM) and
    the three-threads-per-site kernel (variant 15)."""
    dims = (8, 8, 8, 8)
    U, _ = _inputs(dims)
    g = wd.Gauge(ctx, dims, U)
    table = wd.tune_dslash(ctx, g, wd.DF, 18, full=False, with_x=True)
    assert table and {r["variant"] for r in table} <= {0, 1, 15}


def test_df_rejected_where_not_supported(ctx):
    """Double-word storage is a field and operator format: not a solver inner precision."""
    dims = (4, 4, 4, 4)
    g = wd.Gauge(ctx, dims, synth.gauge(dims, seed=1011))
    b = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
    x = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
    b.zero_()
    with pytest.raises(wd.WdError) as e:
        wd.cg_solve(ctx, g, 0.1, x, b, tol=1e-8, inner_prec=wd.DF)
    assert e.value.status == wd.WD_EINVAL
