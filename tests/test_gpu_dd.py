"""Domain-decomposed operator (slabs along t with a halo exchange) against the oracle.

The decomposed operator is D on the global lattice by definition, so the oracle's
global D is the reference.  Slab k's field is the k-th contiguous slice of the
global canonical array (t is the slowest index).
"""
import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import TOL, check_dslash, pack_field, unpack_field
from tests._lattice import rel_max_err, volume

pytestmark = pytest.mark.gpu

DIMS = (4, 6, 4, 8)
MASS = 0.1


@pytest.fixture(scope="module")
def ctx():
    return wd.Context(0)


def _apply_dd(ctx, dims, U, psi, nsub, prec, recon, halo_prec, t_sign=1):
    dd = wd.DomainDecomposition(ctx, dims, nsub, U)
    if t_sign != 1:
        dd.set_boundary(t_sign)
    ld = dd.local_dims()
    assert ld == (dims[0], dims[1], dims[2], dims[3] // nsub)
    vloc = volume(ld)
    ins = [pack_field(ctx, ld, wd.SITES_FULL, prec, psi[k * vloc:(k + 1) * vloc]) for k in range(nsub)]
    outs = [wd.alloc_field(ld, wd.SITES_FULL, prec) for _ in range(nsub)]
    dd.dslash(outs, ins, MASS, prec=prec, recon=recon, halo_prec=halo_prec)
    got = np.concatenate([unpack_field(ctx, ld, wd.SITES_FULL, prec, o) for o in outs])
    dd.close()
    return got


@pytest.mark.parametrize("nsub", [1, 2, 4])
@pytest.mark.parametrize("prec", [wd.F64, wd.F32, wd.F16, wd.BF16])
@pytest.mark.parametrize("recon", [18, 12])
def test_dd_matches_global_operator(ctx, nsub, prec, recon):
    """The boundary pass reads, updates and stores the output of the slab-boundary sites
    again, so 16-bit outputs there are rounded twice (the BF16 bound doubles)."""
    U = synth.gauge(DIMS, seed=1601)
    psi = synth.spinor(DIMS, seed=3601)
    got = _apply_dd(ctx, DIMS, U, psi, nsub, prec, recon, halo_prec=wd.F64 if prec == wd.F64 else wd.F32)
    check_dslash(got, oracle.dirac(DIMS, U, psi, MASS), prec, DIMS, U, psi, recon,
                 lambda u, p: oracle.dirac(DIMS, u, p, MASS), out_roundings=2)


@pytest.mark.parametrize("halo_prec", [wd.F64, wd.F32, wd.F16])
@pytest.mark.parametrize("prec", [wd.F64, wd.F32])
def test_dd_halo_precision(ctx, halo_prec, prec):
    """Faces exchanged in a coarser format: the result is bounded by the coarser of the
    field's and the halo's storage bars (FP16 halos are the paper's compressed exchange)."""
    U = synth.gauge(DIMS, seed=1602)
    psi = synth.spinor(DIMS, seed=3602)
    got = _apply_dd(ctx, DIMS, U, psi, 2, prec, 18, halo_prec)
    err = rel_max_err(got, oracle.dirac(DIMS, U, psi, MASS))
    bar = max(TOL[prec], TOL[halo_prec])
    assert err < bar, err
    if halo_prec == wd.F16:
        assert err > TOL[wd.F32]     # the compression is visible, i.e. the halos are really used


@pytest.mark.parametrize("nsub", [1, 2, 4])
def test_dd_antiperiodic(ctx, nsub):
    U = synth.gauge(DIMS, seed=1603)
    psi = synth.spinor(DIMS, seed=3603)
    got = _apply_dd(ctx, DIMS, U, psi, nsub, wd.F64, 18, wd.F64, t_sign=-1)
    ref = oracle.dirac(DIMS, oracle.antiperiodic_links(DIMS, U), psi, MASS)
    assert rel_max_err(got, ref) < 1e-13


def test_dd_equals_single_domain_kernel(ctx):
    """FP64 fields and halos: the decomposed operator equals the single-domain kernel up to
    the summation order at the slab boundaries."""
    dims = (8, 4, 4, 16)
    U = synth.gauge(dims, seed=1604)
    psi = synth.spinor(dims, seed=3604)
    g = wd.Gauge(ctx, dims, U)
    out = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
    wd.dslash_apply(ctx, g, out, pack_field(ctx, dims, wd.SITES_FULL, wd.F64, psi), MASS, prec=wd.F64)
    single = unpack_field(ctx, dims, wd.SITES_FULL, wd.F64, out)
    for nsub in (2, 4, 8):
        got = _apply_dd(ctx, dims, U, psi, nsub, wd.F64, 18, wd.F64)
        assert rel_max_err(got, single) < 1e-15, nsub


def test_dd_repeated_applications_and_halo_bytes(ctx):
    """Back-to-back applications on the same decomposition (the halo buffers are reused)
    give the same result; the exchanged bytes are 2 faces x 2 parities x nsub slabs."""
    U = synth.gauge(DIMS, seed=1605)
    psi = synth.spinor(DIMS, seed=3605)
    dd = wd.DomainDecomposition(ctx, DIMS, 2, U)
    ld = dd.local_dims()
    vloc = volume(ld)
    ins = [pack_field(ctx, ld, wd.SITES_FULL, wd.F32, psi[k * vloc:(k + 1) * vloc]) for k in range(2)]
    outs = [wd.alloc_field(ld, wd.SITES_FULL, wd.F32) for _ in range(2)]
    res = []
    for _ in range(3):
        dd.dslash(outs, ins, MASS, prec=wd.F32)
        res.append(np.concatenate([unpack_field(ctx, ld, wd.SITES_FULL, wd.F32, o) for o in outs]))
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[1], res[2])
    nf = DIMS[0] * DIMS[1] * DIMS[2] // 2
    assert dd.halo_bytes(wd.F32) == 2 * 2 * 2 * nf * 48
    assert dd.halo_bytes(wd.F16) == 2 * 2 * 2 * nf * 28


def test_dd_arguments(ctx):
    U = synth.gauge(DIMS, seed=1606)
    with pytest.raises(wd.WdError):
        wd.DomainDecomposition(ctx, DIMS, 3, U)      # 3 does not divide L_t = 8
    with pytest.raises(wd.WdError):
        wd.DomainDecomposition(ctx, (4, 6, 4, 6), 2, synth.gauge((4, 6, 4, 6), seed=1))   # local L_t = 3
    dd = wd.DomainDecomposition(ctx, DIMS, 2, U)
    with pytest.raises(wd.WdError):
        dd.set_boundary(2)
    with pytest.raises(wd.WdError):
        dd.halo_bytes(wd.BF16)
