"""Multi right-hand-side operator (links shared by all fields of a launch) against the oracle."""
import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import TOL, check_dslash, pack_field, round_spinor, unpack_field
from tests._lattice import parity, rel_max_err

pytestmark = pytest.mark.gpu

DIMS = (4, 6, 8, 10)


def _fields(ctx, dims, sites, prec, srcs):
    import torch
    return torch.cat([pack_field(ctx, dims, sites, prec, s) for s in srcs])


@pytest.mark.parametrize("prec", [wd.F64, wd.F32, wd.F16, wd.BF16])
@pytest.mark.parametrize("threads", [32, 128, 256])
@pytest.mark.parametrize("recon", [18, 12])
def test_mrhs_full_matches_oracle(prec, threads, recon):
    ctx = wd.Context(0)
    U = synth.gauge(DIMS, seed=1234)
    nrhs = 5
    srcs = [synth.spinor(DIMS, seed=2200 + k) for k in range(nrhs)]
    g = wd.Gauge(ctx, DIMS, U)
    wd.tune_set_dslash(ctx, g, prec, recon, True, True, nrhs, threads, 3)
    fin = _fields(ctx, DIMS, wd.SITES_FULL, prec, srcs)
    fout = wd.alloc_field(DIMS, wd.SITES_FULL, prec, nrhs)
    wd.dslash_apply(ctx, g, fout, fin, 0.1, nrhs=nrhs, prec=prec, recon=recon)
    nb = wd.field_bytes(DIMS, wd.SITES_FULL, prec)
    for k in range(nrhs):
        got = unpack_field(ctx, DIMS, wd.SITES_FULL, prec, fout[k * nb:(k + 1) * nb])
        check_dslash(got, oracle.dirac(DIMS, U, srcs[k], 0.1), prec, DIMS, U, srcs[k], recon,
                     lambda u, p: oracle.dirac(DIMS, u, p, 0.1))


@pytest.mark.parametrize("prec", [wd.F32, wd.F16, wd.BF16])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("with_x", [False, True])
def test_mrhs_eo_matches_oracle(prec, dagger, with_x):
    ctx = wd.Context(0)
    U = synth.gauge(DIMS, seed=1235)
    nrhs = 12
    srcs = [synth.spinor(DIMS, seed=2300 + k) for k in range(nrhs)]
    xs = [synth.spinor(DIMS, seed=2400 + k) for k in range(nrhs)]
    g = wd.Gauge(ctx, DIMS, U)
    fin = _fields(ctx, DIMS, wd.SITES_ODD, prec, srcs)
    fx = _fields(ctx, DIMS, wd.SITES_EVEN, prec, xs) if with_x else None
    fout = wd.alloc_field(DIMS, wd.SITES_EVEN, prec, nrhs)
    a, b = 0.7, -1.3
    wd.dslash_eo_apply(ctx, g, fout, fin, fx, 0, a, b, dagger=dagger, nrhs=nrhs, prec=prec, recon=18)
    par = parity(DIMS)
    nb = wd.field_bytes(DIMS, wd.SITES_EVEN, prec)
    def op(u, src, x):
        src = src.copy()
        src[par == 0] = 0
        if dagger:
            h = oracle.gamma_apply(4, oracle.hop(DIMS, u, oracle.gamma_apply(4, src), out_parity=0))
        else:
            h = oracle.hop(DIMS, u, src, out_parity=0)
        r = b * h + (a * x if with_x else 0)
        return r[par == 0]

    for k in range(nrhs):
        got = unpack_field(ctx, DIMS, wd.SITES_EVEN, prec, fout[k * nb:(k + 1) * nb])[par == 0]
        x_r = round_spinor(xs[k], prec) if prec == wd.BF16 else xs[k]
        check_dslash(got, op(U, srcs[k], xs[k]), prec, DIMS, U, srcs[k], 18, lambda u, p: op(u, p, x_r))


def test_mrhs_equals_single_field_launches():
    """12 fields in one shared-link launch give the single-field results (FP32 rounding)."""
    import torch
    ctx = wd.Context(0)
    dims = (8, 8, 8, 8)
    U = synth.gauge(dims, seed=77)
    g = wd.Gauge(ctx, dims, U)
    nrhs = 12
    srcs = [synth.spinor(dims, seed=2500 + k) for k in range(nrhs)]
    fin = _fields(ctx, dims, wd.SITES_ODD, wd.F32, srcs)
    fout = wd.alloc_field(dims, wd.SITES_EVEN, wd.F32, nrhs)
    wd.dslash_eo_apply(ctx, g, fout, fin, None, 0, 0.0, 1.0, nrhs=nrhs, prec=wd.F32)
    nb = wd.field_bytes(dims, wd.SITES_EVEN, wd.F32)
    for k in range(nrhs):
        one = wd.alloc_field(dims, wd.SITES_EVEN, wd.F32)
        wd.dslash_eo_apply(ctx, g, one, fin[k * nb:(k + 1) * nb], None, 0, 0.0, 1.0, prec=wd.F32)
        a = unpack_field(ctx, dims, wd.SITES_EVEN, wd.F32, one)
        b = unpack_field(ctx, dims, wd.SITES_EVEN, wd.F32, fout[k * nb:(k + 1) * nb])
        assert rel_max_err(b, a) < 1e-6


@pytest.mark.parametrize("dims", [(4, 2, 32, 6), (6, 6, 6, 6), (6, 6, 10, 6)])
@pytest.mark.parametrize("prec", [wd.F64, wd.F32, wd.F16])
@pytest.mark.parametrize("full", [True, False])
def test_mrhs_z_strip_orders(dims, prec, full):
    """Variants 5, 6, 7 visit the (z, t) slices in z-strips of 16, 8, 4: every
    site still computes the same sum, so the output is bit-identical to the
    natural order (variant 3) and within the storage bound of the oracle.
    (4, 2, 32, 6) takes all three widths with slices of 4 sites inside 32-site
    blocks; (6, 6, 6, 6) takes width 4 as strips 4 + 2 with a ragged last block
    (648 sites per parity); (6, 6, 10, 6) takes 8 + 2 and 4 + 4 + 2 (1080)."""
    ctx = wd.Context(0)
    U = synth.gauge(dims, seed=4321)
    nrhs = 5
    srcs = [synth.spinor(dims, seed=2600 + k) for k in range(nrhs)]
    g = wd.Gauge(ctx, dims, U)
    par = parity(dims)
    if full:
        fin = _fields(ctx, dims, wd.SITES_FULL, prec, srcs)
        sites, nb = wd.SITES_FULL, wd.field_bytes(dims, wd.SITES_FULL, prec)
    else:
        fin = _fields(ctx, dims, wd.SITES_ODD, prec, srcs)
        sites, nb = wd.SITES_EVEN, wd.field_bytes(dims, wd.SITES_EVEN, prec)

    def run(variant):
        wd.tune_set_dslash(ctx, g, prec, 18, full, full, nrhs, 128, variant)
        out = wd.alloc_field(dims, sites, prec, nrhs)
        if full:
            wd.dslash_apply(ctx, g, out, fin, 0.1, nrhs=nrhs, prec=prec, recon=18)
        else:
            wd.dslash_eo_apply(ctx, g, out, fin, None, 0, 0.0, 1.0, nrhs=nrhs, prec=prec, recon=18)
        return out

    base = run(3).cpu()
    for variant in (5, 6, 7):
        out = run(variant)
        assert bool((out.cpu() == base).all()), variant
    for k in range(nrhs):
        got = unpack_field(ctx, dims, sites, prec, out[k * nb:(k + 1) * nb])
        if full:
            check_dslash(got, oracle.dirac(dims, U, srcs[k], 0.1), prec, dims, U, srcs[k], 18,
                         lambda u, p: oracle.dirac(dims, u, p, 0.1))
        else:
            def op(u, src):
                src = src.copy()
                src[par == 0] = 0
                return oracle.hop(dims, u, src, out_parity=0)[par == 0]
            check_dslash(got[par == 0], op(U, srcs[k]), prec, dims, U, srcs[k], 18, op)
