"""Antiperiodic boundary conditions in t on the GPU against the oracle.

The oracle's antiperiodic operator is the periodic one on links whose U_t on
the slice t = Lt-1 are negated (pinned on the CPU by half-integer-momentum
plane waves); the GPU applies the sign in its kernels.
"""
import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import check_dslash, pack_field, unpack_field
from tests._lattice import parity, rel_max_err

pytestmark = pytest.mark.gpu

ALL_PREC = [wd.F64, wd.F32, wd.F16, wd.BF16]


@pytest.fixture(scope="module")
def ctx():
    return wd.Context(0)


def _gauge(ctx, dims, seed):
    U = synth.gauge(dims, seed=seed)
    g = wd.Gauge(ctx, dims, U)
    g.set_boundary(-1)
    return U, oracle.antiperiodic_links(dims, U), g


@pytest.mark.parametrize("prec", ALL_PREC)
@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (4, 4, 4, 2)])
def test_full_dslash_antiperiodic(ctx, prec, recon, dims):
    U, Ua, g = _gauge(ctx, dims, 1401)
    psi = synth.spinor(dims, seed=3401)
    out = wd.alloc_field(dims, wd.SITES_FULL, prec)
    wd.dslash_apply(ctx, g, out, pack_field(ctx, dims, wd.SITES_FULL, prec, psi), 0.1, prec=prec, recon=recon)
    got = unpack_field(ctx, dims, wd.SITES_FULL, prec, out)
    ref = oracle.dirac(dims, Ua, psi, 0.1)
    check_dslash(got, ref, prec, dims, U, psi, recon,
                 lambda u, p: oracle.dirac(dims, oracle.antiperiodic_links(dims, u), p, 0.1))
    # and it differs from the periodic operator
    assert rel_max_err(ref, oracle.dirac(dims, U, psi, 0.1)) > 1e-2


@pytest.mark.parametrize("prec", [wd.F64, wd.F32, wd.F16])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_eo_hop_antiperiodic(ctx, prec, dagger, out_parity):
    dims = (4, 6, 4, 6)
    U, Ua, g = _gauge(ctx, dims, 1402)
    psi = synth.spinor(dims, seed=3402)
    xs = synth.spinor(dims, seed=3403)
    par = parity(dims)
    src_sites = wd.SITES_ODD if out_parity == 0 else wd.SITES_EVEN
    out_sites = wd.SITES_EVEN if out_parity == 0 else wd.SITES_ODD
    fin = pack_field(ctx, dims, src_sites, prec, psi)
    fx = pack_field(ctx, dims, out_sites, prec, xs)
    fout = wd.alloc_field(dims, out_sites, prec)
    a, b = 0.3, -0.7
    wd.dslash_eo_apply(ctx, g, fout, fin, fx, out_parity, a, b, dagger=dagger, prec=prec)
    got = unpack_field(ctx, dims, out_sites, prec, fout)[par == out_parity]

    def op(u, src):
        src = src.copy()
        src[par == out_parity] = 0
        ua = oracle.antiperiodic_links(dims, u)
        if dagger:
            h = oracle.gamma_apply(4, oracle.hop(dims, ua, oracle.gamma_apply(4, src), out_parity=out_parity))
        else:
            h = oracle.hop(dims, ua, src, out_parity=out_parity)
        return (a * xs + b * h)[par == out_parity]

    check_dslash(got, op(U, psi), prec, dims, U, psi, 18, op)


@pytest.mark.parametrize("variant", [3, 5, 6, 7])
@pytest.mark.parametrize("full", [True, False])
def test_mrhs_antiperiodic(ctx, variant, full):
    dims = (4, 2, 32, 6)
    U, Ua, g = _gauge(ctx, dims, 1403)
    nrhs = 4
    import torch
    srcs = [synth.spinor(dims, seed=3410 + k) for k in range(nrhs)]
    sites_in = wd.SITES_FULL if full else wd.SITES_ODD
    sites_out = wd.SITES_FULL if full else wd.SITES_EVEN
    fin = torch.cat([pack_field(ctx, dims, sites_in, wd.F32, s) for s in srcs])
    fout = wd.alloc_field(dims, sites_out, wd.F32, nrhs)
    wd.tune_set_dslash(ctx, g, wd.F32, 18, full, full, nrhs, 128, variant)
    if full:
        wd.dslash_apply(ctx, g, fout, fin, 0.1, nrhs=nrhs, prec=wd.F32)
    else:
        wd.dslash_eo_apply(ctx, g, fout, fin, None, 0, 0.0, 1.0, nrhs=nrhs, prec=wd.F32)
    nb = wd.field_bytes(dims, sites_out, wd.F32)
    par = parity(dims)
    for k in range(nrhs):
        got = unpack_field(ctx, dims, sites_out, wd.F32, fout[k * nb:(k + 1) * nb])
        if full:
            ref = oracle.dirac(dims, Ua, srcs[k], 0.1)
        else:
            src = srcs[k].copy()
            src[par == 0] = 0
            ref = oracle.hop(dims, Ua, src, out_parity=0)
            got, ref = got[par == 0], ref[par == 0]
        assert rel_max_err(got, ref) < 1e-5


@pytest.mark.parametrize("solver", ["cg", "bicgstab", "full_bicgstab", "full_cgne"])
def test_solves_antiperiodic(ctx, solver):
    dims, m, tol = (8, 4, 4, 8), 0.1, 1e-10
    U, Ua, g = _gauge(ctx, dims, 1404)
    kw = dict(inner_prec=wd.F16, reliable=True, delta=0.1)
    if solver in ("cg", "bicgstab"):
        b = synth.even_spinor(dims, seed=3404)
        fb = pack_field(ctx, dims, wd.SITES_EVEN, wd.F64, b)
        fx = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
        if solver == "cg":
            wd.cg_solve(ctx, g, m, fx, fb, tol=tol, **kw)
        else:
            wd.bicgstab_solve(ctx, g, m, fx, fb, tol=tol, **kw)
        x = unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, fx)
        ax = oracle.mdagm(dims, Ua, m, x) if solver == "cg" else oracle.mhat(dims, Ua, m, x)
    else:
        b = synth.spinor(dims, seed=3405)
        fb = pack_field(ctx, dims, wd.SITES_FULL, wd.F64, b)
        fx = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
        wd.wilson_solve(ctx, g, m, fx, fb, tol=tol,
                        solver=wd.SOLVER_BICGSTAB if solver == "full_bicgstab" else wd.SOLVER_CGNE, **kw)
        x = unpack_field(ctx, dims, wd.SITES_FULL, wd.F64, fx)
        ax = oracle.dirac(dims, Ua, x, m)
    assert np.linalg.norm(b - ax) / np.linalg.norm(b) <= tol


def test_persistent_batch_antiperiodic(ctx):
    """The persistent multi-solve kernel uses the same hop code and gauge setting."""
    dims, tol = (8, 8, 8, 8), 1e-10
    U, Ua, g = _gauge(ctx, dims, 1405)
    problems = []
    for k, m in enumerate((0.1, 0.3)):
        b = synth.even_spinor(dims, seed=3420 + k)
        problems.append((m, b, pack_field(ctx, dims, wd.SITES_EVEN, wd.F64, b), wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)))
    probs = [dict(gauge=g, mass=m, tol=tol, x=fx, b=fb, inner_prec=wd.F32, reliable=True, delta=0.01)
             for m, b, fb, fx in problems]
    stats = wd.cg_solve_batch(ctx, probs, mode=wd.BATCH_PERSISTENT)
    for (m, b, fb, fx), st in zip(problems, stats):
        assert st["status"] == 0
        x = unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, fx)
        assert np.linalg.norm(b - oracle.mdagm(dims, Ua, m, x)) / np.linalg.norm(b) <= tol


def test_boundary_argument_checked(ctx):
    dims = (4, 4, 4, 4)
    g = wd.Gauge(ctx, dims, synth.gauge(dims, seed=1))
    with pytest.raises(wd.WdError):
        g.set_boundary(0)
    g.set_boundary(-1)
    g.set_boundary(1)


@pytest.mark.parametrize("variant", [0, 11, 12])
@pytest.mark.parametrize("prec", [wd.F32, wd.F16])
def test_single_field_variants_antiperiodic(ctx, variant, prec):
    """Schedules 0 and 1 with links loaded without L1 allocation (variants 11, 12) apply the
    antiperiodic sign like the others, in the full operator and in an even-odd hop."""
    dims = (4, 6, 4, 6)
    U, Ua, g = _gauge(ctx, dims, 1404)
    psi = synth.spinor(dims, seed=3404)
    par = parity(dims)
    for recon in (18, 12):
        wd.tune_set_dslash(ctx, g, prec, recon, True, True, 1, 64, variant)
        wd.tune_set_dslash(ctx, g, prec, recon, False, False, 1, 64, variant)
        out = wd.alloc_field(dims, wd.SITES_FULL, prec)
        wd.dslash_apply(ctx, g, out, pack_field(ctx, dims, wd.SITES_FULL, prec, psi), 0.1, prec=prec, recon=recon)
        check_dslash(unpack_field(ctx, dims, wd.SITES_FULL, prec, out), oracle.dirac(dims, Ua, psi, 0.1), prec,
                     dims, U, psi, recon, lambda u, p: oracle.dirac(dims, oracle.antiperiodic_links(dims, u), p, 0.1))
        fe = wd.alloc_field(dims, wd.SITES_EVEN, prec)
        wd.dslash_eo_apply(ctx, g, fe, pack_field(ctx, dims, wd.SITES_ODD, prec, psi), None, 0, 0.0, 1.0,
                           prec=prec, recon=recon)
        src = psi.copy()
        src[par == 0] = 0
        got = unpack_field(ctx, dims, wd.SITES_EVEN, prec, fe)[par == 0]
        assert rel_max_err(got, oracle.hop(dims, Ua, src, out_parity=0)[par == 0]) < (1e-5 if prec == wd.F32 else 3e-3)
