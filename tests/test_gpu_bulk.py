"""The bulk-copy staged operator kernel (launch variant 10) against the oracle.

The kernel stages each block's forward links, t-forward neighbours and axpy
term in shared memory with cp.async.bulk copies; it applies when the block
size divides a t-slice (Lx/2 * Ly * Lz sites) and falls back to memory
schedule 1 otherwise.  Both paths, every precision and link format, the
antiperiodic t boundary (whose sign the staged t-forward hop applies), several
right-hand sides and the status word of the bounded wait are checked here.
"""
import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import check_dslash, pack_field, unpack_field
from tests._lattice import parity

pytestmark = pytest.mark.gpu

ALL_PREC = [wd.F64, wd.F32, wd.F16, wd.BF16]
BULK = 10


@pytest.fixture(scope="module")
def ctx():
    return wd.Context(0)


def _slice(dims):
    return dims[0] // 2 * dims[1] * dims[2]


@pytest.mark.parametrize("prec", ALL_PREC)
@pytest.mark.parametrize("dims,threads", [((8, 8, 8, 8), 64), ((8, 8, 8, 8), 256), ((4, 6, 8, 10), 32),
                                          ((4, 6, 8, 10), 96), ((4, 6, 8, 10), 64), ((16, 16, 16, 32), 128)])
@pytest.mark.parametrize("tsign", [1, -1])
def test_staged_kernel_full_and_eo(ctx, prec, dims, threads, tsign):
    """Full operator (axpy term staged) and an even-odd hop with axpby, periodic and
    antiperiodic in t.  (4,6,8,10) with 64 threads does not divide its 96-site slice: that
    case checks the fallback to schedule 1."""
    eligible = _slice(dims) % threads == 0
    assert eligible == (dims != (4, 6, 8, 10) or threads != 64)
    U = synth.gauge(dims, seed=1601)
    psi = synth.spinor(dims, seed=3601)
    g = wd.Gauge(ctx, dims, U)
    g.set_boundary(tsign)
    links = (lambda u: oracle.antiperiodic_links(dims, u)) if tsign < 0 else (lambda u: u)
    par = parity(dims)
    for recon in (18, 12):
        wd.tune_set_dslash(ctx, g, prec, recon, True, True, 1, threads, BULK)
        wd.tune_set_dslash(ctx, g, prec, recon, False, True, 1, threads, BULK)
        fin = pack_field(ctx, dims, wd.SITES_FULL, prec, psi)
        fout = wd.alloc_field(dims, wd.SITES_FULL, prec)
        wd.dslash_apply(ctx, g, fout, fin, 0.1, prec=prec, recon=recon)
        full = lambda u, p: oracle.dirac(dims, links(u), p, 0.1)
        check_dslash(unpack_field(ctx, dims, wd.SITES_FULL, prec, fout), full(U, psi), prec, dims, U, psi, recon,
                     full)
        fo = pack_field(ctx, dims, wd.SITES_ODD, prec, psi)
        fx = pack_field(ctx, dims, wd.SITES_EVEN, prec, psi)
        fe = wd.alloc_field(dims, wd.SITES_EVEN, prec)
        wd.dslash_eo_apply(ctx, g, fe, fo, fx, 0, 1.5, -0.25, prec=prec, recon=recon)

        def eo(u, p):
            src = p.copy()
            src[par == 0] = 0
            return (1.5 * p - 0.25 * oracle.hop(dims, links(u), src, out_parity=0))[par == 0]

        got = unpack_field(ctx, dims, wd.SITES_EVEN, prec, fe)
        check_dslash(got[par == 0], eo(U, psi), prec, dims, U, psi, recon, eo)
    assert wd.device_status(ctx) == 0


@pytest.mark.parametrize("prec", [wd.F64, wd.F32, wd.F16])
@pytest.mark.parametrize("dagger", [False, True])
def test_staged_kernel_eo_without_x_odd_output(ctx, prec, dagger):
    """Odd output parity, no axpy term (only links and the t neighbour staged), dagger."""
    dims = (8, 4, 6, 10)
    U = synth.gauge(dims, seed=1602)
    psi = synth.spinor(dims, seed=3602)
    g = wd.Gauge(ctx, dims, U)
    par = parity(dims)
    for recon in (18, 12):
        wd.tune_set_dslash(ctx, g, prec, recon, False, False, 1, 32, BULK)
        fe = pack_field(ctx, dims, wd.SITES_EVEN, prec, psi)
        fo = wd.alloc_field(dims, wd.SITES_ODD, prec)
        wd.dslash_eo_apply(ctx, g, fo, fe, None, 1, 0.0, 1.0, dagger=dagger, prec=prec, recon=recon)
        src = psi.copy()
        src[par == 1] = 0
        if dagger:
            ref = oracle.gamma_apply(4, oracle.hop(dims, U, oracle.gamma_apply(4, src), out_parity=1))
        else:
            ref = oracle.hop(dims, U, src, out_parity=1)
        got = unpack_field(ctx, dims, wd.SITES_ODD, prec, fo)
        check_dslash(got[par == 1], ref[par == 1], prec, dims, U, psi, recon,
                     lambda u, p: _hop_masked(dims, u, p, par, dagger))
    assert wd.device_status(ctx) == 0


def _hop_masked(dims, u, p, par, dagger):
    src = p.copy()
    src[par == 1] = 0
    if dagger:
        return oracle.gamma_apply(4, oracle.hop(dims, u, oracle.gamma_apply(4, src), out_parity=1))[par == 1]
    return oracle.hop(dims, u, src, out_parity=1)[par == 1]


@pytest.mark.parametrize("prec", [wd.F32, wd.F16])
def test_staged_kernel_several_fields(ctx, prec):
    """Three right-hand sides in one launch (grid.y): each field's t neighbour and axpy
    term are staged from its own offset."""
    dims, nrhs = (8, 8, 8, 8), 3
    U = synth.gauge(dims, seed=1603)
    g = wd.Gauge(ctx, dims, U)
    srcs = [synth.spinor(dims, seed=3610 + k) for k in range(nrhs)]
    wd.tune_set_dslash(ctx, g, prec, 18, True, True, nrhs, 64, BULK)
    fin = wd.alloc_field(dims, wd.SITES_FULL, prec, nrhs)
    nb = wd.field_bytes(dims, wd.SITES_FULL, prec)
    for k, s in enumerate(srcs):
        fin[k * nb:(k + 1) * nb].copy_(pack_field(ctx, dims, wd.SITES_FULL, prec, s))
    fout = wd.alloc_field(dims, wd.SITES_FULL, prec, nrhs)
    wd.dslash_apply(ctx, g, fout, fin, 0.2, nrhs=nrhs, prec=prec)
    for k, s in enumerate(srcs):
        got = unpack_field(ctx, dims, wd.SITES_FULL, prec, fout[k * nb:(k + 1) * nb])
        check_dslash(got, oracle.dirac(dims, U, s, 0.2), prec, dims, U, s, 18,
                     lambda u, p: oracle.dirac(dims, u, p, 0.2))
    assert wd.device_status(ctx) == 0


def test_autotuner_includes_staged_kernel(ctx):
    dims = (8, 8, 8, 8)
    g = wd.Gauge(ctx, dims, synth.gauge(dims, seed=1604))
    table = wd.tune_dslash(ctx, g, wd.F32, 18, full=True)
    assert BULK in {t["variant"] for t in table}
    assert all(np.isfinite(t["ms"]) and t["ms"] > 0 for t in table)


def test_bounded_wait_reports_timeout_and_context_recovers(monkeypatch):
    """The barrier is made to expect 16 bytes more than the copies bring (a host-side switch),
    so its phase never completes: every block gives up after its bounded wait (0.1 s here),
    records WD_ETIMEOUT in the context's status word and returns.  The next launch on the
    same context is correct and reports nothing."""
    ctx = wd.Context(0)
    dims = (8, 8, 8, 8)   # 64 blocks of 64 threads: all resident at once
    U = synth.gauge(dims, seed=1605)
    psi = synth.spinor(dims, seed=3605)
    g = wd.Gauge(ctx, dims, U)
    wd.tune_set_dslash(ctx, g, wd.F32, 18, True, True, 1, 64, BULK)
    fin = pack_field(ctx, dims, wd.SITES_FULL, wd.F32, psi)
    fout = wd.alloc_field(dims, wd.SITES_FULL, wd.F32)
    assert wd.device_status(ctx) == 0
    monkeypatch.setenv("WD_FAULT", "bulk_tx")
    monkeypatch.setenv("WD_BULK_TIMEOUT_S", "0.1")
    wd.dslash_apply(ctx, g, fout, fin, 0.1, prec=wd.F32)
    assert wd.device_status(ctx) == wd.WD_ETIMEOUT
    assert wd.device_status(ctx) == 0   # read and cleared
    monkeypatch.delenv("WD_FAULT")
    wd.dslash_apply(ctx, g, fout, fin, 0.1, prec=wd.F32)
    check_dslash(unpack_field(ctx, dims, wd.SITES_FULL, wd.F32, fout), oracle.dirac(dims, U, psi, 0.1), wd.F32,
                 dims, U, psi, 18, lambda u, p: oracle.dirac(dims, u, p, 0.1))
    assert wd.device_status(ctx) == 0
