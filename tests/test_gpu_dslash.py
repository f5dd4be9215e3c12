"""GPU parity of the Wilson-Dirac kernels against the FP64 oracle (through the C ABI).

Tolerances (relative max error over all reals, vs the FP64 oracle on the
unrounded inputs): FP64 1e-13, FP32 1e-5, FP16/BF16 storage 3e-3.
"""
import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import TOL, check_dslash, pack_field, to_dev, unpack_field
from tests._lattice import parity, rel_max_err, volume

pytestmark = pytest.mark.gpu

ALL_PREC = [wd.F64, wd.F32, wd.F16, wd.BF16]
# 8^4 (the small parity case), an uneven all-even lattice, and 16^3x32
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


@pytest.mark.parametrize("prec", ALL_PREC)
def test_pack_unpack_round_trip(ctx, prec):
    dims = (4, 6, 8, 10)
    psi = synth.spinor(dims, seed=2011)
    back = unpack_field(ctx, dims, wd.SITES_FULL, prec, pack_field(ctx, dims, wd.SITES_FULL, prec, psi))
    if prec == wd.F64:
        assert np.array_equal(back, psi)
        return
    # per-site relative error bound: unit roundoff of the storage type
    u = {wd.F32: 2.0 ** -24, wd.F16: 2.0 ** -11, wd.BF16: 2.0 ** -8}[prec]
    site_max = np.max(np.abs(psi.view(np.float64).reshape(-1, 24)), axis=1)
    err = np.max(np.abs((back - psi).view(np.float64).reshape(-1, 24)), axis=1) / site_max
    assert np.max(err) <= u * 1.01


@pytest.mark.parametrize("prec", ALL_PREC)
@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (2, 2, 2, 6), (6, 6, 6, 6)])
def test_full_pack_equals_half_packs(ctx, prec, dims):
    """A full field is packed and unpacked in lexicographic tiles of 128 sites
    (last tile partial for 48 and 1296 sites); half fields go site by site in
    checkerboard order.  The two routes give the same bytes both ways."""
    import torch
    psi = synth.spinor(dims, seed=2013)
    aos = torch.from_numpy(psi.view(np.float64).reshape(-1).copy()).cuda()
    full = wd.alloc_field(dims, wd.SITES_FULL, prec)
    wd.pack(ctx, dims, wd.SITES_FULL, prec, aos, full)
    half = wd.field_bytes(dims, wd.SITES_EVEN, prec)
    ev = wd.alloc_field(dims, wd.SITES_EVEN, prec)
    od = wd.alloc_field(dims, wd.SITES_ODD, prec)
    wd.pack(ctx, dims, wd.SITES_EVEN, prec, aos, ev)
    wd.pack(ctx, dims, wd.SITES_ODD, prec, aos, od)
    torch.cuda.synchronize()
    assert torch.equal(full[:half], ev) and torch.equal(full[half:], od)
    out_full = torch.full_like(aos, float("nan"))
    wd.unpack(ctx, dims, wd.SITES_FULL, prec, full, out_full)
    out_half = torch.full_like(aos, float("nan"))
    wd.unpack(ctx, dims, wd.SITES_EVEN, prec, ev, out_half)
    wd.unpack(ctx, dims, wd.SITES_ODD, prec, od, out_half)
    torch.cuda.synchronize()
    assert torch.equal(out_full, out_half)
    if prec == wd.F64:
        assert torch.equal(out_full, aos)


def test_pack_half_fields_touch_only_their_parity(ctx):
    dims = (4, 4, 4, 6)
    psi = synth.spinor(dims, seed=2012)
    par = parity(dims)
    for sites, p in ((wd.SITES_EVEN, 0), (wd.SITES_ODD, 1)):
        back = unpack_field(ctx, dims, sites, wd.F64, pack_field(ctx, dims, sites, wd.F64, psi))
        assert np.array_equal(back[par == p], psi[par == p])
        assert np.all(back[par != p] == 0)


@pytest.mark.parametrize("prec", ALL_PREC)
@pytest.mark.parametrize("sites", [wd.SITES_FULL, wd.SITES_EVEN])
def test_pack_unpack_with_host_memory(ctx, prec, sites):
    """The canonical array may be pinned host memory (or, on systems where the device can
    access pageable memory, ordinary host memory): the kernels read and write it directly and
    give the same bytes as with a device array.  Device memory is used unchanged."""
    import torch
    dims = (4, 6, 8, 10)
    psi = synth.spinor(dims, seed=2013)
    flat = psi.view(np.float64).reshape(-1)
    dev = torch.from_numpy(flat.copy()).cuda()
    pinned = torch.from_numpy(flat.copy()).pin_memory()
    f_dev = wd.alloc_field(dims, sites, prec)
    f_host = wd.alloc_field(dims, sites, prec)
    wd.pack(ctx, dims, sites, prec, dev, f_dev)
    wd.pack(ctx, dims, sites, prec, pinned, f_host)
    torch.cuda.synchronize()
    assert torch.equal(f_dev, f_host)
    out_dev = torch.zeros_like(dev)
    out_pinned = torch.zeros(flat.size, dtype=torch.float64).pin_memory()
    wd.unpack(ctx, dims, sites, prec, f_dev, out_dev)
    wd.unpack(ctx, dims, sites, prec, f_dev, out_pinned)
    torch.cuda.synchronize()
    assert torch.equal(out_dev.cpu(), out_pinned)
    if wd.device_info(ctx)["pageable_memory_access"]:
        pageable = flat.copy()
        f_pg = wd.alloc_field(dims, sites, prec)
        wd.pack(ctx, dims, sites, prec, pageable.ctypes.data, f_pg)
        torch.cuda.synchronize()
        assert torch.equal(f_dev, f_pg)


@pytest.mark.parametrize("prec", ALL_PREC)
@pytest.mark.parametrize("sites", [wd.SITES_FULL, wd.SITES_ODD])
def test_pack_unpack_fp32_canonical(ctx, prec, sites):
    """wd_pack_f32 / wd_unpack_f32: an FP32 canonical array gives the same field bytes as the
    FP64 path fed the same (FP32-rounded) values, and unpacks to the FP64 result rounded to
    FP32, from device and from pinned host memory."""
    import torch
    dims = (4, 6, 8, 10)
    psi = synth.spinor(dims, seed=2014)
    flat32 = psi.view(np.float64).reshape(-1).astype(np.float32)
    as64 = torch.from_numpy(flat32.astype(np.float64)).cuda()
    f64path = wd.alloc_field(dims, sites, prec)
    wd.pack(ctx, dims, sites, prec, as64, f64path)
    for src in (torch.from_numpy(flat32.copy()).cuda(), torch.from_numpy(flat32.copy()).pin_memory()):
        f32path = wd.alloc_field(dims, sites, prec)
        wd.pack(ctx, dims, sites, prec, src, f32path)
        torch.cuda.synchronize()
        assert torch.equal(f64path, f32path)
    out64 = torch.zeros(flat32.size, dtype=torch.float64, device="cuda")
    wd.unpack(ctx, dims, sites, prec, f64path, out64)
    for dst in (torch.zeros(flat32.size, dtype=torch.float32, device="cuda"),
                torch.zeros(flat32.size, dtype=torch.float32).pin_memory()):
        wd.unpack(ctx, dims, sites, prec, f64path, dst)
        torch.cuda.synchronize()
        assert np.array_equal(dst.cpu().numpy(), out64.cpu().numpy().astype(np.float32))


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("prec", ALL_PREC)
def test_dslash_full_matches_oracle(ctx, dims, recon, prec):
    U, psi = _inputs(dims)
    m = 0.1
    g = wd.Gauge(ctx, dims, U)
    fin = pack_field(ctx, dims, wd.SITES_FULL, prec, psi)
    fout = wd.alloc_field(dims, wd.SITES_FULL, prec)
    wd.dslash_apply(ctx, g, fout, fin, m, prec=prec, recon=recon)
    got = unpack_field(ctx, dims, wd.SITES_FULL, prec, fout)
    ref = oracle.dirac(dims, U, psi, m)
    err = rel_max_err(got, ref)
    assert err < TOL[prec], f"err {err:.3e}"


@pytest.mark.parametrize("prec", ALL_PREC)
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("out_parity", [0, 1])
@pytest.mark.parametrize("with_x", [False, True])
def test_dslash_eo_matches_oracle(ctx, prec, dagger, out_parity, with_x):
    dims = (4, 6, 8, 10)
    U, psi = _inputs(dims)
    xs = synth.spinor(dims, seed=2099)
    a, b = 1.7, -0.35
    g = wd.Gauge(ctx, dims, U)
    p = out_parity
    in_sites = wd.SITES_ODD if p == 0 else wd.SITES_EVEN
    out_sites = wd.SITES_EVEN if p == 0 else wd.SITES_ODD
    fin = pack_field(ctx, dims, in_sites, prec, psi)
    fx = pack_field(ctx, dims, out_sites, prec, xs) if with_x else None
    fout = wd.alloc_field(dims, out_sites, prec)
    wd.dslash_eo_apply(ctx, g, fout, fin, fx, p, a, b, dagger=dagger, prec=prec, recon=18)
    got = unpack_field(ctx, dims, out_sites, prec, fout)
    par = parity(dims)
    src = psi.copy()
    src[par == p] = 0            # only the 1-p half is an input
    if dagger:
        h = oracle.gamma_apply(4, oracle.hop(dims, U, oracle.gamma_apply(4, src), out_parity=p))
    else:
        h = oracle.hop(dims, U, src, out_parity=p)
    ref = b * h + (a * xs if with_x else 0)
    ref[par != p] = 0
    err = rel_max_err(got[par == p], ref[par == p])
    assert err < TOL[prec], f"err {err:.3e}"


def test_dslash_multi_rhs_equals_single(ctx):
    import torch
    dims = (8, 8, 8, 8)
    U, _ = _inputs(dims)
    g = wd.Gauge(ctx, dims, U)
    nrhs = 3
    srcs = [synth.spinor(dims, seed=2100 + k) for k in range(nrhs)]
    nb = wd.field_bytes(dims, wd.SITES_FULL, wd.F32)
    fin = torch.cat([pack_field(ctx, dims, wd.SITES_FULL, wd.F32, s) for s in srcs])
    fout = wd.alloc_field(dims, wd.SITES_FULL, wd.F32, nrhs)
    wd.dslash_apply(ctx, g, fout, fin, 0.1, nrhs=nrhs, prec=wd.F32)
    for k in range(nrhs):
        single = wd.alloc_field(dims, wd.SITES_FULL, wd.F32)
        wd.dslash_apply(ctx, g, single, fin[k * nb:(k + 1) * nb], 0.1, prec=wd.F32)
        a = unpack_field(ctx, dims, wd.SITES_FULL, wd.F32, single)
        b = unpack_field(ctx, dims, wd.SITES_FULL, wd.F32, fout[k * nb:(k + 1) * nb])
        assert rel_max_err(b, a) < 1e-6


def test_dslash_32_4_full_size(ctx):
    """The benchmark launch (32^4, FP32 and FP64, 18 and 12 reals) against the oracle on every site."""
    dims = (32, 32, 32, 32)
    U = synth.gauge(dims, seed=1001)
    psi = synth.spinor(dims, seed=2001)
    ref = oracle.dirac(dims, U, psi, 0.1)
    g = wd.Gauge(ctx, dims, U)
    for prec in (wd.F32, wd.F64):
        fin = pack_field(ctx, dims, wd.SITES_FULL, prec, psi)
        fout = wd.alloc_field(dims, wd.SITES_FULL, prec)
        for recon in (18, 12):
            wd.dslash_apply(ctx, g, fout, fin, 0.1, prec=prec, recon=recon)
            err = rel_max_err(unpack_field(ctx, dims, wd.SITES_FULL, prec, fout), ref)
            assert err < TOL[prec], (prec, recon, err)


def test_argument_errors(ctx):
    import torch
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, seed=1)
    g = wd.Gauge(ctx, dims, U)
    f = wd.alloc_field(dims, wd.SITES_FULL, wd.F32)
    with pytest.raises(wd.WdError) as e:
        wd.dslash_apply(ctx, g, f, f, 0.1)           # aliasing
    assert e.value.status == wd.WD_EINVAL
    big = torch.empty(f.numel() + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(wd.WdError) as e:
        wd.dslash_apply(ctx, g, big[4:].data_ptr(), f, 0.1)   # misaligned
    assert e.value.status == wd.WD_EINVAL
    with pytest.raises(wd.WdError) as e:
        wd.dslash_apply(ctx, g, big, f, 0.1, recon=9)
    assert e.value.status == wd.WD_EINVAL
    with pytest.raises(wd.WdError) as e:
        wd.dslash_eo_apply(ctx, g, big, f, None, 2, 1.0, 1.0)
    assert e.value.status == wd.WD_EINVAL


@pytest.mark.parametrize("prec", ALL_PREC)
@pytest.mark.parametrize("variant", [0, 1, 2, 8, 9, 11, 12, 13, 14, 15])
@pytest.mark.parametrize("threads", [64, 192, 256])
def test_every_launch_variant_matches_oracle(prec, variant, threads):
    """Each memory schedule and block size the autotuner may pick computes the same operator."""
    dims = (4, 6, 8, 10)
    ctx = wd.Context(0)
    U, psi = _inputs(dims)
    g = wd.Gauge(ctx, dims, U)
    for recon in (18, 12):
        wd.tune_set_dslash(ctx, g, prec, recon, True, True, 1, threads, variant)
        wd.tune_set_dslash(ctx, g, prec, recon, False, False, 1, threads, variant)
        fin = pack_field(ctx, dims, wd.SITES_FULL, prec, psi)
        fout = wd.alloc_field(dims, wd.SITES_FULL, prec)
        wd.dslash_apply(ctx, g, fout, fin, 0.1, prec=prec, recon=recon)
        err = rel_max_err(unpack_field(ctx, dims, wd.SITES_FULL, prec, fout), oracle.dirac(dims, U, psi, 0.1))
        assert err < TOL[prec], ("full", recon, err)
        fo = pack_field(ctx, dims, wd.SITES_ODD, prec, psi)
        fe = wd.alloc_field(dims, wd.SITES_EVEN, prec)
        wd.dslash_eo_apply(ctx, g, fe, fo, None, 0, 0.0, 1.0, dagger=True, prec=prec, recon=recon)
        par = parity(dims)
        src = psi.copy()
        src[par == 0] = 0
        ref = oracle.gamma_apply(4, oracle.hop(dims, U, oracle.gamma_apply(4, src), out_parity=0))
        got = unpack_field(ctx, dims, wd.SITES_EVEN, prec, fe)
        assert rel_max_err(got[par == 0], ref[par == 0]) < TOL[prec], ("eo", recon)


def test_autotuner_table_and_choice():
    dims = (8, 8, 8, 8)
    ctx = wd.Context(0)
    U, _ = _inputs(dims)
    g = wd.Gauge(ctx, dims, U)
    table = wd.tune_dslash(ctx, g, wd.F32, 18, full=True)
    # 4 block sizes x 8 single-field variants: schedules 0, 1, 2, the high-occupancy build 4,
    # the shared-memory neighbour window 8, two sites per thread 9 and schedules 0 and 1 with
    # links loaded without L1 allocation (11, 12); 10 is retired, the spin-paired kernels
    # 13, 14 exist for the 16-bit formats only and the one-block-per-SM build 15 for FP64
    assert len(table) == 32
    assert {t["variant"] for t in table} == {0, 1, 2, 4, 8, 9, 11, 12}
    assert all(t["ms"] > 0 for t in table)
    with pytest.raises(wd.WdError):
        wd.tune_set_dslash(ctx, g, wd.F32, 18, True, True, 1, 64, 10)
    table16 = wd.tune_dslash(ctx, g, wd.F16, 18, full=True)
    assert len(table16) == 40
    assert {t["variant"] for t in table16} == {0, 1, 2, 4, 8, 9, 11, 12, 13, 14}


@pytest.mark.parametrize("prec", ALL_PREC)
@pytest.mark.parametrize("dims,threads", [((8, 8, 8, 8), 64), ((16, 16, 16, 32), 256), ((4, 6, 8, 10), 96)])
def test_high_occupancy_variant_matches_oracle(prec, dims, threads):
    """Variant 4: schedule 1 compiled for 3 blocks of 256 threads per SM, with an axpby term."""
    ctx = wd.Context(0)
    U, psi = _inputs(dims)
    g = wd.Gauge(ctx, dims, U)
    for recon in (18, 12):
        wd.tune_set_dslash(ctx, g, prec, recon, True, True, 1, threads, 4)
        wd.tune_set_dslash(ctx, g, prec, recon, False, True, 1, threads, 4)
        fin = pack_field(ctx, dims, wd.SITES_FULL, prec, psi)
        fout = wd.alloc_field(dims, wd.SITES_FULL, prec)
        wd.dslash_apply(ctx, g, fout, fin, 0.1, prec=prec, recon=recon)
        check_dslash(unpack_field(ctx, dims, wd.SITES_FULL, prec, fout), oracle.dirac(dims, U, psi, 0.1), prec,
                     dims, U, psi, recon, lambda u, p: oracle.dirac(dims, u, p, 0.1))
        fo = pack_field(ctx, dims, wd.SITES_ODD, prec, psi)
        fx = pack_field(ctx, dims, wd.SITES_EVEN, prec, psi)
        fe = wd.alloc_field(dims, wd.SITES_EVEN, prec)
        wd.dslash_eo_apply(ctx, g, fe, fo, fx, 0, 1.5, -0.25, prec=prec, recon=recon)
        par = parity(dims)

        def eo(u, p):
            src = p.copy()
            src[par == 0] = 0
            return (1.5 * p - 0.25 * oracle.hop(dims, u, src, out_parity=0))[par == 0]

        got = unpack_field(ctx, dims, wd.SITES_EVEN, prec, fe)
        check_dslash(got[par == 0], eo(U, psi), prec, dims, U, psi, recon, eo)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 6), (6, 2, 2, 2), (2, 2, 10, 2)])
@pytest.mark.parametrize("prec", ALL_PREC)
@pytest.mark.parametrize("threads,variant", [(32, 0), (64, 1), (256, 2), (192, 4), (32, 8), (128, 8), (64, 9), (96, 9), (64, 11), (128, 12), (32, 13), (64, 13), (96, 14), (128, 14), (128, 15), (256, 15)])
def test_degenerate_extents_and_ragged_tails(dims, prec, threads, variant):
    """L_mu = 2 (x+mu and x-mu are the same site, both terms added) and half-lattice sizes far
    below or not a multiple of the block size."""
    ctx = wd.Context(0)
    U = synth.gauge(dims, seed=1111)
    psi = synth.spinor(dims, seed=2222)
    g = wd.Gauge(ctx, dims, U)
    for recon in (18, 12):
        wd.tune_set_dslash(ctx, g, prec, recon, True, True, 1, threads, variant)
        fin = pack_field(ctx, dims, wd.SITES_FULL, prec, psi)
        fout = wd.alloc_field(dims, wd.SITES_FULL, prec)
        wd.dslash_apply(ctx, g, fout, fin, 0.3, prec=prec, recon=recon)
        check_dslash(unpack_field(ctx, dims, wd.SITES_FULL, prec, fout), oracle.dirac(dims, U, psi, 0.3), prec,
                     dims, U, psi, recon, lambda u, p: oracle.dirac(dims, u, p, 0.3))


@pytest.mark.parametrize("prec", ALL_PREC)
@pytest.mark.parametrize("recon", [18, 12])
def test_dagger_is_paper_convention(ctx, prec, recon):
    """D^dagger = (m+4) - D_h / 2 with D_h the hopping term of Eq. (1) as printed
    (the oracle's convention 1, pinned against gamma5 H gamma5 on the CPU)."""
    dims = (4, 6, 8, 10)
    U = synth.gauge(dims, seed=1501)
    psi = synth.spinor(dims, seed=3501)
    g = wd.Gauge(ctx, dims, U)
    out = wd.alloc_field(dims, wd.SITES_FULL, prec)
    wd.dslash_apply_dagger(ctx, g, out, pack_field(ctx, dims, wd.SITES_FULL, prec, psi), 0.1, prec=prec, recon=recon)
    got = unpack_field(ctx, dims, wd.SITES_FULL, prec, out)
    fn = lambda u, p: 4.1 * p - 0.5 * oracle.hop(dims, u, p, convention=1)
    check_dslash(got, fn(U, psi), prec, dims, U, psi, recon, fn)
    # <x, D y> = <D^dagger x, y> with the GPU operators (FP64)
    if prec == wd.F64:
        y = synth.spinor(dims, seed=3502)
        dy = wd.alloc_field(dims, wd.SITES_FULL, prec)
        wd.dslash_apply(ctx, g, dy, pack_field(ctx, dims, wd.SITES_FULL, prec, y), 0.1, prec=prec, recon=recon)
        lhs = np.vdot(psi, unpack_field(ctx, dims, wd.SITES_FULL, prec, dy))
        rhs = np.vdot(got, y)
        assert abs(lhs - rhs) / abs(lhs) < 1e-13

