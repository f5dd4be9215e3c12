"""Parity at the benchmark's full sizes, in the launch configurations the benchmark times.

Each test repeats one benchmark configuration (its lattice, seeds, options and the
autotuner's launch shapes) and checks the GPU result against the FP64 oracle on every
site, or, for solves, by the oracle operator's true residual on the GPU solution.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import TOL, pack_field, unpack_field
from tests._lattice import parity, rel_max_err, volume

pytestmark = pytest.mark.gpu

L32 = (32, 32, 32, 32)
L16 = (16, 16, 16, 32)
L24 = (24, 24, 24, 48)


@pytest.fixture(scope="module")
def ctx():
    return wd.Context(0)


_inputs = {}


def _links_and_source(dims):
    if dims not in _inputs:
        seed_l, seed_s = (1001, 2001) if dims == L32 else (1002, 2002)
        _inputs[dims] = (synth.gauge(dims, seed=seed_l), synth.spinor(dims, seed=seed_s))
    return _inputs[dims]


@pytest.mark.parametrize("dims", [L32, L16])
@pytest.mark.parametrize("prec", [wd.F64, wd.F32, wd.F16, wd.BF16])
def test_operator_variants_at_benchmark_sizes(ctx, dims, prec):
    """Full and even-odd, 18 and 12 reals, with the tuned launch shapes of the variants table."""
    U, psi = _links_and_source(dims)
    g = wd.Gauge(ctx, dims, U)
    par = parity(dims)
    ref_full = oracle.dirac(dims, U, psi, 0.1)
    src = psi.copy()
    src[par == 0] = 0
    ref_eo = oracle.hop(dims, U, src, out_parity=0)[par == 0]
    fin = pack_field(ctx, dims, wd.SITES_FULL, prec, psi)
    half = wd.field_bytes(dims, wd.SITES_EVEN, prec)
    fout = wd.alloc_field(dims, wd.SITES_FULL, prec)
    eo_out = wd.alloc_field(dims, wd.SITES_EVEN, prec)
    for recon in (18, 12):
        g.prepare(prec, recon)
        wd.tune_dslash(ctx, g, prec, recon, full=True)
        wd.tune_dslash(ctx, g, prec, recon, full=False, with_x=False)
        wd.dslash_apply(ctx, g, fout, fin, 0.1, prec=prec, recon=recon)
        err = rel_max_err(unpack_field(ctx, dims, wd.SITES_FULL, prec, fout), ref_full)
        assert err < TOL[prec], ("full", recon, err)
        wd.dslash_eo_apply(ctx, g, eo_out, fin[half:], None, wd.EVEN, 0.0, 1.0, prec=prec, recon=recon)
        got = unpack_field(ctx, dims, wd.SITES_EVEN, prec, eo_out)[par == 0]
        err = rel_max_err(got, ref_eo)
        assert err < TOL[prec], ("eo", recon, err)


@pytest.mark.parametrize("full", [False, True])
def test_twelve_fields_sharing_links_32_4(ctx, full):
    """12 right-hand sides on 32^4 in FP32 with the tuned shared-link launch (z-strip order),
    each against the oracle (distinct sources, unlike the timing run, which repeats one)."""
    dims, nrhs = L32, 12
    U, _ = _links_and_source(dims)
    g = wd.Gauge(ctx, dims, U)
    par = parity(dims)
    srcs = [synth.spinor(dims, seed=2100 + k) for k in range(nrhs)]
    sites_in = wd.SITES_FULL if full else wd.SITES_ODD
    sites_out = wd.SITES_FULL if full else wd.SITES_EVEN
    fin = torch.cat([pack_field(ctx, dims, sites_in, wd.F32, s) for s in srcs])
    fout = wd.alloc_field(dims, sites_out, wd.F32, nrhs)
    table = wd.tune_dslash(ctx, g, wd.F32, 18, full=full, with_x=False, nrhs=nrhs)
    assert min(table, key=lambda t: t["ms"])["variant"] in (3, 5, 6, 7)
    if full:
        wd.dslash_apply(ctx, g, fout, fin, 0.1, nrhs=nrhs, prec=wd.F32)
    else:
        wd.dslash_eo_apply(ctx, g, fout, fin, None, wd.EVEN, 0.0, 1.0, nrhs=nrhs, prec=wd.F32)
    nb = wd.field_bytes(dims, sites_out, wd.F32)
    for k in (0, 5, 11):
        got = unpack_field(ctx, dims, sites_out, wd.F32, fout[k * nb:(k + 1) * nb])
        if full:
            ref = oracle.dirac(dims, U, srcs[k], 0.1)
        else:
            s = srcs[k].copy()
            s[par == 0] = 0
            ref = oracle.hop(dims, U, s, out_parity=0)
            got, ref = got[par == 0], ref[par == 0]
        assert rel_max_err(got, ref) < TOL[wd.F32], k


_cg = {}


def _cg_problem(ctx):
    if "p" not in _cg:
        U = synth.gauge(L24, seed=1003)
        b = synth.even_spinor(L24, seed=3001)
        g = wd.Gauge(ctx, L24, U)
        _cg["p"] = (U, b, g, pack_field(ctx, L24, wd.SITES_EVEN, wd.F64, b))
    return _cg["p"]


@pytest.mark.parametrize("mass", [0.1, 0.05])
@pytest.mark.parametrize("kw", [dict(inner_prec=wd.F64), dict(inner_prec=wd.F16, delta=0.01),
                                dict(inner_prec=wd.BF16, delta=0.01),
                                dict(inner_prec=wd.F16, delta=0.01, use_graph=True)],
                         ids=["fp64", "fp16", "bf16", "fp16_graph"])
def test_cg_24_3x48(ctx, mass, kw):
    """The CG configuration: even-odd normal equations on 24^3x48 to a 1e-10 true residual."""
    U, b, g, fb = _cg_problem(ctx)
    fx = wd.alloc_field(L24, wd.SITES_EVEN, wd.F64)
    st = wd.cg_solve(ctx, g, mass, fx, fb, tol=1e-10, autotune=True, **kw)
    x = unpack_field(ctx, L24, wd.SITES_EVEN, wd.F64, fx)
    rel = float(np.linalg.norm(b - oracle.mdagm(L24, U, mass, x)) / np.linalg.norm(b))
    assert st["status"] == 0 and rel <= 1e-10, (st, rel)


@pytest.mark.parametrize("solver,kw", [(wd.SOLVER_BICGSTAB, dict(inner_prec=wd.F16, delta=0.01)),
                                       (wd.SOLVER_CGNE, dict(inner_prec=wd.F16, delta=0.01, use_graph=True))],
                         ids=["bicgstab_fp16", "cgne_fp16_graph"])
def test_full_solve_24_3x48(ctx, solver, kw):
    U = synth.gauge(L24, seed=1003)
    b = synth.spinor(L24, seed=3201)
    g = wd.Gauge(ctx, L24, U)
    fb = pack_field(ctx, L24, wd.SITES_FULL, wd.F64, b)
    fx = wd.alloc_field(L24, wd.SITES_FULL, wd.F64)
    st = wd.wilson_solve(ctx, g, 0.1, fx, fb, tol=1e-10, solver=solver, **kw)
    x = unpack_field(ctx, L24, wd.SITES_FULL, wd.F64, fx)
    rel = float(np.linalg.norm(b - oracle.dirac(L24, U, x, 0.1)) / np.linalg.norm(b))
    assert st["status"] == 0 and rel <= 1e-10, (st, rel)


@pytest.mark.parametrize("mode,inner", [(wd.BATCH_GRAPH, wd.F32), (wd.BATCH_PERSISTENT, wd.F32),
                                        (wd.BATCH_PERSISTENT, wd.F16)])
def test_uneven_batch_benchmark_configuration(ctx, mode, inner):
    """The 24 solves of the batch benchmark (8 each of 8^4, 16^4, 24^3x48; masses U[0.05, 0.5],
    seed 4001; FP32 or FP16 inner, delta 0.01), every solve checked by the oracle operator."""
    rng = np.random.default_rng(4001)
    lattices = [(8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 48)]
    gauges, probs, host = {}, [], []
    for k in range(24):
        dims = lattices[k // 8]
        if dims not in gauges:
            U = synth.gauge(dims, seed=1000 + 10 + k // 8)
            gauges[dims] = (U, wd.Gauge(ctx, dims, U))
        U, g = gauges[dims]
        b = synth.even_spinor(dims, seed=3200 + k)
        mass = float(rng.uniform(0.05, 0.5))
        probs.append(dict(gauge=g, mass=mass, tol=1e-10, b=pack_field(ctx, dims, wd.SITES_EVEN, wd.F64, b),
                          x=wd.alloc_field(dims, wd.SITES_EVEN, wd.F64), inner_prec=inner, delta=0.01))
        host.append((dims, U, mass, b))
    stats = wd.cg_solve_batch(ctx, probs, mode=mode)
    for k, (st, (dims, U, mass, b)) in enumerate(zip(stats, host)):
        assert st["status"] == 0, (k, st)
        x = unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, probs[k]["x"])
        rel = float(np.linalg.norm(b - oracle.mdagm(dims, U, mass, x)) / np.linalg.norm(b))
        assert rel <= 1e-10, (k, rel)


@pytest.mark.parametrize("halo_prec", [wd.F32, wd.F16])
def test_decomposed_operator_32_4(ctx, halo_prec):
    """The decomposition benchmark: 32^4 FP32 in 4 slabs."""
    U, psi = _links_and_source(L32)
    dd = wd.DomainDecomposition(ctx, L32, 4, U)
    ld = dd.local_dims()
    vloc = volume(ld)
    ins = [pack_field(ctx, ld, wd.SITES_FULL, wd.F32, psi[k * vloc:(k + 1) * vloc]) for k in range(4)]
    outs = [wd.alloc_field(ld, wd.SITES_FULL, wd.F32) for _ in range(4)]
    dd.dslash(outs, ins, 0.1, prec=wd.F32, halo_prec=halo_prec)
    got = np.concatenate([unpack_field(ctx, ld, wd.SITES_FULL, wd.F32, o) for o in outs])
    err = rel_max_err(got, oracle.dirac(L32, U, psi, 0.1))
    assert err < max(TOL[wd.F32], TOL[halo_prec]), err


def test_stream_products_benchmark_size(ctx):
    """2^26 complex numbers (1 GiB arrays), a sample of 2^20 elements against the oracle."""
    n = 1 << 26
    gen = torch.Generator(device="cuda").manual_seed(6001)
    x = torch.randn(2 * n, dtype=torch.float64, device="cuda", generator=gen)
    y = torch.randn(2 * n, dtype=torch.float64, device="cuda", generator=gen)
    z = torch.randn(2 * n, dtype=torch.float64, device="cuda", generator=gen)
    idx = torch.from_numpy(np.random.default_rng(61).choice(n, 1 << 20, replace=False)).cuda()
    pick = lambda a: torch.stack([a[2 * idx], a[2 * idx + 1]], 1).reshape(-1).cpu().numpy()
    xs, ys, zs = pick(x), pick(y), pick(z)
    for kind in (wd.STREAM_CPLX_MUL, wd.STREAM_CPLX_CONJ_MADD):
        out = torch.empty_like(z) if kind == wd.STREAM_CPLX_MUL else z.clone()
        wd.stream_mul(ctx, kind, n, x, y, out)
        ref = oracle.stream_mul(kind, xs, ys, zs)
        got = pick(out)
        assert np.max(np.abs(got - ref)) <= 1e-15 * np.max(np.abs(ref)) * 8, kind
    out = torch.empty_like(x)
    wd.stream_mul(ctx, wd.STREAM_REAL_MUL, 2 * n, x, y, out)
    ridx = torch.from_numpy(np.random.default_rng(62).choice(2 * n, 1 << 20, replace=False)).cuda()
    assert np.array_equal(out[ridx].cpu().numpy(), oracle.stream_mul(wd.STREAM_REAL_MUL, x[ridx].cpu().numpy(),
                                                                      y[ridx].cpu().numpy()))
