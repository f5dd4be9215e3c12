"""Mixed-precision solves whose reliable updates recompute the true residual with the
double-word FP32 operator (outer_prec = WD_DF), judged by the FP64 oracle.

Each GPU solution x is checked by the oracle's own residual |b - A x| / |b| <= tol with
no slack: the solver's double-word residual has errors of order 2^-48 |A| |x| (a few
1e-15 |b| for these sources), far below the 10 % margin of its stopping test.
"""
import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import pack_field, unpack_field

pytestmark = pytest.mark.gpu

L24 = (24, 24, 24, 48)
L8 = (8, 8, 8, 8)


@pytest.fixture(scope="module")
def ctx():
    return wd.Context(0)


_p = {}


def _problem(ctx, dims, seed_l, seed_b):
    key = (dims, seed_l, seed_b)
    if key not in _p:
        U = synth.gauge(dims, seed=seed_l)
        b = synth.even_spinor(dims, seed=seed_b)
        g = wd.Gauge(ctx, dims, U)
        _p[key] = (U, b, g, pack_field(ctx, dims, wd.SITES_EVEN, wd.F64, b))
    return _p[key]


def _rel(dims, U, mass, b, x):
    return float(np.linalg.norm(b - oracle.mdagm(dims, U, mass, x)) / np.linalg.norm(b))


@pytest.mark.parametrize("tol", [1e-10, 1e-12])
@pytest.mark.parametrize("kw", [dict(inner_prec=wd.F16), dict(inner_prec=wd.F32), dict(inner_prec=wd.BF16),
                                dict(inner_prec=wd.F16, use_graph=True), dict(inner_prec=wd.F16, reliable=False)],
                         ids=["fp16", "fp32", "bf16", "fp16_graph", "fp16_refine"])
def test_cg_df_updates_24_3x48(ctx, tol, kw):
    U, b, g, fb = _problem(ctx, L24, 1003, 3001)
    fx = wd.alloc_field(L24, wd.SITES_EVEN, wd.F64)
    st = wd.cg_solve(ctx, g, 0.1, fx, fb, tol=tol, delta=0.01, outer_prec=wd.DF, autotune=True, **kw)
    rel = _rel(L24, U, 0.1, b, unpack_field(ctx, L24, wd.SITES_EVEN, wd.F64, fx))
    assert st["status"] == 0 and rel <= tol, (st, rel)
    assert st["reliable_updates"] >= 2


def test_cg_df_updates_12_real_links(ctx):
    U, b, g, fb = _problem(ctx, L8, 1004, 3002)
    fx = wd.alloc_field(L8, wd.SITES_EVEN, wd.F64)
    st = wd.cg_solve(ctx, g, 0.05, fx, fb, tol=1e-10, inner_prec=wd.F16, inner_recon=12, outer_recon=12,
                     outer_prec=wd.DF)
    rel = _rel(L8, U, 0.05, b, unpack_field(ctx, L8, wd.SITES_EVEN, wd.F64, fx))
    assert st["status"] == 0 and rel <= 1e-10, (st, rel)


def test_bicgstab_and_full_solve_df_updates(ctx):
    U = synth.gauge(L24, seed=1003)
    g = wd.Gauge(ctx, L24, U)
    be = synth.even_spinor(L24, seed=3101)
    fb = pack_field(ctx, L24, wd.SITES_EVEN, wd.F64, be)
    fx = wd.alloc_field(L24, wd.SITES_EVEN, wd.F64)
    st = wd.bicgstab_solve(ctx, g, 0.1, fx, fb, tol=1e-10, inner_prec=wd.F16, outer_prec=wd.DF)
    x = unpack_field(ctx, L24, wd.SITES_EVEN, wd.F64, fx)
    rel = float(np.linalg.norm(be - oracle.mhat(L24, U, 0.1, x)) / np.linalg.norm(be))
    assert st["status"] == 0 and rel <= 1e-10, (st, rel)
    b = synth.spinor(L24, seed=3201)
    fbf = pack_field(ctx, L24, wd.SITES_FULL, wd.F64, b)
    fxf = wd.alloc_field(L24, wd.SITES_FULL, wd.F64)
    for solver in (wd.SOLVER_BICGSTAB, wd.SOLVER_CGNE):
        st = wd.wilson_solve(ctx, g, 0.1, fxf, fbf, tol=1e-10, solver=solver, inner_prec=wd.F16, outer_prec=wd.DF)
        x = unpack_field(ctx, L24, wd.SITES_FULL, wd.F64, fxf)
        rel = float(np.linalg.norm(b - oracle.dirac(L24, U, x, 0.1)) / np.linalg.norm(b))
        assert st["status"] == 0 and rel <= 1e-10, (solver, st, rel)


def test_batch_graph_df_updates_bitwise_alone(ctx):
    """Graph-mode batch with double-word updates: every solve meets tol by the oracle and gives
    the same bits alone (a batch of one) as in the batch."""
    lattices = [(8, 8, 8, 8), (16, 16, 16, 16)]
    probs, host = [], []
    for k in range(6):
        dims = lattices[k % 2]
        U, b, g, fb = _problem(ctx, dims, 1010 + k % 2, 3300 + k)
        mass = 0.1 + 0.05 * k
        probs.append(dict(gauge=g, mass=mass, tol=1e-10, b=fb, x=wd.alloc_field(dims, wd.SITES_EVEN, wd.F64),
                          inner_prec=wd.F16, delta=0.01, outer_prec=wd.DF))
        host.append((dims, U, mass, b))
    stats = wd.cg_solve_batch(ctx, probs, mode=wd.BATCH_GRAPH)
    for k, (st, (dims, U, mass, b)) in enumerate(zip(stats, host)):
        assert st["status"] == 0, (k, st)
        x = unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, probs[k]["x"])
        assert _rel(dims, U, mass, b, x) <= 1e-10, k
        alone = dict(probs[k])
        alone["x"] = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
        st1 = wd.cg_solve_batch(ctx, [alone], mode=wd.BATCH_GRAPH)[0]
        assert st1["iters"] == st["iters"], (k, st1, st)
        assert np.array_equal(unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, alone["x"]), x), k


def test_persistent_batch_rejects_df_updates(ctx):
    U, b, g, fb = _problem(ctx, L8, 1004, 3002)
    p = dict(gauge=g, mass=0.1, tol=1e-10, b=fb, x=wd.alloc_field(L8, wd.SITES_EVEN, wd.F64), inner_prec=wd.F16,
             outer_prec=wd.DF)
    with pytest.raises(wd.WdError) as e:
        wd.cg_solve_batch(ctx, [p], mode=wd.BATCH_PERSISTENT)
    assert e.value.status == wd.WD_EINVAL


def test_bad_outer_precision_rejected(ctx):
    U, b, g, fb = _problem(ctx, L8, 1004, 3002)
    fx = wd.alloc_field(L8, wd.SITES_EVEN, wd.F64)
    for op in (wd.F32, wd.F16, 7):
        with pytest.raises(wd.WdError) as e:
            wd.cg_solve(ctx, g, 0.1, fx, fb, tol=1e-10, inner_prec=wd.F16, outer_prec=op)
        assert e.value.status == wd.WD_EINVAL


def test_queue_df_updates_same_alone_as_in_mix(ctx):
    """Requests with double-word updates through the serving queue: results by the oracle and
    bit for bit the same alone as in a mix of six on two gauges."""
    q = wd.Queue(ctx, 8 << 30, 8)
    reqs, host = [], []
    for k in range(6):
        dims = (8, 8, 8, 8) if k % 2 else (16, 16, 16, 16)
        U, b, g, fb = _problem(ctx, dims, 1020 + k % 2, 3400 + k)
        mass = 0.1 + 0.03 * k
        p = dict(gauge=g, mass=mass, tol=1e-10, b=fb, x=wd.alloc_field(dims, wd.SITES_EVEN, wd.F64),
                 inner_prec=wd.F16, delta=0.01, outer_prec=wd.DF)
        reqs.append((q.submit(p), p))
        host.append((dims, U, mass, b))
    xs = []
    for (t, p), (dims, U, mass, b) in zip(reqs, host):
        r = q.wait(t, timeout_ms=60000)
        assert r["status"] == 0, r
        x = unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, p["x"])
        assert _rel(dims, U, mass, b, x) <= 1e-10
        xs.append(x)
    q.close()
    for k, ((t, p), (dims, U, mass, b)) in enumerate(zip(reqs, host)):
        q1 = wd.Queue(ctx, 8 << 30, 1)
        alone = dict(p)
        alone["x"] = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
        r = q1.wait(q1.submit(alone), timeout_ms=60000)
        q1.close()
        assert r["status"] == 0
        assert np.array_equal(unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, alone["x"]), xs[k]), k


@pytest.mark.parametrize("use_graph", [False, True])
def test_cg_df_updates_light_mass_tight_tol(ctx, use_graph):
    """A light mass (m = 0.02, |x| / |b| large) at tol 1e-12: the double-word residual's noise
    is then within a few orders of the target, and the FP64 convergence checks still end the
    solve with the oracle's residual <= tol."""
    dims = (16, 16, 16, 32)
    U, b, g, fb = _problem(ctx, dims, 1030, 3500)
    fx = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
    st = wd.cg_solve(ctx, g, 0.02, fx, fb, tol=1e-12, inner_prec=wd.F16, delta=0.01, outer_prec=wd.DF,
                     use_graph=use_graph, maxiter=40000)
    rel = _rel(dims, U, 0.02, b, unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, fx))
    assert st["status"] == 0 and rel <= 1e-12, (st, rel)
