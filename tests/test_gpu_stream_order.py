"""Solves that run on their own streams (graph-driven CG, batch graph mode, CGNE with
graphs) must see the work the caller queued on its stream before the call.

The source is written on the current stream behind a ~20 ms spin kernel, and the solve
is called at once: a solve that started early would read the zeros that were there.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import pack_field, unpack_field

pytestmark = pytest.mark.gpu

DIMS, MASS, TOL_SOLVE = (8, 8, 8, 8), 0.1, 1e-10


@pytest.fixture(scope="module")
def ctx():
    return wd.Context(0)


def _late_source(ctx, b, sites):
    real = pack_field(ctx, DIMS, sites, wd.F64, b)
    fb = torch.zeros_like(real)
    torch.cuda.synchronize()
    torch.cuda._sleep(40_000_000)      # bounded spin on the current stream
    fb.copy_(real)                     # queued behind it
    return fb


def test_graph_cg_waits_for_the_callers_stream(ctx):
    U = synth.gauge(DIMS, seed=1701)
    b = synth.even_spinor(DIMS, seed=3701)
    g = wd.Gauge(ctx, DIMS, U)
    g.prepare(wd.F64, 18)
    g.prepare(wd.F16, 18)
    fx = wd.alloc_field(DIMS, wd.SITES_EVEN, wd.F64)
    fb = _late_source(ctx, b, wd.SITES_EVEN)
    wd.cg_solve(ctx, g, MASS, fx, fb, tol=TOL_SOLVE, inner_prec=wd.F16, reliable=True, delta=0.1, use_graph=True)
    x = unpack_field(ctx, DIMS, wd.SITES_EVEN, wd.F64, fx)
    assert np.linalg.norm(b - oracle.mdagm(DIMS, U, MASS, x)) / np.linalg.norm(b) <= TOL_SOLVE


def test_graph_batch_waits_for_the_callers_stream(ctx):
    U = synth.gauge(DIMS, seed=1702)
    b = synth.even_spinor(DIMS, seed=3702)
    g = wd.Gauge(ctx, DIMS, U)
    g.prepare(wd.F64, 18)
    g.prepare(wd.F32, 18)
    fx = wd.alloc_field(DIMS, wd.SITES_EVEN, wd.F64)
    fb = _late_source(ctx, b, wd.SITES_EVEN)
    wd.cg_solve_batch(ctx, [dict(gauge=g, mass=MASS, tol=TOL_SOLVE, x=fx, b=fb, inner_prec=wd.F32)],
                      mode=wd.BATCH_GRAPH)
    x = unpack_field(ctx, DIMS, wd.SITES_EVEN, wd.F64, fx)
    assert np.linalg.norm(b - oracle.mdagm(DIMS, U, MASS, x)) / np.linalg.norm(b) <= TOL_SOLVE


def test_cgne_with_graph_waits_for_its_own_operator(ctx):
    """The full solve's CGNE applies Mhat^dagger on the caller's stream and then starts the
    graph-driven CG on that result."""
    U = synth.gauge(DIMS, seed=1703)
    b = synth.spinor(DIMS, seed=3703)
    g = wd.Gauge(ctx, DIMS, U)
    fx = wd.alloc_field(DIMS, wd.SITES_FULL, wd.F64)
    fb = _late_source(ctx, b, wd.SITES_FULL)
    wd.wilson_solve(ctx, g, MASS, fx, fb, tol=TOL_SOLVE, solver=wd.SOLVER_CGNE, inner_prec=wd.F16, reliable=True,
                    delta=0.1, use_graph=True)
    x = unpack_field(ctx, DIMS, wd.SITES_FULL, wd.F64, fx)
    assert np.linalg.norm(b - oracle.dirac(DIMS, U, x, MASS)) / np.linalg.norm(b) <= TOL_SOLVE
