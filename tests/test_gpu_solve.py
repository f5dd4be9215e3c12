"""BiCGStab on Mhat and the full-system solve D x = b on the GPU against the FP64 oracle.

A solve is judged by its true residual computed with the oracle's own operator on
the GPU solution (the bar: the tolerance asked for), and by the distance to the
oracle's solution, which agrees to about cond * tol.
"""
import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import pack_field, unpack_field
from tests._lattice import golden_gammas, parity, plane_wave, rel_max_err, volume

pytestmark = pytest.mark.gpu

PREC_CASES = [
    dict(inner_prec=wd.F64),
    dict(inner_prec=wd.F32, reliable=True, delta=0.1),
    dict(inner_prec=wd.F16, reliable=True, delta=0.1),
    dict(inner_prec=wd.BF16, reliable=True, delta=0.1),
    dict(inner_prec=wd.F16, inner_recon=12, outer_recon=12, reliable=True, delta=0.01),
    dict(inner_prec=wd.F16, reliable=False, delta=1e-2),
]


def _ids(kw):
    return "-".join(f"{a}{b}" for a, b in kw.items())


@pytest.fixture(scope="module")
def ctx():
    return wd.Context(0)


_cache = {}


def _schur_problem(dims, mass):
    key = ("schur", dims, mass)
    if key not in _cache:
        U = synth.gauge(dims, seed=1100 + volume(dims) % 997)
        b = synth.even_spinor(dims, seed=3101)
        xo, it, rel = oracle.bicgstab(dims, U, mass, b, tol=1e-12)
        assert it > 0 and rel <= 1e-12
        _cache[key] = (U, b, xo)
    return _cache[key]


def _full_problem(dims, mass):
    key = ("full", dims, mass)
    if key not in _cache:
        U = synth.gauge(dims, seed=1200 + volume(dims) % 997)
        b = synth.spinor(dims, seed=3201)
        xo, it, rel = oracle.solve_full(dims, U, mass, b, tol=1e-12)
        assert it > 0 and rel <= 1e-12
        _cache[key] = (U, b, xo)
    return _cache[key]


@pytest.mark.parametrize("kw", PREC_CASES, ids=_ids)
@pytest.mark.parametrize("dims,mass", [((8, 8, 8, 8), 0.1), ((4, 6, 8, 10), 0.05)])
def test_bicgstab_reaches_true_residual(ctx, dims, mass, kw):
    tol = 1e-10
    U, b, xo = _schur_problem(dims, mass)
    g = wd.Gauge(ctx, dims, U)
    fb = pack_field(ctx, dims, wd.SITES_EVEN, wd.F64, b)
    fx = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
    st = wd.bicgstab_solve(ctx, g, mass, fx, fb, tol=tol, **kw)
    x = unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, fx)
    assert st["status"] == 0 and st["true_rel_resid"] <= tol
    true_rel = float(np.linalg.norm(b - oracle.mhat(dims, U, mass, x)) / np.linalg.norm(b))
    assert true_rel <= tol, true_rel
    assert np.all(x[parity(dims) == 1] == 0)
    assert rel_max_err(x, xo) < 1e-7


@pytest.mark.parametrize("solver", [wd.SOLVER_BICGSTAB, wd.SOLVER_CGNE])
@pytest.mark.parametrize("kw", PREC_CASES[:4] + [dict(inner_prec=wd.F16, reliable=True, delta=0.01, use_graph=True)],
                         ids=_ids)
@pytest.mark.parametrize("dims,mass", [((8, 8, 8, 8), 0.1), ((4, 6, 8, 10), 0.05)])
def test_wilson_solve_full_system(ctx, dims, mass, solver, kw):
    if solver == wd.SOLVER_BICGSTAB and kw.get("use_graph"):
        kw = {k: v for k, v in kw.items() if k != "use_graph"}
    tol = 1e-10
    U, b, xo = _full_problem(dims, mass)
    g = wd.Gauge(ctx, dims, U)
    fb = pack_field(ctx, dims, wd.SITES_FULL, wd.F64, b)
    fx = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
    st = wd.wilson_solve(ctx, g, mass, fx, fb, tol=tol, solver=solver, **kw)
    x = unpack_field(ctx, dims, wd.SITES_FULL, wd.F64, fx)
    assert st["status"] == 0 and st["true_rel_resid"] <= tol
    true_rel = float(np.linalg.norm(b - oracle.dirac(dims, U, x, mass)) / np.linalg.norm(b))
    assert true_rel <= tol, true_rel
    assert rel_max_err(x, xo) < 1e-7


@pytest.mark.parametrize("solver", [wd.SOLVER_BICGSTAB, wd.SOLVER_CGNE])
def test_wilson_solve_free_field_closed_form(ctx, solver):
    """Unit links: D(p)^{-1} = (a - i gamma.s) / (a^2 + |s|^2) on a plane wave."""
    G = golden_gammas()
    I4 = np.eye(4)
    dims, m = (8, 4, 4, 8), 0.05
    U = synth.unit_gauge(dims)
    n = (3, 1, 2, 5)
    p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
    a = m + np.sum(1 - np.cos(p))
    gs = sum(G[mu] * np.sin(p[mu]) for mu in range(4))
    dinv = (a * I4 - 1j * gs) / (a * a + np.sum(np.sin(p) ** 2))
    rng = np.random.default_rng(31)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    b = plane_wave(dims, n, u)
    g = wd.Gauge(ctx, dims, U)
    fb = pack_field(ctx, dims, wd.SITES_FULL, wd.F64, b)
    fx = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
    wd.wilson_solve(ctx, g, m, fx, fb, tol=1e-12, solver=solver, inner_prec=wd.F32, reliable=True, delta=0.1)
    x = unpack_field(ctx, dims, wd.SITES_FULL, wd.F64, fx)
    assert rel_max_err(x, plane_wave(dims, n, dinv @ u)) < 1e-10


@pytest.mark.parametrize("solver", [wd.SOLVER_BICGSTAB, wd.SOLVER_CGNE])
@pytest.mark.parametrize("which", ["even_only", "odd_only"])
def test_wilson_solve_one_parity_sources(ctx, solver, which):
    """A source on one parity only: b^_e = b_e (odd part zero) or b^_e = H_eo b_o / (2(m+4))."""
    dims, m = (4, 4, 4, 6), 0.1
    U = synth.gauge(dims, seed=1301)
    b = synth.spinor(dims, seed=3301)
    par = parity(dims)
    b[par == (1 if which == "even_only" else 0)] = 0
    g = wd.Gauge(ctx, dims, U)
    fb = pack_field(ctx, dims, wd.SITES_FULL, wd.F64, b)
    fx = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
    st = wd.wilson_solve(ctx, g, m, fx, fb, tol=1e-10, solver=solver, inner_prec=wd.F16, reliable=True,
                         delta=0.1)
    x = unpack_field(ctx, dims, wd.SITES_FULL, wd.F64, fx)
    assert st["status"] == 0
    assert np.linalg.norm(b - oracle.dirac(dims, U, x, m)) / np.linalg.norm(b) <= 1e-10


def test_wilson_solve_zero_source(ctx):
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, seed=5)
    g = wd.Gauge(ctx, dims, U)
    fb = pack_field(ctx, dims, wd.SITES_FULL, wd.F64, np.zeros((volume(dims), 4, 3), np.complex128))
    fx = pack_field(ctx, dims, wd.SITES_FULL, wd.F64, synth.spinor(dims, seed=6))
    for solver in (wd.SOLVER_BICGSTAB, wd.SOLVER_CGNE):
        st = wd.wilson_solve(ctx, g, 0.1, fx, fb, tol=1e-10, solver=solver, inner_prec=wd.F16)
        assert st["iters"] == 0 and st["true_rel_resid"] == 0.0
        assert np.all(unpack_field(ctx, dims, wd.SITES_FULL, wd.F64, fx) == 0)


def test_bicgstab_not_converged_and_bad_arguments(ctx):
    dims, m = (8, 8, 8, 8), 0.1
    U, b, _ = _schur_problem(dims, m)
    g = wd.Gauge(ctx, dims, U)
    fb = pack_field(ctx, dims, wd.SITES_EVEN, wd.F64, b)
    fx = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
    st = wd.bicgstab_solve(ctx, g, m, fx, fb, tol=1e-10, inner_prec=wd.F64, maxiter=3, check=False)
    assert st["status"] == wd.WD_ENOCONV and st["iters"] == 3
    assert 1e-10 < st["true_rel_resid"] < 1.0
    with pytest.raises(wd.WdError):
        wd.bicgstab_solve(ctx, g, m, fb, fb, tol=1e-10)          # x aliases b
    with pytest.raises(wd.WdError):
        wd.bicgstab_solve(ctx, g, m, fx, fb, tol=0.0)
    ff = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
    fbf = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
    with pytest.raises(wd.WdError):
        wd.wilson_solve(ctx, g, m, ff, fbf, tol=1e-10, solver=7)


def test_bicgstab_iterations_compared_with_cg(ctx):
    """Both solve the same even system; BiCGStab needs two Mhat per iteration, CG on the
    normal equations two as well, and on this well-conditioned case BiCGStab needs fewer
    iterations than CGNE (cond(Mhat) vs cond(Mhat)^2)."""
    dims, m = (8, 8, 8, 8), 0.1
    U, b, _ = _full_problem(dims, m)
    g = wd.Gauge(ctx, dims, U)
    fb = pack_field(ctx, dims, wd.SITES_FULL, wd.F64, b)
    fx = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
    sb = wd.wilson_solve(ctx, g, m, fx, fb, tol=1e-10, solver=wd.SOLVER_BICGSTAB, inner_prec=wd.F64)
    sc = wd.wilson_solve(ctx, g, m, fx, fb, tol=1e-10, solver=wd.SOLVER_CGNE, inner_prec=wd.F64)
    assert sb["iters"] < sc["iters"]
