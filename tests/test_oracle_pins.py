"""Pins of the FP64 oracle against facts other than its own formula (CPU only).

What each pin catches (arXiv:1901.07294 Sec. II-A, Eq. (1), plus the readings
listed in the oracle's header):
  * Clifford algebra / golden basis ........ wrong gamma entries
  * free-field plane waves (closed form) .... projector signs, factor 1/2, mass
                                              term, wrap, direction order
  * golden 2^4 free spectrum ................ the same, eigenvalue multiplicities
  * gauge covariance ........................ link placement and daggers
  * gamma5-hermiticity ...................... consistency of the two hops
  * Eq. (1) identity ........................ D_h(paper) = gamma5 H gamma5
  * dense brute force ....................... the whole operator, entry by entry
  * Schur complement / dense solve / free CG  even-odd operator and CG
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from tests._lattice import (coords, golden_gammas, parity, plane_wave, rel_max_err,
                            shift_index, volume)

G = golden_gammas()
I4 = np.eye(4)


def test_golden_basis_clifford_algebra():
    for mu in range(4):
        g = G[mu]
        assert np.allclose(g, g.conj().T)                      # Hermitian
        for nu in range(4):
            anti = g @ G[nu] + G[nu] @ g
            assert np.allclose(anti, 2 * (mu == nu) * I4)      # {g_mu, g_nu} = 2 delta
        assert np.linalg.matrix_rank(I4 - g) == 2 and np.linalg.matrix_rank(I4 + g) == 2
    g5 = G[0] @ G[1] @ G[2] @ G[3]
    assert np.allclose(g5, G[5])
    assert np.allclose(G[5], np.diag([1, 1, -1, -1]))          # chiral: gamma5 diagonal


def test_oracle_gammas_match_golden_basis():
    for mu in range(4):
        assert np.array_equal(oracle.gamma(mu), G[mu])
    assert np.array_equal(oracle.gamma(4), G[5])


def _random_u(rng):
    return rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 6, 2, 8), (6, 2, 4, 2)])
def test_free_field_plane_waves(dims):
    """U = 1: D exp(ip.x) u = exp(ip.x) [m + sum(1-cos p) + i sum gamma sin p] u."""
    rng = np.random.default_rng(7)
    m = 0.1
    U = synth.unit_gauge(dims)
    for trial in range(4):
        n = [rng.integers(0, L) for L in dims]
        p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
        u = _random_u(rng)
        psi = plane_wave(dims, n, u)
        dp = (m + np.sum(1 - np.cos(p))) * I4 + 1j * sum(G[mu] * np.sin(p[mu]) for mu in range(4))
        expect = plane_wave(dims, n, dp @ u)
        got = oracle.dirac(dims, U, psi, m)
        assert rel_max_err(got, expect) < 1e-14


def test_free_field_constant_field_gives_mass():
    dims = (4, 4, 2, 2)
    U = synth.unit_gauge(dims)
    psi = np.broadcast_to(_random_u(np.random.default_rng(1)), (volume(dims), 4, 3))
    assert rel_max_err(oracle.dirac(dims, U, psi, 0.37), 0.37 * psi) < 1e-14


def _dense_from_oracle(dims, fn):
    v = volume(dims)
    n = 12 * v
    cols = []
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1.0
        cols.append(fn(e.reshape(v, 4, 3)).reshape(n))
    return np.stack(cols, axis=1)


def _golden_spectrum():
    rows = []
    from tests._lattice import GOLDEN
    import os
    with open(os.path.join(GOLDEN, "free_field_2x2x2x2_spectrum.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return rows


def test_free_field_spectrum_2x2x2x2_golden():
    dims, m = (2, 2, 2, 2), 0.25
    U = synth.unit_gauge(dims)
    D = _dense_from_oracle(dims, lambda p: oracle.dirac(dims, U, p, m))
    ev = np.linalg.eigvals(D)
    assert np.max(np.abs(ev.imag)) < 1e-12
    vals = np.round(ev.real - m, 10)
    for k, shift, mult in _golden_spectrum():
        assert np.sum(np.abs(vals - shift) < 1e-9) == mult


def test_free_field_spectrum_closed_form_4x4x2x2():
    """Eigenvalues m + sum(1-cos p) +- i sqrt(sum sin^2 p), each 6-fold per momentum."""
    dims, m = (4, 4, 2, 2), 0.1
    U = synth.unit_gauge(dims)
    D = _dense_from_oracle(dims, lambda p: oracle.dirac(dims, U, p, m))
    ev = np.sort_complex(np.round(np.linalg.eigvals(D), 9))
    expect = []
    for n in itertools.product(*[range(L) for L in dims]):
        p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
        a = m + np.sum(1 - np.cos(p))
        s = math.sqrt(np.sum(np.sin(p) ** 2))
        expect += [a + 1j * s] * 6 + [a - 1j * s] * 6
    expect = np.sort_complex(np.round(np.asarray(expect), 9))
    assert np.max(np.abs(ev - expect)) < 1e-8


def _dense_numpy(dims, U, m):
    """Explicit 12V x 12V matrix assembled block by block (site, spin, colour)."""
    v = volume(dims)
    D = (m + 4) * np.eye(12 * v, dtype=np.complex128)
    for mu in range(4):
        fwd = shift_index(dims, mu, +1)
        bwd = shift_index(dims, mu, -1)
        for s in range(v):
            sp, sm = fwd[s], bwd[s]
            D[12 * s:12 * s + 12, 12 * sp:12 * sp + 12] += -0.5 * np.kron(I4 - G[mu], U[s, mu])
            D[12 * s:12 * s + 12, 12 * sm:12 * sm + 12] += -0.5 * np.kron(I4 + G[mu], U[sm, mu].conj().T)
    return D


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4), (4, 4, 2, 2)])
def test_dense_brute_force(dims):
    U = synth.gauge(dims, seed=1000 + volume(dims))
    m = 0.1
    D = _dense_numpy(dims, U, m)
    psi = synth.spinor(dims, seed=2001)
    got = oracle.dirac(dims, U, psi, m).reshape(-1)
    assert np.max(np.abs(got - D @ psi.reshape(-1))) < 1e-13


def test_gamma5_hermiticity():
    dims = (4, 4, 4, 4)
    U = synth.gauge(dims, seed=1003)
    x = synth.spinor(dims, seed=2002)
    y = synth.spinor(dims, seed=2003)
    m = 0.1
    lhs = np.vdot(x, oracle.dirac(dims, U, y, m))
    g5dg5x = oracle.gamma_apply(4, oracle.dirac(dims, U, oracle.gamma_apply(4, x), m))
    rhs = np.vdot(g5dg5x, y)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


def test_gauge_covariance():
    """U'_mu(x) = G(x) U_mu(x) G(x+mu)^dagger, psi' = G psi  =>  D[U'] psi' = G D[U] psi."""
    dims = (4, 2, 4, 6)
    v = volume(dims)
    U = synth.gauge(dims, seed=1004)
    Gx = synth.su3(v, 1.5, seed=7777)
    Up = np.empty_like(U)
    for mu in range(4):
        fwd = shift_index(dims, mu, +1)
        Up[:, mu] = Gx @ U[:, mu] @ Gx[fwd].conj().transpose(0, 2, 1)
    psi = synth.spinor(dims, seed=2004)
    psip = np.einsum("sij,saj->sai", Gx, psi)
    lhs = oracle.dirac(dims, Up, psip, 0.2)
    rhs = np.einsum("sij,saj->sai", Gx, oracle.dirac(dims, U, psi, 0.2))
    assert rel_max_err(lhs, rhs) < 1e-13


def test_paper_convention_identity():
    """Eq. (1) as printed equals gamma5 H gamma5 (gamma5 gamma_mu gamma5 = -gamma_mu)."""
    dims = (4, 2, 2, 4)
    U = synth.gauge(dims, seed=1005)
    psi = synth.spinor(dims, seed=2005)
    dh = oracle.hop(dims, U, psi, convention=1)
    g5hg5 = oracle.gamma_apply(4, oracle.hop(dims, U, oracle.gamma_apply(4, psi), convention=0))
    assert rel_max_err(dh, g5hg5) < 1e-14
    assert rel_max_err(dh, oracle.hop(dims, U, psi, convention=0)) > 1e-2


def test_even_odd_blocks_sum_to_full_hop():
    dims = (4, 4, 2, 6)
    U = synth.gauge(dims, seed=1006)
    psi = synth.spinor(dims, seed=2006)
    par = parity(dims)
    full = oracle.hop(dims, U, psi)
    he = oracle.hop(dims, U, psi, out_parity=0)
    ho = oracle.hop(dims, U, psi, out_parity=1)
    assert np.all(he[par == 1] == 0) and np.all(ho[par == 0] == 0)
    assert rel_max_err(he + ho, full) < 1e-15
    # H_{eo} only reads odd sites
    psi_o = psi.copy()
    psi_o[par == 0] = 0
    assert rel_max_err(oracle.hop(dims, U, psi_o, out_parity=0), he) < 1e-15


def _eo_perm(dims):
    par = parity(dims)
    ev = np.where(par == 0)[0]
    od = np.where(par == 1)[0]
    idx = lambda sites: (12 * sites[:, None] + np.arange(12)[None, :]).reshape(-1)
    return idx(ev), idx(od)


def test_schur_complement_against_dense_inverse():
    dims = (4, 2, 2, 4)
    U = synth.gauge(dims, seed=1007)
    m = 0.1
    D = _dense_numpy(dims, U, m)
    e, o = _eo_perm(dims)
    schur = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    x = synth.even_spinor(dims, seed=2007)
    got = oracle.mhat(dims, U, m, x)
    assert np.max(np.abs(got.reshape(-1)[o])) == 0
    assert np.max(np.abs(got.reshape(-1)[e] - schur @ x.reshape(-1)[e])) < 1e-12
    gotd = oracle.mhat(dims, U, m, x, dagger=True)
    assert np.max(np.abs(gotd.reshape(-1)[e] - schur.conj().T @ x.reshape(-1)[e])) < 1e-12


def test_cg_against_dense_solve():
    dims = (4, 2, 2, 4)
    U = synth.gauge(dims, seed=1008)
    m = 0.05
    D = _dense_numpy(dims, U, m)
    e, o = _eo_perm(dims)
    schur = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    A = schur.conj().T @ schur
    b = synth.even_spinor(dims, seed=3001)
    x, it, rel = oracle.cg(dims, U, m, b, tol=1e-12)
    assert it > 0 and rel <= 1e-12
    xd = np.linalg.solve(A, b.reshape(-1)[e])
    assert rel_max_err(x.reshape(-1)[e], xd) < 1e-9
    assert np.all(x.reshape(-1)[o] == 0)


def test_cg_free_field_momentum_space():
    """Free field: even-restricted plane waves are eigenvectors of Mhat with the
    4x4 symbol (m+4) - H(p)^2 / (4(m+4)), H(p) = 2 sum cos p - 2i sum gamma sin p."""
    dims = (4, 4, 4, 8)
    m = 0.1
    U = synth.unit_gauge(dims)
    par = parity(dims)
    n = (1, 3, 2, 5)
    p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
    Hp = 2 * np.sum(np.cos(p)) * I4 - 2j * sum(G[mu] * np.sin(p[mu]) for mu in range(4))
    Mp = (m + 4) * I4 - Hp @ Hp / (4 * (m + 4))
    u = _random_u(np.random.default_rng(3))
    b = plane_wave(dims, n, u)
    b[par == 1] = 0
    mb = oracle.mhat(dims, U, m, b)
    expect = plane_wave(dims, n, Mp @ u)
    expect[par == 1] = 0
    assert rel_max_err(mb, expect) < 1e-13
    x, it, rel = oracle.cg(dims, U, m, b, tol=1e-12)
    assert it > 0 and rel <= 1e-12
    xs = plane_wave(dims, n, np.linalg.solve(Mp.conj().T @ Mp, u))
    xs[par == 1] = 0
    assert rel_max_err(x, xs) < 1e-10


def test_planted_sign_error_is_caught():
    """A projector-sign mistake (Eq. (1) convention used as H) fails the free-field pin."""
    dims = (4, 4, 2, 2)
    U = synth.unit_gauge(dims)
    n = (1, 1, 0, 1)
    p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
    u = _random_u(np.random.default_rng(11))
    psi = plane_wave(dims, n, u)
    m = 0.1
    wrong = (m + 4) * psi - 0.5 * oracle.hop(dims, U, psi, convention=1)
    dp = (m + np.sum(1 - np.cos(p))) * I4 + 1j * sum(G[mu] * np.sin(p[mu]) for mu in range(4))
    assert rel_max_err(wrong, plane_wave(dims, n, dp @ u)) > 1e-2


def test_bicgstab_against_dense_solve():
    """BiCGStab on Mhat (not Hermitian) reaches the dense solution of the Schur system."""
    dims = (4, 2, 2, 4)
    U = synth.gauge(dims, seed=1009)
    m = 0.05
    D = _dense_numpy(dims, U, m)
    e, o = _eo_perm(dims)
    schur = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    b = synth.even_spinor(dims, seed=3002)
    x, it, rel = oracle.bicgstab(dims, U, m, b, tol=1e-12)
    assert it > 0 and rel <= 1e-12
    xd = np.linalg.solve(schur, b.reshape(-1)[e])
    assert rel_max_err(x.reshape(-1)[e], xd) < 1e-10
    assert np.all(x.reshape(-1)[o] == 0)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_solve_full_against_dense_solve(dims):
    """Source reduction, Schur solve and odd reconstruction together give D^{-1} b."""
    U = synth.gauge(dims, seed=1010)
    m = 0.1
    D = _dense_numpy(dims, U, m)
    b = synth.spinor(dims, seed=3003)
    x, it, rel = oracle.solve_full(dims, U, m, b, tol=1e-12)
    assert it > 0 and rel <= 1e-12
    xd = np.linalg.solve(D, b.reshape(-1))
    assert rel_max_err(x.reshape(-1), xd) < 1e-10


def test_solve_full_free_field_inverse():
    """Free field: D(p) = a + i gamma.s with a = m + sum(1 - cos p), s = sin p, so
    D(p)^{-1} = (a - i gamma.s) / (a^2 + |s|^2) on a plane wave."""
    dims = (8, 4, 4, 8)
    m = 0.05
    U = synth.unit_gauge(dims)
    n = (3, 1, 2, 5)
    p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
    a = m + np.sum(1 - np.cos(p))
    gs = sum(G[mu] * np.sin(p[mu]) for mu in range(4))
    dinv = (a * I4 - 1j * gs) / (a * a + np.sum(np.sin(p) ** 2))
    u = _random_u(np.random.default_rng(21))
    b = plane_wave(dims, n, u)
    x, it, rel = oracle.solve_full(dims, U, m, b, tol=1e-12)
    assert it > 0 and rel <= 1e-12
    assert rel_max_err(x, plane_wave(dims, n, dinv @ u)) < 1e-10


@pytest.mark.parametrize("dims", [(4, 4, 2, 6), (2, 2, 2, 2)])
def test_antiperiodic_free_field_half_integer_momenta(dims):
    """Antiperiodic in t: exp(i p.x) u with p_t = (2 n_t + 1) pi / L_t changes sign
    around t and is an eigenvector with the same symbol D(p) = a + i gamma.s."""
    m = 0.1
    U = oracle.antiperiodic_links(dims, synth.unit_gauge(dims))
    n = (1, 1, 0, 0.5)                     # p_t = pi / L_t
    p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
    u = _random_u(np.random.default_rng(41))
    psi = plane_wave(dims, n, u)
    dp = (m + np.sum(1 - np.cos(p))) * I4 + 1j * sum(G[mu] * np.sin(p[mu]) for mu in range(4))
    assert rel_max_err(oracle.dirac(dims, U, psi, m), plane_wave(dims, n, dp @ u)) < 1e-13
    # the periodic operator does not have this eigenvector
    assert rel_max_err(oracle.dirac(dims, synth.unit_gauge(dims), psi, m), plane_wave(dims, n, dp @ u)) > 1e-2


def test_antiperiodic_links_touch_only_the_last_time_slice():
    dims = (4, 2, 2, 6)
    U = synth.gauge(dims, seed=1011)
    A = oracle.antiperiodic_links(dims, U)
    t = coords(dims)[:, 3]
    assert np.array_equal(A[t < 5], U[t < 5])
    assert np.array_equal(A[t == 5][:, :3], U[t == 5][:, :3])
    assert np.array_equal(A[t == 5][:, 3], -U[t == 5][:, 3])


def test_antiperiodic_full_solve_free_field():
    """D^{-1} on an antiperiodic plane wave is (a - i gamma.s) / (a^2 + |s|^2)."""
    dims = (4, 4, 4, 8)
    m = 0.05
    U = oracle.antiperiodic_links(dims, synth.unit_gauge(dims))
    n = (1, 3, 2, 2.5)
    p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
    a = m + np.sum(1 - np.cos(p))
    gs = sum(G[mu] * np.sin(p[mu]) for mu in range(4))
    dinv = (a * I4 - 1j * gs) / (a * a + np.sum(np.sin(p) ** 2))
    u = _random_u(np.random.default_rng(42))
    x, it, rel = oracle.solve_full(dims, U, m, plane_wave(dims, n, u), tol=1e-12)
    assert it > 0 and rel <= 1e-12
    assert rel_max_err(x, plane_wave(dims, n, dinv @ u)) < 1e-10


def test_stream_products_against_python_complex():
    """The written-out complex products agree with Python's own complex arithmetic
    (an independent implementation) element by element, and the identities
    conj(x) x = |x|^2, x i = (-Im x, Re x) hold."""
    rng = np.random.default_rng(51)
    n = 257
    x = rng.standard_normal(2 * n)
    y = rng.standard_normal(2 * n)
    z = rng.standard_normal(2 * n)
    cx = [complex(x[2 * k], x[2 * k + 1]) for k in range(n)]
    cy = [complex(y[2 * k], y[2 * k + 1]) for k in range(n)]
    cz = [complex(z[2 * k], z[2 * k + 1]) for k in range(n)]
    expect = {
        oracle.STREAM_CPLX_MUL: [a * b for a, b in zip(cx, cy)],
        oracle.STREAM_CPLX_CONJ_MUL: [a.conjugate() * b for a, b in zip(cx, cy)],
        oracle.STREAM_CPLX_MADD: [c + a * b for a, b, c in zip(cx, cy, cz)],
        oracle.STREAM_CPLX_CONJ_MADD: [c + a.conjugate() * b for a, b, c in zip(cx, cy, cz)],
    }
    for kind, ref in expect.items():
        got = oracle.stream_mul(kind, x, y, z)
        ref = np.array([[v.real, v.imag] for v in ref]).reshape(-1)
        assert np.max(np.abs(got - ref)) <= 1e-15 * np.max(np.abs(ref)), kind
    assert np.array_equal(oracle.stream_mul(oracle.STREAM_REAL_MUL, x, y), np.array([a * b for a, b in zip(x, y)]))
    xx = oracle.stream_mul(oracle.STREAM_CPLX_CONJ_MUL, x, x)
    assert np.all(xx[1::2] == 0) and np.allclose(xx[0::2], x[0::2] ** 2 + x[1::2] ** 2, rtol=1e-15)
    i_unit = np.tile([0.0, 1.0], n)
    xi = oracle.stream_mul(oracle.STREAM_CPLX_MUL, x, i_unit)
    assert np.array_equal(xi[0::2], -x[1::2]) and np.array_equal(xi[1::2], x[0::2])
