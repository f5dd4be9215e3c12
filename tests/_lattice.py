"""Test-side lattice helpers (numpy): geometry, golden gamma matrices, error metric.

Independent of both the oracle and the CUDA library.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

_TOK = {"0": 0, "1": 1, "-1": -1, "i": 1j, "-i": -1j}


def golden_gammas() -> dict[int, np.ndarray]:
    """Dirac matrices from tests/golden/gamma_chiral_basis.txt; key 5 is gamma5."""
    out, cur, rows = {}, None, []
    with open(os.path.join(GOLDEN, "gamma_chiral_basis.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("gamma"):
                cur, rows = int(line.split()[1]), []
                continue
            rows.append([_TOK[t] for t in line.split()])
            if len(rows) == 4:
                out[cur] = np.array(rows, dtype=np.complex128)
    return out


def volume(dims) -> int:
    return int(np.prod([int(d) for d in dims]))


def coords(dims) -> np.ndarray:
    """(V, 4) integer coordinates (x, y, z, t) in lexicographic order."""
    lx, ly, lz, lt = (int(d) for d in dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1)


def lex(dims, c) -> np.ndarray:
    lx, ly, lz, _ = (int(d) for d in dims)
    return c[..., 0] + lx * (c[..., 1] + ly * (c[..., 2] + lz * c[..., 3]))


def shift_index(dims, mu: int, step: int) -> np.ndarray:
    """Lexicographic index of x + step*mu-hat for every site x (periodic)."""
    c = coords(dims).copy()
    c[:, mu] = (c[:, mu] + step) % int(dims[mu])
    return lex(dims, c)


def parity(dims) -> np.ndarray:
    return coords(dims).sum(axis=1) & 1


def rel_max_err(y, yref) -> float:
    """max_i |y_i - yref_i| / max_i |yref_i| over all real components."""
    y = np.asarray(y).view(np.float64) if np.iscomplexobj(y) else np.asarray(y)
    yref = np.asarray(yref).view(np.float64) if np.iscomplexobj(yref) else np.asarray(yref)
    return float(np.max(np.abs(y - yref)) / np.max(np.abs(yref)))


def plane_wave(dims, n, u) -> np.ndarray:
    """psi(x) = exp(i p.x) u with p_mu = 2 pi n_mu / L_mu; u is (4,3)."""
    p = 2 * np.pi * np.asarray(n, dtype=np.float64) / np.asarray(dims, dtype=np.float64)
    ph = np.exp(1j * (coords(dims) @ p))
    return ph[:, None, None] * np.asarray(u)[None, :, :]
