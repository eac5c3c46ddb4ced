"""Exact discrete solutions of the 5-point Dirichlet problem, built independently of
the oracle's stencil loops, used to pin it.

* ``matrix``: the 5-point operator assembled as a Kronecker sum of 1D second
  differences, T_x (x) I + beta^2 I (x) T_y, with T = tridiag(-1, 2, -1).
* ``dense_solve``: numpy/LAPACK solve of that system (grids up to ~30 x 30).
* ``dst_solve``: the same system diagonalised by the type-I discrete sine
  transform (scipy.fft), any size.
* ``sine_mode``: the closed form for one sine mode on one edge.
"""
from __future__ import annotations

import numpy as np
import scipy.fft


def second_difference(N: int) -> np.ndarray:
    return 2.0 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)


def matrix(m: int, n: int, beta: float = 1.0) -> np.ndarray:
    """dx^2 * (-Laplacian) on the (n-2) x (m-2) interior, unknowns row-major (j, i)."""
    mi, ni = m - 2, n - 2
    return np.kron(np.eye(ni), second_difference(mi)) + beta ** 2 * np.kron(
        second_difference(ni), np.eye(mi))


def ring_rhs(psi: np.ndarray, beta: float = 1.0) -> np.ndarray:
    """Right-hand side from the Dirichlet ring: interior nodes next to the ring get the
    ring value (weight 1 across x, beta^2 across y)."""
    n, m = psi.shape
    b = np.zeros((n - 2, m - 2))
    b[:, 0] += psi[1:-1, 0]
    b[:, -1] += psi[1:-1, -1]
    b[0, :] += beta ** 2 * psi[0, 1:-1]
    b[-1, :] += beta ** 2 * psi[-1, 1:-1]
    return b


def dense_solve(psi: np.ndarray, beta: float = 1.0, source: np.ndarray | None = None) -> np.ndarray:
    """Exact solution with the ring of psi; ``source`` q adds (E+W)+b2(N+S)-d u + q = 0."""
    n, m = psi.shape
    b = ring_rhs(psi, beta)
    if source is not None:
        b = b + source[1:-1, 1:-1]
    u = np.linalg.solve(matrix(m, n, beta), b.ravel())
    out = psi.copy()
    out[1:-1, 1:-1] = u.reshape(n - 2, m - 2)
    return out


def dst_solve(psi: np.ndarray, beta: float = 1.0, source: np.ndarray | None = None) -> np.ndarray:
    """Same solution via the eigen-decomposition of T: T = S diag(4 sin^2(k pi / 2(N+1))) S."""
    n, m = psi.shape
    mi, ni = m - 2, n - 2
    b = ring_rhs(psi, beta)
    if source is not None:
        b = b + source[1:-1, 1:-1]
    lx = 4.0 * np.sin(np.arange(1, mi + 1) * np.pi / (2 * (mi + 1))) ** 2
    ly = 4.0 * np.sin(np.arange(1, ni + 1) * np.pi / (2 * (ni + 1))) ** 2
    bh = scipy.fft.dstn(b, type=1, norm="ortho")
    uh = bh / (lx[None, :] + beta ** 2 * ly[:, None])
    out = psi.copy()
    out[1:-1, 1:-1] = scipy.fft.idstn(uh, type=1, norm="ortho")
    return out


def sine_mode(m: int, n: int, k: int, beta: float = 1.0) -> np.ndarray:
    """Exact 5-point solution for psi(i, 0) = sin(k pi i / (m-1)), zero on the other edges:
    psi_ij = sin(k pi i/(m-1)) sinh(theta (n-1-j)) / sinh(theta (n-1)),
    cosh(theta) = 1 + (1 - cos(k pi/(m-1))) / beta^2."""
    i = np.arange(m)[None, :]
    j = np.arange(n)[:, None]
    theta = np.arccosh(1.0 + (1.0 - np.cos(k * np.pi / (m - 1))) / beta ** 2)
    # sinh ratio written with exponentials that cannot overflow
    ratio = (np.exp(-theta * j) - np.exp(-theta * (2 * (n - 1) - j))) / (1.0 - np.exp(-2 * theta * (n - 1)))
    out = np.sin(k * np.pi * i / (m - 1)) * ratio
    out[:, 0] = 0.0
    out[:, -1] = 0.0
    out[-1, :] = 0.0
    return out


def iteration_matrix(step, m: int, n: int) -> np.ndarray:
    """Matrix of a linear homogeneous iteration on the interior, by brute force: column k is
    the interior of step(e_k) for the unit field e_k with a zero ring."""
    N = (m - 2) * (n - 2)
    T = np.empty((N, N))
    for k in range(N):
        e = np.zeros((n, m))
        e[1 + k // (m - 2), 1 + k % (m - 2)] = 1.0
        T[:, k] = step(e)[1:-1, 1:-1].ravel()
    return T


def spectral_radius(T: np.ndarray) -> float:
    return float(np.max(np.abs(np.linalg.eigvals(T))))
