"""Seeded synthetic inputs for the Laplace solvers (boundary rings and initial guesses).

This module holds input generation only -- none of the solvers' arithmetic -- so
that the CUDA path and the CPU oracle can be fed the very same arrays. It imports
numpy only.

A field is a float64 array of shape (n, m): ``psi[j, i]`` is psi_{i,j} of the paper,
i along x (m points), j along y (n points). The outer ring carries the Dirichlet
data, the interior the initial guess (zero, as in the paper).

Recipes (seed = 20220804 + config index unless given):
  chamber       the paper's problem (Problem Definition): 25 x 17, dx = dy = 0.25 m,
                psi = 1 on the non-corner nodes of wall AB (the bottom wall, j = 0),
                0 on every other wall. Each gap CA / BD spans one cell, so the
                linear variation across it touches no interior node; corners are 0
                and never enter the 5-point stencil.
  chamber_sym   the second verification set (Results and Discussion): the top wall
                carries the same values as the bottom wall.
  sine_edges    each edge carries sum_{k=1..8} a_k sin(k pi s), a_k ~ U[-1, 1] drawn
                per edge, s in [0, 1] the normalised arclength (increasing with i or
                j); corners are 0. Used for the 4097^2 and 8193^2 grids.
  random_ring   i.i.d. U[0, 1] on every ring node (batched and serving workloads).
  polynomial    ring = P(x, y) at x = i dx, y = j dy (harmonic test data).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20220804

CHAMBER_M, CHAMBER_N, CHAMBER_H = 25, 17, 0.25
N_MODES = 8


def empty(m: int, n: int) -> np.ndarray:
    return np.zeros((n, m), dtype=np.float64)


def chamber(m: int = CHAMBER_M, n: int = CHAMBER_N, symmetric: bool = False) -> np.ndarray:
    psi = empty(m, n)
    psi[0, 1:m - 1] = 1.0
    if symmetric:
        psi[n - 1, 1:m - 1] = 1.0
    return psi


def sine_coefficients(seed: int, modes: int = N_MODES) -> np.ndarray:
    """a_{e,k} for the four edges (bottom, top, left, right), shape (4, modes)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(4, modes))


def sine_edges(m: int, n: int, seed: int = SEED_BASE + 1, modes: int = N_MODES) -> np.ndarray:
    a = sine_coefficients(seed, modes)
    k = np.arange(1, modes + 1)[:, None]
    sx = np.arange(m)[None, :] / (m - 1)
    sy = np.arange(n)[None, :] / (n - 1)
    ex = np.sin(np.pi * k * sx)   # (modes, m)
    ey = np.sin(np.pi * k * sy)   # (modes, n)
    psi = empty(m, n)
    psi[0, :] = a[0] @ ex
    psi[n - 1, :] = a[1] @ ex
    psi[:, 0] = a[2] @ ey
    psi[:, m - 1] = a[3] @ ey
    for j, i in ((0, 0), (0, m - 1), (n - 1, 0), (n - 1, m - 1)):
        psi[j, i] = 0.0
    return psi


def random_ring(m: int, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    psi = empty(m, n)
    ring = rng.uniform(0.0, 1.0, size=2 * m + 2 * (n - 2))
    psi[0, :] = ring[:m]
    psi[n - 1, :] = ring[m:2 * m]
    psi[1:n - 1, 0] = ring[2 * m:2 * m + n - 2]
    psi[1:n - 1, m - 1] = ring[2 * m + n - 2:]
    return psi


def polynomial(m: int, n: int, dx: float, dy: float, fn, interior: str = "zero") -> np.ndarray:
    """Ring = fn(x, y); interior zero (``interior='zero'``) or fn itself ('exact')."""
    x = np.arange(m)[None, :] * dx
    y = np.arange(n)[:, None] * dy
    full = np.broadcast_to(fn(x, y), (n, m)).astype(np.float64).copy()
    if interior == "zero":
        full[1:n - 1, 1:m - 1] = 0.0
    return full


def random_interior(psi: np.ndarray, seed: int, scale: float = 1.0) -> np.ndarray:
    """Copy of psi with a U[-scale, scale] interior (iterate-level parity tests)."""
    out = psi.copy()
    rng = np.random.default_rng(seed)
    out[1:-1, 1:-1] = rng.uniform(-scale, scale, size=(psi.shape[0] - 2, psi.shape[1] - 2))
    return out


def batch_shapes(count: int, seed: int, kmin: int = 5, kmax: int = 9, max_aspect_log2: int = 2):
    """(m, n) pairs with m, n in {2^k + 1}, k ~ U{kmin..kmax} independently, redrawn
    while the aspect ratio exceeds 2^max_aspect_log2 (the batched workload)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        km, kn = rng.integers(kmin, kmax + 1, size=2)
        if abs(int(km) - int(kn)) <= max_aspect_log2:
            out.append((2 ** int(km) + 1, 2 ** int(kn) + 1))
    return out


def w_opt_sor(m: int, n: int, beta: float = 1.0) -> float:
    """Optimal SOR factor 2 / (1 + sqrt(1 - rho_J^2)) from the Jacobi spectral radius
    rho_J = (cos(pi/(m-1)) + beta^2 cos(pi/(n-1))) / (1 + beta^2). For a square
    grid with m = n this is 2 / (1 + sin(pi/(m-1)))."""
    if m == n and beta == 1.0:
        return float(2.0 / (1.0 + np.sin(np.pi / (m - 1))))
    b2 = beta * beta
    rho = (np.cos(np.pi / (m - 1)) + b2 * np.cos(np.pi / (n - 1))) / (1.0 + b2)
    return float(2.0 / (1.0 + np.sqrt(1.0 - rho * rho)))


def w_opt_slor(m: int, n: int, beta: float = 1.0) -> float:
    """Optimal factor of zebra line SOR by x-lines, 2 / (1 + sqrt(1 - rho^2)), from the
    spectral radius of line Jacobi by x-lines, rho = beta^2 cos(pi/(n-1)) /
    (1 + beta^2 - cos(pi/(m-1))) (its slowest mode sin(pi x) sin(pi y)); zebra ordering
    is consistently ordered, so Young's formula applies."""
    b2 = beta * beta
    rho = b2 * np.cos(np.pi / (n - 1)) / (1.0 + b2 - np.cos(np.pi / (m - 1)))
    return float(2.0 / (1.0 + np.sqrt(1.0 - rho * rho)))
