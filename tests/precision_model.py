"""A numpy model of the mixed-precision solver (FP64 defect correction around V(2,2) cycles
on the correction equation) whose cycle runs in a chosen storage precision: FP64, FP32, or
FP32 arithmetic with the coarse levels' correction and source stored in BF16.

It serves the storage-precision study only (is BF16 for the coarse levels accurate
enough?), not parity: the arithmetic follows the V-cycle of the Multigrid section (steps
1-11: red-black Gauss-Seidel smoothing, residual, full-weighting restriction scaled to the
coarse equation, exact coarsest solve, bilinear interpolation) in numpy's rounding, not the
kernels' or the oracle's operation order."""
import numpy as np


def to_bf16(a):
    """FP32 values rounded to the nearest BF16 value (ties to even), kept in FP32 storage."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _colour_masks(m, n):
    j, i = np.meshgrid(np.arange(n), np.arange(m), indexing="ij")
    out = []
    for c in (0, 1):
        msk = (i + j) % 2 == c
        msk[0, :] = msk[-1, :] = False
        msk[:, 0] = msk[:, -1] = False
        out.append(msk)
    return out


def _neighbours(u, b2):
    return (u[1:-1, :-2] + u[1:-1, 2:]) + b2 * (u[:-2, 1:-1] + u[2:, 1:-1])


def _smooth(u, q, b2, d, masks, store):
    for msk in masks:  # red, then black (Eq. 6 with the source of the coarse equation)
        new = np.zeros_like(u)
        new[1:-1, 1:-1] = (_neighbours(u, b2) + q[1:-1, 1:-1]) / d
        u[msk] = new[msk]
        if store is not None:
            u[:] = store(u)


def residual(u, q, b2, d):
    """r = (E + W) + beta^2 (N + S) - d u + q on the interior (Eqs. 11-12, scaled)."""
    r = np.zeros_like(u)
    r[1:-1, 1:-1] = _neighbours(u, b2) - d * u[1:-1, 1:-1] + q[1:-1, 1:-1]
    return r


def _restrict(r):
    # full weighting, times 4 for the coarse equation's doubled spacing
    n, m = r.shape
    qc = np.zeros(((n - 1) // 2 + 1, (m - 1) // 2 + 1), r.dtype)
    c = r[2:-2:2, 2:-2:2]
    e = (r[2:-2:2, 1:-3:2] + r[2:-2:2, 3:-1:2]) + (r[1:-3:2, 2:-2:2] + r[3:-1:2, 2:-2:2])
    k = (r[1:-3:2, 1:-3:2] + r[1:-3:2, 3:-1:2]) + (r[3:-1:2, 1:-3:2] + r[3:-1:2, 3:-1:2])
    qc[1:-1, 1:-1] = (4 * c + 2 * e + k) / 4
    return qc


def _prolong_add(ec, u):
    f = np.zeros_like(u)
    f[::2, ::2] = ec
    f[::2, 1::2] = 0.5 * (ec[:, :-1] + ec[:, 1:])
    f[1::2, ::2] = 0.5 * (ec[:-1, :] + ec[1:, :])
    f[1::2, 1::2] = 0.25 * ((ec[:-1, :-1] + ec[:-1, 1:]) + (ec[1:, :-1] + ec[1:, 1:]))
    u[1:-1, 1:-1] += f[1:-1, 1:-1]


def _coarsest(q, b2, d):
    n, m = q.shape
    mi, ni = m - 2, n - 2
    A = np.zeros((mi * ni, mi * ni))
    for j in range(ni):
        for i in range(mi):
            k = j * mi + i
            A[k, k] = -d
            if i > 0:
                A[k, k - 1] = 1.0
            if i < mi - 1:
                A[k, k + 1] = 1.0
            if j > 0:
                A[k, k - mi] = b2
            if j < ni - 1:
                A[k, k + mi] = b2
    u = np.zeros((n, m))
    u[1:-1, 1:-1] = np.linalg.solve(A, -q[1:-1, 1:-1].astype(np.float64).reshape(-1)).reshape(ni, mi)
    return u


def _vcycle(u, q, lev, shapes, masks, b2, d, dtype, coarse_store, nu):
    store = coarse_store if lev > 0 else None
    if lev == len(shapes) - 1:
        u[:] = _coarsest(q, float(b2), float(d)).astype(dtype)
        if store is not None:
            u[:] = store(u)
        return
    for _ in range(nu):
        _smooth(u, q, b2, d, masks[lev], store)
    qc = _restrict(residual(u, q, b2, d)).astype(dtype)
    if coarse_store is not None:
        qc = coarse_store(qc)
    uc = np.zeros((shapes[lev + 1][1], shapes[lev + 1][0]), dtype)
    _vcycle(uc, qc, lev + 1, shapes, masks, b2, d, dtype, coarse_store, nu)
    _prolong_add(uc, u)
    if store is not None:
        u[:] = store(u)
    for _ in range(nu):
        _smooth(u, q, b2, d, masks[lev], store)


def mixed_solve(psi, dtype=np.float32, coarse_store=None, tol=1e-10, max_iter=40, nu=2):
    """Defect correction with beta = 1: r = FP64 residual of psi; e = one V(nu, nu) cycle on
    the correction equation in `dtype` from e = 0 (coarse levels passed through coarse_store
    after every write); psi += e in FP64; until ||r||_2 <= tol ||r_0||_2. Returns psi and the
    relative residual after each iteration."""
    n, m = psi.shape
    shapes = [(m, n)]
    while ((shapes[-1][0] - 1) % 2 == 0 and (shapes[-1][1] - 1) % 2 == 0
           and (shapes[-1][0] - 1) // 2 + 1 >= 5 and (shapes[-1][1] - 1) // 2 + 1 >= 5):
        shapes.append(((shapes[-1][0] - 1) // 2 + 1, (shapes[-1][1] - 1) // 2 + 1))
    masks = [_colour_masks(a, b) for (a, b) in shapes]
    b2, d = dtype(1.0), dtype(4.0)
    psi = np.array(psi, dtype=np.float64)
    zero = np.zeros_like(psi)
    r = residual(psi, zero, 1.0, 4.0)
    r0 = np.linalg.norm(r)
    hist = []
    for _ in range(max_iter):
        e = np.zeros(psi.shape, dtype)
        _vcycle(e, r.astype(dtype), 0, shapes, masks, b2, d, dtype, coarse_store, nu)
        psi += e.astype(np.float64)
        r = residual(psi, zero, 1.0, 4.0)
        hist.append(float(np.linalg.norm(r) / r0))
        if hist[-1] <= tol:
            break
    return psi, hist
