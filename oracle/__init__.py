"""Python access to the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code with
the CUDA path of ``paper_2208_02427_gb300`` and is never used as a fallback.

Fields are numpy float64 arrays of shape (n, m): row j (y index) holds the m
values along x, so ``psi[j, i]`` is the paper's psi_{i,j}.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_SRC_MT = os.path.join(_HERE, "timing_mt.c")
_LIB_MT = os.path.join(_HERE, "liboracle_mt.so")

LEX, RB = 0, 1
LINES_SUCCESSIVE, LINES_ZEBRA = 0, 1
FORM_A, FORM_B = 0, 1
JACOBI, GS, SOR, SLOR, ADI, MG = range(6)
NORM_L2_REL, NORM_L2_ABS, NORM_MAXDELTA = 0, 1, 2
COARSE_DIRECT, COARSE_GS = 0, 1
SUM_PAPER, SUM_DIAGONAL = 0, 1
STATUS = {0: "converged", 1: "max_iter", 2: "diverged"}


def build(force: bool = False) -> str:
    """Compile liboracle.so with contraction off (explicit fma() only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        )
    if force or not os.path.exists(_LIB_MT) or os.path.getmtime(_LIB_MT) < os.path.getmtime(_SRC_MT):
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-pthread", "-o", _LIB_MT, _SRC_MT, "-lm"]
        )
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("method", C.c_int), ("ordering", C.c_int), ("line_order", C.c_int), ("form", C.c_int),
        ("w", C.c_double), ("norm", C.c_int), ("tol", C.c_double), ("max_iter", C.c_long),
        ("check_every", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
        ("coarsest_min", C.c_int), ("max_levels", C.c_int), ("coarse", C.c_int),
        ("sum_order", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        i, d = C.c_int, C.c_double
        sig = {
            "ora_defect": (None, [i, i, d, dp, dp, dp]),
            "ora_defect_norm_l2": (d, [i, i, d, dp, dp]),
            "ora_jacobi_sweep": (None, [i, i, d, dp, dp]),
            "ora_gs_sweep": (None, [i, i, d, i, dp, dp]),
            "ora_sor_sweep": (None, [i, i, d, d, i, dp, dp]),
            "ora_gs_sweep_ordered": (i, [i, i, d, i, i, dp, dp]),
            "ora_sor_sweep_ordered": (i, [i, i, d, d, i, i, dp, dp]),
            "ora_thomas": (None, [i, dp, dp, dp, dp, dp, dp, dp]),
            "ora_line_sweep": (None, [i, i, d, d, i, i, i, dp]),
            "ora_adi_iteration": (None, [i, i, d, d, i, i, dp]),
            "ora_restrict_fw": (None, [i, i, dp, dp]),
            "ora_prolong_add": (None, [i, i, dp, i, i, dp]),
            "ora_coarse_direct": (i, [i, i, d, dp, dp]),
            "ora_mg_levels": (i, [i, i, i, i]),
            "ora_solve": (i, [i, i, d, d, dp, C.POINTER(_Params), C.POINTER(C.c_long), dp, dp,
                              dp, C.c_long]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


_lib_mt = None


def lib_mt():
    """The threaded red-black SOR timing wrapper (timing_mt.c), for the all-cores baseline."""
    global _lib_mt
    if _lib_mt is None:
        build()
        _lib_mt = C.CDLL(_LIB_MT)
        _lib_mt.ora_mt_sor_rb_sweeps.restype = C.c_int
        _lib_mt.ora_mt_sor_rb_sweeps.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                                 C.POINTER(C.c_double), C.c_int]
    return _lib_mt


def mt_sor_rb_sweeps(psi, w, nsweeps, beta=1.0, threads=1):
    """nsweeps red-black SOR sweeps on `threads` host threads (returns a copy)."""
    psi = _field(psi).copy()
    n, m = psi.shape
    if lib_mt().ora_mt_sor_rb_sweeps(m, n, beta, w, nsweeps, _ptr(psi), threads) != 0:
        raise RuntimeError("could not start the timing threads")
    return psi


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _field(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.ndim == 2 and a.shape[0] >= 3 and a.shape[1] >= 3
    return a


# ---- building blocks --------------------------------------------------------

def defect(psi, beta=1.0, q=None):
    psi = _field(psi)
    n, m = psi.shape
    r = np.zeros_like(psi)
    lib().ora_defect(m, n, beta, _ptr(psi), _ptr(None if q is None else _field(q)), _ptr(r))
    return r


def defect_norm(psi, beta=1.0, q=None):
    psi = _field(psi)
    n, m = psi.shape
    return lib().ora_defect_norm_l2(m, n, beta, _ptr(psi), _ptr(None if q is None else _field(q)))


def jacobi_sweep(psi, beta=1.0):
    psi = _field(psi)
    n, m = psi.shape
    out = np.empty_like(psi)
    lib().ora_jacobi_sweep(m, n, beta, _ptr(psi), _ptr(out))
    return out


def gs_sweep(psi, beta=1.0, ordering=RB, q=None, sum_order=SUM_PAPER):
    psi = _field(psi).copy()
    n, m = psi.shape
    rc = lib().ora_gs_sweep_ordered(m, n, beta, ordering, sum_order, _ptr(psi),
                                    _ptr(None if q is None else _field(q)))
    if rc:
        raise ValueError("the diagonal summation order needs beta = 1")
    return psi


def sor_sweep(psi, w, beta=1.0, ordering=RB, q=None, sum_order=SUM_PAPER):
    psi = _field(psi).copy()
    n, m = psi.shape
    rc = lib().ora_sor_sweep_ordered(m, n, beta, w, ordering, sum_order, _ptr(psi),
                                     _ptr(None if q is None else _field(q)))
    if rc:
        raise ValueError("the diagonal summation order needs beta = 1")
    return psi


def thomas(a, b, c, d):
    N = len(d)
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, d)]
    x, cp, dp = np.empty(N), np.empty(N), np.empty(N)
    lib().ora_thomas(N, *[_ptr(v) for v in arrs], _ptr(x), _ptr(cp), _ptr(dp))
    return x


def line_sweep(psi, w, direction, beta=1.0, form=FORM_A, line_order=LINES_ZEBRA):
    psi = _field(psi).copy()
    n, m = psi.shape
    lib().ora_line_sweep(m, n, beta, w, form, direction, line_order, _ptr(psi))
    return psi


def adi_iteration(psi, w, beta=1.0, form=FORM_A, line_order=LINES_ZEBRA):
    psi = _field(psi).copy()
    n, m = psi.shape
    lib().ora_adi_iteration(m, n, beta, w, form, line_order, _ptr(psi))
    return psi


def restrict_fw(r):
    r = _field(r)
    nf, mf = r.shape
    qc = np.zeros(((nf - 1) // 2 + 1, (mf - 1) // 2 + 1))
    lib().ora_restrict_fw(mf, nf, _ptr(r), _ptr(qc))
    return qc


def prolong_add(ec, uf):
    ec, uf = _field(ec), _field(uf).copy()
    nc, mc = ec.shape
    nf, mf = uf.shape
    lib().ora_prolong_add(mc, nc, _ptr(ec), mf, nf, _ptr(uf))
    return uf


def coarse_direct(u, beta=1.0, q=None):
    u = _field(u).copy()
    n, m = u.shape
    rc = lib().ora_coarse_direct(m, n, beta, _ptr(u), _ptr(None if q is None else _field(q)))
    if rc:
        raise ValueError("coarse system too large for the dense oracle solve")
    return u


def mg_levels(m, n, coarsest_min=5, max_levels=0):
    return lib().ora_mg_levels(m, n, coarsest_min, max_levels)


# ---- driver -----------------------------------------------------------------

def solve(psi, method, dx=1.0, dy=1.0, w=1.0, tol=1e-10, norm=NORM_L2_REL, max_iter=100000,
          check_every=1, ordering=RB, line_order=LINES_ZEBRA, form=FORM_A, nu1=2, nu2=2,
          coarsest_min=5, max_levels=0, coarse=COARSE_DIRECT, history=False, sum_order=SUM_PAPER):
    """Run ``ora_solve``; returns (psi, info) with info = dict(status, iters, r0, r_final[, hist])."""
    psi = _field(psi).copy()
    n, m = psi.shape
    p = _Params(method, ordering, line_order, form, w, norm, tol, max_iter, check_every, nu1,
                nu2, coarsest_min, max_levels, coarse, sum_order)
    iters, r0, rf = C.c_long(0), C.c_double(0), C.c_double(0)
    hist = np.zeros(max(1, max_iter // check_every + 1)) if history else None
    rc = lib().ora_solve(m, n, dx, dy, _ptr(psi), C.byref(p), C.byref(iters), C.byref(r0),
                         C.byref(rf), _ptr(hist), 0 if hist is None else len(hist))
    if rc < 0:
        raise ValueError(f"ora_solve rejected its arguments (rc={rc})")
    info = {"status": STATUS.get(rc, rc), "iters": iters.value, "r0": r0.value,
            "r_final": rf.value}
    if history:
        info["hist"] = hist[: (iters.value + check_every - 1) // check_every] if iters.value else hist[:0]
    return psi, info
