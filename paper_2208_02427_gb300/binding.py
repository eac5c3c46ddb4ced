"""Python binding of liblaplace.so (include/laplace.h), argument marshalling only.

Every step of a solve runs in the library's CUDA kernels; this module turns torch
tensors into (pointer, m, n, pitch) triples and calls the C ABI through ctypes. There
is no CPU path: if the library cannot be loaded, every call raises.

A field is a 2-D torch.float64 CUDA tensor of shape (n, m) whose rows may be padded:
``psi[j, i]`` is psi_{i,j}; its row stride is the pitch. ``field(m, n)`` allocates one
with a 32-element-aligned pitch.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

c_int32, c_int64, c_double, c_void_p = C.c_int32, C.c_int64, C.c_double, C.c_void_p

METHODS = {"jacobi": 0, "gs": 1, "sor": 2, "adi": 3, "mg": 4, "mg_mixed": 5, "slor": 6, "mg_fp32": 9,
           "gs_lex": 7, "sor_lex": 8}
NORMS = {"l2_rel": 0, "l2_abs": 1, "maxdelta": 2}
FORMS = {"A": 0, "B": 1}
SUM_ORDERS = {"paper": 0, "diagonal": 1}
GRID_MAX_M = 1 << 28  # LAP_GRID_MAX_M: the widest grid (points along x)
GRID_MAX_N = 131070  # LAP_GRID_MAX_N: the tallest grid (points along y)
STATUS = {0: "converged", 1: "max_iter", 2: "diverged"}
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EUNSUPPORTED"}


class LapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblaplace {ERRORS.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("m", c_int32), ("n", c_int32), ("dx", c_double), ("dy", c_double),
                ("pitch", c_int64)]


class Params(C.Structure):
    _fields_ = [("method", c_int32), ("w", c_double), ("tol", c_double), ("norm", c_int32),
                ("max_iter", c_int64), ("check_every", c_int32), ("nu1", c_int32),
                ("nu2", c_int32), ("coarsest_min", c_int32), ("max_levels", c_int32),
                ("smoother_w", c_double), ("line_form", c_int32), ("inner_cycles", c_int32),
                ("tail_size", c_int32), ("unfused", c_int32), ("tiling", c_int32),
                ("item_points", c_int32), ("persistent", c_int32), ("sum_order", c_int32)]


class Result(C.Structure):
    _fields_ = [("status", c_int32), ("iters", c_int64), ("r0", c_double), ("r_final", c_double),
                ("last_check", c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load():
    """Load liblaplace.so (building it first if the sources are newer). Raises if the
    CUDA library cannot be built or loaded: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        try:
            path = _build.build()
        except Exception as exc:  # no nvcc, or a compile error
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"liblaplace.so is not built and cannot be built: {exc}") from exc
            path = _build.LIB
        lib = C.CDLL(path)
        P, G, R = C.POINTER(Params), C.POINTER(Grid), C.POINTER(Result)
        sig = {
            "lap_default_params": (None, [P]),
            "lap_create": (C.c_int, [C.POINTER(c_void_p), C.c_size_t, C.c_int]),
            "lap_destroy": (None, [c_void_p]),
            "lap_workspace_bytes": (C.c_int, [G, P, C.POINTER(C.c_size_t)]),
            "lap_solve": (C.c_int, [c_void_p, G, c_void_p, P, R, c_void_p]),
            "lap_solve_host": (C.c_int, [c_void_p, G, c_void_p, C.c_int64, P, R, c_void_p]),
            "lap_residual": (C.c_int, [c_void_p, G, c_void_p, c_void_p, C.POINTER(c_double), c_void_p]),
            "lap_smooth": (C.c_int, [G, c_void_p, c_void_p, c_double, C.c_int, c_void_p]),
            "lap_jacobi_sweep": (C.c_int, [G, c_void_p, c_void_p, c_void_p]),
            "lap_restrict": (C.c_int, [G, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64,
                                       c_void_p]),
            "lap_prolong_add": (C.c_int, [G, c_void_p, c_void_p, c_int64, c_void_p]),
            "lap_coarse_solve": (C.c_int, [c_void_p, G, c_void_p, c_void_p, c_void_p]),
            "lap_line_sweep": (C.c_int, [c_void_p, G, c_void_p, c_double, C.c_int, C.c_int, c_void_p]),
            "lap_set_graphs": (C.c_int, [c_void_p, C.c_int]),
            "lap_solve_batched": (C.c_int, [c_void_p, C.c_int, G, C.POINTER(c_void_p), P, R, c_void_p]),
            "lap_server_create": (C.c_int, [C.POINTER(c_void_p), c_void_p, C.c_size_t, P, C.c_int, C.c_int]),
            "lap_server_destroy": (None, [c_void_p]),
            "lap_server_submit": (C.c_int, [c_void_p, G, c_void_p, C.c_int, c_double, c_double, c_int64,
                                            C.POINTER(c_int64)]),
            "lap_server_step": (C.c_int, [c_void_p, c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "lap_server_poll": (C.c_int, [c_void_p, c_int64, R]),
            "lap_server_drain": (C.c_int, [c_void_p, C.POINTER(c_int64), R, C.c_int, C.POINTER(C.c_int)]),
            "lap_strerror": (C.c_char_p, [C.c_int]),
            "lap_last_error": (C.c_char_p, []),
            "lap_kernel_launches": (c_int64, []),
            "lap_check_rounding": (C.c_int, [c_void_p, c_int64, C.c_uint64, C.POINTER(c_int64)]),
            "lap_fp64_rate": (C.c_int, [c_void_p, C.POINTER(c_double)]),
            "lap_last_batch_config": (C.c_int, [c_void_p, C.POINTER(c_int32), C.POINTER(c_int32),
                                                C.POINTER(c_int32), C.POINTER(c_int32),
                                                C.POINTER(c_int32)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(code: int):
    if code != 0:
        raise LapError(code, load().lap_last_error().decode())


def kernel_launches() -> int:
    return int(load().lap_kernel_launches())


# ---- fields --------------------------------------------------------------------------

def field(m: int, n: int, device=None, align: int = 32) -> torch.Tensor:
    """Zeroed (n, m) float64 CUDA field with the row pitch rounded up to `align`."""
    pitch = (m + align - 1) // align * align
    return torch.zeros((n, pitch), dtype=torch.float64, device=device or "cuda")[:, :m]


def to_field(a, device=None) -> torch.Tensor:
    t = torch.as_tensor(a, dtype=torch.float64)
    f = field(t.shape[1], t.shape[0], device)
    f.copy_(t)
    return f


def _grid(t: torch.Tensor, dx: float, dy: float) -> Grid:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or t.dim() != 2:
        raise TypeError("a field is a 2-D float64 CUDA tensor")
    if t.stride(1) != 1 or t.stride(0) < t.shape[1]:
        raise TypeError("a field needs unit column stride and row stride >= its width")
    return Grid(t.shape[1], t.shape[0], float(dx), float(dy), t.stride(0))


def _same_layout(a: torch.Tensor, b: torch.Tensor, what: str):
    if b.shape != a.shape or b.stride() != a.stride() or b.device != a.device or b.dtype != a.dtype:
        raise TypeError(f"{what} must have the field's shape, pitch, dtype and device")


def _ptr(t):
    return None if t is None else c_void_p(t.data_ptr())


def _stream(stream, device):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return c_void_p(s.cuda_stream)


def params(method="sor", w=1.0, tol=1e-10, norm="l2_rel", max_iter=100000, check_every=1,
           nu1=2, nu2=2, coarsest_min=5, max_levels=0, smoother_w=1.0, line_form="A",
           inner_cycles=1, tail_size=0, unfused=False, tiling=0, item_points=0,
           persistent=0, sum_order="paper") -> Params:
    return Params(METHODS[method], float(w), float(tol), NORMS[norm], int(max_iter),
                  int(check_every), int(nu1), int(nu2), int(coarsest_min), int(max_levels),
                  float(smoother_w), FORMS[line_form], int(inner_cycles), int(tail_size),
                  1 if unfused else 0, int(tiling), int(item_points), int(persistent),
                  SUM_ORDERS[sum_order])


class Batch:
    """The C-ABI descriptors of a list of fields for lap_solve_batched (grid array and pointer
    array), marshalled once so that repeated solves of the same batch pay for it once. The
    fields stay referenced; their sizes and storage must not change while the Batch is used.
    dx, dy: scalars or one value per field."""

    def __init__(self, fields, dx=1.0, dy=1.0):
        self.fields = list(fields)
        n = self.count = len(self.fields)
        if n == 0:
            raise ValueError("empty batch")
        dxs = dx if hasattr(dx, "__len__") else [dx] * n
        dys = dy if hasattr(dy, "__len__") else [dy] * n
        self.grids = (Grid * n)(*[_grid(f, a, c) for f, a, c in zip(self.fields, dxs, dys)])
        self.ptrs = (c_void_p * n)(*[f.data_ptr() for f in self.fields])
        self.device = self.fields[0].device


class Laplace:
    """A handle of the library on one CUDA device (scratch memory, cached tables)."""

    def __init__(self, device=None, hbm_budget: int = 0):
        self._lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        h = c_void_p()
        _check(self._lib.lap_create(C.byref(h), int(hbm_budget), self.device.index))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def check_rounding(self, count: int, seed: int = 1) -> int:
        """Mismatches of the kernels' integer-pipe FP64 -> FP32 rounding and multiply by
        2^-s against the instructions they replace, over `count` seeded doubles (0 expected)."""
        out = c_int64(0)
        _check(self._lib.lap_check_rounding(self._h, int(count), int(seed), C.byref(out)))
        return int(out.value)

    def fp64_rate(self) -> float:
        """FP64 fused multiply-adds per second on this handle's device (a probe kernel)."""
        out = c_double(0)
        _check(self._lib.lap_fp64_rate(self._h, C.byref(out)))
        return out.value

    def set_graphs(self, enabled: bool):
        """Replay each check period as a CUDA graph (default) or launch kernels one by one."""
        _check(self._lib.lap_set_graphs(self._h, 1 if enabled else 0))

    def workspace_bytes(self, psi, dx=1.0, dy=1.0, **kw) -> int:
        """Scratch bytes lap_solve needs for the field psi, or for a grid shape (m, n) (row
        pitch m) before any field is allocated; LapError where the solve would refuse."""
        if isinstance(psi, torch.Tensor):
            g = _grid(psi, dx, dy)
        else:
            m, n = (int(v) for v in psi)
            g = Grid(m, n, float(dx), float(dy), m)
        out = C.c_size_t(0)
        _check(self._lib.lap_workspace_bytes(C.byref(g), C.byref(params(**kw)), C.byref(out)))
        return out.value

    def solve(self, psi: torch.Tensor, dx=1.0, dy=1.0, stream=None, **kw) -> dict:
        """Solve in place on the device field psi; returns status, iterations and norms."""
        res = Result()
        _check(self._lib.lap_solve(self._h, C.byref(_grid(psi, dx, dy)), _ptr(psi),
                                   C.byref(params(**kw)), C.byref(res), _stream(stream, psi.device)))
        return {"status": STATUS.get(res.status, res.status), "iters": res.iters, "r0": res.r0,
                "r_final": res.r_final, "last_check": res.last_check}

    def solve_batched(self, fields, dx=1.0, dy=1.0, stream=None, **kw) -> list:
        """Solve many fields (different sizes allowed) with the V-cycle in batched launches.
        fields: a list of fields (dx, dy: scalars or one value per field) or a Batch (its own
        spacings). Returns one result dict per field."""
        batch = fields if isinstance(fields, Batch) else Batch(fields, dx, dy)
        res = (Result * batch.count)()
        _check(self._lib.lap_solve_batched(self._h, batch.count, batch.grids, batch.ptrs,
                                           C.byref(params(**kw)), res, _stream(stream, batch.device)))
        return [{"status": STATUS.get(r.status, r.status), "iters": r.iters, "r0": r.r0,
                 "r_final": r.r_final, "last_check": r.last_check} for r in res]

    def last_batch_config(self) -> dict:
        """The launch configuration the last batched cycle ran, and whether the choice by timing
        had finished (see lap_last_batch_config)."""
        v = [c_int32(0) for _ in range(5)]
        _check(self._lib.lap_last_batch_config(self._h, *[C.byref(x) for x in v]))
        return {"tail_size": v[0].value, "tiling": v[1].value, "item_points": v[2].value,
                "persistent": v[3].value, "tuned": bool(v[4].value)}

    def solve_host(self, psi_host: torch.Tensor, dx=1.0, dy=1.0, stream=None, align: int = 32,
                   **kw):
        """End-to-end solve of a host array through lap_solve_host: the library copies it to
        a device field of its own (row pitch rounded up to `align`), solves and copies the
        result back into psi_host, in place. Pinned host memory lets the copies overlap."""
        t = psi_host
        if (not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or t.dim() != 2
                or t.stride(1) != 1 or t.stride(0) < t.shape[1]):
            raise TypeError("psi_host is a 2-D float64 host tensor with unit column stride")
        m, n = t.shape[1], t.shape[0]
        g = Grid(m, n, float(dx), float(dy), (m + align - 1) // align * align)
        res = Result()
        _check(self._lib.lap_solve_host(self._h, C.byref(g), _ptr(t), t.stride(0),
                                        C.byref(params(**kw)), C.byref(res),
                                        _stream(stream, self.device)))
        return {"status": STATUS.get(res.status, res.status), "iters": res.iters, "r0": res.r0,
                "r_final": res.r_final, "last_check": res.last_check}

    def residual(self, psi, dx=1.0, dy=1.0, q=None, stream=None) -> float:
        if q is not None:
            _same_layout(psi, q, "q")
        out = c_double(0)
        _check(self._lib.lap_residual(self._h, C.byref(_grid(psi, dx, dy)), _ptr(psi), _ptr(q),
                                      C.byref(out), _stream(stream, psi.device)))
        return out.value

    def coarse_solve(self, u, dx=1.0, dy=1.0, q=None, stream=None):
        if q is not None:
            _same_layout(u, q, "q")
        _check(self._lib.lap_coarse_solve(self._h, C.byref(_grid(u, dx, dy)), _ptr(u), _ptr(q),
                                          _stream(stream, u.device)))

    def line_sweep(self, psi, w, form="A", direction=0, dx=1.0, dy=1.0, stream=None):
        _check(self._lib.lap_line_sweep(self._h, C.byref(_grid(psi, dx, dy)), _ptr(psi), float(w),
                                        FORMS[form], int(direction), _stream(stream, psi.device)))


# ---- handle-free kernels -------------------------------------------------------------

def smooth(psi, q=None, w=1.0, nsweeps=1, dx=1.0, dy=1.0, stream=None):
    if q is not None:
        _same_layout(psi, q, "q")
    _check(load().lap_smooth(C.byref(_grid(psi, dx, dy)), _ptr(psi), _ptr(q), float(w), int(nsweeps),
                             _stream(stream, psi.device)))


def jacobi_sweep(src, dst, dx=1.0, dy=1.0, stream=None):
    _same_layout(src, dst, "dst")
    _check(load().lap_jacobi_sweep(C.byref(_grid(src, dx, dy)), _ptr(src), _ptr(dst),
                                   _stream(stream, src.device)))


def restrict(u, qc, r, q=None, ec=None, dx=1.0, dy=1.0, stream=None):
    _same_layout(u, r, "r")
    if q is not None:
        _same_layout(u, q, "q")
    mc, nc = (u.shape[1] - 1) // 2 + 1, (u.shape[0] - 1) // 2 + 1
    if qc.shape != (nc, mc) or qc.stride(1) != 1 or (ec is not None and ec.stride() != qc.stride()):
        raise TypeError("qc/ec must be coarse fields of shape ((n-1)/2+1, (m-1)/2+1) with one pitch")
    _check(load().lap_restrict(C.byref(_grid(u, dx, dy)), _ptr(u), _ptr(q), _ptr(r), _ptr(qc),
                               _ptr(ec), qc.stride(0), _stream(stream, u.device)))


def prolong_add(u, ec, dx=1.0, dy=1.0, stream=None):
    mc, nc = (u.shape[1] - 1) // 2 + 1, (u.shape[0] - 1) // 2 + 1
    if ec.shape != (nc, mc) or ec.stride(1) != 1:
        raise TypeError("ec must be a coarse field of shape ((n-1)/2+1, (m-1)/2+1)")
    _check(load().lap_prolong_add(C.byref(_grid(u, dx, dy)), _ptr(u), _ptr(ec), ec.stride(0),
                                  _stream(stream, u.device)))


class Server:
    """Continuous-batching solve server on one Laplace handle (see lap_server_* in laplace.h).

    submit() queues a request on a caller-owned device field (kept referenced here until its
    result is polled); step() admits what fits the HBM budget and runs one iteration of every
    running request in shared launches; poll() returns the result dict once finished."""

    def __init__(self, lap: Laplace, hbm_budget: int, max_running: int = 1024, sor_sweeps: int = 50,
                 **mg_kw):
        self._lap = lap
        self._lib = lap._lib
        h = c_void_p()
        _check(self._lib.lap_server_create(C.byref(h), lap._h, int(hbm_budget),
                                           C.byref(params(method="mg", **mg_kw)), int(max_running),
                                           int(sor_sweeps)))
        self._h = h
        self._fields = {}

    def submit(self, psi, dx=1.0, dy=1.0, method="mg_mixed", w=1.0, tol=1e-10,
               max_iter=100000) -> int:
        rid = c_int64(0)
        _check(self._lib.lap_server_submit(self._h, C.byref(_grid(psi, dx, dy)), _ptr(psi),
                                           METHODS[method], float(w), float(tol), int(max_iter),
                                           C.byref(rid)))
        self._fields[rid.value] = psi
        return rid.value

    def step(self, stream=None):
        running, queued = C.c_int(0), C.c_int(0)
        _check(self._lib.lap_server_step(self._h, _stream(stream, self._lap.device),
                                         C.byref(running), C.byref(queued)))
        return running.value, queued.value

    def poll(self, rid: int):
        res = Result()
        rc = self._lib.lap_server_poll(self._h, int(rid), C.byref(res))
        if rc < 0:
            _check(rc)
        if rc == 0:
            return None
        self._fields.pop(rid, None)
        return {"status": STATUS.get(res.status, res.status), "iters": res.iters, "r0": res.r0,
                "r_final": res.r_final, "last_check": res.last_check}

    def drain(self, capacity: int = 4096) -> list:
        """(id, result dict) of the requests finished so far, oldest first (see lap_server_drain)."""
        out = []
        ids = (c_int64 * capacity)()
        res = (Result * capacity)()
        n = C.c_int(0)
        while True:
            _check(self._lib.lap_server_drain(self._h, ids, res, capacity, C.byref(n)))
            for k in range(n.value):
                r = res[k]
                self._fields.pop(ids[k], None)
                out.append((ids[k], {"status": STATUS.get(r.status, r.status), "iters": r.iters,
                                     "r0": r.r0, "r_final": r.r_final, "last_check": r.last_check}))
            if n.value < capacity:
                return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lap_server_destroy(self._h)
            self._h = None
            self._fields.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
