"""lap_residual_noalloc: the residual norm for callers that cannot allocate device memory
(their memory is fully reserved by another allocator or budget, or they cannot afford the
synchronisation of cudaMalloc/cudaFree, or they hold no lap_handle). It must give the
same norm as lap_residual, call after call, while its scratch is a fixed array inside
the library. This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_lap_residual_on_consecutive_calls():
    from paper_2208_02427_gb300 import binding as b
    from paper_2208_02427_gb300 import workloads as wl

    lib = b.load()
    fn = lib.lap_residual_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(b.Grid), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")

    def noalloc(psi, q, dx, dy):
        g = b.Grid(psi.shape[1], psi.shape[0], dx, dy, psi.stride(0))
        rc = fn(C.byref(g), C.c_void_p(psi.data_ptr()),
                None if q is None else C.c_void_p(q.data_ptr()), C.c_void_p(out.data_ptr()),
                C.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.lap_last_error().decode()
        torch.cuda.synchronize()
        return out.item()

    big = b.to_field(wl.sine_edges(4097, 4097, seed=wl.SEED_BASE + 1))
    small_np = wl.random_interior(wl.random_ring(129, 65, seed=5), seed=6)
    small = b.to_field(small_np)
    q = b.to_field(wl.random_interior(np.zeros((65, 129)), seed=7))
    # the large grid fills all partial sums, the small one only 63: stale entries of the
    # first call must not leak into the second
    cases = [(big, None, 1 / 4096, 1 / 4096), (small, q, 0.7, 1.0)]
    with b.Laplace() as lap:
        for psi, qq, dx, dy in cases:  # two calls in a row
            got = noalloc(psi, qq, dx, dy)
            want = lap.residual(psi, dx, dy, qq)
            # the same kernels, blocks and summation order: the same bits
            assert got == want, (got, want)
        # and the calls make no device allocation of their own
        noalloc(big, None, 1 / 4096, 1 / 4096)
        free_before = torch.cuda.mem_get_info()[0]
        again = noalloc(small, q, 0.7, 1.0)
        assert torch.cuda.mem_get_info()[0] == free_before
        assert again == lap.residual(small, 0.7, 1.0, q)
