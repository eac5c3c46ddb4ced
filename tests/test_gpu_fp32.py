"""The V-cycle entirely in FP32 (LAP_MG_FP32), the plain-FP32 comparison point of the
mixed-precision solver: it reaches a 1e-5 relative residual, its solution is within FP32
accuracy of the exact discrete solution, it cannot reach 1e-10, and its tile kernels and
small-level tail give the same iterates as the one-kernel-per-pass cycle."""
import numpy as np
import pytest
import torch

from paper_2208_02427_gb300 import workloads as wl
from tests import exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    from paper_2208_02427_gb300 import binding
    binding.load()
    return binding


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().copy()


@pytest.mark.parametrize("shape", [(1025, 1025), (257, 513), (65, 33)])
def test_fp32_reaches_its_tolerance_and_fp32_accuracy(b, shape):
    m, n = shape
    lap = b.Laplace()
    x = wl.sine_edges(m, n, seed=31)
    want = exact.dst_solve(x)
    f = b.to_field(x)
    r = lap.solve(f, 1.0, 1.0, method="mg_fp32", tol=1e-5, max_iter=40)
    assert r["status"] == "converged" and 2 <= r["iters"] <= 12
    got = host(f)
    assert np.array_equal(got[0], x[0]) and np.array_equal(got[:, 0], x[:, 0])  # ring untouched
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert 1e-9 < err < 1e-4, err  # FP32 accuracy: not FP64's
    lap.close()


def test_fp32_stalls_before_1e10(b):
    lap = b.Laplace()
    x = wl.sine_edges(1025, 1025, seed=32)
    f = b.to_field(x)
    r = lap.solve(f, 1.0, 1.0, method="mg_fp32", tol=1e-10, max_iter=25)
    assert r["status"] == "max_iter"
    assert r["r_final"] / r["r0"] > 1e-9  # the FP64 residual of the FP32 solution
    lap.close()


@pytest.mark.parametrize("shape", [(513, 513), (129, 257), (9, 9), (3, 3), (24, 17)])
def test_fp32_fused_and_tail_equal_per_pass_kernels(b, shape):
    m, n = shape
    lap = b.Laplace()
    x = wl.random_ring(m, n, seed=33 + m)
    outs = []
    for kw in (dict(unfused=True, tail_size=-1), dict(tail_size=-1), dict(tail_size=65),
               dict(tail_size=100000), dict(tail_size=0)):
        f = b.to_field(x)
        r = lap.solve(f, 1.0, 1.0, method="mg_fp32", tol=0.0, max_iter=3, **kw)
        outs.append((host(f), r["r_final"]))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and o[1] == outs[0][1]
    lap.close()


def test_fp32_rejects_maxdelta(b):
    lap = b.Laplace()
    f = b.to_field(wl.random_ring(33, 33, seed=1))
    with pytest.raises(b.LapError):
        lap.solve(f, method="mg_fp32", norm="maxdelta")
    lap.close()
