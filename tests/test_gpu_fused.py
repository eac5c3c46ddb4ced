"""The FP32 cycle's shared-memory tile kernels (one descent and one ascent kernel per level)
against the same cycle run one kernel per pass: every value is computed by the same
expression, so the iterates must be equal bit for bit, for ragged tile edges, beta != 1,
SOR smoothers, any nu1/nu2 the halos allow, several inner cycles, with or without the
small-level tail, single-grid and batched."""
import numpy as np
import pytest
import torch

from paper_2208_02427_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    from paper_2208_02427_gb300 import binding
    binding.load()
    return binding


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().copy()


def solve(b, lap, x, dx, **kw):
    f = b.to_field(x)
    r = lap.solve(f, dx, 1.0, method="mg_mixed", **kw)
    return host(f), r


@pytest.mark.parametrize("shape", [(1025, 1025), (257, 129), (129, 513), (65, 65), (33, 65),
                                   (9, 9), (5, 5), (17, 9), (1025, 33)])
@pytest.mark.parametrize("dx", [1.0, 0.7])
def test_fused_equals_unfused(b, shape, dx):
    m, n = shape
    lap = b.Laplace()
    x = wl.random_ring(m, n, seed=700 + m + 3 * n)
    for tail in (-1, 0):
        kw = dict(tol=0.0, max_iter=3, tail_size=tail)
        ref, r_ref = solve(b, lap, x, dx, unfused=True, **kw)
        got, r = solve(b, lap, x, dx, **kw)
        assert np.array_equal(got, ref), (shape, dx, tail)
        assert r["iters"] == r_ref["iters"] and r["r_final"] == r_ref["r_final"]
    lap.close()


@pytest.mark.parametrize("nu", [(2, 2), (1, 1), (0, 2), (2, 0), (3, 3), (4, 1), (1, 4), (0, 1)])
@pytest.mark.parametrize("smoother_w", [1.0, 1.3])
def test_fused_smoothing_parameters(b, nu, smoother_w):
    lap = b.Laplace()
    x = wl.sine_edges(513, 257, seed=9)
    kw = dict(tol=0.0, max_iter=2, nu1=nu[0], nu2=nu[1], smoother_w=smoother_w, tail_size=-1)
    ref, _ = solve(b, lap, x, 1.0, unfused=True, **kw)
    got, _ = solve(b, lap, x, 1.0, **kw)
    assert np.array_equal(got, ref), (nu, smoother_w)
    lap.close()


@pytest.mark.parametrize("inner", [1, 2, 3])
def test_fused_inner_cycles_to_convergence(b, inner):
    lap = b.Laplace()
    x = wl.sine_edges(1025, 513, seed=10)
    kw = dict(tol=1e-10, max_iter=30, inner_cycles=inner)
    ref, r_ref = solve(b, lap, x, 1.0, unfused=True, **kw)
    got, r = solve(b, lap, x, 1.0, **kw)
    assert r["status"] == r_ref["status"] == "converged"
    assert r["iters"] == r_ref["iters"]
    assert np.array_equal(got, ref)
    lap.close()


def test_fused_batched_equals_unfused(b):
    shapes = [(33, 33), (65, 129), (129, 65), (257, 257), (513, 129), (3, 3), (9, 17), (513, 513)]
    inputs = [wl.random_ring(m, n, seed=900 + k) for k, (m, n) in enumerate(shapes)]
    lap = b.Laplace()
    outs = []
    for unfused in (True, False):
        fields = [b.to_field(x) for x in inputs]
        res = lap.solve_batched(fields, 1.0, 1.0, method="mg_mixed", tol=1e-10, max_iter=40,
                                unfused=unfused)
        assert all(r["status"] == "converged" for r in res)
        outs.append(([host(f) for f in fields], [r["iters"] for r in res]))
    assert outs[0][1] == outs[1][1]
    for k in range(len(shapes)):
        assert np.array_equal(outs[0][0][k], outs[1][0][k]), shapes[k]
    lap.close()
