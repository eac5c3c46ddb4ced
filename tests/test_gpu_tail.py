"""The small-level tail of the V-cycle: the levels at or below a size run as one single-CTA
kernel per cycle. It changes the launch structure and not the arithmetic, so every tail
size (none, some levels, the whole cycle) and the timing-based choice must give the same
iterates bit for bit, single-grid and batched, FP64 and mixed precision."""
import numpy as np
import pytest
import torch

from paper_2208_02427_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TAILS = [-1, 3, 5, 9, 17, 33, 65, 129, 100000]


@pytest.fixture(scope="module")
def b():
    from paper_2208_02427_gb300 import binding
    binding.load()
    return binding


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().copy()


def run(b, lap, x, dx, **kw):
    f = b.to_field(x)
    r = lap.solve(f, dx, 1.0, **kw)
    return host(f), r


@pytest.mark.parametrize("method", ["mg", "mg_mixed"])
@pytest.mark.parametrize("shape", [(1025, 1025), (257, 129), (65, 65), (33, 129), (9, 9),
                                   (3, 3), (24, 17), (17, 5)])
def test_single_grid_tail_sizes_are_bitwise_equal(b, method, shape):
    m, n = shape
    lap = b.Laplace()
    x = wl.random_ring(m, n, seed=300 + m + n)
    dx = 1.0 if m % 2 else 0.7
    k0 = b.kernel_launches()
    ref, r_ref = run(b, lap, x, dx, method=method, tol=0.0, max_iter=3, tail_size=-1)
    launches = {-1: b.kernel_launches() - k0}
    for t in TAILS[1:]:
        k0 = b.kernel_launches()
        got, r = run(b, lap, x, dx, method=method, tol=0.0, max_iter=3, tail_size=t)
        launches[t] = b.kernel_launches() - k0
        assert r["iters"] == r_ref["iters"] == 3
        assert np.array_equal(got, ref), (shape, t)
        assert r["r_final"] == r_ref["r_final"]
    # the whole cycle in the tail: one kernel per V-cycle replaces the per-level launches
    if m >= 65 and n >= 65:
        assert launches[100000] < launches[-1] // 2, launches
    lap.close()


@pytest.mark.parametrize("method", ["mg", "mg_mixed"])
def test_tail_with_other_smoothing_parameters(b, method):
    lap = b.Laplace()
    x = wl.random_ring(129, 257, seed=41)
    kw = dict(method=method, tol=0.0, max_iter=2, nu1=3, nu2=1, smoother_w=1.15)
    ref, _ = run(b, lap, x, 1.0, tail_size=-1, **kw)
    for t in (9, 33, 129, 257):
        got, _ = run(b, lap, x, 1.0, tail_size=t, **kw)
        assert np.array_equal(got, ref), t
    kw.update(nu1=0, nu2=2, smoother_w=1.0)
    ref, _ = run(b, lap, x, 1.0, tail_size=-1, **kw)
    got, _ = run(b, lap, x, 1.0, tail_size=65, **kw)
    assert np.array_equal(got, ref)
    lap.close()


@pytest.mark.parametrize("method", ["mg", "mg_mixed"])
def test_tuned_tail_gives_the_untuned_iterates(b, method):
    """tail_size 0: successive periods try the candidates while timing them; every solve of
    the shape, during and after tuning, has the iterates of the solve without a tail."""
    lap = b.Laplace()
    x = wl.sine_edges(513, 513, seed=12)
    ref, r_ref = run(b, lap, x, 1.0, method=method, tol=1e-10, max_iter=50, tail_size=-1)
    for _ in range(4):
        got, r = run(b, lap, x, 1.0, method=method, tol=1e-10, max_iter=50, tail_size=0)
        assert r["status"] == "converged" and r["iters"] == r_ref["iters"]
        assert np.array_equal(got, ref)
    lap.close()


@pytest.mark.parametrize("method", ["mg", "mg_mixed"])
def test_batched_tail_sizes_are_bitwise_equal(b, method):
    shapes = [(33, 33), (65, 129), (129, 65), (257, 257), (513, 129), (3, 3), (9, 17), (24, 17)]
    inputs = [wl.random_ring(m, n, seed=500 + k) for k, (m, n) in enumerate(shapes)]
    lap = b.Laplace()
    ref = None
    for t in (-1, 17, 65, 129, 513, 0, 0):
        fields = [b.to_field(x) for x in inputs]
        res = lap.solve_batched(fields, 1.0, 1.0, method=method, tol=1e-10, max_iter=40,
                                tail_size=t)
        assert all(r["status"] == "converged" for r in res)
        out = [host(f) for f in fields]
        its = [r["iters"] for r in res]
        if ref is None:
            ref = (out, its)
            continue
        assert its == ref[1], t
        for k in range(len(shapes)):
            assert np.array_equal(out[k], ref[0][k]), (t, shapes[k])
    lap.close()


def test_tail_size_is_validated(b):
    lap = b.Laplace()
    f = b.to_field(wl.random_ring(33, 33, seed=1))
    for bad in (-2, 1, 2):
        with pytest.raises(b.LapError):
            lap.solve(f, method="mg", tail_size=bad)
    lap.close()


@pytest.mark.parametrize("method", ["mg", "mg_mixed"])
def test_batched_tuning_gives_the_same_results(b, method):
    """The batched tuner times the tail sizes on the cycles in which every problem is still
    running, across successive solves of the same batch: every solve, while tuning and
    after, has the same iterates and iteration counts."""
    shapes = [(65, 65), (129, 257), (257, 129), (513, 513), (33, 129), (17, 17)]
    inputs = [wl.random_ring(m, n, seed=800 + k) for k, (m, n) in enumerate(shapes)]
    lap = b.Laplace()
    ref = None
    for _ in range(5):
        fields = [b.to_field(x) for x in inputs]
        res = lap.solve_batched(fields, 1.0, 1.0, method=method, tol=1e-10, max_iter=40)
        assert all(r["status"] == "converged" for r in res)
        out = ([host(f) for f in fields], [r["iters"] for r in res])
        if ref is None:
            ref = out
            continue
        assert out[1] == ref[1]
        for k in range(len(shapes)):
            assert np.array_equal(out[0][k], ref[0][k]), shapes[k]
    lap.close()
