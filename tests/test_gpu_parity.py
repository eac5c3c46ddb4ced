"""GPU (through the C ABI) against the FP64 oracle, element by element, on the same
seeded inputs.

Bar: bitwise equality where the library evaluates the oracle's expression with the
same roundings (Jacobi, red-black Gauss-Seidel / SOR, smoother with source, residual
field, restriction, interpolation, and whole point-method solves); max |gpu - oracle| /
max |oracle| <= 1e-12 (REL) where it reassociates (line solves, coarsest-grid inverse,
multigrid cycles that contain it, norms)."""
import numpy as np
import pytest
import torch

import oracle as ora
from paper_2208_02427_gb300 import workloads as wl
from tests import exact

pytestmark = pytest.mark.gpu
REL = 1e-12


@pytest.fixture(scope="module")
def b():
    from paper_2208_02427_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def lap(b):
    h = b.Laplace()
    yield h
    h.close()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().copy()


def relerr(got, want):
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


def rand_field(m, n, seed, scale=1.0):
    return wl.random_interior(wl.random_ring(m, n, seed), seed + 7, scale)


def ora_kw(method, w=1.0, line_form="A", nu1=2, nu2=2, coarsest_min=5, max_levels=0,
           smoother_w=1.0, **_):
    if method == "jacobi":
        return dict(method=ora.JACOBI)
    if method == "gs":
        return dict(method=ora.GS, ordering=ora.RB)
    if method == "sor":
        return dict(method=ora.SOR, ordering=ora.RB, w=w)
    if method == "gs_lex":
        return dict(method=ora.GS, ordering=ora.LEX)
    if method == "sor_lex":
        return dict(method=ora.SOR, ordering=ora.LEX, w=w)
    if method in ("adi", "slor"):
        return dict(method=ora.ADI if method == "adi" else ora.SLOR, w=w,
                    form=ora.FORM_A if line_form == "A" else ora.FORM_B, line_order=ora.LINES_ZEBRA)
    return dict(method=ora.MG, ordering=ora.RB, w=smoother_w, nu1=nu1, nu2=nu2,
                coarsest_min=coarsest_min, max_levels=max_levels, coarse=ora.COARSE_DIRECT)


NORMS = {"l2_rel": ora.NORM_L2_REL, "l2_abs": ora.NORM_L2_ABS, "maxdelta": ora.NORM_MAXDELTA}


def both(lap, b, psi, dx=1.0, dy=1.0, **kw):
    """Run the same solve on the GPU and in the oracle."""
    t = b.to_field(psi)
    g = lap.solve(t, dx, dy, **kw)
    o_sol, o = ora.solve(psi, dx=dx, dy=dy, tol=kw.get("tol", 1e-10),
                         norm=NORMS[kw.get("norm", "l2_rel")], max_iter=kw.get("max_iter", 100000),
                         check_every=kw.get("check_every", 1), **ora_kw(**kw))
    return host(t), g, o_sol, o


SHAPES = [(3, 3), (5, 4), (25, 17), (67, 45), (130, 97), (257, 33)]


# ---- single kernels -----------------------------------------------------------------

@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("beta", [1.0, 0.7])
def test_jacobi_sweep_is_bitwise(b, shape, beta):
    m, n = shape
    psi = rand_field(m, n, 1)
    src, dst = b.to_field(psi), b.field(m, n)
    b.jacobi_sweep(src, dst, dx=beta, dy=1.0)
    assert np.array_equal(host(dst), ora.jacobi_sweep(psi, beta))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("beta", [1.0, 1.3])
@pytest.mark.parametrize("w", [1.0, 1.7])
@pytest.mark.parametrize("with_q", [False, True])
def test_red_black_sweeps_are_bitwise(b, shape, beta, w, with_q):
    m, n = shape
    psi = rand_field(m, n, 2)
    q = wl.random_interior(np.zeros((n, m)), 3, 0.5) if with_q else None
    t = b.to_field(psi)
    b.smooth(t, None if q is None else b.to_field(q), w=w, nsweeps=3, dx=beta, dy=1.0)
    want = psi
    for _ in range(3):
        want = (ora.gs_sweep(want, beta, ora.RB, q) if w == 1.0 else
                ora.sor_sweep(want, w, beta, ora.RB, q))
    assert np.array_equal(host(t), want)


@pytest.mark.parametrize("shape", SHAPES)
def test_residual_norm(lap, b, shape):
    m, n = shape
    psi = rand_field(m, n, 4)
    q = wl.random_interior(np.zeros((n, m)), 5)
    for beta, qq in ((1.0, None), (0.6, q)):
        got = lap.residual(b.to_field(psi), beta, 1.0, None if qq is None else b.to_field(qq))
        want = ora.defect_norm(psi, beta, qq)
        assert abs(got - want) <= 1e-13 * want


@pytest.mark.parametrize("shape", [(5, 5), (9, 9), (33, 17), (65, 129), (257, 33)])
@pytest.mark.parametrize("beta", [1.0, 1.4])
def test_restriction_is_bitwise(b, shape, beta):
    m, n = shape
    u = rand_field(m, n, 6)
    q = wl.random_interior(np.zeros((n, m)), 8)
    mc, nc = (m - 1) // 2 + 1, (n - 1) // 2 + 1
    tu, tq, tr = b.to_field(u), b.to_field(q), b.field(m, n)
    qc, ec = b.field(mc, nc), b.to_field(np.full((nc, mc), 3.0))
    b.restrict(tu, qc, tr, q=tq, ec=ec, dx=beta, dy=1.0)
    want = ora.restrict_fw(ora.defect(u, beta, q))
    got = host(qc)
    assert np.array_equal(got[1:-1, 1:-1], want[1:-1, 1:-1])
    e = host(ec)
    assert np.all(e[1:-1, 1:-1] == 0.0) and np.all(e[0] == 3.0)


@pytest.mark.parametrize("shape", [(5, 5), (9, 9), (33, 17), (65, 129), (257, 33)])
def test_interpolation_is_bitwise(b, shape):
    m, n = shape
    mc, nc = (m - 1) // 2 + 1, (n - 1) // 2 + 1
    u = rand_field(m, n, 9)
    ec = rand_field(mc, nc, 10)
    tu = b.to_field(u)
    b.prolong_add(tu, b.to_field(ec))
    assert np.array_equal(host(tu), ora.prolong_add(ec, u))


@pytest.mark.parametrize("shape", [(3, 3), (5, 5), (7, 5), (5, 17), (9, 9), (17, 9), (33, 33)])
@pytest.mark.parametrize("beta", [1.0, 0.8])
def test_coarsest_solve(lap, b, shape, beta):
    m, n = shape
    u = wl.random_ring(m, n, 11)
    q = wl.random_interior(np.zeros((n, m)), 12)
    t = b.to_field(u)
    lap.coarse_solve(t, beta, 1.0, b.to_field(q))
    assert relerr(host(t), ora.coarse_direct(u, beta, q)) <= 1e-13


# x-lines of 3072 unknowns or more are cut into up to 64 chunks (two warps), shorter ones into
# up to 32: (3073, 5) and (3075, 5) sit on either side, (4097, 5) is the full 64-chunk cut
LINE_SHAPES = [(3, 3), (25, 17), (300, 41), (41, 300), (1003, 7), (7, 1003), (4097, 5), (5, 4097),
               (1025, 385), (36, 20), (20, 36), (3073, 5), (3075, 5), (5, 3075)]


@pytest.mark.parametrize("shape", LINE_SHAPES)
@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("form", ["A", "B"])
@pytest.mark.parametrize("w", [1.0, 1.3])
def test_line_sweep(lap, b, shape, direction, form, w):
    m, n = shape
    psi = rand_field(m, n, 13)
    beta = 1.0 if shape[0] % 2 else 1.2
    t = b.to_field(psi)
    lap.line_sweep(t, w, form, direction, beta, 1.0)
    want = ora.line_sweep(psi, w, direction, beta, ora.FORM_A if form == "A" else ora.FORM_B,
                          ora.LINES_ZEBRA)
    assert relerr(host(t), want) <= 1e-13


@pytest.mark.parametrize("shape", [(130, 97), (97, 130), (33, 2049), (3200, 9)])
@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("form,w", [("A", 1.95), ("B", 1.95), ("B", 1.6)])
@pytest.mark.parametrize("beta", [0.3, 3.0])
def test_line_sweep_extreme_coefficients(lap, b, shape, direction, form, w, beta):
    """Relaxation near 2 (form B: the line matrix close to singular, so its chunk influence
    vectors barely decay) and strongly anisotropic grids (beta^2 = 0.09 and 9 along and across
    the lines)."""
    m, n = shape
    psi = rand_field(m, n, 31)
    t = b.to_field(psi)
    lap.line_sweep(t, w, form, direction, beta, 1.0)
    want = ora.line_sweep(psi, w, direction, beta, ora.FORM_A if form == "A" else ora.FORM_B,
                          ora.LINES_ZEBRA)
    assert relerr(host(t), want) <= REL


def test_line_sweeps_reuse_scratch_across_shapes(lap, b):
    """y-line sweeps of different shapes in a row (the handle's scratch grows, and is reused
    by a smaller shape) give the same values as on a fresh handle."""
    for shape in ((65, 1025), (1025, 65), (33, 33), (65, 1025)):
        psi = rand_field(*shape, 32)
        t = b.to_field(psi)
        lap.line_sweep(t, 1.3, "A", 1, 1.0, 1.0)
        fresh = b.Laplace()
        u = b.to_field(psi)
        fresh.line_sweep(u, 1.3, "A", 1, 1.0, 1.0)
        fresh.close()
        assert np.array_equal(host(t), host(u)), shape


# ---- whole solves -------------------------------------------------------------------

@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("method,w", [("jacobi", 1.0), ("gs", 1.0), ("sor", 1.0), ("sor", 1.8)])
def test_point_solves_fixed_iterations_bitwise(lap, b, shape, method, w):
    m, n = shape
    psi = rand_field(m, n, 14)
    got, g, want, o = both(lap, b, psi, 1.0, 0.8, method=method, w=w, tol=0.0, max_iter=7,
                           check_every=3)
    assert g["iters"] == o["iters"] == 7
    assert np.array_equal(got, want)
    assert abs(g["r_final"] - o["r_final"]) <= 1e-13 * o["r_final"]


@pytest.mark.parametrize("method,w", [("jacobi", 1.0), ("gs", 1.0), ("sor", 1.5), ("sor", 1.75),
                                      ("sor", 1.9)])
@pytest.mark.parametrize("norm,tol", [("l2_rel", 1e-10), ("maxdelta", 1e-9)])
def test_chamber_solves_match_oracle(lap, b, method, w, norm, tol):
    psi = wl.chamber()
    got, g, want, o = both(lap, b, psi, 0.25, 0.25, method=method, w=w, norm=norm, tol=tol)
    assert g["status"] == o["status"] == "converged"
    assert g["iters"] == o["iters"]
    assert np.array_equal(got, want)


@pytest.mark.parametrize("shape", [(3, 3), (25, 17), (67, 45), (130, 97)])
@pytest.mark.parametrize("form", ["A", "B"])
@pytest.mark.parametrize("w", [1.0, 1.25])
def test_adi_fixed_iterations(lap, b, shape, form, w):
    m, n = shape
    psi = rand_field(m, n, 15)
    got, g, want, o = both(lap, b, psi, 1.0, 0.9, method="adi", w=w, line_form=form, tol=0.0,
                           max_iter=5)
    assert g["iters"] == 5
    assert relerr(got, want) <= REL


@pytest.mark.parametrize("shape,beta", [((25, 17), 1.0), ((65, 65), 1.0), ((129, 33), 1.0),
                                        ((33, 65), 0.8), ((9, 9), 1.0), ((24, 17), 1.0)])
@pytest.mark.parametrize("cfg", [dict(nu1=2, nu2=2), dict(nu1=3, nu2=1, smoother_w=1.2),
                                 dict(nu1=1, nu2=1, max_levels=2)])
def test_multigrid_fixed_cycles(lap, b, shape, beta, cfg):
    m, n = shape
    psi = rand_field(m, n, 16)
    got, g, want, o = both(lap, b, psi, beta, 1.0, method="mg", tol=0.0, max_iter=4, **cfg)
    assert g["iters"] == 4
    assert relerr(got, want) <= REL


def test_multigrid_chamber_cycles_match_oracle(lap, b):
    psi = wl.chamber()
    got, g, want, o = both(lap, b, psi, 0.25, 0.25, method="mg", tol=1e-10)
    assert g["status"] == "converged" and g["iters"] == o["iters"]
    assert relerr(got, want) <= REL


@pytest.mark.parametrize("form,w", [("A", 1.3), ("B", 1.25)])
def test_adi_chamber_matches_oracle(lap, b, form, w):
    got, g, want, o = both(lap, b, wl.chamber(), 0.25, 0.25, method="adi", line_form=form, w=w,
                           tol=1e-10)
    assert g["status"] == "converged" and abs(g["iters"] - o["iters"]) <= 1
    assert relerr(got, want) <= 1e-10


# ---- full size (4097 x 4097, the benchmark's grid and launch shapes) ---------------------

@pytest.fixture(scope="module")
def big():
    return wl.sine_edges(4097, 4097, seed=wl.SEED_BASE + 1)


def test_full_size_sor_sweeps_bitwise(lap, b, big):
    w = wl.w_opt_sor(4097, 4097)
    got, g, want, o = both(lap, b, big, 1 / 4096, 1 / 4096, method="sor", w=w, tol=0.0,
                           max_iter=3, check_every=3)
    assert np.array_equal(got, want)


def test_full_size_jacobi_bitwise(lap, b, big):
    got, g, want, o = both(lap, b, big, 1 / 4096, 1 / 4096, method="jacobi", tol=0.0, max_iter=2,
                           check_every=2)
    assert np.array_equal(got, want)


def test_full_size_adi_iteration(lap, b, big):
    got, g, want, o = both(lap, b, big, 1 / 4096, 1 / 4096, method="adi", w=1.5, tol=0.0,
                           max_iter=1)
    assert relerr(got, want) <= REL


@pytest.mark.parametrize("form", ["A", "B"])
def test_full_size_slor_iterations(lap, b, big, form):
    """Zebra line SOR on the full 4097^2 field at the line-SOR optimum (the bench's solve),
    two iterations against the oracle."""
    w = wl.w_opt_slor(4097, 4097)
    got, g, want, o = both(lap, b, big, 1 / 4096, 1 / 4096, method="slor", w=w, line_form=form,
                           tol=0.0, max_iter=2)
    assert g["iters"] == o["iters"] == 2
    assert relerr(got, want) <= REL


def test_fp64_rate_probe(lap):
    """lap_fp64_rate: the FP64 fma issue rate the bench's ALU roofline divides by. GB300 is
    specified at 1.25 TFLOP/s FP64 (0.625 T fma/s); a measurement far outside means the probe
    does not measure what it claims."""
    r = lap.fp64_rate()
    assert 2e11 < r < 2e12, r


def test_full_size_multigrid_cycle(lap, b, big):
    got, g, want, o = both(lap, b, big, 1 / 4096, 1 / 4096, method="mg", tol=0.0, max_iter=1)
    assert relerr(got, want) <= REL


def test_full_size_multigrid_converges_to_exact_solution(lap, b, big):
    t = b.to_field(big)
    g = lap.solve(t, 1 / 4096, 1 / 4096, method="mg", tol=1e-10)
    assert g["status"] == "converged" and g["iters"] <= 20
    err = np.max(np.abs(host(t) - exact.dst_solve(big)))
    # residual reduced 1e10 times from ||r0|| ~ boundary size: error at the 1e-9 level
    assert err <= 1e-8, err


# ---- edge cases and failure handling ---------------------------------------------------

@pytest.mark.parametrize("shape", [(3, 3), (3, 9), (9, 3), (4, 4)])
@pytest.mark.parametrize("method", ["jacobi", "gs", "sor", "adi", "mg"])
def test_tiny_grids_converge_to_dense_solution(lap, b, shape, method):
    m, n = shape
    psi = wl.random_ring(m, n, 17)
    t = b.to_field(psi)
    g = lap.solve(t, method=method, w=1.2 if method in ("sor", "adi") else 1.0, tol=1e-13)
    assert g["status"] == "converged"
    assert relerr(host(t), exact.dense_solve(psi)) <= 1e-11


def test_zero_iterations_and_exact_start(lap, b):
    psi = rand_field(33, 17, 18)
    t = b.to_field(psi)
    g = lap.solve(t, method="sor", w=1.5, max_iter=0)
    assert g["iters"] == 0 and g["status"] == "max_iter" and np.array_equal(host(t), psi)
    exact_field = wl.polynomial(33, 17, 0.1, 0.1, lambda x, y: x * y, interior="exact")
    t = b.to_field(exact_field)
    g = lap.solve(t, 0.1, 0.1, method="mg", norm="l2_abs", tol=1e-12)
    assert g["status"] == "converged" and g["iters"] == 0


def test_non_finite_boundary_is_reported_as_divergence(lap, b):
    psi = wl.chamber()
    psi[0, 5] = np.nan
    for method in ("sor", "mg", "adi"):
        g = lap.solve(b.to_field(psi), 0.25, 0.25, method=method, w=1.5, tol=1e-10, max_iter=20)
        assert g["status"] == "diverged"
    g = lap.solve(b.to_field(wl.chamber()), 0.25, 0.25, method="adi", line_form="B", w=1.95,
                  norm="maxdelta", tol=1e-9, max_iter=2000)
    assert g["status"] == "diverged"


def test_invalid_arguments_are_rejected(lap, b):
    good = b.field(9, 9)
    with pytest.raises(b.LapError) as e:
        lap.solve(good, method="sor", w=2.5)
    assert e.value.code == -1
    with pytest.raises(b.LapError):
        lap.solve(good, dx=-1.0)
    with pytest.raises(b.LapError) as e:
        lap.solve(b.field(9, 9), method="mg", coarsest_min=2)
    assert e.value.code == -1
    # a host pointer is refused before any kernel sees it
    import ctypes as C
    host_buf = np.zeros((9, 9))
    res = b.Result()
    rc = b.load().lap_solve(lap._h, C.byref(b.Grid(9, 9, 1.0, 1.0, 9)),
                            C.c_void_p(host_buf.ctypes.data), C.byref(b.params()), C.byref(res), None)
    assert rc == -1


def test_hbm_budget_is_enforced(b):
    small = b.Laplace(hbm_budget=1 << 20)
    try:
        with pytest.raises(b.LapError) as e:
            small.solve(b.field(1025, 1025), method="jacobi", max_iter=1)
        assert e.value.code == -2
    finally:
        small.close()


def test_solves_are_deterministic_and_count_launches(lap, b, big):
    before = b.kernel_launches()
    outs = []
    for _ in range(2):
        t = b.to_field(big[:1025, :1025].copy())
        g = lap.solve(t, method="mg", tol=1e-10)
        outs.append((host(t), g["r_final"], g["iters"]))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1:] == outs[1][1:]
    assert b.kernel_launches() > before


def test_host_buffer_solve_equals_device_solve(lap, b):
    """lap_solve_host (host field in, the library's copies, host field out) gives lap_solve's
    iterates bit for bit: pinned and pageable memory, a host row stride wider than the grid,
    the library's device field grown for a larger grid and reused for a smaller one."""
    for shape, kw in (((257, 129), dict(method="mg", tol=1e-10)),
                      ((513, 257), dict(method="sor", w=1.9, max_iter=40, check_every=10)),
                      ((65, 33), dict(method="adi", w=1.3, max_iter=3)),
                      ((129, 65), dict(method="mg_mixed", tol=1e-10))):
        psi = wl.sine_edges(*shape, seed=3 + shape[0])
        t = b.to_field(psi)
        want = lap.solve(t, **kw)
        for pin in (True, False):
            wide = torch.zeros((shape[1], shape[0] + 7), dtype=torch.float64)
            if pin:
                wide = wide.pin_memory()
            hv = wide[:, :shape[0]]
            hv.copy_(torch.from_numpy(psi))
            got = lap.solve_host(hv, **kw)
            assert (got["iters"], got["status"], got["r_final"]) == \
                (want["iters"], want["status"], want["r_final"]), (shape, pin)
            assert np.array_equal(hv.numpy(), host(t)), (shape, pin)
            assert np.all(wide[:, shape[0]:].numpy() == 0.0)  # the padding is not written
    with pytest.raises(TypeError):
        lap.solve_host(b.field(33, 33), method="mg")
    # a device pointer given as the host field is refused by the library itself
    d = b.field(33, 33)
    g = b.Grid(33, 33, 1.0, 1.0, d.stride(0))
    r = b.Result()
    rc = lap._lib.lap_solve_host(lap._h, b.C.byref(g), b.c_void_p(d.data_ptr()), d.stride(0),
                                 b.C.byref(b.params(method="mg")), b.C.byref(r),
                                 b.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert b.ERRORS.get(rc) == "EINVAL"


@pytest.mark.parametrize("kw", [
    dict(method="jacobi", max_iter=23, check_every=5),
    dict(method="jacobi", max_iter=20, check_every=4, norm="maxdelta", tol=0.0),
    dict(method="sor", w=1.7, max_iter=25, check_every=7),
    dict(method="gs", max_iter=9, check_every=3, norm="maxdelta", tol=0.0),
    dict(method="adi", w=1.2, line_form="B", max_iter=5, check_every=2),
    dict(method="mg", max_iter=4, check_every=1),
    dict(method="mg", max_iter=3, check_every=2, norm="maxdelta", tol=0.0),
])
def test_graph_replay_equals_direct_launches(b, kw):
    kw = dict(kw)
    kw.setdefault("tol", 0.0)
    if kw["method"] == "mg":
        kw["tail_size"] = -1  # a fixed launch structure (the timed choice varies per period)
    psi = rand_field(65, 33, 21)
    outs = []
    t = b.field(65, 33)  # one field: the third solve replays the graph the second captured
    h = b.Laplace()
    for graphs in (False, True, True):  # direct, graph capture, graph replay from cache
        h.set_graphs(graphs)
        t.copy_(torch.from_numpy(psi))
        before = b.kernel_launches()
        g = h.solve(t, 0.9, 1.0, **kw)
        outs.append((host(t), (g["iters"], g["r_final"], g["last_check"]), h,
                     b.kernel_launches() - before))
    outs[0][2].close()
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and o[1] == outs[0][1]
    # a replayed graph counts the kernels it runs; with graphs the stopping test of whole
    # check periods runs on the device (one more kernel per period)
    assert outs[1][3] == outs[2][3] >= outs[0][3]


@pytest.mark.parametrize("shape", [(3, 3), (25, 17), (67, 45), (130, 97)])
@pytest.mark.parametrize("form,w", [("A", 1.0), ("A", 1.65), ("B", 1.25)])
def test_slor_fixed_iterations(lap, b, shape, form, w):
    m, n = shape
    psi = rand_field(m, n, 22)
    got, g, want, o = both(lap, b, psi, 1.0, 1.1, method="slor", w=w, line_form=form, tol=0.0,
                           max_iter=6)
    assert g["iters"] == 6
    assert relerr(got, want) <= REL


@pytest.mark.parametrize("form,w", [("A", 1.65), ("B", 1.25)])
def test_slor_chamber_matches_oracle(lap, b, form, w):
    """The paper's stopping rule on the chamber (the one-CTA line solver): the oracle's
    stopping iteration, its iterate to rounding."""
    got, g, want, o = both(lap, b, wl.chamber(), 0.25, 0.25, method="slor", line_form=form, w=w,
                           norm="maxdelta", tol=1e-9)
    assert g["status"] == o["status"] == "converged" and g["iters"] == o["iters"]
    assert relerr(got, want) <= REL


@pytest.mark.parametrize("shape", [(3, 3), (25, 17), (67, 45), (130, 97), (33, 257)])
@pytest.mark.parametrize("method,w", [("gs_lex", 1.0), ("sor_lex", 1.0), ("sor_lex", 1.8)])
def test_lexicographic_fixed_iterations_bitwise(lap, b, shape, method, w):
    m, n = shape
    psi = rand_field(m, n, 23)
    got, g, want, o = both(lap, b, psi, 1.0, 0.8, method=method, w=w, tol=0.0, max_iter=11,
                           check_every=4)
    assert g["iters"] == 11 and np.array_equal(got, want)


def test_paper_chamber_counts_on_the_gpu(lap, b):
    """The paper's own orderings on its chamber problem (stop at max|dpsi| <= 1e-9), run on
    the GPU and bitwise equal to the oracle: Jacobi, lexicographic GS, and the SOR w sweep
    whose optimum the paper prints (1.75)."""
    kw = dict(norm="maxdelta", tol=1e-9)
    for method in ("jacobi", "gs_lex"):
        got, g, want, o = both(lap, b, wl.chamber(), 0.25, 0.25, method=method, **kw)
        assert g["iters"] == o["iters"] and np.array_equal(got, want)
    its = []
    for w in np.round(np.arange(1.0, 1.951, 0.05), 2):
        got, g, want, o = both(lap, b, wl.chamber(), 0.25, 0.25, method="sor_lex", w=float(w), **kw)
        assert g["iters"] == o["iters"] and np.array_equal(got, want)
        its.append(g["iters"])
    assert np.round(np.arange(1.0, 1.951, 0.05), 2)[int(np.argmin(its))] == 1.75


def test_lexicographic_refuses_grids_beyond_one_sm(lap, b):
    with pytest.raises(b.LapError) as e:
        lap.solve(b.field(257, 257), method="gs_lex", max_iter=1)
    assert e.value.code == -4


# ---- the whole solve in one CTA (small grids, the stopping rule of Eq. 16) -------------

@pytest.mark.parametrize("method", ["slor", "adi"])
@pytest.mark.parametrize("form,w", [("A", 1.3), ("B", 1.25), ("A", 1.0)])
@pytest.mark.parametrize("every,max_iter,tol", [(1, 400, 1e-9), (3, 10, 0.0), (4, 23, 0.0),
                                                (5, 1000, 1e-8)])
@pytest.mark.parametrize("shape,beta", [((25, 17), 1.0), ((33, 65), 0.8), ((3, 3), 1.0),
                                        ((4, 61), 1.3)])
def test_one_cta_line_solve_matches_oracle(lap, b, method, form, w, every, max_iter, tol, shape, beta):
    """SLOR and ADI on grids of at most 4096 points with the stopping rule of Eq. 16 run the
    whole solve in one kernel: the oracle's iterates to rounding (tabulated pivots instead of
    the serial solver's divisions), its stopping iteration, for any period length and cap."""
    m, n = shape
    psi = rand_field(m, n, 41 + m)
    t = b.to_field(psi)
    torch.cuda.synchronize()
    before = b.kernel_launches()
    g = lap.solve(t, beta, 1.0, method=method, w=w, line_form=form, norm="maxdelta", tol=tol,
                  check_every=every, max_iter=max_iter)
    # one kernel for the whole solve, beside the initial and final residual norms
    assert b.kernel_launches() - before <= 5
    want, o = ora.solve(psi, dx=beta, dy=1.0, tol=tol, norm=ora.NORM_MAXDELTA, max_iter=max_iter,
                        check_every=every, history=True, **ora_kw(method, w=w, line_form=form))
    assert g["status"] == o["status"]
    assert g["iters"] == o["iters"]
    assert relerr(host(t), want) <= REL
    if g["iters"]:
        assert abs(g["last_check"] - o["hist"][-1]) <= 1e-10 * o["hist"][-1] + 1e-15


@pytest.mark.parametrize("method,w", [("jacobi", 1.0), ("gs", 1.0), ("sor", 1.6), ("gs_lex", 1.0),
                                      ("sor_lex", 1.6)])
@pytest.mark.parametrize("every,max_iter,tol", [(1, 400, 1e-7), (3, 10, 0.0), (4, 23, 0.0),
                                                (7, 1000, 1e-8), (5, 5, 0.0)])
@pytest.mark.parametrize("shape,beta", [((25, 17), 1.0), ((33, 65), 0.8), ((3, 3), 1.0)])
def test_one_cta_solve_matches_oracle(lap, b, method, w, every, max_iter, tol, shape, beta):
    """Point methods on grids of at most 4096 points with max|psi^{k+1} - psi^k| <= tol run
    the whole solve (periods and tests) in one kernel: the same iterates, stopping
    iteration and test value as the oracle, for any period length and iteration cap."""
    m, n = shape
    psi = rand_field(m, n, 23 + m)
    t = b.to_field(psi)
    g = lap.solve(t, beta, 1.0, method=method, w=w, norm="maxdelta", tol=tol, check_every=every,
                  max_iter=max_iter)
    want, o = ora.solve(psi, dx=beta, dy=1.0, tol=tol, norm=ora.NORM_MAXDELTA, max_iter=max_iter,
                        check_every=every, history=True, **ora_kw(method, w=w))
    assert g["status"] == o["status"]
    assert g["iters"] == o["iters"]
    assert np.array_equal(host(t), want)
    if g["iters"]:
        assert g["last_check"] == o["hist"][-1]


# ---- the diagonal summation order: (W + S) + (E + N), beta = 1 ----------------------

DIAG_SHAPES = [(3, 3), (4, 5), (25, 17), (67, 45), (130, 97), (257, 33), (40, 300), (600, 21)]


@pytest.mark.parametrize("shape", DIAG_SHAPES)
@pytest.mark.parametrize("method,w", [("gs", 1.0), ("sor", 1.0), ("sor", 1.8)])
@pytest.mark.parametrize("norm", ["l2_rel", "maxdelta"])
def test_diagonal_order_fixed_iterations_bitwise(lap, b, shape, method, w, norm):
    """The diagonal-pair kernel (threads walking 16-point diagonal runs) against the oracle's
    sweeps in the same summation order: the same bits for every launch shape and tail."""
    m, n = shape
    psi = rand_field(m, n, 31 + m)
    t = b.to_field(psi)
    g = lap.solve(t, 1.0, 1.0, method=method, w=w, tol=0.0, max_iter=7, check_every=3, norm=norm,
                  sum_order="diagonal")
    want, o = ora.solve(psi, tol=0.0, max_iter=7, check_every=3, norm=NORMS[norm],
                        sum_order=ora.SUM_DIAGONAL, **ora_kw(method, w=w))
    # (a 3 x 3 grid is solved exactly by one Gauss-Seidel sweep: both stop at the first test)
    assert g["status"] == o["status"]
    assert g["iters"] == o["iters"] == (3 if shape == (3, 3) and w == 1.0 else 7)
    assert np.array_equal(host(t), want)


@pytest.mark.parametrize("method,w", [("gs", 1.0), ("sor", 1.75), ("sor", 1.9)])
@pytest.mark.parametrize("norm,tol", [("l2_rel", 1e-10), ("maxdelta", 1e-9)])
def test_diagonal_order_chamber_solves_match_oracle(lap, b, method, w, norm, tol):
    psi = wl.chamber()
    t = b.to_field(psi)
    g = lap.solve(t, 0.25, 0.25, method=method, w=w, norm=norm, tol=tol, sum_order="diagonal")
    want, o = ora.solve(psi, dx=0.25, dy=0.25, tol=tol, norm=NORMS[norm],
                        sum_order=ora.SUM_DIAGONAL, **ora_kw(method, w=w))
    assert g["status"] == o["status"] == "converged"
    assert g["iters"] == o["iters"]
    assert np.array_equal(host(t), want)


def test_diagonal_order_full_size_sweeps_bitwise(lap, b, big):
    w = wl.w_opt_sor(4097, 4097)
    t = b.to_field(big)
    lap.solve(t, 1 / 4096, 1 / 4096, method="sor", w=w, tol=0.0, max_iter=3, check_every=3,
              sum_order="diagonal")
    want, _ = ora.solve(big, dx=1 / 4096, dy=1 / 4096, tol=0.0, max_iter=3, check_every=3,
                        sum_order=ora.SUM_DIAGONAL, **ora_kw("sor", w=w))
    assert np.array_equal(host(t), want)


def test_diagonal_order_stays_within_rounding_of_the_paper_order(lap, b):
    """Many sweeps in either order: the iterates part only by accumulated rounding."""
    m, n = 513, 385
    psi = wl.sine_edges(m, n, seed=wl.SEED_BASE + 5)
    w = wl.w_opt_sor(m, n)
    a, c = b.to_field(psi), b.to_field(psi)
    ga = lap.solve(a, 1.0, 1.0, method="sor", w=w, tol=1e-10, check_every=25, sum_order="diagonal")
    gc = lap.solve(c, 1.0, 1.0, method="sor", w=w, tol=1e-10, check_every=25)
    assert ga["status"] == gc["status"] == "converged"
    assert ga["iters"] == gc["iters"]
    assert 0.0 < relerr(host(a), host(c)) <= REL


def test_diagonal_order_refuses_other_methods_and_beta(lap, b):
    good = b.to_field(rand_field(33, 33, 3))
    with pytest.raises(b.LapError) as e:
        lap.solve(good, 1.0, 0.5, method="sor", w=1.5, max_iter=2, sum_order="diagonal")
    assert "EUNSUPPORTED" in str(e.value)
    for method in ("jacobi", "mg", "adi", "mg_mixed"):
        with pytest.raises(b.LapError) as e:
            lap.solve(good, 1.0, 1.0, method=method, max_iter=2, sum_order="diagonal")
        assert "EINVAL" in str(e.value)


# ---- size limits ---------------------------------------------------------------------

@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("form", ["A", "B"])
def test_longest_lines(lap, b, direction, form):
    """Lines of 16383 unknowns, the longest the line solver takes (x-lines: 64 chunks of 255 in
    131 KB of shared memory per CTA; y-lines: 32 chunks of 511), against the oracle; one more
    unknown is refused with EUNSUPPORTED."""
    shape = (16385, 5) if direction == 0 else (5, 16385)
    psi = rand_field(*shape, 41)
    t = b.to_field(psi)
    lap.line_sweep(t, 1.3, form, direction, 1.0, 1.0)
    want = ora.line_sweep(psi, 1.3, direction, 1.0, ora.FORM_A if form == "A" else ora.FORM_B,
                          ora.LINES_ZEBRA)
    assert relerr(host(t), want) <= 1e-13
    big = b.to_field(rand_field(*((16386, 5) if direction == 0 else (5, 16386)), 42))
    with pytest.raises(b.LapError) as e:
        lap.line_sweep(big, 1.3, form, direction, 1.0, 1.0)
    assert "EUNSUPPORTED" in str(e.value)


def test_tallest_grid(lap, b):
    """The tallest grid the library takes, LAP_GRID_MAX_N rows (the point kernels' launch grids
    reach 65535 CTA rows), against the oracle: Jacobi and red-black SOR in both summation
    orders, bit for bit. One more row is refused with EUNSUPPORTED before anything runs."""
    N = b.GRID_MAX_N
    psi = rand_field(5, N, 43)
    cases = [(dict(method="jacobi"), dict(method=ora.JACOBI)),
             (dict(method="sor", w=1.5), dict(method=ora.SOR, ordering=ora.RB, w=1.5)),
             (dict(method="sor", w=1.5, sum_order="diagonal"),
              dict(method=ora.SOR, ordering=ora.RB, w=1.5, sum_order=ora.SUM_DIAGONAL))]
    for kw, okw in cases:
        t = b.to_field(psi)
        g = lap.solve(t, 1.0, 1.0, tol=0.0, max_iter=2, **kw)
        want, o = ora.solve(psi, dx=1.0, dy=1.0, tol=0.0, max_iter=2, **okw)
        assert g["iters"] == o["iters"] == 2, kw
        assert np.array_equal(host(t), want), kw
    with pytest.raises(b.LapError) as e:
        lap.solve(b.to_field(rand_field(5, N + 1, 44)), 1.0, 1.0, method="jacobi", tol=0.0,
                  max_iter=1)
    assert "EUNSUPPORTED" in str(e.value)


def test_largest_coarsest_solve(lap, b):
    """The exact coarsest-level solve at its limit of 1024 interior unknowns (34 x 34 field),
    against the oracle's Gaussian elimination; 35 x 34 (1056 unknowns) is refused."""
    u = wl.random_ring(34, 34, 13)
    q = wl.random_interior(np.zeros((34, 34)), 14)
    t = b.to_field(u)
    lap.coarse_solve(t, 1.0, 1.0, b.to_field(q))
    assert relerr(host(t), ora.coarse_direct(u, 1.0, q)) <= 1e-12
    with pytest.raises(b.LapError) as e:
        lap.coarse_solve(b.to_field(wl.random_ring(35, 34, 15)), 1.0, 1.0,
                         b.to_field(np.zeros((34, 35))))
    assert "EUNSUPPORTED" in str(e.value)
