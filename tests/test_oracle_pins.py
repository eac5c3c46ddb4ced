"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics,
never against the oracle itself: exact discrete-harmonic data, dense and DST direct
solves, closed-form spectra of every iteration (Jacobi, Gauss-Seidel, SOR, line
relaxation in both forms and both orderings), the adjointness of the multigrid
transfer operators, multigrid's grid-independent convergence, the discrete maximum
principle and the symmetry of the paper's second verification case."""
import numpy as np
import pytest

import oracle as ora
from paper_2208_02427_gb300 import workloads as wl
from tests import exact

HARMONIC = {
    "one": lambda x, y: 1.0 + 0.0 * x * y,
    "x": lambda x, y: x + 0.0 * y,
    "y": lambda x, y: y + 0.0 * x,
    "x2-y2": lambda x, y: x ** 2 - y ** 2,
    "xy": lambda x, y: x * y,
    "x3-3xy2": lambda x, y: x ** 3 - 3 * x * y ** 2,
}
NOT_HARMONIC = lambda x, y: x ** 4 - 6 * x ** 2 * y ** 2 + y ** 4  # L = 2 (dx^2 + dy^2)

METHODS = {
    "jacobi": dict(method=ora.JACOBI),
    "gs-lex": dict(method=ora.GS, ordering=ora.LEX),
    "gs-rb": dict(method=ora.GS, ordering=ora.RB),
    "sor-lex": dict(method=ora.SOR, ordering=ora.LEX, w=1.5),
    "sor-rb": dict(method=ora.SOR, ordering=ora.RB, w=1.5),
    "slorA": dict(method=ora.SLOR, form=ora.FORM_A, line_order=ora.LINES_SUCCESSIVE, w=1.3),
    "slorB": dict(method=ora.SLOR, form=ora.FORM_B, line_order=ora.LINES_SUCCESSIVE, w=1.3),
    "adiA-zebra": dict(method=ora.ADI, form=ora.FORM_A, line_order=ora.LINES_ZEBRA, w=1.2),
    "adiB-zebra": dict(method=ora.ADI, form=ora.FORM_B, line_order=ora.LINES_ZEBRA, w=1.2),
    "adiB-succ": dict(method=ora.ADI, form=ora.FORM_B, line_order=ora.LINES_SUCCESSIVE, w=1.2),
    "mg": dict(method=ora.MG, nu1=2, nu2=2, coarsest_min=3),
    "mg-lex-gscoarse": dict(method=ora.MG, nu1=3, nu2=3, ordering=ora.LEX, coarse=ora.COARSE_GS,
                            coarsest_min=3),
}


# ---- exact discrete-harmonic data --------------------------------------------

@pytest.mark.parametrize("poly", sorted(HARMONIC))
@pytest.mark.parametrize("meth", sorted(METHODS))
def test_harmonic_polynomials_are_fixed_points(poly, meth):
    m, n, dx, dy = 17, 13, 0.3, 0.2
    exact_field = wl.polynomial(m, n, dx, dy, HARMONIC[poly], interior="exact")
    scale = np.max(np.abs(exact_field))
    # started at the exact values, one iteration moves nothing beyond rounding
    once, _ = ora.solve(exact_field, dx=dx, dy=dy, max_iter=1, tol=0.0, **METHODS[meth])
    assert np.max(np.abs(once - exact_field)) <= 1e-13 * scale
    # started from a zero interior, the iteration converges to the polynomial
    start = wl.polynomial(m, n, dx, dy, HARMONIC[poly], interior="zero")
    sol, info = ora.solve(start, dx=dx, dy=dy, tol=1e-13, max_iter=20000, **METHODS[meth])
    assert info["status"] == "converged"
    assert np.max(np.abs(sol - exact_field)) <= 1e-9 * scale


def test_non_harmonic_quartic_is_not_reproduced():
    m, n, dx, dy = 17, 13, 0.3, 0.2
    exact_field = wl.polynomial(m, n, dx, dy, NOT_HARMONIC, interior="exact")
    sol, info = ora.solve(wl.polynomial(m, n, dx, dy, NOT_HARMONIC), dx=dx, dy=dy, tol=1e-13,
                          method=ora.MG, coarsest_min=3)
    assert info["status"] == "converged"
    assert np.max(np.abs(sol - exact_field)) > 1e-5 * np.max(np.abs(exact_field))
    # the oracle's scaled defect of the quartic is the closed form 2 dx^2 (dx^2 + dy^2)
    r = ora.defect(exact_field, beta=dx / dy)
    assert np.allclose(r[1:-1, 1:-1], 2.0 * dx ** 2 * (dx ** 2 + dy ** 2), rtol=1e-9, atol=0)


# ---- exact direct solves --------------------------------------------------------

@pytest.mark.parametrize("shape", [(3, 3), (3, 5), (5, 3), (9, 9), (5, 9), (9, 7)])
@pytest.mark.parametrize("beta", [1.0, 1.5])
@pytest.mark.parametrize("meth", sorted(METHODS))
def test_converges_to_dense_direct_solution(shape, beta, meth):
    m, n = shape
    psi = wl.random_ring(m, n, seed=100 + m * 10 + n)
    ref = exact.dense_solve(psi, beta)
    sol, info = ora.solve(psi, dx=beta, dy=1.0, tol=1e-14, max_iter=20000, **METHODS[meth])
    assert info["status"] == "converged"
    assert np.max(np.abs(sol - ref)) <= 1e-11


@pytest.mark.parametrize("shape", [(3, 3), (7, 5), (9, 9), (5, 17)])
def test_coarse_direct_solve_matches_lapack(shape):
    m, n = shape
    rng = np.random.default_rng(7)
    u = wl.random_ring(m, n, seed=3)
    q = np.zeros((n, m))
    q[1:-1, 1:-1] = rng.standard_normal((n - 2, m - 2))
    got = ora.coarse_direct(u, beta=0.7, q=q)
    ref = exact.dense_solve(u, 0.7, source=q)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_exact_helpers_agree_with_closed_form():
    # the test's own exact solvers are pinned to the closed form before they pin the oracle
    for (m, n, k, beta) in [(17, 9, 1, 1.0), (33, 17, 3, 1.0), (21, 31, 5, 0.8)]:
        psi = exact.sine_mode(m, n, k, beta)
        ring = psi.copy()
        ring[1:-1, 1:-1] = 0.0
        assert np.max(np.abs(exact.dst_solve(ring, beta) - psi)) <= 1e-13
    psi = wl.random_ring(9, 7, seed=5)
    assert np.max(np.abs(exact.dst_solve(psi, 1.3) - exact.dense_solve(psi, 1.3))) <= 1e-13


def test_mg_converges_to_dst_solution_large():
    m, n = 129, 65
    psi = wl.sine_edges(m, n, seed=wl.SEED_BASE + 1)
    ref = exact.dst_solve(psi)
    sol, info = ora.solve(psi, method=ora.MG, tol=1e-13, max_iter=60)
    assert info["status"] == "converged"
    assert np.max(np.abs(sol - ref)) <= 1e-10


# ---- spectra of the iterations -----------------------------------------------

def young_radius(w, mu):
    """Spectral radius of SOR for a consistently ordered matrix with Jacobi radius mu."""
    w_opt = 2.0 / (1.0 + np.sqrt(1.0 - mu * mu))
    if w >= w_opt:
        return w - 1.0
    root = (w * mu + np.sqrt(w * w * mu * mu - 4.0 * (w - 1.0))) / 2.0
    return root * root


@pytest.mark.parametrize("shape,beta", [((7, 6), 1.3), ((9, 9), 1.0), ((6, 10), 0.7)])
def test_jacobi_spectrum_is_closed_form(shape, beta):
    m, n = shape
    T = exact.iteration_matrix(lambda e: ora.jacobi_sweep(e, beta), m, n)
    got = np.sort(np.linalg.eigvals(T).real)
    k = np.arange(1, m - 1)[None, :]
    l = np.arange(1, n - 1)[:, None]
    want = np.sort(((np.cos(k * np.pi / (m - 1)) + beta ** 2 * np.cos(l * np.pi / (n - 1)))
                    / (1.0 + beta ** 2)).ravel())
    assert np.max(np.abs(got - want)) <= 1e-12
    if m == n and beta == 1.0:
        assert abs(exact.spectral_radius(T) - np.cos(np.pi / (m - 1))) <= 1e-12


def jacobi_radius(m, n, beta):
    return (np.cos(np.pi / (m - 1)) + beta ** 2 * np.cos(np.pi / (n - 1))) / (1.0 + beta ** 2)


@pytest.mark.parametrize("ordering", [ora.LEX, ora.RB])
@pytest.mark.parametrize("w", [0.8, 1.0, 1.2, 1.9])
def test_sor_spectral_radius_follows_young(ordering, w):
    m, n, beta = 9, 7, 1.2
    T = exact.iteration_matrix(lambda e: ora.sor_sweep(e, w, beta, ordering), m, n)
    mu = jacobi_radius(m, n, beta)
    assert abs(exact.spectral_radius(T) - young_radius(w, mu)) <= 1e-8


@pytest.mark.parametrize("ordering", [ora.LEX, ora.RB])
def test_gauss_seidel_radius_is_jacobi_squared(ordering):
    m, n, beta = 9, 7, 1.2
    T = exact.iteration_matrix(lambda e: ora.gs_sweep(e, beta, ordering), m, n)
    assert abs(exact.spectral_radius(T) - jacobi_radius(m, n, beta) ** 2) <= 1e-10


def line_spectrum(m, n, beta, w, form, direction):
    """All eigenvalues of line relaxation (zebra or successive lines; both orders are
    consistently ordered) from the Fourier pair (k along the line, l across it):
    [(d - 2 c_a cos_k) lam - (1 - w)_B d]^2 = w^2 g_l^2 lam (form B), block SOR (form A)."""
    b2 = beta ** 2
    d = 2.0 * (1.0 + b2)
    along, across = ((m, n) if direction == 0 else (n, m))
    off, cross = ((1.0, b2) if direction == 0 else (b2, 1.0))
    out = []
    for k in range(1, along - 1):
        ck = np.cos(k * np.pi / (along - 1))
        for l in range(1, across - 1):
            g = 2.0 * cross * np.cos(l * np.pi / (across - 1))
            if form == ora.FORM_A:
                mu = g / (d - 2.0 * off * ck)
                # block SOR: (lam + w - 1)^2 = lam w^2 mu^2
                out.extend(np.roots([1.0, 2.0 * (w - 1.0) - w * w * mu * mu, (w - 1.0) ** 2]))
            else:
                D = d - 2.0 * w * off * ck
                c0 = (1.0 - w) * d
                out.extend(np.roots([D * D, -(2.0 * D * c0 + w * w * g * g), c0 * c0]))
    return np.array(out)


@pytest.mark.parametrize("form", [ora.FORM_A, ora.FORM_B])
@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("order", [ora.LINES_ZEBRA, ora.LINES_SUCCESSIVE])
@pytest.mark.parametrize("w", [1.0, 1.3, 1.8])
def test_line_relaxation_radius_is_closed_form(form, direction, order, w):
    m, n, beta = 9, 8, 1.3
    T = exact.iteration_matrix(lambda e: ora.line_sweep(e, w, direction, beta, form, order), m, n)
    want = np.max(np.abs(line_spectrum(m, n, beta, w, form, direction)))
    assert abs(exact.spectral_radius(T) - want) <= 1e-7


def test_adi_is_x_sweep_then_y_sweep():
    psi = wl.random_interior(wl.random_ring(11, 9, seed=1), seed=2)
    for form in (ora.FORM_A, ora.FORM_B):
        a = ora.adi_iteration(psi, 1.3, 0.9, form)
        b = ora.line_sweep(ora.line_sweep(psi, 1.3, 0, 0.9, form), 1.3, 1, 0.9, form)
        assert np.array_equal(a, b)


def test_line_forms_coincide_at_w_one():
    psi = wl.random_interior(wl.random_ring(11, 9, seed=4), seed=5)
    for direction in (0, 1):
        a = ora.line_sweep(psi, 1.0, direction, 1.1, ora.FORM_A)
        b = ora.line_sweep(psi, 1.0, direction, 1.1, ora.FORM_B)
        assert np.max(np.abs(a - b)) <= 1e-14


@pytest.mark.parametrize("N", [1, 2, 3, 17, 100])
def test_thomas_matches_lapack(N):
    rng = np.random.default_rng(N)
    a, c = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    b = 2.5 + rng.uniform(0, 1, N)
    d = rng.standard_normal(N)
    A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    assert np.max(np.abs(ora.thomas(a, b, c, d) - np.linalg.solve(A, d))) <= 1e-14


# ---- multigrid -------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(9, 9), (17, 9), (9, 13)])
def test_full_weighting_is_adjoint_of_bilinear(shape):
    mf, nf = shape
    mc, nc = (mf - 1) // 2 + 1, (nf - 1) // 2 + 1
    Nc, Nf = (mc - 2) * (nc - 2), (mf - 2) * (nf - 2)
    P = np.zeros((Nf, Nc))
    for k in range(Nc):
        ec = np.zeros((nc, mc))
        ec[1 + k // (mc - 2), 1 + k % (mc - 2)] = 1.0
        P[:, k] = ora.prolong_add(ec, np.zeros((nf, mf)))[1:-1, 1:-1].ravel()
    R = np.zeros((Nc, Nf))
    for k in range(Nf):
        rf = np.zeros((nf, mf))
        rf[1 + k // (mf - 2), 1 + k % (mf - 2)] = 1.0
        R[:, k] = ora.restrict_fw(rf)[1:-1, 1:-1].ravel()
    # q_coarse = (2h)^2 FW(R) = 4 * (1/4) P^T r = P^T r exactly
    assert np.array_equal(R, P.T)
    assert set(np.unique(P)) <= {0.0, 0.25, 0.5, 1.0}


def test_transfer_operators_are_exact_on_bilinear_fields():
    mf, nf = 17, 13
    mc, nc = 9, 7
    f = lambda X, Y: 0.3 + 1.7 * X - 0.4 * Y + 0.9 * X * Y
    Xc, Yc = np.meshgrid(np.arange(mc) * 2.0, np.arange(nc) * 2.0)
    Xf, Yf = np.meshgrid(np.arange(mf) * 1.0, np.arange(nf) * 1.0)
    up = ora.prolong_add(f(Xc, Yc), np.zeros((nf, mf)))
    assert np.max(np.abs(up[1:-1, 1:-1] - f(Xf, Yf)[1:-1, 1:-1])) <= 1e-12
    lin = lambda X, Y: 0.5 - 0.25 * X + 2.0 * Y
    q = ora.restrict_fw(lin(Xf, Yf))
    assert np.max(np.abs(q[1:-1, 1:-1] - 4.0 * lin(Xc, Yc)[1:-1, 1:-1])) <= 1e-12


def cycle_factor(m, n, seed):
    psi = wl.random_ring(m, n, seed)
    _, info = ora.solve(psi, method=ora.MG, tol=0.0, max_iter=7, history=True)
    h = info["hist"]
    return float((h[-1] / h[1]) ** (1.0 / (len(h) - 2)))


@pytest.mark.slow
def test_mg_v22_factor_is_small_and_grid_independent():
    factors = [cycle_factor(m, n, 11) for (m, n) in [(33, 33), (65, 65), (129, 129), (257, 129)]]
    assert max(factors) < 0.2, factors
    assert max(factors) / min(factors) < 2.0, factors


def test_two_grid_with_exact_coarse_solve_beats_smoothing():
    m = n = 33
    psi = wl.random_ring(m, n, 12)
    _, two = ora.solve(psi, method=ora.MG, tol=0.0, max_iter=3, max_levels=2, history=True)
    _, smooth = ora.solve(psi, method=ora.GS, tol=0.0, max_iter=3 * 4, history=True)
    assert two["hist"][-1] < 1e-3 * smooth["hist"][-1]


def test_mg_level_count():
    assert ora.mg_levels(4097, 4097, 5, 0) == 11
    assert ora.mg_levels(25, 17, 5, 0) == 3  # 25x17, 13x9, 7x5 as in the paper
    assert ora.mg_levels(33, 129, 5, 0) == 4
    assert ora.mg_levels(24, 17, 5, 0) == 1


# ---- maximum principle and symmetry -----------------------------------------------

@pytest.mark.parametrize("meth", ["jacobi", "gs-lex", "gs-rb"])
def test_iterates_obey_maximum_principle(meth):
    psi = wl.random_ring(21, 15, seed=9)
    ring = np.concatenate([psi[0, 1:-1], psi[-1, 1:-1], psi[1:-1, 0], psi[1:-1, -1]])
    lo, hi = ring.min(), ring.max()
    cur = psi.copy()
    cur[1:-1, 1:-1] = 0.5 * (lo + hi)
    for _ in range(30):
        cur, _ = ora.solve(cur, max_iter=5, tol=0.0, **METHODS[meth])
        inner = cur[1:-1, 1:-1]
        assert inner.min() >= lo and inner.max() <= hi


def test_converged_solution_obeys_maximum_principle():
    psi = wl.random_ring(33, 17, seed=10)
    sol, _ = ora.solve(psi, method=ora.SOR, w=1.8, tol=1e-12)
    ring = np.concatenate([psi[0, 1:-1], psi[-1, 1:-1], psi[1:-1, 0], psi[1:-1, -1]])
    assert sol[1:-1, 1:-1].min() >= ring.min() and sol[1:-1, 1:-1].max() <= ring.max()


def test_verification_cases_are_symmetric():
    for sym in (False, True):
        psi = wl.chamber(symmetric=sym)
        sol, info = ora.solve(psi, method=ora.MG, tol=1e-13, dx=0.25, dy=0.25)
        assert info["status"] == "converged"
        assert np.max(np.abs(sol - sol[:, ::-1])) <= 1e-11
        if sym:
            assert np.max(np.abs(sol - sol[::-1, :])) <= 1e-11


def test_orderings_reach_the_same_solution():
    psi = wl.chamber()
    a, _ = ora.solve(psi, method=ora.GS, ordering=ora.LEX, tol=1e-13)
    b, _ = ora.solve(psi, method=ora.GS, ordering=ora.RB, tol=1e-13)
    c, _ = ora.solve(psi, method=ora.ADI, form=ora.FORM_B, w=1.3, tol=1e-13)
    assert np.max(np.abs(a - b)) <= 1e-11 and np.max(np.abs(a - c)) <= 1e-11


# ---- the visiting order of each sweep ----------------------------------------------
# One sweep leaves a defect that only the neighbours visited *after* a node explain:
# these identities fix the ordering, which the spectra above cannot (every
# consistently ordered ordering shares Young's spectrum and the fixed point).

def _field(seed, m=13, n=10):
    return wl.random_interior(wl.random_ring(m, n, seed=seed), seed=seed + 1)


def test_red_black_gs_is_jacobi_on_red_then_black():
    beta = 1.3
    psi = _field(21)
    n, m = psi.shape
    jj, ii = np.mgrid[0:n, 0:m]
    red = ((ii + jj) % 2 == 0)
    red[0, :] = red[-1, :] = red[:, 0] = red[:, -1] = False
    black = ((ii + jj) % 2 == 1)
    black[0, :] = black[-1, :] = black[:, 0] = black[:, -1] = False
    rb = ora.gs_sweep(psi, beta, ora.RB)
    half = psi.copy()
    half[red] = ora.jacobi_sweep(psi, beta)[red]
    assert np.array_equal(rb[red], half[red])
    assert np.array_equal(rb[black], ora.jacobi_sweep(half, beta)[black])


def test_lexicographic_gs_defect_comes_from_later_neighbours():
    beta = 0.8
    psi = _field(23)
    new = ora.gs_sweep(psi, beta, ora.LEX)
    delta = new - psi
    r = ora.defect(new, beta)
    # node (i,j) was solved exactly with E = (i+1,j) and N = (i,j+1) still old
    want = delta[1:-1, 2:] + beta ** 2 * delta[2:, 1:-1]
    assert np.max(np.abs(r[1:-1, 1:-1] - want)) <= 1e-13


@pytest.mark.parametrize("order", [ora.LINES_ZEBRA, ora.LINES_SUCCESSIVE])
@pytest.mark.parametrize("direction", [0, 1])
def test_line_sweep_defect_comes_from_later_lines(order, direction):
    beta = 1.2
    psi = _field(25)
    new = ora.line_sweep(psi, 1.0, direction, beta, ora.FORM_A, order)
    delta = new - psi
    r = ora.defect(new, beta)
    n, m = psi.shape
    # work with lines as rows: transpose for y-lines; weight of the cross neighbours
    if direction == 1:
        delta, r = delta.T, r.T
    cross = beta ** 2 if direction == 0 else 1.0
    nlines = r.shape[0] - 2
    for l in range(1, nlines + 1):
        if order == ora.LINES_SUCCESSIVE:
            later = [l + 1]
        else:  # odd lines first: odd lines see both (even) neighbours change afterwards
            later = [l - 1, l + 1] if l % 2 == 1 else []
        want = sum(cross * delta[k, 1:-1] for k in later)
        assert np.max(np.abs(r[l, 1:-1] - want)) <= 1e-13, (l, order, direction)


def test_slor_optimum_minimises_the_oracle_radius():
    """w_opt_slor (the bench's zebra line-SOR factor) from the x-line Jacobi radius: at it the
    oracle's zebra SLOR (form A) iteration matrix has radius w_opt - 1 (Young's optimum for a
    consistently ordered splitting), and nearby factors converge more slowly."""
    m, n, beta = 9, 8, 1.3
    w = wl.w_opt_slor(m, n, beta)

    def radius(wv):
        T = exact.iteration_matrix(lambda e: ora.line_sweep(e, wv, 0, beta, ora.FORM_A, ora.LINES_ZEBRA),
                                   m, n)
        return exact.spectral_radius(T)

    # the optimum is a double eigenvalue (a Jordan block): computed to about sqrt(eps)
    assert abs(radius(w) - (w - 1.0)) <= 1e-6
    assert radius(w - 0.05) > radius(w) + 1e-3
    assert radius(w + 0.05) > radius(w) + 1e-3


@pytest.mark.parametrize("shape,beta,threads", [((33, 17), 1.0, 1), ((65, 40), 1.3, 3),
                                                ((257, 129), 1.0, 8), ((9, 5), 0.7, 16)])
def test_threaded_timing_sweeps_equal_the_oracle(shape, beta, threads):
    """The all-cores CPU baseline's threaded red-black SOR sweeps are the oracle's sweeps bit
    for bit (same update expression; rows split across threads, a barrier per colour)."""
    m, n = shape
    psi = wl.random_interior(wl.random_ring(m, n, seed=m + n), seed=m * n)
    want = psi.copy()
    for _ in range(5):
        want = ora.sor_sweep(want, 1.7, beta, ora.RB)
    got = ora.mt_sor_rb_sweeps(psi, 1.7, 5, beta, threads)
    assert np.array_equal(got, want)


# ---- the diagonal summation order (W + S) + (E + N), beta = 1 ---------------------

def integer_field(m, n, seed):
    """Values that are small integers: every partial sum of four of them is exact, so any
    order of the neighbour sum gives the same bits, and a wrong neighbour gives another value."""
    rng = np.random.default_rng(seed)
    return rng.integers(-1000, 1001, size=(n, m)).astype(np.float64)


@pytest.mark.parametrize("shape", [(3, 3), (7, 5), (16, 9), (33, 20)])
@pytest.mark.parametrize("w", [1.0, 0.75, 1.5])
def test_diagonal_order_equals_paper_order_on_exact_sums(shape, w):
    m, n = shape
    psi = integer_field(m, n, 40 + m)
    q = integer_field(m, n, 41 + m)
    for qq in (None, q):
        if w == 1.0:
            a = ora.gs_sweep(psi, 1.0, ora.RB, qq, sum_order=ora.SUM_DIAGONAL)
            ref = ora.gs_sweep(psi, 1.0, ora.RB, qq)
        else:
            a = ora.sor_sweep(psi, w, 1.0, ora.RB, qq, sum_order=ora.SUM_DIAGONAL)
            ref = ora.sor_sweep(psi, w, 1.0, ora.RB, qq)
        assert np.array_equal(a, ref)
        # and both are Eq. 6 / 7 written out for the red-black order (exact sums)
        want = psi.copy()
        for colour in (0, 1):
            for j in range(1, n - 1):
                for i in range(1, m - 1):
                    if (i + j) % 2 != colour:
                        continue
                    s = want[j, i - 1] + want[j, i + 1] + want[j - 1, i] + want[j + 1, i]
                    if qq is not None:
                        s += qq[j, i]
                    want[j, i] = (1 - w) * want[j, i] + w * 0.25 * s if w != 1.0 else 0.25 * s
        assert np.allclose(a, want, rtol=0, atol=1e-9 * np.max(np.abs(want)))


def test_diagonal_order_differs_from_paper_order_only_in_rounding():
    m, n = 40, 31
    psi = wl.random_interior(wl.random_ring(m, n, seed=3), seed=4)
    a = ora.sor_sweep(psi, 1.7, 1.0, ora.RB, sum_order=ora.SUM_DIAGONAL)
    ref = ora.sor_sweep(psi, 1.7, 1.0, ora.RB)
    diff = np.max(np.abs(a - ref))
    assert 0.0 < diff <= 8 * np.finfo(float).eps * np.max(np.abs(ref))


def test_diagonal_order_converges_to_dense_solution_and_keeps_harmonics():
    for m, n in [(9, 9), (7, 5)]:
        psi = wl.random_ring(m, n, seed=200 + m)
        ref = exact.dense_solve(psi, 1.0)
        for method, w in ((ora.GS, 1.0), (ora.SOR, 1.4)):
            sol, info = ora.solve(psi, method=method, ordering=ora.RB, w=w, tol=1e-14,
                                  max_iter=20000, sum_order=ora.SUM_DIAGONAL)
            assert info["status"] == "converged"
            assert np.max(np.abs(sol - ref)) <= 1e-11
    # x^2 - y^2 on unit spacing is discrete-harmonic with exact sums: a fixed point
    m, n = 12, 9
    x, y = np.meshgrid(np.arange(m, dtype=float), np.arange(n, dtype=float))
    h = x ** 2 - y ** 2
    start = h.copy()
    start[1:-1, 1:-1] = 0.0
    sol, info = ora.solve(start, method=ora.SOR, ordering=ora.RB, w=1.5, tol=1e-15,
                          max_iter=20000, sum_order=ora.SUM_DIAGONAL)
    assert np.max(np.abs(sol - h)) <= 1e-9
    again = ora.sor_sweep(h, 1.5, 1.0, ora.RB, sum_order=ora.SUM_DIAGONAL)
    assert np.array_equal(again, h)


def test_diagonal_order_needs_unit_beta_and_a_point_method():
    psi = wl.random_ring(9, 9, seed=5)
    with pytest.raises(ValueError):
        ora.sor_sweep(psi, 1.5, 0.8, ora.RB, sum_order=ora.SUM_DIAGONAL)
    with pytest.raises(ValueError):
        ora.solve(psi, method=ora.MG, sum_order=ora.SUM_DIAGONAL)
    with pytest.raises(ValueError):
        ora.solve(psi, method=ora.SOR, w=1.5, dx=0.5, dy=1.0, sum_order=ora.SUM_DIAGONAL)


@pytest.mark.parametrize("w", [0.7, 1.0, 1.5, 1.9])
@pytest.mark.parametrize("order", [ora.SUM_PAPER, ora.SUM_DIAGONAL])
def test_sor_black_defect_is_one_minus_w_times_the_pass_defect(w, order):
    """Eq. 7 in red-black order: a black point's neighbours are all red, so during the black
    pass its defect is that of the field with the new reds and the old blacks, and after its
    update the defect is (1 - w) times that. Both fields' defects come from the oracle's
    residual, the sweep from its SOR; nothing here re-implements the update. A wrong blend
    (sign, w or 1 - w swapped), a colour swept twice or in the wrong order breaks it."""
    m, n = 23, 17
    psi0 = wl.random_interior(wl.random_ring(m, n, seed=60), seed=61)
    psi1 = ora.sor_sweep(psi0, w, 1.0, ora.RB, sum_order=order)
    jj, ii = np.meshgrid(np.arange(n), np.arange(m), indexing="ij")
    black = ((ii + jj) % 2 == 1)
    black[0, :] = black[-1, :] = black[:, 0] = black[:, -1] = False
    mid = np.where(black, psi0, psi1)  # new reds, old blacks (the ring is the same in both)
    r_pass = ora.defect(mid, beta=1.0)[black]
    r_after = ora.defect(psi1, beta=1.0)[black]
    scale = np.max(np.abs(r_pass))
    assert scale > 0
    assert np.max(np.abs(r_after - (1.0 - w) * r_pass)) <= 1e-13 * scale
