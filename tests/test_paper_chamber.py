"""The oracle against the numbers the paper prints for its chamber problem
(tests/golden/paper_chamber.txt). The geometry figures are missing from the paper,
so the boundary follows the reading stated in the workloads module (psi = 1 on the
non-corner nodes of the bottom wall AB). Under that reading the optimal relaxation
factors of SOR, SLORB and ADI are reproduced exactly; iteration counts come out a
few per cent below the printed ones and are checked with a stated tolerance."""
import os

import numpy as np
import pytest

import oracle as ora
from paper_2208_02427_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_chamber.txt")
W_GRID = np.round(np.arange(1.0, 1.951, 0.05), 2)  # w swept 1.0..1.95 in steps of 0.05
PAPER_STOP = dict(dx=0.25, dy=0.25, norm=ora.NORM_MAXDELTA, tol=1e-9, max_iter=100000)
# the paper's own orderings: lexicographic points, successive lines
PAPER_METHODS = {
    "sor": dict(method=ora.SOR, ordering=ora.LEX),
    "slora": dict(method=ora.SLOR, form=ora.FORM_A, line_order=ora.LINES_SUCCESSIVE),
    "slorb": dict(method=ora.SLOR, form=ora.FORM_B, line_order=ora.LINES_SUCCESSIVE),
    "adi": dict(method=ora.ADI, form=ora.FORM_B, line_order=ora.LINES_SUCCESSIVE),
}


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            key, value = line.split()[:2]
            out[key] = value
    return out


def iterations(**kw):
    sol, info = ora.solve(wl.chamber(), **PAPER_STOP, **kw)
    return info["iters"] if info["status"] == "converged" else np.inf


@pytest.mark.parametrize("name", ["sor", "slorb", "adi"])
def test_optimal_relaxation_factor_matches_paper(name):
    its = [iterations(w=float(w), **PAPER_METHODS[name]) for w in W_GRID]
    assert W_GRID[int(np.argmin(its))] == float(golden()[f"opt_w.{name}"])


def test_unrelaxed_sor_is_gauss_seidel():
    g = golden()
    assert g["iters.sor_w1"] == g["iters.gs"]
    a, _ = ora.solve(wl.chamber(), method=ora.GS, ordering=ora.LEX, max_iter=40, tol=0.0)
    b, _ = ora.solve(wl.chamber(), method=ora.SOR, ordering=ora.LEX, w=1.0, max_iter=40, tol=0.0)
    assert np.array_equal(a, b)


def test_unrelaxed_iteration_counts_near_paper():
    g = golden()
    jac = iterations(method=ora.JACOBI)
    gs = iterations(method=ora.GS, ordering=ora.LEX)
    slor = iterations(method=ora.SLOR, w=1.0, **{k: v for k, v in PAPER_METHODS["slora"].items()
                                               if k != "method"})
    for ours, key in ((jac, "iters.jacobi"), (gs, "iters.gs"), (slor, "iters.slor_w1")):
        assert abs(ours / float(g[key]) - 1.0) < 0.07, (key, ours)
    # Jacobi needs about twice the Gauss-Seidel iterations
    assert abs(jac / gs - float(g["iters.jacobi"]) / float(g["iters.gs"])) < 0.05


def test_adi_beats_slorb_at_their_optima():
    g = golden()
    adi = iterations(w=float(g["opt_w.adi"]), **PAPER_METHODS["adi"])
    slorb = iterations(w=float(g["opt_w.slorb"]), **PAPER_METHODS["slorb"])
    paper = float(g["iters.adi_opt"]) / float(g["iters.slorb_opt"])
    assert adi < slorb and abs(adi / slorb - paper) < 0.1
    assert abs(adi / float(g["iters.adi_opt"]) - 1.0) < 0.1


def test_multigrid_levels_and_cycles():
    g = golden()
    sizes = []
    m, n = wl.CHAMBER_M, wl.CHAMBER_N
    for _ in range(ora.mg_levels(m, n, 5, 0)):
        sizes.append(f"{m}x{n}")
        m, n = (m - 1) // 2 + 1, (n - 1) // 2 + 1
    assert ",".join(sizes) == g["levels.mg"]
    # the paper's cycle: 3 Gauss-Seidel sweeps before and after, Gauss-Seidel on the
    # coarsest mesh until it stops changing
    cycles = iterations(method=ora.MG, nu1=3, nu2=3, ordering=ora.LEX, coarse=ora.COARSE_GS)
    assert abs(cycles - int(g["cycles.mg"])) <= 2


def test_divergence_is_reported():
    # SLORB beyond its stability limit (the product of its two roots exceeds one)
    _, info = ora.solve(wl.chamber(), w=1.95, **PAPER_STOP, **PAPER_METHODS["slorb"])
    assert info["status"] == "diverged"
    bad = wl.chamber()
    bad[0, 3] = np.nan
    for norm in (ora.NORM_MAXDELTA, ora.NORM_L2_REL):
        _, info = ora.solve(bad, method=ora.SOR, w=1.5, norm=norm, tol=1e-9, max_iter=50)
        assert info["status"] == "diverged"
