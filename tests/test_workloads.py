"""The seeded input generators follow their stated recipes (CPU): the fields the parity tests
and the bench feed to both the oracle and the CUDA path are what the workload descriptions
say they are."""
import numpy as np
import pytest

from paper_2208_02427_gb300 import workloads as wl


def test_chamber_is_the_papers_problem():
    """25 x 17; psi = 1 on the 23 non-corner nodes of the bottom wall AB, 0 elsewhere (the
    Problem Definition read as psi = 1 on AB); the second set adds the same top wall."""
    psi = wl.chamber()
    assert psi.shape == (17, 25)
    assert np.array_equal(psi[0, 1:24], np.ones(23))
    assert psi.sum() == 23.0
    sym = wl.chamber(symmetric=True)
    assert np.array_equal(sym[16], sym[0]) and sym.sum() == 46.0


@pytest.mark.parametrize("m,n", [(65, 33), (129, 129), (257, 65)])
def test_sine_edges_carry_their_sine_series(m, n):
    """Each edge is sum_k a_k sin(k pi s) with the drawn a_k: DST-I orthogonality on the
    m - 1 intervals recovers the coefficients from the bottom and top edges (and from the
    left and right ones on n - 1); corners and interior are 0; |a_k| <= 1."""
    seed = wl.SEED_BASE + 1
    psi = wl.sine_edges(m, n, seed=seed)
    a = wl.sine_coefficients(seed)
    assert np.all(np.abs(a) <= 1.0)
    assert np.all(psi[1:-1, 1:-1] == 0.0)
    assert psi[0, 0] == psi[0, -1] == psi[-1, 0] == psi[-1, -1] == 0.0

    def coefficients(edge, length):
        s = np.arange(length) / (length - 1)
        k = np.arange(1, wl.N_MODES + 1)[:, None]
        return 2.0 / (length - 1) * (np.sin(np.pi * k * s) @ edge)

    for e, edge, length in ((0, psi[0, :], m), (1, psi[-1, :], m), (2, psi[:, 0], n), (3, psi[:, -1], n)):
        assert np.allclose(coefficients(edge, length), a[e], atol=1e-12), e


def test_generators_are_deterministic_per_seed():
    for make in (lambda s: wl.sine_edges(33, 17, seed=s), lambda s: wl.random_ring(33, 17, s),
                 lambda s: wl.random_interior(wl.random_ring(9, 9, 1), s)):
        assert np.array_equal(make(7), make(7))
        assert not np.array_equal(make(7), make(8))
    assert wl.batch_shapes(64, seed=3) == wl.batch_shapes(64, seed=3)


def test_random_ring_is_uniform_on_the_ring_and_zero_inside():
    psi = wl.random_ring(65, 33, seed=11)
    ring = np.concatenate([psi[0], psi[-1], psi[1:-1, 0], psi[1:-1, -1]])
    assert ring.size == 2 * 65 + 2 * 31
    assert np.all((ring >= 0.0) & (ring < 1.0))
    assert abs(ring.mean() - 0.5) < 0.1 and len(np.unique(ring)) == ring.size
    assert np.all(psi[1:-1, 1:-1] == 0.0)


def test_batch_shapes_follow_the_batched_workload():
    """m, n in {2^k + 1 : k = 5..9}, k drawn independently and redrawn while the aspect ratio
    exceeds 4; every k occurs on both axes."""
    shapes = wl.batch_shapes(4096, seed=wl.SEED_BASE + 2)
    assert len(shapes) == 4096
    sides = {33, 65, 129, 257, 513}
    assert all(m in sides and n in sides for m, n in shapes)
    assert all(max(m - 1, n - 1) // min(m - 1, n - 1) <= 4 for m, n in shapes)
    assert {m for m, _ in shapes} == sides and {n for _, n in shapes} == sides


def test_optimal_sor_factor():
    """2 / (1 + sin(pi / (m - 1))) on square grids is the general formula with the Jacobi
    radius rho = cos(pi / (m - 1)); 4097^2 gives 1.998467 and the chamber 1.7152 (the paper's
    grid search lands on 1.75)."""
    assert wl.w_opt_sor(4097, 4097) == pytest.approx(1.998467, abs=1e-6)
    rho = np.cos(np.pi / 4096)
    assert wl.w_opt_sor(4097, 4097) == pytest.approx(2 / (1 + np.sqrt(1 - rho * rho)), rel=1e-12)
    assert wl.w_opt_sor(25, 17) == pytest.approx(1.7152, abs=1e-4)
