"""Storage precision of the mixed solver's coarse levels (CPU model, tests/precision_model.py).

The design keeps every level of the inner V-cycle in FP32. BF16 storage for the coarse
levels would halve their bytes, but it has to leave the refined result within 1e-10 of the
FP64 solver's. These tests record the measurement behind that choice, on the 513^2
sine-edge problem at the 1e-10 stopping rule:
* FP32 cycles track the FP64 cycles one for one (7 iterations, iterates within 1e-14),
  which is what the GPU solver shows too;
* BF16 coarse levels still converge, but slow each cycle on smooth modes: the solve takes
  one iteration more (8), and after the FP64 solver's 7 cycles the iterate is 3e-10 away from
  the FP64 one, outside the 1e-10 bar. So BF16 buys no accuracy-neutral bandwidth, and the
  coarse levels it would shrink are latency-bound anyway (the FP32 tile kernels)."""
import numpy as np
import pytest

from paper_2208_02427_gb300 import workloads as wl
from tests import precision_model as pm


@pytest.fixture(scope="module")
def runs():
    psi = wl.sine_edges(513, 513, seed=wl.SEED_BASE + 1)
    out = {}
    for name, dtype, store in (("fp64", np.float64, None), ("fp32", np.float32, None),
                               ("bf16", np.float32, pm.to_bf16)):
        out[name] = pm.mixed_solve(psi, dtype, store)
        out[name + "_at7"] = pm.mixed_solve(psi, dtype, store, tol=0.0, max_iter=7)[0]
    return out


def test_bf16_rounding_is_round_to_nearest_even():
    # BF16 keeps 7 fraction bits: the spacing above 1 is 2^-7
    x = np.array([1.0, 1.0 + 2.0**-8, 1.0 + 3 * 2.0**-9, 1.0 + 2.0**-9, 1.0 + 3 * 2.0**-8, -2.5],
                 np.float32)
    want = [1.0,               # exact
            1.0,               # halfway between 1 and 1 + 2^-7: to the even one, 1
            1.0 + 2.0**-7,     # above halfway
            1.0,               # below halfway
            1.0 + 2.0**-6,     # halfway between 1 + 2^-7 and 1 + 2^-6: to the even one
            -2.5]              # exact
    got = pm.to_bf16(x)
    assert got.tolist() == want
    assert np.all(pm.to_bf16(got) == got)  # idempotent


def test_fp32_cycles_track_fp64_cycles(runs):
    p64, h64 = runs["fp64"]
    p32, h32 = runs["fp32"]
    assert len(h64) == len(h32) == 7
    assert np.max(np.abs(p32 - p64)) / np.max(np.abs(p64)) < 1e-13


def test_bf16_coarse_levels_miss_the_bar(runs):
    p64, h64 = runs["fp64"]
    pbf, hbf = runs["bf16"]
    assert hbf[-1] <= 1e-10  # it converges ...
    assert len(hbf) == len(h64) + 1  # ... one iteration later
    scale = np.max(np.abs(runs["fp64_at7"]))
    gap = np.max(np.abs(runs["bf16_at7"] - runs["fp64_at7"])) / scale
    assert gap > 1e-10  # outside the bar after the FP64 solver's cycles
    assert np.max(np.abs(runs["fp32_at7"] - runs["fp64_at7"])) / scale < 1e-13
