"""The surrogate's data generator on the GPU.

* The reach crop of a cement case (the z cells within 1.6 m of its source
  and receivers) reproduces the whole well's receiver traces over all 6000
  steps: a wave that leaves the span and returns travels at most
  5900 m/s x 0.486 ms = 2.87 m, so nothing outside the crop reaches the
  receivers inside the window, and the crop's end layers absorb what leaves.
* The refined-grid generator (the crop on the paper's azimuthally refined
  grid, sampled at the uniform grid's times) against the plain solver
  (uniform grid, whole well) on the reflected window: the two
  discretisations of the same well agree far within the surrogate's 5 %
  tolerance.
"""
import numpy as np
import pytest

from paper_2302_13907_gb300 import workloads as W
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1000, 9003])
def test_reach_crop_equals_the_whole_well(seed):
    from paper_2302_13907_gb300.binding import Simulation, time_step
    sc = W.scenario_case(seed, surrogate_inputs=True)
    crop = W.reach_crop(sc)
    assert crop.grid.nz < sc.grid.nz
    dt = time_step(sc)
    with Simulation(sc, graph_chunk=200) as a, Simulation(crop, graph_chunk=200, dt=dt) as b:
        a.step(sc.steps)
        b.step(sc.steps)
        ta, tb = a.traces(), b.traces()
    err = rel_l2(tb, ta)
    print(f"seed {seed}: crop {crop.grid.nz} of {sc.grid.nz} cells, traces rel-L2 {err:.2e}")
    assert err <= 1e-5, err


@pytest.mark.parametrize("seed", [1000, 9003])
def test_refined_window_against_the_plain_solver(seed):
    from paper_2302_13907_gb300.binding import Simulation
    from paper_2302_13907_gb300.surrogate_data import WINDOW, refined_window
    sc = W.scenario_case(seed, surrogate_inputs=True)
    with Simulation(sc, graph_chunk=200) as a:
        a.step(sc.steps)
        plain = a.traces()[:, sc.steps - WINDOW:]
    ref = refined_window(sc)
    assert ref.shape == plain.shape == (8, WINDOW)
    err = rel_l2(ref, plain)
    print(f"seed {seed}: refined-crop window vs plain solver rel-L2 {err:.3e}")
    assert err <= 0.01, err
