"""Host-side parity of the library with the oracle, without a GPU:

* the refined grid's interface maps, which the library's host code builds
  from the closed form of trigonometric interpolation (simr_interface_matrix
  makes no device call) and the oracle builds by the paper's DFT steps
  (Sec. 3);
* the time step (reading R7) the library's host code takes (sim_time_step,
  no device call) against the oracle's, on every workload family.
"""
import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import workloads as W


@pytest.mark.parametrize("na", [4, 8, 16, 32])
def test_library_interface_maps_equal_the_oracle(na):
    """The refined grid's host code builds its interface maps from the closed
    form (simr_interface_matrix, no device call); the oracle builds them by the
    paper's DFT steps.  Element by element, both staggerings and directions."""
    from paper_2302_13907_gb300 import binding as B
    nb = 2 * na
    for half in (False, True):
        P = np.stack([oracle.fft_interp(np.eye(na)[j], nb, half) for j in range(na)], axis=1)
        assert np.abs(B.interface_matrix(na, half, False) - P).max() < 1e-13
        assert np.abs(B.interface_matrix(na, half, True) - 0.5 * P.T).max() < 1e-13


@pytest.mark.parametrize("make", [W.config1, lambda: W.scenario_case(3), lambda: W.small_cement_case(5),
                                  lambda: W.reach_crop(W.scenario_case(4))])
def test_library_time_step_equals_the_oracle(make):
    """sim_time_step (host only) and the oracle's R7 time step agree bit for
    bit (the same formula, minimum over the same cells); a reach crop keeps
    the whole well's step (its axis ring limits both)."""
    from paper_2302_13907_gb300 import binding as B
    sc = make()
    assert B.time_step(sc) == oracle.cfl_dt(sc.medium, sc.cfl)
    assert B.time_step(sc, dt=1.5e-7) == 1.5e-7


def test_time_step_rejects_bad_input():
    from paper_2302_13907_gb300 import binding as B
    sc = W.config1()
    bad = W.Scenario("bad", W.Medium(sc.grid, sc.medium.cell_id, sc.medium.rho[:1], sc.medium.vp[:1],
                                     sc.medium.vs[:1]), sc.source, sc.receivers)
    with pytest.raises(B.SimError) as ei:
        B.time_step(bad)
    assert ei.value.code == B.SIM_EINVAL
