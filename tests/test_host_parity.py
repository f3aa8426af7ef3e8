"""Host-side parity of the library with the oracle, without a GPU: the
refined grid's interface maps, which the library's host code builds from the
closed form of trigonometric interpolation (simr_interface_matrix makes no
device call) and the oracle builds by the paper's DFT steps (Sec. 3)."""
import numpy as np
import pytest

import oracle
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

