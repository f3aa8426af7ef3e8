"""Storage precision on the GPU against the FP64 oracle: the Nz = 1024 crop of
the 20 m well (same rock noise), traces compared with the oracle traces
stored by tests/golden/make_crop_reference.py (a script that calls only the
oracle and the workload generator)."""
import hashlib
import os

import numpy as np
import pytest

from paper_2302_13907_gb300 import workloads as W
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu
REF = os.path.join(os.path.dirname(__file__), "golden", "crop1024_oracle_traces.npz")


def medium_hash(med):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(med.cell_id).tobytes())
    for a in (med.rho, med.vp, med.vs):
        h.update(np.ascontiguousarray(a, np.float64).tobytes())
    return h.hexdigest()


@pytest.fixture(scope="module")
def crop():
    if not os.path.exists(REF):
        pytest.skip("oracle reference traces not generated")
    ref = np.load(REF)
    sc = W.config3_crop()
    assert medium_hash(sc.medium) == str(ref["medium_sha256"]), "generator did not reproduce the reference medium"
    return sc, ref


def test_fp32_long_window_matches_oracle(crop):
    """20000 steps of the 13.2 M-cell crop in FP32: trace rel-L2 <= 1e-4."""
    from paper_2302_13907_gb300.binding import Simulation
    sc, ref = crop
    n = int(ref["steps"])
    with Simulation(sc, max_steps=n, graph_chunk=200) as s:
        assert s.dt == pytest.approx(float(ref["dt"]), rel=1e-14)
        s.step(n)
        got = s.traces()
    assert rel_l2(got, ref["traces"]) <= 1e-4


def test_reduced_storage_error_is_finite_and_ordered(crop):
    """BF16 / FP16 storage with FP32 arithmetic over the whole 20000-step
    window (the direct arrivals reach the receivers after about 4000 steps).
    A step changes a field by roughly 2 pi / (steps per source period) of its
    amplitude, about 0.2 % here, which is of the order of BF16's resolution
    (2^-8) and a few times FP16's (2^-11): increments are partly rounded away,
    so the error against the FP64 oracle is large, and larger for BF16 than
    for FP16.  The test pins that ordering and loose bounds around the
    measured values (BF16 about 0.7, FP16 about 0.13 relative L2);
    precision_report gives the per-receiver figures."""
    from paper_2302_13907_gb300.binding import Simulation
    sc, ref = crop
    n = int(ref["steps"])
    err = {}
    for storage in ("bf16", "f16"):
        with Simulation(sc, storage=storage, max_steps=n, graph_chunk=200) as s:
            s.step(n)
            got = s.traces()
        assert np.all(np.isfinite(got)), storage
        assert np.abs(got).max() > 0, storage
        err[storage] = rel_l2(got, ref["traces"])
    assert err["f16"] < err["bf16"], err
    assert err["f16"] <= 0.3 and err["bf16"] <= 1.0, err
