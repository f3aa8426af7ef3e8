"""Host logic of the surrogate pipeline (no GPU): the parameter layout, the
BF16 packing of the weights, the gate's nearest-neighbour rule and the
leave-one-out choice of its margin."""
import numpy as np
import pytest

from oracle import surrogate_ref as Ref
from paper_2302_13907_gb300 import surrogate_run as R
from paper_2302_13907_gb300.binding import SURROGATE_DEFAULT


def test_layout_matches_the_reference_network():
    assert R.surrogate_shapes(SURROGATE_DEFAULT) == Ref.shapes()


def test_bf16_packing_rounds_weights_and_keeps_biases():
    shp = R.surrogate_shapes(SURROGATE_DEFAULT)
    n = sum(int(np.prod(s)) for _, s in shp)
    th = np.random.default_rng(1).standard_normal(n).astype(np.float32)
    bits, b = R.pack_params(th, SURROGATE_DEFAULT)
    u = R.unpack_params(bits, b, SURROGATE_DEFAULT)
    o = 0
    torch = __import__("pytest").importorskip("torch")
    for _, s in shp:
        k = int(np.prod(s))
        seg, got = th[o:o + k], u[o:o + k]
        if len(s) > 1:  # round to nearest even, as torch's bfloat16 conversion
            ref = torch.from_numpy(seg).to(torch.bfloat16).to(torch.float32).numpy()
            assert np.array_equal(got, ref)
        else:
            assert np.array_equal(got, seg)
        o += k


def test_knn_worst_against_brute_force():
    rng = np.random.default_rng(2)
    Xr, e = rng.standard_normal((40, 6)), rng.random(40)
    Xq = rng.standard_normal((7, 6))
    got = R.knn_worst(Xq, Xr, e, 3)
    for q in range(7):
        d = [np.sum((Xq[q] - x) ** 2) for x in Xr]
        assert got[q] == max(e[np.argsort(d)[:3]])
    loo = R.knn_worst(Xr, Xr, e, 3, exclude_self=True)
    for q in range(40):
        d = [np.sum((Xr[q] - x) ** 2) if i != q else np.inf for i, x in enumerate(Xr)]
        assert loo[q] == max(e[np.argsort(d)[:3]])


def test_margin_is_the_largest_that_admits_no_bad_validation_case():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((60, 6))
    e = 0.01 + 0.02 * rng.random(60)
    e[5] = 0.08  # one case above the 5 % tolerance
    m = R.choose_margin(X, e, 3)
    worst = R.knn_worst(X, X, e, 3, exclude_self=True)
    assert np.all(e[worst <= m * R.TOL] <= R.TOL)
    if m < 1.0:  # the next step would admit a bad case
        assert np.any(e[worst <= (m + 0.05) * R.TOL] > R.TOL)
    e_ok = np.full(60, 0.01)
    assert R.choose_margin(X, e_ok, 3) == 1.0


def test_two_signal_gate_admits_no_bad_validation_case_and_uses_the_sensitivity():
    """choose_gate: whatever margin and bound it returns, the gate (neighbour
    rule leave one out, sensitivity bound) accepts no validation case above
    the tolerance and the reported share is the share it accepts; a bad case
    that sits among good neighbours but has a high sensitivity no longer
    forces the tiny margin the neighbour rule alone needs."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((200, 6))
    e = 0.005 + 0.005 * rng.random(200)
    sens = 0.01 + 0.01 * rng.random(200)
    e[[7, 60]] = [0.09, 0.12]       # two bad cases among good neighbours
    sens[[7, 60]] = [0.08, 0.11]    # with high sensitivity
    m, smax, acc = R.choose_gate(X, e, sens, 3)
    worst = R.knn_worst(X, X, e, 3, exclude_self=True)
    a = (worst <= m * R.TOL) & (sens <= smax)
    assert np.all(e[a] <= R.TOL)
    assert acc == pytest.approx(a.mean())
    assert smax < 0.08 and acc > 0.9
    m_knn = R.choose_margin(X, e, 3)
    assert m_knn < m
    assert acc > np.mean(worst <= m_knn * R.TOL)
    # no bad case at all: no bound needed
    m2, smax2, acc2 = R.choose_gate(X, np.full(200, 0.01), sens, 3)
    assert np.isinf(smax2) and acc2 == 1.0
