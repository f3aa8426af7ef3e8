"""What the trained surrogate gains over the simulator alone, end to end.

A miniature of the cement-hardening family (same six inputs, same source and
receiver placement relative to the cement top, 5 mm cells, 1200 steps, last
256 samples of 4 axis receivers): the simulator generates the training set
in one batched launch per kernel per step, the network is trained by the
library's own BF16 tensor-core kernels, the kNN gate decides per held-out
case whether the network's answer is trusted (5 % relative L2), and rejected
cases fall back to the simulator.  The test measures both routes on the
same held-out cases: accuracy against the simulator and wall time."""
import time

import numpy as np
import pytest

from paper_2302_13907_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 0.05
WINDOW = 256
STEPS = 1200


def mini_case(seed):
    sc = W.small_cement_case(seed, steps=STEPS)
    return sc, W.surrogate_features(sc)


def rel_err(pred, true):
    d = (pred - true).reshape(len(true), -1)
    t = true.reshape(len(true), -1)
    return np.linalg.norm(d, axis=1) / np.linalg.norm(t, axis=1)


def batch_traces(cases):
    from paper_2302_13907_gb300.binding import BatchSimulation
    with BatchSimulation(cases, graph_chunk=200, max_steps=STEPS) as b:
        b.run(STEPS)
        b.sync()
        return np.stack([b.traces(c)[:, STEPS - WINDOW:] for c in range(len(cases))])


def simulate_one(sc):
    from paper_2302_13907_gb300.binding import Simulation
    with Simulation(sc, graph_chunk=200, max_steps=STEPS) as s:
        s.step(STEPS)
        return s.traces()[:, STEPS - WINDOW:]


def test_surrogate_with_fallback_beats_the_plain_solver_at_stated_error():
    from paper_2302_13907_gb300.binding import Surrogate
    train = [mini_case(s) for s in range(192)]
    test = [mini_case(s) for s in range(5000, 5032)]
    X = np.stack([x for _, x in train])
    Y = batch_traces([sc for sc, _ in train])
    Xt = np.stack([x for _, x in test])

    # the method without the network: every held-out case simulated
    simulate_one(test[0][0])  # warm (library load, autotune cache)
    t0 = time.perf_counter()
    Yt = np.stack([simulate_one(sc) for sc, _ in test])
    t_plain = time.perf_counter() - t0

    rng = np.random.default_rng(0)
    perm = rng.permutation(len(X))
    iv, it = perm[:32], perm[32:]
    x_mean, x_scale = X[it].mean(axis=0), np.maximum(X[it].std(axis=0), 1e-12)
    y_scale = float(np.sqrt(np.mean(Y[it].astype(np.float64) ** 2)))
    arch = dict(in_dim=6, h1=64, h2=128, l0=16, chans=(32, 32, 16, 16, 8), out_ch=4)
    with Surrogate(max_batch=64, seed=5, **arch) as S:
        assert S.out_len == WINDOW
        S.set_normalization(x_mean, x_scale, y_scale)
        hist = S.train(X[it], Y[it], epochs=600, batch=16, lr=2e-3, seed=1)
        assert hist[-1] < 0.05 * hist[0]
        S.gate_fit(X[iv], rel_err(S.forward(X[iv]), Y[iv]))
        S.forward(Xt[:2])  # warm
        # the method with the network: surrogate answers, gate, simulator fallback
        t0 = time.perf_counter()
        P = S.forward(Xt)
        acc = S.gate(Xt, k=3, tol=TOL)
        for q in np.flatnonzero(~acc):
            P[q] = simulate_one(test[q][0])
        t_with = time.perf_counter() - t0
    e_net = rel_err(P, Yt)
    speedup = t_plain / t_with
    print(f"accepted {acc.mean():.2f}, accepted within 5 %: {np.mean(e_net[acc] <= TOL) if acc.any() else None}, "
          f"final within 5 %: {np.mean(e_net <= TOL + 1e-7):.2f}, plain {t_plain:.3f} s, "
          f"with surrogate {t_with:.3f} s, speedup {speedup:.2f}")
    assert acc.mean() >= 0.5
    assert np.mean(e_net[acc] <= TOL) >= 0.9
    assert np.mean(e_net <= TOL + 1e-7) >= 0.9
    assert speedup > 1.5
