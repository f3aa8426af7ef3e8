"""Surrogate kernels on the GPU against the FP64 reference (oracle/surrogate_ref.py)."""
import numpy as np
import pytest

from oracle import surrogate_ref as R

pytestmark = pytest.mark.gpu


def to_bf16_bits(a):
    """Round-to-nearest-even FP32 -> BF16 bit patterns."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return r


def bf16_value(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def bf16_round(a):
    a = np.asarray(a)
    return bf16_value(to_bf16_bits(a.astype(np.float32))).reshape(a.shape)


def cosine(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


@pytest.mark.parametrize("path", ["mma", "tcgen05"])
@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
@pytest.mark.parametrize("M,N,K", [(37, 70, 45), (128, 64, 32), (5, 3, 200), (300, 130, 17), (257, 300, 129),
                                   (1024, 16, 64)])
def test_tensor_core_gemm_against_fp64(path, ta, tb, M, N, K):
    """Both tensor-core kernels (mma.sync; tcgen05 with the accumulator in
    tensor memory) against the FP64 product of the same BF16 inputs, over
    every transpose combination and ragged M, N, K (tiles of 64 / 128)."""
    from paper_2302_13907_gb300.binding import gemm_bf16
    rng = np.random.default_rng(M * 7 + N + K)
    A = to_bf16_bits(rng.standard_normal((K, M) if ta else (M, K)))
    B = to_bf16_bits(rng.standard_normal((N, K) if tb else (K, N)))
    C = gemm_bf16(A, B, ta, tb, path=path)
    a, b = bf16_value(A), bf16_value(B)
    ref = (a.T if ta else a) @ (b.T if tb else b)
    assert np.abs(C - ref).max() <= 1e-5 * np.abs(ref).max() * max(1.0, K / 64)


def _bf16_theta(th, shp):
    """Weight matrices rounded to BF16 (as the GPU's GEMMs see them), biases FP32."""
    out = th.astype(np.float64).copy()
    o = 0
    for name, sh in shp:
        n = int(np.prod(sh))
        if len(sh) > 1:
            out[o:o + n] = bf16_value(to_bf16_bits(th[o:o + n]))
        o += n
    return out


def test_forward_and_gradient_match_fp64_reference():
    from paper_2302_13907_gb300.binding import Surrogate
    shp = R.shapes()
    rng = np.random.default_rng(11)
    X = rng.uniform(-1, 1, (4, 6)).astype(np.float32)
    with Surrogate(max_batch=8, seed=3) as s:
        th = s.params()
        assert th.size == sum(int(np.prod(x)) for _, x in shp)
        Y = s.forward(X)
        thb = _bf16_theta(th, shp)
        ref = R.forward(thb, X.astype(np.float64), shp)
        assert Y.shape == ref.shape == (4, 8, 2048)
        rel = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
        assert rel <= 2e-2, rel
        # a target near the output (a trained-network regime) and a random one
        for T in (ref * (1 + 0.1 * rng.standard_normal(ref.shape)),
                  rng.standard_normal(ref.shape) * np.abs(ref).max()):
            T = T.astype(np.float32)
            loss, g = s.loss_grad(X, T)
            lref, gref = R.loss_and_grad(thb, X.astype(np.float64), T.astype(np.float64), shp)
            # the same contraction operands rounded to BF16 as on the GPU
            lq, gq = R.loss_and_grad(thb, X.astype(np.float64), T.astype(np.float64), shp, q=bf16_round)
            assert abs(loss - lref) <= 2e-2 * lref
            per = {}
            o = 0
            for name, sh in shp:
                nn = int(np.prod(sh))
                a, b, c = g[o:o + nn], gq[o:o + nn], gref[o:o + nn]
                per[name] = (cosine(a, b), cosine(a, c))
                o += nn
            assert cosine(g, gq) >= 0.999, per
            assert min(v[0] for v in per.values()) >= 0.99, per
            assert cosine(g, gref) >= 0.99, per


def test_training_reduces_loss_on_a_smooth_map():
    from paper_2302_13907_gb300.binding import Surrogate
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, (64, 6)).astype(np.float32)
    t = np.linspace(0, 1, 2048)
    # a smooth family of damped oscillations parameterised by the inputs
    Y = np.stack([[np.sin(2 * np.pi * (3 + x[0] + 0.3 * c) * t + x[1]) * np.exp(-t * (1 + x[2] ** 2))
                   for c in range(8)] for x in X]).astype(np.float32)
    with Surrogate(max_batch=32, seed=7) as s:
        hist = s.train(X, Y, epochs=40, batch=16, lr=2e-3, seed=1)
        assert np.all(np.isfinite(hist))
        assert hist[-1] < 0.5 * hist[0], hist


def test_forward_elementwise_against_bf16_rounded_reference():
    """The GPU forward pass element by element against the FP64 reference
    that rounds every contraction operand to BF16 where the GPU does (weights,
    inputs, activations): what is left is FP32 accumulation and FP32 GELU,
    plus the rare activation that FP32 and FP64 round to neighbouring BF16
    values."""
    from paper_2302_13907_gb300.binding import Surrogate
    shp = R.shapes()
    rng = np.random.default_rng(12)
    X = rng.uniform(-1, 1, (6, 6)).astype(np.float32)
    with Surrogate(max_batch=8, seed=4) as s:
        th = s.params()
        Y = s.forward(X).astype(np.float64)
    ref = R.forward(_bf16_theta(th, shp), X.astype(np.float64), shp, q=bf16_round)
    ref_exact = R.forward(_bf16_theta(th, shp), X.astype(np.float64), shp)
    err = np.abs(Y - ref)
    scale = np.abs(ref).max()
    rel = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    rel_exact = np.linalg.norm(ref_exact - ref) / np.linalg.norm(ref)
    print(f"forward: max elementwise {err.max() / scale:.3e} of max, rel-L2 {rel:.3e}; "
          f"unrounded reference {rel_exact:.3e}")
    assert err.max() <= 8e-3 * scale, err.max() / scale
    assert rel <= 2e-3, rel
    # the rounded reference is the closer one: BF16 rounding points are reproduced
    assert rel <= 0.5 * rel_exact, (rel, rel_exact)


def test_adam_steps_match_fp64_adam():
    """Two training steps on one sample (so the minibatch gradient is the one
    sur_loss_grad returns, bit for bit) against the FP64 Adam of the reference
    (beta = (0.9, 0.999), eps = 1e-8; learning rate lr on the first step of
    each one-epoch call of the cosine schedule): each FP32 weight within
    1e-6 of itself plus 1e-4 lr of the FP64 update."""
    from paper_2302_13907_gb300.binding import Surrogate
    rng = np.random.default_rng(21)
    X = rng.uniform(-1, 1, (1, 6)).astype(np.float32)
    T = (rng.standard_normal((1, 8, 2048)) * 0.05).astype(np.float32)
    lr = 1e-3
    with Surrogate(max_batch=4, seed=9) as s:
        w = s.params().astype(np.float64)
        m = np.zeros_like(w)
        v = np.zeros_like(w)
        for t in (1, 2):
            _, g = s.loss_grad(X, T)
            s.train(X, T, epochs=1, batch=1, lr=lr, seed=t)
            w_gpu = s.params().astype(np.float64)
            w_ref, m, v = R.adam_step(w, g.astype(np.float64), m, v, t, lr)
            bad = np.abs(w_gpu - w_ref) > 1e-6 * np.abs(w_ref) + 1e-4 * lr
            assert not bad.any(), (t, int(bad.sum()), float(np.abs(w_gpu - w_ref).max()))
            assert np.abs(w_gpu - w).max() > 0.5 * lr  # the step moved the weights
            w = w_gpu


def test_sensitivity_against_the_reference_network():
    """sur_sensitivity (the gate's second signal) against the same quantity
    from the FP64 reference with the GPU's BF16 rounding points: for each
    query the largest relative output change over moves of 0.1 along each
    input, over queries split across several device batches."""
    from paper_2302_13907_gb300.binding import Surrogate
    shp = R.shapes()
    rng = np.random.default_rng(13)
    X = rng.uniform(-1, 1, (10, 6)).astype(np.float32)
    with Surrogate(max_batch=4, seed=5) as s:
        th = s.params()
        sens = s.sensitivity(X, step=0.1)
    thb = _bf16_theta(th, shp)

    def f(x):
        return R.forward(thb, x.astype(np.float64), shp, q=bf16_round).reshape(len(x), -1)

    y0 = f(X)
    ref = np.zeros(len(X))
    for d in range(6):
        Xp = X.copy()
        Xp[:, d] += np.float32(0.1)  # the move as the library makes it, in FP32
        ref = np.maximum(ref, np.linalg.norm(f(Xp) - y0, axis=1) / np.linalg.norm(y0, axis=1))
    print("sensitivity", sens.round(4), "reference", ref.round(4))
    assert np.all(ref > 0)
    assert np.all(np.abs(sens - ref) <= 0.05 * ref + 1e-3), (sens, ref)
