"""Pins of the FP64 surrogate reference (oracle/surrogate_ref.py): library
routines (PyTorch CPU, float64) for the transposed convolution, GELU and the
whole forward pass; brute-force loops; central finite differences."""
import numpy as np
import pytest

from oracle import surrogate_ref as R

torch = pytest.importorskip("torch")
TINY = dict(in_dim=6, h1=8, h2=12, c0=4, l0=4, chans=(4, 4, 3, 3, 2), out_ch=8)


def tiny_theta(seed=0):
    shp = R.shapes(**TINY)
    n = sum(int(np.prod(s)) for _, s in shp)
    return shp, np.random.default_rng(seed).standard_normal(n) * 0.4


def test_conv_t_matches_brute_force_and_library():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 5, 3))
    W = rng.standard_normal((3, 4, 4))
    b = rng.standard_normal(4)
    y = R.conv_t(x, W, b)
    # brute force from the definition t = 2 s - 1 + q
    ref = np.zeros((2, 10, 4)) + b
    for bb in range(2):
        for s in range(5):
            for q in range(4):
                t = 2 * s - 1 + q
                if 0 <= t < 10:
                    ref[bb, t] += x[bb, s] @ W[:, :, q]
    assert np.allclose(y, ref, atol=1e-13)
    lib = torch.nn.functional.conv_transpose1d(torch.tensor(x).permute(0, 2, 1), torch.tensor(W), torch.tensor(b),
                                               stride=2, padding=1)
    assert np.allclose(y, lib.permute(0, 2, 1).numpy(), atol=1e-13)


def test_gelu_matches_library():
    x = np.linspace(-6, 6, 1001)
    lib = torch.nn.functional.gelu(torch.tensor(x), approximate="tanh").numpy()
    assert np.allclose(R.gelu(x), lib, atol=1e-15)
    # derivative by central differences
    h = 1e-6
    assert np.allclose(R.gelu_grad(x), (R.gelu(x + h) - R.gelu(x - h)) / (2 * h), atol=1e-8)


def test_forward_matches_library_network():
    shp, th = tiny_theta(2)
    P = R.unpack(th, shp)
    x = np.random.default_rng(3).standard_normal((3, 6))
    y = R.forward(th, x, shp, c0=TINY["c0"], l0=TINY["l0"])
    F = torch.nn.functional
    t = lambda a: torch.tensor(a)
    h = F.gelu(F.linear(t(x), t(P["W1"]).T, t(P["b1"])), approximate="tanh")
    h = F.gelu(F.linear(h, t(P["W2"]).T, t(P["b2"])), approximate="tanh")
    z = F.linear(h, t(P["W3"]).T, t(P["b3"])).reshape(3, TINY["l0"], TINY["c0"]).permute(0, 2, 1)
    a = F.gelu(z, approximate="tanh")
    for i in range(5):
        a = F.gelu(F.conv_transpose1d(a, t(P[f"T{i}"]), t(P[f"t{i}"]), stride=2, padding=1), approximate="tanh")
    out = F.conv1d(a, t(P["Wf"]).T.unsqueeze(-1), t(P["bf"]))
    assert out.shape == (3, 8, TINY["l0"] * 32)
    assert np.allclose(y, out.numpy(), atol=1e-12)


def test_gradient_matches_finite_differences():
    shp, th = tiny_theta(4)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 6))
    target = rng.standard_normal((2, 8, TINY["l0"] * 32))
    loss, g = R.loss_and_grad(th, x, target, shp, c0=TINY["c0"], l0=TINY["l0"])
    idx = rng.choice(th.size, size=60, replace=False)
    h = 1e-6
    for q in idx:
        tp, tm = th.copy(), th.copy()
        tp[q] += h
        tm[q] -= h
        lp, _ = R.loss_and_grad(tp, x, target, shp, c0=TINY["c0"], l0=TINY["l0"])
        lm, _ = R.loss_and_grad(tm, x, target, shp, c0=TINY["c0"], l0=TINY["l0"])
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(fd)), (q, fd, g[q])


def test_full_size_parameter_count():
    n = sum(int(np.prod(s)) for _, s in R.shapes())
    assert 2.0e6 < n < 2.6e6  # "~2M parameters"


def test_adam_step_matches_torch_optim_adam():
    """Three Adam steps of the reference against torch.optim.Adam (float64,
    beta = (0.9, 0.999), eps = 1e-8) on changing gradients."""
    rng = np.random.default_rng(5)
    w0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) * s for s in (1.0, 0.3, 2.0)]
    lr = 1e-2
    p = torch.nn.Parameter(torch.tensor(w0, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        w, m, v = R.adam_step(w, g, m, v, t, lr)
        assert np.allclose(w, p.detach().numpy(), rtol=1e-13, atol=1e-15), t
