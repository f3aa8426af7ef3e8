"""FP64 reference of the trace surrogate's forward and backward pass.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): the CUDA surrogate
kernels are checked against it; it shares no code with them.

Network (inputs normalised by the caller):
    h1 = gelu(x W1 + b1)                      6 -> H1
    h2 = gelu(h1 W2 + b2)                     H1 -> H2
    a0 = gelu(reshape(h2 W3 + b3, [L0, C0]))  H2 -> L0 x C0 (channels last)
    a_{l+1} = gelu(convT(a_l; W_l, b_l))      5 transposed convolutions,
                                              kernel 4, stride 2, padding 1:
                                              length doubles, C_l -> C_{l+1}
    y = a_5 Wf + bf                           1x1 convolution C_5 -> 8,
                                              output [8][L0 * 32]
gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).

Transposed convolution, written from its definition: for every input
position s and tap q the input x[s, :] W[:, :, q] lands on output position
t = 2 s - 1 + q (positions outside [0, L_out) are dropped).

Parameter vector order: W1, b1, W2, b2, W3, b3, then (W_l [C_l][C_{l+1}][4],
b_l) for each transposed convolution, then Wf [C_5][8], bf.
Loss: mean over the batch and all outputs of (y - target)^2.

Optimiser: Adam (Kingma and Ba, 2015, Algorithm 1), written out in
`adam_step`: first and second moment estimates with decay rates beta1,
beta2, bias-corrected by 1 - beta^t, step lr * m_hat / (sqrt(v_hat) + eps).
"""
from __future__ import annotations

import numpy as np

SQ2PI = np.sqrt(2.0 / np.pi)


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(SQ2PI * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    u = SQ2PI * (x + 0.044715 * x ** 3)
    t = np.tanh(u)
    du = SQ2PI * (1.0 + 3 * 0.044715 * x ** 2)
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * du


def shapes(in_dim=6, h1=256, h2=512, c0=64, l0=64, chans=(64, 64, 32, 32, 16), out_ch=8):
    s = [("W1", (in_dim, h1)), ("b1", (h1,)), ("W2", (h1, h2)), ("b2", (h2,)), ("W3", (h2, l0 * c0)),
         ("b3", (l0 * c0,))]
    cin = c0
    for i, c in enumerate(chans):
        s += [(f"T{i}", (cin, c, 4)), (f"t{i}", (c,))]
        cin = c
    s += [("Wf", (cin, out_ch)), ("bf", (out_ch,))]
    return s


def unpack(theta, shp):
    out, o = {}, 0
    for name, sh in shp:
        n = int(np.prod(sh))
        out[name] = theta[o:o + n].reshape(sh)
        o += n
    assert o == theta.size
    return out


def conv_t(x, W, b):
    """x [B, L, Cin], W [Cin, Cout, 4] -> [B, 2L, Cout], by the definition."""
    B, L, _ = x.shape
    y = np.zeros((B, 2 * L, W.shape[1])) + b
    for q in range(4):
        contrib = np.einsum("bsc,cd->bsd", x, W[:, :, q])
        t = 2 * np.arange(L) - 1 + q
        ok = (t >= 0) & (t < 2 * L)
        y[:, t[ok], :] += contrib[:, ok, :]
    return y


def conv_t_backward(x, W, dy):
    B, L, _ = x.shape
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for q in range(4):
        t = 2 * np.arange(L) - 1 + q
        ok = (t >= 0) & (t < 2 * L)
        g = np.zeros((B, L, W.shape[1]))
        g[:, ok, :] = dy[:, t[ok], :]
        dx += np.einsum("bsd,cd->bsc", g, W[:, :, q])
        dW[:, :, q] += np.einsum("bsc,bsd->cd", x, g)
    return dx, dW, dy.sum(axis=(0, 1))


def _ident(a):
    return a


def forward(theta, x, shp, c0=64, l0=64, keep=False, q=_ident):
    """`q` is applied to every operand of a contraction (identity: exact FP64;
    a BF16 rounding reproduces the rounding points of a BF16 implementation)."""
    P = unpack(theta, shp)
    cache = {}
    xq = q(x)
    z1 = xq @ P["W1"] + P["b1"]
    h1 = q(gelu(z1))
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = q(gelu(z2))
    z3 = (h2 @ P["W3"] + P["b3"]).reshape(x.shape[0], l0, c0)
    a = q(gelu(z3))
    cache.update(x=xq, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, a=[a], z=[])
    i = 0
    while f"T{i}" in P:
        z = conv_t(a, P[f"T{i}"], P[f"t{i}"])
        a = q(gelu(z))
        cache["z"].append(z)
        cache["a"].append(a)
        i += 1
    y = a @ P["Wf"] + P["bf"]  # [B, L, 8]
    y = np.transpose(y, (0, 2, 1))  # [B, 8, L]
    return (y, cache) if keep else y


def loss_and_grad(theta, x, target, shp, c0=64, l0=64, q=_ident):
    y, c = forward(theta, x, shp, c0, l0, keep=True, q=q)
    P = unpack(theta, shp)
    n = y.size
    loss = np.sum((y - target) ** 2) / n
    dy = 2.0 * (y - target) / n
    dy = np.transpose(dy, (0, 2, 1))  # [B, L, 8]
    G = {}
    a = c["a"][-1]
    G["bf"] = dy.sum(axis=(0, 1))
    dyq = q(dy)
    G["Wf"] = np.einsum("blc,blo->co", a, dyq)
    da = dyq @ P["Wf"].T
    nT = len(c["z"])
    for i in reversed(range(nT)):
        dz = da * gelu_grad(c["z"][i])
        G[f"t{i}"] = dz.sum(axis=(0, 1))
        dx, G[f"T{i}"], _ = conv_t_backward(c["a"][i], P[f"T{i}"], q(dz))
        da = dx
    dz3 = (da * gelu_grad(c["z3"])).reshape(x.shape[0], -1)
    G["b3"] = dz3.sum(axis=0)
    dz3 = q(dz3)
    G["W3"] = c["h2"].T @ dz3
    dh2 = dz3 @ P["W3"].T
    dz2 = dh2 * gelu_grad(c["z2"])
    G["b2"] = dz2.sum(axis=0)
    dz2 = q(dz2)
    G["W2"] = c["h1"].T @ dz2
    dh1 = dz2 @ P["W2"].T
    dz1 = dh1 * gelu_grad(c["z1"])
    G["b1"] = dz1.sum(axis=0)
    G["W1"] = c["x"].T @ q(dz1)
    grad = np.concatenate([G[name].ravel() for name, _ in shp])
    return loss, grad


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1 (Kingma and Ba, Algorithm 1), FP64.
    Returns the new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return w - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
