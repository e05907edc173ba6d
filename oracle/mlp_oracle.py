"""CPU oracle of the control-variate network (TEST INFRASTRUCTURE ONLY; the
library never calls it).

Network: x -> [W0, b0] -> GELU -> [W1, b1] -> GELU -> [W2, b2] -> GELU ->
[w3, b3] -> y, GELU(z) = z Phi(z), Phi the standard normal CDF; loss
(1/B) sum_b (y_b - t_b)^2. Forward and backward by the chain rule in
float64. With bf16=True the values are rounded to bfloat16 (round to
nearest, ties to even) at the points where the GPU kernels store bfloat16:
the input, the weights of the three hidden layers, every hidden activation
and every hidden pre-activation gradient used by a matrix product.
Parameter layout: W0 [w][n_in], b0 [w], W1 [w][w], b1, W2 [w][w], b2,
w3 [w], b3 [1].
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def to_bf16(a):
    """Round float64 values to bfloat16 (through float32), ties to even."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_d(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def unpack(p, n_in, width):
    shapes = [(width, n_in), (width,), (width, width), (width,), (width, width), (width,), (width,), (1,)]
    out, off = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        out.append(np.asarray(p[off:off + n], dtype=np.float64).reshape(sh))
        off += n
    assert off == len(p)
    return out


def n_params(n_in, width):
    return width * n_in + width + 2 * (width * width + width) + width + 1


def forward(p, x, n_in, width, bf16=False):
    W0, b0, W1, b1, W2, b2, w3, b3 = unpack(p, n_in, width)
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    a = r(x)
    zs, hs = [], [a]
    for W, b in ((W0, b0), (W1, b1), (W2, b2)):
        z = a @ r(W).T + b
        a = r(gelu(z))
        zs.append(z)
        hs.append(a)
    y = a @ w3 + b3[0]
    return y, zs, hs


def loss_and_grad(p, x, t, n_in, width, bf16=False):
    W0, b0, W1, b1, W2, b2, w3, b3 = unpack(p, n_in, width)
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, zs, hs = forward(p, x, n_in, width, bf16)
    B = x.shape[0]
    d = y - t
    loss = np.mean(d * d)
    dy = 2.0 * d / B
    g_w3 = hs[3].T @ dy
    g_b3 = np.array([dy.sum()])
    dz = np.outer(dy, w3) * gelu_d(zs[2])
    grads = {}
    Ws = [W0, W1, W2]
    for l in (2, 1, 0):
        grads[("W", l)] = r(dz).T @ hs[l]
        grads[("b", l)] = dz.sum(axis=0)
        if l:
            dh = r(dz) @ r(Ws[l])
            dz = dh * gelu_d(zs[l - 1])
    g = np.concatenate([grads[("W", 0)].ravel(), grads[("b", 0)], grads[("W", 1)].ravel(), grads[("b", 1)],
                        grads[("W", 2)].ravel(), grads[("b", 2)], g_w3, g_b3])
    return loss, g
