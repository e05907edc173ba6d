"""Pins of the network oracle (CPU): GELU closed forms, gradients against
central finite differences in float64, bfloat16 rounding."""
import numpy as np

from oracle import mlp_oracle as mo


def test_gelu_closed_forms():
    assert abs(mo.gelu(1.0) - 0.8413447460685429) < 1e-15          # Phi(1)
    assert abs(mo.gelu(-1.0) + 0.15865525393145707) < 1e-15
    assert mo.gelu(0.0) == 0.0 and abs(mo.gelu_d(0.0) - 0.5) < 1e-16
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    assert np.max(np.abs((mo.gelu(z + h) - mo.gelu(z - h)) / (2 * h) - mo.gelu_d(z))) < 1e-8


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, width, B = 8, 6, 5
    p = rng.standard_normal(mo.n_params(n_in, width)) * 0.5
    x = rng.standard_normal((B, n_in))
    t = rng.standard_normal(B)
    loss, g = mo.loss_and_grad(p, x, t, n_in, width)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p); e[i] = h
        fd[i] = (mo.loss_and_grad(p + e, x, t, n_in, width)[0] - mo.loss_and_grad(p - e, x, t, n_in, width)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-7 * max(1.0, np.max(np.abs(g)))
    y, _, _ = mo.forward(p, x, n_in, width)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-14


def test_bf16_rounding():
    # 8 significant bits: the spacing at 1 is 2^-7
    assert mo.to_bf16(1.0) == 1.0
    assert mo.to_bf16(1.0 + 2 ** -9) == 1.0                  # below half a spacing
    assert mo.to_bf16(1.0 + 2 ** -8) == 1.0                  # tie: to the even neighbour
    assert mo.to_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6    # tie: to the even neighbour (up)
    assert mo.to_bf16(1.0 + 5 * 2 ** -9) == 1.0 + 2 ** -7    # above half a spacing
    x = np.random.default_rng(1).standard_normal(1000)
    assert np.max(np.abs(mo.to_bf16(x) - x) / np.abs(x)) <= 2 ** -8
