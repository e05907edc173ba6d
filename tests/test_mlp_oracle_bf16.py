"""The control-variate network oracle's BF16 mode against PyTorch on the CPU:
its rounding (round to nearest, ties to even) against torch's bfloat16
conversion, and its loss and gradients against automatic differentiation
of the same network in float64 with the values rounded at the same points:
the input, the hidden-layer weights and activations (straight through for
the gradient), and the hidden pre-activation gradients that enter matrix
products (a gradient hook on the product, so that the bias gradient stays
unrounded). A rounding point that the oracle misses or adds shows up as a
mismatch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_oracle as mo


def _bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


def test_rounding_matches_torch_bfloat16():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))
    # exact ties of the 8-bit mantissa, both parities
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 2.0 + 2.0 ** -7])
    for v in (x, ties):
        want = _bf16(torch.from_numpy(v.astype(np.float32).astype(np.float64))).numpy()
        assert np.array_equal(mo.to_bf16(v), want)


def _torch_loss_and_grad(p, x, t, n_in, width):
    W0, b0, W1, b1, W2, b2, w3, b3 = [torch.tensor(a, dtype=torch.float64, requires_grad=True)
                                      for a in mo.unpack(p, n_in, width)]

    def st(v):   # rounded value, identity gradient
        return v + (_bf16(v) - v).detach()

    a = _bf16(torch.from_numpy(x))
    for W, b in ((W0, b0), (W1, b1), (W2, b2)):
        zw = a @ st(W).T
        zw.register_hook(lambda g: _bf16(g))      # rounded for the products, not for the bias
        z = zw + b
        a = st(0.5 * z * (1.0 + torch.erf(z / np.sqrt(2.0))))
    y = a @ w3 + b3[0]
    loss = torch.mean((y - torch.from_numpy(t)) ** 2)
    loss.backward()
    g = torch.cat([W0.grad.reshape(-1), b0.grad, W1.grad.reshape(-1), b1.grad, W2.grad.reshape(-1), b2.grad,
                   w3.grad, b3.grad])
    return loss.item(), g.numpy()


@pytest.mark.parametrize("n_in,width,batch,seed", [(7, 16, 5, 1), (12, 32, 9, 2)])
def test_bf16_loss_and_gradients_match_autograd(n_in, width, batch, seed):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mo.n_params(n_in, width)) * 0.3
    x = rng.standard_normal((batch, n_in))
    t = rng.standard_normal(batch)
    loss, g = mo.loss_and_grad(p, x, t, n_in, width, bf16=True)
    tl, tg = _torch_loss_and_grad(p, x, t, n_in, width)
    assert abs(loss - tl) <= 1e-12 * abs(tl)
    assert np.allclose(g, tg, rtol=1e-10, atol=1e-12 * np.abs(tg).max())
    # the unrounded network differs: the rounding points matter at this size
    _, g64 = mo.loss_and_grad(p, x, t, n_in, width, bf16=False)
    assert not np.allclose(g64, tg, rtol=1e-6, atol=1e-6 * np.abs(tg).max())
