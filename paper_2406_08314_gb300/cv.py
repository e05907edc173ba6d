"""Learned control variate for the local energy (the paper has no
counterpart): a small MLP f on features x of the reference Green's function
(its non-zero rows) predicts Re E_L; on a walker population the estimator

    E_cv = mean_i f(x_i) + mean_{i in S} (E_L,i - f(x_i)),

with S a uniform random subsample, is unbiased for mean_i E_L,i and needs the
exact local energy only on S. Training uses local energies the library
computes; every forward, backward and optimiser step runs in the library's
kernels (BF16 weights and activations, FP32 accumulation on the tensor
cores). Python here only loops, shuffles indices and marshals arguments.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import msd as _msd

_lib = _msd.lib()


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


class MLP:
    """msd_mlp: n_in -> 3 x width (GELU) -> 1."""

    def __init__(self, n_in: int, width: int = 256, device: int = 0, seed: int = 0):
        h = ctypes.c_void_p()
        rc = _lib.msd_mlp_create(ctypes.byref(h), n_in, width, device)
        if rc:
            raise _msd.MSDError(rc, "msd_mlp_create failed (n_in, width multiples of 64?)")
        self._h = h
        self.n_in, self.width, self.device = n_in, width, device
        self.n_params = int(_lib.msd_mlp_param_count(h))
        self.set_params(self.init_params(seed))
        # standardisation of the target (applied outside the network)
        self.t_mean, self.t_std = 0.0, 1.0

    def init_params(self, seed):
        """He-normal hidden weights, small output layer, zero biases."""
        rng = np.random.default_rng(seed)
        n, w = self.n_in, self.width
        parts = [rng.standard_normal(w * n) * np.sqrt(2.0 / n), np.zeros(w)]
        for _ in range(2):
            parts += [rng.standard_normal(w * w) * np.sqrt(2.0 / w), np.zeros(w)]
        parts += [rng.standard_normal(w) * np.sqrt(1.0 / w), np.zeros(1)]
        return np.concatenate(parts).astype(np.float32)

    def _check(self, rc):
        if rc:
            raise _msd.MSDError(rc, _lib.msd_mlp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _lib.msd_mlp_destroy(self._h)
            self._h = None

    __del__ = close

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.n_params
        self._check(_lib.msd_mlp_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p)))

    def params(self):
        p = np.empty(self.n_params, np.float32)
        self._check(_lib.msd_mlp_get_params(self._h, p.ctypes.data_as(ctypes.c_void_p)))
        return p

    def raw_forward(self, x, stream=None):
        import torch
        y = torch.empty((x.shape[0],), dtype=torch.float32, device=x.device)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream if stream is None else int(stream))
        self._check(_lib.msd_mlp_forward(self._h, x.shape[0], _vp(x), _vp(y), st))
        return y

    def predict(self, x, stream=None):
        """Predicted Re E_L (target units)."""
        return self.raw_forward(x, stream) * self.t_std + self.t_mean

    def grad(self, x, t, stream=None):
        import torch
        g = torch.empty((self.n_params,), dtype=torch.float32, device=x.device)
        loss = torch.empty((1,), dtype=torch.float32, device=x.device)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream if stream is None else int(stream))
        self._check(_lib.msd_mlp_grad(self._h, x.shape[0], _vp(x), _vp(t), _vp(g), _vp(loss), st))
        return loss, g

    def fit(self, x, e, epochs=30, batch=1024, lr=1e-3, lr_final=1e-4, seed=0, val=None):
        """Adam on the mean squared error of the standardised target.
        x: [n][n_in] FP32, e: [n] target (device tensors). Returns the
        per-epoch training loss (and validation loss if val=(xv, ev))."""
        import torch
        self.t_mean = float(e.mean())
        self.t_std = float(e.std()) or 1.0
        t = ((e - self.t_mean) / self.t_std).float().contiguous()
        n = x.shape[0]
        gen = torch.Generator(device=x.device)
        gen.manual_seed(seed)
        hist = []
        steps = epochs * ((n + batch - 1) // batch)
        k = 0
        loss = torch.empty((1,), dtype=torch.float32, device=x.device)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for ep in range(epochs):
            perm = torch.randperm(n, device=x.device, generator=gen)
            tot = torch.zeros((), dtype=torch.float64, device=x.device)
            for i in range(0, n, batch):
                idx = perm[i:i + batch]
                xb, tb = x[idx].contiguous(), t[idx].contiguous()
                rate = lr * (lr_final / lr) ** (k / max(1, steps - 1))
                self._check(_lib.msd_mlp_grad(self._h, xb.shape[0], _vp(xb), _vp(tb), None, _vp(loss), st))
                self._check(_lib.msd_mlp_adam_step(self._h, float(rate), 0.9, 0.999, 1e-8, st))
                tot += loss[0].double() * xb.shape[0]
                k += 1
            rec = {"epoch": ep, "train_mse": float(tot) / n}
            if val is not None:
                xv, ev = val
                pv = self.predict(xv)
                rec["val_mse_std"] = float(((pv - ev) / self.t_std).pow(2).mean())
            hist.append(rec)
        return hist


def cv_estimate(f_all, e_sub, f_sub):
    """Control-variate estimate of mean E_L: mean(f) + mean over the
    subsample of (E_L - f)."""
    return float(np.mean(f_all) + np.mean(np.asarray(e_sub) - np.asarray(f_sub)))


def estimator_study(e_all, f_all, frac=0.125, draws=4000, seed=0):
    """Bias and variance of the control-variate estimator against the plain
    subsample mean at the same number of exact evaluations, over random
    subsamples of one population (e_all exact, f_all surrogate)."""
    rng = np.random.default_rng(seed)
    e_all = np.asarray(e_all, np.float64)
    f_all = np.asarray(f_all, np.float64)
    n = e_all.size
    k = max(1, int(round(frac * n)))
    plain = np.empty(draws)
    cv = np.empty(draws)
    for d in range(draws):
        s = rng.choice(n, k, replace=False)
        plain[d] = e_all[s].mean()
        cv[d] = f_all.mean() + (e_all[s] - f_all[s]).mean()
    exact = e_all.mean()
    return {"n": n, "subsample": k, "exact_mean": exact,
            "plain_var": float(plain.var()), "cv_var": float(cv.var()),
            "variance_reduction": float(plain.var() / max(cv.var(), 1e-300)),
            "cv_bias": float(cv.mean() - exact), "cv_bias_stderr": float(cv.std() / np.sqrt(draws)),
            "plain_bias": float(plain.mean() - exact)}


def propagated_pairs(ctx, phi_a, phi_b, n_steps, dt=0.005, seed=0, qr_every=5, order=6):
    """Features and exact local energies of a walker population along a
    phaseless AFQMC run (msd_propagate: Gaussian fields, force bias,
    Taylor propagator, phaseless weights, a QR every qr_every steps; Sec.
    II A), one (features, Re E_L) pair per walker and step, all computed by
    the library on the device. phi_a, phi_b: device walkers (modified in
    place). Returns (features [n_steps n_w][ld] FP32, energies [n_steps n_w]
    FP32, weights [n_steps n_w] FP64)."""
    import torch
    n_w = phi_a.shape[0]
    gen = torch.Generator(device=phi_a.device)
    gen.manual_seed(int(seed))
    w = torch.ones(n_w, dtype=torch.float64, device=phi_a.device)
    xs, es, ws = [], [], []
    for step in range(n_steps):
        x = torch.randn((n_w, ctx.n_chol), dtype=torch.float64, device=phi_a.device, generator=gen)
        ctx.propagate(phi_a, phi_b, w, x, dt, order, (step + 1) % qr_every == 0)
        xs.append(ctx.features_rows(phi_a, phi_b))
        es.append(ctx.local_energy(phi_a, phi_b).real.float())
        ws.append(w.clone())
    return torch.cat(xs), torch.cat(es), torch.cat(ws)
