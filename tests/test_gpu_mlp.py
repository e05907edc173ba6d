"""The learned control variate: the network's GPU forward pass and gradients
against the CPU oracle (same bfloat16 rounding points, float64 arithmetic),
training on local energies the library computes, and the unbiased
control-variate estimator against the plain subsample estimator."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_2406_08314_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2406_08314_gb300 import build
    build.build()
    from paper_2406_08314_gb300 import cv, msd
    return msd, cv


def test_forward_and_gradients_match_oracle(mods):
    import torch
    msd, cv = mods
    n_in, width, B = 256, 256, 300          # B not a multiple of the 64-row padding
    net = cv.MLP(n_in, width, seed=3)
    rng = np.random.default_rng(4)
    p = net.params().astype(np.float64)
    p[-1] = 0.3
    p[width * n_in: width * n_in + width] = 0.05 * rng.standard_normal(width)   # nonzero biases
    net.set_params(p.astype(np.float32))
    p = net.params().astype(np.float64)
    x = rng.standard_normal((B, n_in)).astype(np.float32)
    t = rng.standard_normal(B).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = net.raw_forward(xd).cpu().numpy()
    y_ref, _, _ = mo.forward(p, x.astype(np.float64), n_in, width, bf16=True)
    assert np.max(np.abs(y - y_ref)) <= 2e-3 * np.max(np.abs(y_ref)), np.max(np.abs(y - y_ref))
    loss, g = net.grad(xd, td)
    g = g.cpu().numpy()
    loss_ref, g_ref = mo.loss_and_grad(p, x.astype(np.float64), t.astype(np.float64), n_in, width, bf16=True)
    assert abs(float(loss.item()) - loss_ref) <= 2e-3 * loss_ref
    # per parameter block: W0 b0 W1 b1 W2 b2 w3 b3
    sizes = [width * n_in, width, width * width, width, width * width, width, width, 1]
    off = 0
    for k, n in enumerate(sizes):
        a, b = g[off:off + n], g_ref[off:off + n]
        err = np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30)
        assert err <= 1e-2, (k, err)
        off += n


@pytest.fixture(scope="module")
def cu2o2_data(mods):
    """Reference-Green's-function features and exact local energies of
    walkers of the copper-oxo-shaped system near the trial, all computed by
    the library."""
    import torch
    msd, cv = mods
    s, _ = synth.config_system("cu2o2", seed=0, n_w=1)
    ctx = msd.Context(s, "mixed")
    rng = np.random.default_rng(11)
    feats, ens = [], []
    for _ in range(6):                      # 6 x 4096 walkers
        w = synth.make_walkers_varied(rng, s.M, s.n_alpha, s.n_beta, 4096, noise_range=(0.02, 0.15))
        da, db = torch.from_numpy(w.phi_a).cuda(), torch.from_numpy(w.phi_b).cuda()
        feats.append(ctx.features_rows(da, db))
        ens.append(ctx.local_energy(da, db).real.float())
    ctx.close()
    return torch.cat(feats), torch.cat(ens)


def test_training_and_control_variate(mods, cu2o2_data):
    """The trained surrogate on every walker plus the exact correction on a
    random eighth: unbiased, and far less variance than the exact local
    energy on the same eighth alone (the estimator without the network)."""
    msd, cv = mods
    x, e = cu2o2_data
    n_train = x.shape[0] - 4096
    net = cv.MLP(x.shape[1], 256, seed=1)
    hist = net.fit(x[:n_train], e[:n_train], epochs=20, batch=512, lr=1e-3, lr_final=3e-5,
                   val=(x[n_train:], e[n_train:]))
    assert hist[-1]["train_mse"] < 0.2 * hist[0]["train_mse"]
    f = net.predict(x[n_train:]).cpu().numpy()
    ex = e[n_train:].cpu().numpy()
    r2 = 1 - np.mean((f - ex) ** 2) / np.var(ex)
    study = cv.estimator_study(ex[:640], f[:640], frac=0.125, draws=4000, seed=2)
    print("train", hist[0], hist[-1], "r2", r2, "study", study)
    assert r2 > 0.8, r2
    assert study["variance_reduction"] > 5.0, study
    assert abs(study["cv_bias"]) < 5 * study["cv_bias_stderr"] + 1e-12, study


def test_control_variate_on_propagated_walkers(mods):
    """Training pairs from the method's own runs: two seeded phaseless AFQMC
    runs of the copper-oxo-shaped system (640 walkers x 20 steps, dt =
    0.005, msd_propagate); held out: a third run's walkers after 20 steps.
    The estimator stays unbiased and the surrogate removes most of the
    variance of the exact local energy."""
    import torch
    msd, cv = mods
    s, w0 = synth.config_system("cu2o2", seed=0, n_w=640)
    ctx = msd.Context(s, "mixed")
    xs, es = [], []
    for run in range(2):
        da, db = torch.from_numpy(w0.phi_a).cuda(), torch.from_numpy(w0.phi_b).cuda()
        x_r, e_r, w_r = cv.propagated_pairs(ctx, da, db, 20, dt=0.005, seed=run)
        assert x_r.shape[0] == 640 * 20 and torch.all(torch.isfinite(e_r))
        assert torch.all(w_r >= 0)
        xs.append(x_r)
        es.append(e_r)
    x, e = torch.cat(xs), torch.cat(es)
    net = cv.MLP(x.shape[1], 256, seed=1)
    net.fit(x, e, epochs=20, batch=512, lr=1e-3, lr_final=3e-5)
    da, db = torch.from_numpy(w0.phi_a).cuda(), torch.from_numpy(w0.phi_b).cuda()
    cv.propagated_pairs(ctx, da, db, 20, dt=0.005, seed=7)
    ex = ctx.local_energy(da, db).real.double().cpu().numpy()
    f = net.predict(ctx.features_rows(da, db)).double().cpu().numpy()
    ctx.close()
    study = cv.estimator_study(ex, f, frac=0.125, draws=4000, seed=2)
    print("propagated", study, "r2", 1 - np.mean((f - ex) ** 2) / np.var(ex))
    assert abs(study["cv_bias"]) < 5 * study["cv_bias_stderr"] + 1e-12, study
    assert study["variance_reduction"] > 2.0, study
