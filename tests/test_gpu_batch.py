"""Batched uneven systems (msd_batch_*): one persistent launch for the
per-determinant terms of all systems, recorded as a CUDA graph. Results must
equal the per-system path (same arithmetic, same partial-sum slots) and the
oracle; graph replays must read the current contents of the walker buffers;
the autotuner must keep the results and reuse its cache."""
import numpy as np
import pytest

import oracle
from paper_2406_08314_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msd():
    from paper_2406_08314_gb300 import build
    build.build()
    from paper_2406_08314_gb300 import msd as m
    return m


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _np(t):
    return t.cpu().numpy()


def _systems(n, seed0, n_w):
    # the batched recipe (M uniform, N = M // 6 per spin, log-uniform N_det,
    # N_chol = 4 M) at sizes the oracle finishes quickly
    return synth.batched_systems(n_systems=n, seed0=seed0, n_w=n_w, m_range=(24, 60),
                                 det_range=(200, 3000))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_per_system_oracle_and_replays(msd, precision):
    import torch
    sysw = _systems(6, 100, 8)
    ctxs = [msd.Context(s, precision) for s, _ in sysw]
    walkers = [(_cuda(w.phi_a), _cuda(w.phi_b)) for _, w in sysw]
    batch = msd.Batch(ctxs)
    outs = batch.evaluate(walkers)
    torch.cuda.synchronize()
    assert batch.graph_ready()
    got = [tuple(_np(x) for x in o) for o in outs]
    for i, ((s, w), c, (a, b)) in enumerate(zip(sysw, ctxs, walkers)):
        o2, v2, e2 = (_np(x) for x in c.evaluate(a, b))
        o1, v1, e1 = got[i]
        assert np.allclose(e1, e2, rtol=1e-12, atol=0), i
        assert np.allclose(o1, o2, rtol=1e-12, atol=0), i
        assert np.allclose(v1, v2, rtol=1e-12, atol=1e-14 * np.abs(v2).max()), i
    # oracle on two walkers of three systems
    for i in (0, 2, 4):
        s, w = sysw[i]
        ref = oracle.msd(s, w.phi_a[:2], w.phi_b[:2], energy=True, vbias=True, per_det=True)
        cO = s.coeff[None, :] * ref["det_ovlp"]
        scale_e = np.sum(np.abs(cO * ref["det_e"]), axis=1) / np.abs(ref["ovlp"])
        tol = 1e-10 if precision == "fp64" else 2e-6
        assert np.all(np.abs(got[i][2][:2] - ref["e_loc"]) <= tol * scale_e), i
        assert np.all(np.abs(got[i][0][:2] - ref["ovlp"]) <= 1e-10 * np.sum(np.abs(cO), axis=1)), i
    # replay: new walkers written into the same buffers
    sysw2 = _systems(6, 100, 8)
    rng = np.random.default_rng(7)
    for (a, b), (s, w) in zip(walkers, sysw2):
        pa = synth.make_walkers(rng, s.M, s.n_alpha, s.n_beta, 8, noise=0.2)
        a.copy_(_cuda(pa.phi_a))
        b.copy_(_cuda(pa.phi_b))
    outs = batch.evaluate(walkers, outs)         # graph replay
    torch.cuda.synchronize()
    for i, (c, (a, b)) in enumerate(zip(ctxs, walkers)):
        o2, v2, e2 = (_np(x) for x in c.evaluate(a, b))
        assert np.allclose(_np(outs[i][2]), e2, rtol=1e-12, atol=0), i
        assert np.allclose(_np(outs[i][0]), o2, rtol=1e-12, atol=0), i
    batch.close()
    for c in ctxs:
        c.close()


def test_batch_autotune_keeps_results_and_caches(msd, tmp_path):
    import torch
    sysw = _systems(4, 200, 16)
    ctxs = [msd.Context(s, "mixed") for s, _ in sysw]
    walkers = [(_cuda(w.phi_a), _cuda(w.phi_b)) for _, w in sysw]
    batch = msd.Batch(ctxs)
    ref = [tuple(_np(x) for x in o) for o in batch.evaluate(walkers)]
    cache = tmp_path / "tune.txt"
    cfg = batch.autotune(walkers, cache_path=str(cache))
    assert cfg["tile_n"] in (128, 256) and cfg["ctas_per_sm"] in (1, 2, 4) and cfg["order"] in (0, 1, 2)
    assert cache.read_text().split()[1:4] == [str(cfg["tile_n"]), str(cfg["ctas_per_sm"]), str(cfg["order"])]
    out = batch.evaluate(walkers)
    torch.cuda.synchronize()
    for (o1, v1, e1), o in zip(ref, out):
        assert np.allclose(_np(o[2]), e1, rtol=1e-6, atol=0)
        assert np.allclose(_np(o[0]), o1, rtol=1e-12, atol=0)
    # a second batch with the same shapes takes the cached choice
    batch2 = msd.Batch(ctxs)
    batch2.set_config(128, 1, 0)
    assert batch2.autotune(walkers, cache_path=str(cache)) == cfg
    assert len(cache.read_text().strip().splitlines()) == 1
    batch.close()
    batch2.close()


def test_batch_at_spec_sizes(msd):
    """Systems of the batched workload's full size range (M up to 160,
    N_det up to 1e5, N_chol = 4 M): the batch against the per-system path on
    all walkers, and with each trial cut to a sample of 200 determinants
    against the oracle on two walkers."""
    import copy
    import torch
    sysw = synth.batched_systems(n_systems=4, seed0=11, n_w=16)
    Ms = [s.M for s, _ in sysw]
    dets = [s.n_det for s, _ in sysw]
    assert max(Ms) >= 120 and max(dets) >= 3e4, (Ms, dets)
    ctxs = [msd.Context(s, "mixed") for s, _ in sysw]
    walkers = [(_cuda(w.phi_a), _cuda(w.phi_b)) for _, w in sysw]
    batch = msd.Batch(ctxs)
    outs = batch.evaluate(walkers)
    torch.cuda.synchronize()
    for i, (c, (a, b)) in enumerate(zip(ctxs, walkers)):
        o2, v2, e2 = (_np(x) for x in c.evaluate(a, b))
        assert np.allclose(_np(outs[i][2]), e2, rtol=1e-12, atol=0), i
        assert np.allclose(_np(outs[i][0]), o2, rtol=1e-12, atol=0), i
        assert np.allclose(_np(outs[i][1]), v2, rtol=1e-12, atol=1e-14 * np.abs(v2).max()), i
    batch.close()
    for c in ctxs:
        c.close()
    # sampled trials at the same sizes against the oracle
    subs = []
    rng = np.random.default_rng(5)
    for s, w in sysw:
        idx = np.concatenate([[0], np.sort(rng.choice(np.arange(1, s.n_det), 199, replace=False))])
        t = copy.copy(s)
        t.coeff = np.ascontiguousarray(s.coeff[idx])
        t.occ_a = np.ascontiguousarray(s.occ_a[idx])
        t.occ_b = np.ascontiguousarray(s.occ_b[idx])
        subs.append((t, w))
    for precision, tol in (("fp64", 1e-10), ("mixed", 2e-6)):
        ctxs = [msd.Context(t, precision) for t, _ in subs]
        walkers = [(_cuda(w.phi_a[:2]), _cuda(w.phi_b[:2])) for _, w in subs]
        batch = msd.Batch(ctxs)
        outs = batch.evaluate(walkers)
        torch.cuda.synchronize()
        for i, (t, w) in enumerate(subs):
            ref = oracle.msd(t, w.phi_a[:2], w.phi_b[:2], energy=True, vbias=True, per_det=True)
            cO = t.coeff[None, :] * ref["det_ovlp"]
            scale_e = np.sum(np.abs(cO * ref["det_e"]), axis=1) / np.abs(ref["ovlp"])
            assert np.all(np.abs(_np(outs[i][2]) - ref["e_loc"]) <= tol * scale_e), (precision, i)
            assert np.all(np.abs(_np(outs[i][0]) - ref["ovlp"]) <= 1e-10 * np.sum(np.abs(cO), axis=1)), i
        batch.close()
        for c in ctxs:
            c.close()
