"""The copper-oxo-shaped system at N_det = 1e6 (the paper's largest
expansion, Sec. III) in the 10-walker regime: sampled per-determinant ratios
against the oracle's full determinants, additivity of the numerators over a
split of the determinant list (which ties the full-size sums to the subset
parity of the other tests), mixed against FP64, and a workspace budget that
splits the walkers into chunks without changing any result."""
import copy

import numpy as np
import pytest

import oracle
from paper_2406_08314_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def msd():
    from paper_2406_08314_gb300 import build
    build.build()
    from paper_2406_08314_gb300 import msd as m
    return m


@pytest.fixture(scope="module")
def big():
    return synth.config_system("cu2o2_1e6", seed=0, n_w=10)


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _np(t):
    return t.cpu().numpy()


def _subtrial(s, idx):
    t = copy.copy(s)
    t.coeff = np.ascontiguousarray(s.coeff[idx])
    t.occ_a = np.ascontiguousarray(s.occ_a[idx])
    t.occ_b = np.ascontiguousarray(s.occ_b[idx])
    return t


def test_1e6_sampled_ratios(msd, big):
    s, w = big
    assert s.n_det == 1000000
    ctx = msd.Context(s, "fp64")
    r = ctx.det_ratios(_cuda(w.phi_a), _cuda(w.phi_b))
    rng = np.random.default_rng(3)
    for wk in rng.choice(w.n_w, 3, replace=False):
        o0, _ = oracle.det_terms(s.M, s.occ_a[0], s.occ_b[0], s.h1, s.e0, s.L[:1], w.phi_a[wk], w.phi_b[wk])
        for I in rng.choice(s.n_det, 40, replace=False):
            oi, _ = oracle.det_terms(s.M, s.occ_a[I], s.occ_b[I], s.h1, s.e0, s.L[:1], w.phi_a[wk], w.phi_b[wk])
            assert abs(complex(r[wk, I].item()) - oi / o0) <= TOL * max(1, abs(oi / o0))
    ctx.close()


def test_1e6_additivity(msd, big):
    s, w = big
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    rng = np.random.default_rng(9)
    rest = rng.permutation(np.arange(1, s.n_det))
    A = np.concatenate([[0], np.sort(rest[: s.n_det // 2])])
    B = np.concatenate([[0], np.sort(rest[s.n_det // 2:])])
    tB = _subtrial(s, B)
    tB.coeff = tB.coeff.copy()
    tB.coeff[0] = 0.0
    res = {}
    for name, t in (("full", s), ("A", _subtrial(s, A)), ("B", tB)):
        ctx = msd.Context(t, "fp64")
        _, R = ctx.overlap(da, db, ratio_sum=True)
        e = ctx.local_energy(da, db)
        v = ctx.force_bias(da, db)
        res[name] = (_np(R), _np(e), _np(v))
        ctx.close()
    RA, eA, vA = res["A"]
    RB, eB, vB = res["B"]
    R, e, v = res["full"]
    assert np.allclose(RA + RB, R, rtol=1e-11, atol=0)
    canc = (np.abs(RA) + np.abs(RB)) / np.abs(R)
    e_comb = (eA * RA + eB * RB) / R
    assert np.all(np.abs(e_comb - e) <= 1e-10 * canc * (np.abs(eA) + np.abs(eB)))
    v_comb = (vA * RA[:, None] + vB * RB[:, None]) / R[:, None]
    assert np.all(np.abs(v_comb - v) <= 1e-10 * canc[:, None] * np.max(np.abs(v), axis=1, keepdims=True))


def test_1e6_mixed_against_fp64(msd, big):
    s, w = big
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    out = {}
    for prec in ("fp64", "mixed"):
        ctx = msd.Context(s, prec)
        ctx.set_timing(True)
        e, o = ctx.local_energy(da, db, ovlp=True)
        out[prec] = (_np(e), _np(o), _np(ctx.force_bias(da, db)))
        # ~80 determinants per string: the opposite-spin term over runs
        # sharing a string (projections)
        assert "k_pair_run" in ctx.kernel_stats() and "k_pair_cross" not in ctx.kernel_stats()
        ctx.close()
    (e64, o64, v64), (em, om, vm) = out["fp64"], out["mixed"]
    assert np.all(np.abs(em - e64) <= 1e-6), np.abs(em - e64).max()
    assert np.allclose(om, o64, rtol=1e-12, atol=0)
    assert np.all(np.abs(vm - v64).max(axis=1) <= 1e-4 * np.abs(v64).max(axis=1))


def test_1e6_workspace_budget(msd, big):
    """A workspace budget of a quarter of what the 10 walkers take at once
    forces walker chunks at N_det = 1e6; the per-walker workspace does not
    grow with N_det (it is set by the distinct strings, at most C(16, 8) =
    12870 per spin here), so every walker still fits, the workspace stays
    within the budget, and the results equal the unchunked ones."""
    s, w = big
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    ref = msd.Context(s, "mixed")
    e0, o0 = ref.local_energy(da, db, ovlp=True)
    assert ref.info("walker_chunk") == w.n_w
    full = ref.info("workspace_bytes")
    v0 = ref.force_bias(da, db)
    ref.close()
    budget = full // 4
    ctx = msd.Context(s, "mixed")
    ctx.set_workspace_limit(budget)
    e1, o1 = ctx.local_energy(da, db, ovlp=True)
    assert 1 <= ctx.info("walker_chunk") < w.n_w
    assert ctx.info("workspace_bytes") <= budget + (1 << 20)
    v1 = ctx.force_bias(da, db)
    ctx.close()
    assert np.allclose(_np(e1), _np(e0), rtol=1e-13, atol=0)
    assert np.allclose(_np(o1), _np(o0), rtol=1e-13, atol=0)
    assert np.allclose(_np(v1), _np(v0), rtol=1e-13, atol=0)


def test_1e6_pair_forms_agree(msd, big):
    """The three forms of the opposite-spin term at 1e6 determinants (runs
    with projections, per beta string, per determinant): the same sum in a
    different FP32 order."""
    s, w = big
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    ctx = msd.Context(s, "mixed")
    out = {}
    for form in (2, 1, 0):
        ctx.set_pair_form(form)
        out[form] = _np(ctx.local_energy(da, db))
    ctx.close()
    for form in (1, 0):
        assert np.all(np.abs(out[form] - out[2]) <= 1e-7), (form, np.abs(out[form] - out[2]).max())
