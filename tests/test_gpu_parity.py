"""CUDA path (through the C-ABI) against the CPU oracle, element by element on
the same seeded inputs. FP64 mode must match within 1e-10 relative to the
cancellation scale of each quantity:
  |dO_T|  <= 1e-10 * sum_I |c_I O_I|
  |dE_L|  <= 1e-10 * sum_I |c_I O_I E_I| / |O_T|
  |dv_g|  <= 1e-10 * (sum_I |c_I O_I| / |O_T|) * max_g |v_g|
  |dr_I|  <= 1e-10 * max(1, |r_I|)
"""
import numpy as np
import pytest

import oracle
from paper_2406_08314_gb300 import synth
from tiny import tiny_system, tiny_walkers

pytestmark = pytest.mark.gpu

TOL = 1e-10


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
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


def _ref(sys_, pa, pb):
    out = oracle.msd(sys_, pa, pb, energy=True, vbias=True, per_det=True)
    cO = sys_.coeff[None, :] * out["det_ovlp"]
    out["scale_o"] = np.sum(np.abs(cO), axis=1)
    out["scale_e"] = np.sum(np.abs(cO * out["det_e"]), axis=1) / np.abs(out["ovlp"])
    out["canc"] = out["scale_o"] / np.abs(out["ovlp"])
    return out


def _check_all(m, sys_, pa, pb, ref, precision="fp64", tol=TOL, tol_e=None):
    ctx = m.Context(sys_, precision)
    da, db = _cuda(pa), _cuda(pb)
    ov, rs = ctx.overlap(da, db, ratio_sum=True)
    ov = _np(ov)
    assert np.all(np.abs(ov - ref["ovlp"]) <= tol * ref["scale_o"]), \
        np.max(np.abs(ov - ref["ovlp"]) / ref["scale_o"])
    r, o0 = ctx.det_ratios(da, db, ref_ovlp=True)
    r = _np(r)
    want_r = ref["det_ovlp"] / ref["det_ovlp"][:, :1]
    assert np.all(np.abs(r - want_r) <= tol * np.maximum(1, np.abs(want_r))), \
        np.max(np.abs(r - want_r) / np.maximum(1, np.abs(want_r)))
    assert np.allclose(_np(o0), ref["det_ovlp"][:, 0], rtol=tol, atol=0)
    v = _np(ctx.force_bias(da, db))
    vt = tol * ref["canc"] * np.max(np.abs(ref["vbias"]), axis=1)
    assert np.all(np.abs(v - ref["vbias"]) <= vt[:, None]), \
        np.max(np.abs(v - ref["vbias"]) / vt[:, None] * tol)
    e, o2 = ctx.local_energy(da, db, ovlp=True)
    e = _np(e)
    te = (tol_e or tol) * ref["scale_e"]
    assert np.all(np.abs(e - ref["e_loc"]) <= te), np.max(np.abs(e - ref["e_loc"]) / ref["scale_e"])
    assert np.all(np.abs(_np(o2) - ref["ovlp"]) <= tol * ref["scale_o"])
    # the combined entry point shares the overlap part; same results
    o3, v3, e3 = (_np(x) for x in ctx.evaluate(da, db))
    assert np.allclose(e3, e, rtol=1e-14, atol=0) and np.allclose(o3, ov, rtol=1e-14, atol=0)
    assert np.allclose(v3, v, rtol=1e-13, atol=1e-15 * np.abs(v).max())
    ctx.close()
    return dict(e=e, v=v, ov=ov)


def test_small_workload_fp64(msd):
    s, w = synth.config_system("small", seed=0)
    ref = _ref(s, w.phi_a, w.phi_b)
    _check_all(msd, s, w.phi_a, w.phi_b, ref)


def _relabel(sys_, pa, pb, seed):
    """Permute orbital labels so the reference is not the first N orbitals."""
    perm = np.random.default_rng(seed).permutation(sys_.M)
    inv = np.argsort(perm)
    sys_.h1 = sys_.h1[:, perm][:, :, perm]
    sys_.L = np.ascontiguousarray(sys_.L[:, perm][:, :, perm])
    sys_.occ_a = np.sort(inv[sys_.occ_a], axis=1).astype(np.int32)
    sys_.occ_b = np.sort(inv[sys_.occ_b], axis=1).astype(np.int32)
    return sys_, np.ascontiguousarray(pa[:, perm]), np.ascontiguousarray(pb[:, perm])


@pytest.mark.parametrize("M,na,nb,n_det,max_level,seed", [
    (12, 5, 4, 150, 4, 0),
    (13, 7, 6, 300, 12, 1),     # levels up to 6 per spin
    (9, 1, 3, 40, None, 2),     # a single alpha electron
])
def test_tiny_systems_any_reference(msd, M, na, nb, n_det, max_level, seed):
    s = tiny_system(seed, M, na, nb, n_chol=7, n_det=n_det, max_level=max_level)
    pa, pb = tiny_walkers(seed, M, na, nb, n_w=3, noise=0.6)
    s, pa, pb = _relabel(s, pa, pb, seed)
    ref = _ref(s, pa, pb)
    _check_all(msd, s, pa, pb, ref)


def test_cu2o2_shaped_fp64(msd):
    s, w = synth.config_system("cu2o2", seed=0, n_w=2)
    ref = _ref(s, w.phi_a, w.phi_b)
    _check_all(msd, s, w.phi_a, w.phi_b, ref)


@pytest.fixture(scope="module")
def fe2s2():
    return synth.config_system("fe2s2", seed=0, n_w=640)


def _subtrial(s, idx):
    import copy
    t = copy.copy(s)
    t.coeff = np.ascontiguousarray(s.coeff[idx])
    t.occ_a = np.ascontiguousarray(s.occ_a[idx])
    t.occ_b = np.ascontiguousarray(s.occ_b[idx])
    return t


def test_fe2s2_shaped_subset_fp64(msd, fe2s2):
    """Full Hamiltonian, orbital and Cholesky sizes; 300 determinants drawn
    across all levels; 2 walkers."""
    s, w = fe2s2
    idx = np.concatenate([[0], np.sort(np.random.default_rng(5).choice(
        np.arange(1, s.n_det), 299, replace=False))])
    t = _subtrial(s, idx)
    pa, pb = w.phi_a[:2], w.phi_b[:2]
    ref = _ref(t, pa, pb)
    _check_all(msd, t, pa, pb, ref)


def test_fe2s2_full_size_sampled_ratios(msd, fe2s2):
    """Full size, bench launch configuration: sampled per-determinant ratios
    against the oracle's full N x N determinants."""
    s, w = fe2s2
    ctx = msd.Context(s, "fp64")
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    r = ctx.det_ratios(da, db)
    rng = np.random.default_rng(3)
    for wk in rng.choice(w.n_w, 3, replace=False):
        o0, _ = oracle.det_terms(s.M, s.occ_a[0], s.occ_b[0], s.h1, s.e0, s.L[:1],
                                 w.phi_a[wk], w.phi_b[wk])
        for I in rng.choice(s.n_det, 40, replace=False):
            oi, _ = oracle.det_terms(s.M, s.occ_a[I], s.occ_b[I], s.h1, s.e0, s.L[:1],
                                     w.phi_a[wk], w.phi_b[wk])
            got = complex(r[wk, I].item())
            assert abs(got - oi / o0) <= TOL * max(1, abs(oi / o0))
    ctx.close()


def test_fe2s2_full_size_additivity(msd, fe2s2):
    """Full size: the numerators sum_I c_I r_I (E_I, v_I) are additive over a
    split of the determinant list, so E_L and vbias of the full trial follow
    from two half trials (each keeps D0 first; the second with c_0 = 0)."""
    s, w = fe2s2
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
    e_comb = (eA * RA + eB * RB) / R
    canc = (np.abs(RA) + np.abs(RB)) / np.abs(R)
    assert np.all(np.abs(e_comb - e) <= 1e-10 * canc * (np.abs(eA) + np.abs(eB)))
    v_comb = (vA * RA[:, None] + vB * RB[:, None]) / R[:, None]
    assert np.all(np.abs(v_comb - v) <= 1e-10 * canc[:, None] * np.max(np.abs(v), axis=1, keepdims=True))


# ------------------------------------------------------------------ edges
def test_edge_cases(msd):
    s, w = synth.config_system("small", seed=1)
    ctx = msd.Context(s, "fp64")
    import torch
    empty = torch.empty((0, s.M, s.n_alpha), dtype=torch.complex128, device="cuda")
    empty_b = torch.empty((0, s.M, s.n_beta), dtype=torch.complex128, device="cuda")
    assert ctx.local_energy(empty, empty_b).shape == (0,)
    # singular reference block: walker orthogonal to the reference orbitals
    pa = w.phi_a[:2].copy()
    pa[1, : s.n_alpha, :] = 0.0
    with pytest.raises(msd.MSDError) as ei:
        ctx.local_energy(_cuda(pa), _cuda(w.phi_b[:2]))
    assert ei.value.name == "MSD_ERR_REF_SINGULAR"
    # opposite-spin form: -1, 0, 1 or 2
    with pytest.raises(msd.MSDError) as ei:
        ctx.set_pair_form(3)
    assert ei.value.name == "MSD_ERR_ARG"
    ctx.set_pair_form("auto")
    # unsorted occupations
    bad = s.occ_a.copy()
    bad[3] = bad[3][::-1]
    with pytest.raises(msd.MSDError) as ei:
        ctx.set_trial(s.coeff, bad, s.occ_b)
    assert ei.value.name == "MSD_ERR_ARG"
    ctx.close()


def test_single_determinant_and_host_buffers(msd):
    s, w = synth.config_system("small", seed=2)
    t = _subtrial(s, np.array([0]))
    ref = _ref(t, w.phi_a, w.phi_b)
    ctx = msd.Context(t, "fp64")
    e = ctx.local_energy(w.phi_a, w.phi_b)          # numpy in, numpy out (host path)
    assert isinstance(e, np.ndarray)
    assert np.all(np.abs(e - ref["e_loc"]) <= TOL * ref["scale_e"])
    v = ctx.force_bias(w.phi_a, w.phi_b)
    assert np.allclose(v, ref["vbias"], rtol=1e-10, atol=1e-12)
    ctx.close()


def test_walker_chunking_matches(msd):
    s, w = synth.config_system("cu2o2", seed=0, n_w=24)
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    ctx = msd.Context(s, "fp64")
    e1, v1 = _np(ctx.local_energy(da, db)), _np(ctx.force_bias(da, db))
    ctx.set_workspace_limit(4 << 20)                # forces several walker chunks
    e2 = _np(ctx.local_energy(da, db))
    assert ctx.info("walker_chunk") < 24
    v2 = _np(ctx.force_bias(da, db))
    assert ctx.info("walker_chunk") < 24
    assert np.allclose(e1, e2, rtol=1e-13, atol=0) and np.allclose(v1, v2, rtol=1e-13, atol=1e-15)
    ctx.close()


# ------------------------------------------------------------ mixed mode
# Mixed precision: the Cholesky contractions run as 3xTF32 on the tensor
# cores with FP32 accumulation and the per-determinant energy terms in FP32;
# the reference inverse, the minor determinants, the reference-determinant
# energy (its Cholesky sums by the exact-integer split on the tensor cores)
# and the reductions stay FP64-accurate. Stated bound:
#   |dE_L| <= 2e-6 * sum_I |c_I O_I E_I| / |O_T|  and  |dE_L| <= 1e-6 Ha,
#   |dv_g| <= 1e-4 * max_g |v_g|,  overlaps and ratios as in FP64 mode.
MIX_E_REL, MIX_E_ABS, MIX_V = 2e-6, 1e-6, 1e-4


def _check_mixed(m, sys_, pa, pb, ref, fused=True, per_beta=True, e_abs=MIX_E_ABS, tensor_gram=False):
    ctx = m.Context(sys_, "mixed")
    ctx.set_fused(fused)
    ctx.set_pair_form(per_beta)
    ctx.set_tensor_gram(tensor_gram)
    assert ctx.info("exact_reference") == 1
    da, db = _cuda(pa), _cuda(pb)
    e, o = ctx.local_energy(da, db, ovlp=True)
    e, o = _np(e), _np(o)
    de = np.abs(e - ref["e_loc"])
    assert np.all(de <= MIX_E_REL * ref["scale_e"]), np.max(de / ref["scale_e"])
    assert np.all(de <= e_abs), de.max()
    assert np.all(np.abs(o - ref["ovlp"]) <= TOL * ref["scale_o"])
    v = _np(ctx.force_bias(da, db))
    dv = np.abs(v - ref["vbias"]).max(axis=1) / np.abs(ref["vbias"]).max(axis=1)
    assert np.all(dv <= MIX_V), dv.max()
    r = _np(ctx.det_ratios(da, db))
    want_r = ref["det_ovlp"] / ref["det_ovlp"][:, :1]
    assert np.all(np.abs(r - want_r) <= TOL * np.maximum(1, np.abs(want_r)))
    ctx.close()


# fused: the energy's Cholesky contraction and its epilogue in one
# persistent tensor-core kernel (default); unfused: GEMM + epilogue kernel.
# pairY: the opposite-spin term formed per beta string (default); perdet:
# the double sum per determinant.
FUSED = pytest.mark.parametrize("fused,per_beta", [(True, True), (False, True), (True, False), (True, 2)],
                                ids=["fused-pairY", "unfused-pairY", "fused-perdet", "fused-runs"])


@FUSED
def test_small_workload_mixed(msd, fused, per_beta):
    s, w = synth.config_system("small", seed=0)
    _check_mixed(msd, s, w.phi_a, w.phi_b, _ref(s, w.phi_a, w.phi_b), fused, per_beta)


@FUSED
@pytest.mark.parametrize("M,na,nb,n_det,max_level,seed", [(12, 5, 4, 150, 4, 0), (13, 7, 6, 300, 12, 1)])
def test_tiny_systems_mixed(msd, M, na, nb, n_det, max_level, seed, fused, per_beta):
    s = tiny_system(seed, M, na, nb, n_chol=7, n_det=n_det, max_level=max_level)
    pa, pb = tiny_walkers(seed, M, na, nb, n_w=3, noise=0.3)
    s, pa, pb = _relabel(s, pa, pb, seed)
    # unnormalised N(0, 1) Cholesky vectors: local energies of 10-500 Ha with
    # large per-determinant corrections; the FP32 per-determinant terms hold
    # the relative bound here, not 1e-6 Ha (measured up to 6e-5 Ha)
    _check_mixed(msd, s, pa, pb, _ref(s, pa, pb), fused, per_beta, e_abs=np.inf)


@FUSED
def test_cu2o2_shaped_mixed(msd, fused, per_beta):
    s, w = synth.config_system("cu2o2", seed=0, n_w=2)
    _check_mixed(msd, s, w.phi_a, w.phi_b, _ref(s, w.phi_a, w.phi_b), fused, per_beta)


@FUSED
def test_fe2s2_shaped_subset_mixed(msd, fe2s2, fused, per_beta):
    s, w = fe2s2
    idx = np.concatenate([[0], np.sort(np.random.default_rng(6).choice(
        np.arange(1, s.n_det), 299, replace=False))])
    t = _subtrial(s, idx)
    pa, pb = w.phi_a[:2], w.phi_b[:2]
    _check_mixed(msd, t, pa, pb, _ref(t, pa, pb), fused, per_beta)


# Chemical energy scale: the Cholesky vectors scaled so that the mean
# on-site Coulomb integral (pp|pp) is 1 Ha (local energies of 5-500 Ha), and
# the slow-decay stress spectrum exp(-g / (N_chol / 6)), both without any
# rescaling of the inputs to fit the bound.
def test_small_workload_chemical_scale_mixed(msd):
    s, w = synth.config_system("small", seed=0, onsite=1.0)
    ref = _ref(s, w.phi_a, w.phi_b)
    assert np.abs(ref["e_loc"]).min() > 1.0
    _check_mixed(msd, s, w.phi_a, w.phi_b, ref)


def _fe2s2_subset(seed, n_w, **kw):
    s, w = synth.config_system("fe2s2", seed=0, n_w=n_w, **kw)
    idx = np.concatenate([[0], np.sort(np.random.default_rng(seed).choice(
        np.arange(1, s.n_det), 299, replace=False))])
    return _subtrial(s, idx), w


@pytest.mark.parametrize("kw", [dict(onsite=1.0), dict(decay=800 / 6), dict(decay=800 / 6, onsite=1.0)],
                         ids=["chemical", "slow-decay", "slow-decay-chemical"])
def test_fe2s2_subset_stress_mixed(msd, kw):
    t, w = _fe2s2_subset(6, 4, **kw)
    ref = _ref(t, w.phi_a, w.phi_b)
    _check_mixed(msd, t, w.phi_a, w.phi_b, ref)


def test_exact_reference_off_keeps_relative_bound(msd):
    """With the reference sums from the FP32 traces (msd_set_exact_reference
    0) the error grows with the energy scale: the relative bound still holds
    at chemical scale, the absolute one no longer does; switching back
    restores it."""
    t, w = _fe2s2_subset(6, 4, onsite=1.0)
    ref = _ref(t, w.phi_a, w.phi_b)
    ctx = msd.Context(t, "mixed")
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    ctx.set_exact_reference(False)
    assert ctx.info("exact_reference") == 0
    e_off = _np(ctx.local_energy(da, db))
    ctx.set_exact_reference(True)
    e_on = _np(ctx.local_energy(da, db))
    ctx.close()
    d_off, d_on = np.abs(e_off - ref["e_loc"]), np.abs(e_on - ref["e_loc"])
    assert np.all(d_off <= 20 * MIX_E_REL * ref["scale_e"])
    assert d_off.max() > MIX_E_ABS and np.all(d_on <= MIX_E_ABS)


@pytest.mark.parametrize("spin", [0, 1])
def test_one_spin_excitations_mixed(msd, spin):
    """Trial whose excited determinants all keep one spin's reference string:
    the opposite-spin term has nothing to add (the per-beta-string kernel
    still forms Y_b for the excited beta strings, then skips every
    determinant, or has no excited beta string at all)."""
    import copy
    s, w = synth.config_system("small", seed=3)
    # the trial's distinct strings of the other spin, each paired with this
    # spin's reference string (the reference determinant first)
    other = s.occ_b if spin == 0 else s.occ_a
    _, first = np.unique(other, axis=0, return_index=True)
    idx = np.sort(first)
    assert idx[0] == 0 and len(idx) > 5
    t = copy.copy(s)
    t.coeff = np.ascontiguousarray(s.coeff[idx])
    keep = (s.occ_a if spin == 0 else s.occ_b)[0]
    fixed = np.ascontiguousarray(np.repeat(keep[None, :], len(idx), axis=0))
    if spin == 0:
        t.occ_a, t.occ_b = fixed, np.ascontiguousarray(s.occ_b[idx])
    else:
        t.occ_a, t.occ_b = np.ascontiguousarray(s.occ_a[idx]), fixed
    pa, pb = w.phi_a[:4], w.phi_b[:4]
    _check_mixed(msd, t, pa, pb, _ref(t, pa, pb))


def test_fe2s2_full_size_mixed_vs_fp64(msd, fe2s2):
    """Full size, bench launch configuration (640 walkers, 1.2e5
    determinants): mixed against the FP64 GPU path, which the tests above
    tie to the oracle."""
    s, w = fe2s2
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    out = {}
    for prec in ("fp64", "mixed"):
        ctx = msd.Context(s, prec)
        e, o = ctx.local_energy(da, db, ovlp=True)
        v = ctx.force_bias(da, db)
        out[prec] = (_np(e), _np(o), _np(v))
        ctx.close()
    (e64, o64, v64), (em, om, vm) = out["fp64"], out["mixed"]
    assert np.all(np.abs(em - e64) <= MIX_E_ABS), np.abs(em - e64).max()
    assert np.allclose(om, o64, rtol=1e-12, atol=0)
    dv = np.abs(vm - v64).max(axis=1) / np.abs(v64).max(axis=1)
    assert np.all(dv <= MIX_V), dv.max()


def test_fe2s2_full_size_fused_matches_unfused(msd, fe2s2):
    """Full size (640 walkers, 800 Cholesky vectors, 1.2e5 determinants):
    the fused contraction + epilogue against the separate GEMM and epilogue
    kernels. Same TF32 splits and FP32 rounding points; only the order of
    the FP32 sums differs, so the local energies agree far inside the mixed
    bound."""
    s, w = fe2s2
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    ctx = msd.Context(s, "mixed")
    ctx.set_fused(False)
    e0 = _np(ctx.local_energy(da, db))
    ctx.set_fused(True)
    e1 = _np(ctx.local_energy(da, db))
    ctx.close()
    assert np.all(np.isfinite(e1))
    assert np.all(np.abs(e1 - e0) <= 0.1 * MIX_E_ABS), np.abs(e1 - e0).max()


def test_fe2s2_full_size_stream_overlap_identical(msd, fe2s2):
    """Full size, bench launch configuration: the energy's second stage on
    its own stream (the default) against every kernel on the caller's
    stream. The same kernels compute the same values in the same order, so
    overlaps, force biases and local energies agree bit for bit: with device
    buffers, with host buffers, and with walker chunks smaller than the
    batch (one fork and join per chunk)."""
    s, w = fe2s2
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    ctx = msd.Context(s, "mixed")
    ctx.set_stream_overlap(False)
    ref = [_np(x) for x in ctx.evaluate(da, db)]
    ctx.set_stream_overlap(True)
    for got in ([_np(x) for x in ctx.evaluate(da, db)],
                [_np(x) for x in ctx.evaluate(w.phi_a, w.phi_b)]):
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)
    ctx.set_workspace_limit(3 << 30)
    got = [_np(x) for x in ctx.evaluate(da, db)]
    assert ctx.info("walker_chunk") < 640
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    ctx.close()


def test_fe2s2_full_size_pair_forms_agree(msd, fe2s2):
    """Full size, bench launch configuration: the opposite-spin term over
    runs sharing a string (the default here), per beta string and per
    determinant. All FP32 with FP64 slot sums; only the order of the FP32
    sums differs."""
    s, w = fe2s2
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    ctx = msd.Context(s, "mixed")
    ctx.set_timing(True)
    ea = _np(ctx.local_energy(da, db))
    # ~10 determinants per string: the cost model prefers the runs form
    assert "k_pair_run" in ctx.kernel_stats() and "k_pair_y" not in ctx.kernel_stats()
    out = {}
    for form in (0, 1, 2):
        ctx.set_pair_form(form)
        out[form] = _np(ctx.local_energy(da, db))
    e2 = _np(ctx.local_energy(da, db))
    ctx.close()
    assert np.array_equal(ea, out[2]) and np.array_equal(e2, out[2])   # deterministic
    for form in (0, 1):
        assert np.all(np.isfinite(out[form]))
        assert np.all(np.abs(out[form] - out[2]) <= 0.1 * MIX_E_ABS), (form, np.abs(out[form] - out[2]).max())


def test_fe2s2_full_size_chemical_scale_mixed_vs_fp64(msd):
    """Full iron-sulfur size at chemical scale (|E_L| ~ 400 Ha), 64 walkers,
    all 1.2e5 determinants: mixed against the FP64 GPU path. The reference
    part is FP64-accurate; what remains comes from the FP32 per-determinant
    terms (measured max 3.1e-6 Ha, median 8e-7 Ha, a relative 8e-9)."""
    s, w = synth.config_system("fe2s2", seed=0, n_w=64, onsite=1.0)
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    out = {}
    for prec in ("fp64", "mixed"):
        ctx = msd.Context(s, prec)
        out[prec] = _np(ctx.local_energy(da, db))
        ctx.close()
    de = np.abs(out["mixed"] - out["fp64"])
    assert np.all(de <= 2e-8 * np.abs(out["fp64"])), (de / np.abs(out["fp64"])).max()
    assert np.median(de) <= 2e-6, np.median(de)


@pytest.mark.parametrize("name", ["small", "cu2o2"])
def test_tensor_gram_mixed(msd, name):
    """The Gram matrices on the tensor cores (transposed Lambda rows, 3xTF32
    products, one or two M-tiles) against the oracle: the small workload
    (2X = 50: one tile) and the copper-oxo-shaped one (2X = 128)."""
    s, w = synth.config_system(name, seed=0, n_w=2 if name == "cu2o2" else 16)
    _check_mixed(msd, s, w.phi_a, w.phi_b, _ref(s, w.phi_a, w.phi_b), tensor_gram=True)


def test_fe2s2_full_size_tensor_gram_matches_fma_gram(msd, fe2s2):
    """Full size: the Gram matrices on the tensor cores (3xTF32, FP32
    accumulation in TMEM) against the FP32-FMA kernel. Both are within
    FP32 rounding of each other, far inside the mixed bound."""
    s, w = fe2s2
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    ctx = msd.Context(s, "mixed")
    e0 = _np(ctx.local_energy(da, db))      # the default: FP32 FMAs
    ctx.set_tensor_gram(True)
    ctx.set_timing(True)
    e1 = _np(ctx.local_energy(da, db))
    assert ctx.kernel_stats()["tc_gram"][0] == 1
    ctx.close()
    assert np.all(np.isfinite(e1))
    assert np.all(np.abs(e1 - e0) <= 0.1 * MIX_E_ABS), np.abs(e1 - e0).max()
