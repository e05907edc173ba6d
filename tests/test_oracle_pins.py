"""Pins of the CPU oracle against results fixed by the mathematics, not by the
oracle itself: brute-force Fock-space expectation values, the textbook
Slater-Condon rules, closed forms and invariants (CPU only)."""
import itertools

import numpy as np
import pytest

import oracle
from fock_brute import _annihilate, _create, brute_force
from tiny import tiny_system, tiny_walkers


def _rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


@pytest.mark.parametrize("M,na,nb,n_det,max_level,seed", [
    (5, 2, 2, None, None, 0),      # full CI space, 100 determinants
    (6, 3, 2, 60, None, 1),        # unequal spins, random subset up to quintuples
    (6, 2, 3, None, 3, 2),         # every determinant up to triples
])
def test_brute_force_fock(M, na, nb, n_det, max_level, seed):
    """O_T, E_L, the force-bias numerators and G_T equal brute-force
    <Psi_T|X|phi>/<Psi_T|phi> in Fock space (Sec. II A-B)."""
    sys = tiny_system(seed, M, na, nb, n_chol=3, n_det=n_det, max_level=max_level)
    pa, pb = tiny_walkers(seed, M, na, nb, n_w=1)
    ov, en, vb, G = brute_force(M, sys.h1, sys.e0, sys.L, sys.coeff, sys.occ_a, sys.occ_b,
                                pa[0], pb[0])
    out = oracle.msd(sys, pa, pb, energy=True, vbias=True, green=True)
    assert _rel(out["ovlp"][0], ov) < 1e-12
    assert abs(out["e_loc"][0] - en) < 1e-11 * max(1.0, abs(en))
    assert _rel(out["vbias"][0], vb) < 1e-11
    assert _rel(out["G_T"][0], G) < 1e-11


def _eri(L):
    return np.einsum("gpq,grs->pqrs", L, L)


def _slater_condon(M, h, e0, eri, occ_a, occ_b, ref_a, ref_b):
    """<D_I|H|D_0> for orthonormal orbitals by the Slater-Condon rules, in
    spin orbitals (alpha p -> p, beta p -> M + p), [pq|rs] = (pq|rs) when
    p, q share a spin and r, s share a spin."""
    D0 = sorted(list(ref_a) + [M + p for p in ref_b])
    DI = sorted(list(occ_a) + [M + p for p in occ_b])
    spin = lambda x: x // M
    sp = lambda x: x % M

    def g(p, q, r, s):
        if spin(p) != spin(q) or spin(r) != spin(s):
            return 0.0
        return eri[sp(p), sp(q), sp(r), sp(s)]

    def hh(p, q):
        return h[sp(p), sp(q)] if spin(p) == spin(q) else 0.0

    holes = sorted(set(D0) - set(DI))
    parts = sorted(set(DI) - set(D0))
    mask0 = sum(1 << x for x in D0)
    if not holes:
        e = e0 + sum(hh(i, i) for i in D0)
        e += 0.5 * sum(g(i, i, j, j) - g(i, j, j, i) for i in D0 for j in D0)
        return e
    if len(holes) == 1:
        (i,), (a,) = holes, parts
        s1, m = _annihilate(mask0, i)
        s2, m = _create(m, a)
        assert m == sum(1 << x for x in DI)
        return s1 * s2 * (hh(a, i) + sum(g(a, i, j, j) - g(a, j, j, i) for j in D0))
    if len(holes) == 2:
        (i, j), (a, b) = holes, parts
        # |D_I> = sign * a+_a a+_b a_j a_i |D_0>
        s1, m = _annihilate(mask0, i)
        s2, m = _annihilate(m, j)
        s3, m = _create(m, b)
        s4, m = _create(m, a)
        assert m == sum(1 << x for x in DI)
        return s1 * s2 * s3 * s4 * (g(a, i, b, j) - g(a, j, b, i))
    return 0.0


def test_slater_condon_rules_match_brute_force():
    """The textbook rules used below agree with the Fock-space brute force."""
    from fock_brute import apply_one_body, apply_two_body, det_state, dot
    sys = tiny_system(3, 5, 2, 2, n_chol=2, n_det=40)
    eri = _eri(sys.L)
    ref_a, ref_b = sys.occ_a[0], sys.occ_b[0]
    d0 = det_state(5, ref_a, ref_b)
    hd0 = apply_one_body(d0, sys.h1[0], 5)
    vd0 = apply_two_body(d0, eri, 5)
    for oa, ob in zip(sys.occ_a, sys.occ_b):
        di = det_state(5, oa, ob)
        want = sys.e0 * dot(di, d0) + dot(di, hd0) + dot(di, vd0)
        got = _slater_condon(5, sys.h1[0], sys.e0, eri, oa, ob, ref_a, ref_b)
        assert abs(got - want) < 1e-12


def test_hartree_fock_closed_form():
    """N_det = 1 and phi = D0 R: E_L is the Hartree-Fock energy
    e0 + sum_i h_ii + 1/2 sum_ij (ii|jj) - 1/2 sum_{ij same spin} (ij|ji),
    and O_T = det(R_a) det(R_b), exactly (Sec. II A, single-determinant case)."""
    rng = np.random.default_rng(7)
    M, na, nb = 12, 4, 3
    sys = tiny_system(7, M, na, nb, n_chol=5, n_det=1)
    eri = _eri(sys.L)
    Ra = rng.standard_normal((na, na)) + 1j * rng.standard_normal((na, na))
    Rb = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
    pa = np.zeros((1, M, na), complex); pa[0, :na] = Ra
    pb = np.zeros((1, M, nb), complex); pb[0, :nb] = Rb
    out = oracle.msd(sys, pa, pb)
    h = sys.h1[0]
    occ = [(p, 0) for p in range(na)] + [(p, 1) for p in range(nb)]
    e = sys.e0 + sum(h[p, p] for p, _ in occ)
    for p, s in occ:
        for q, t in occ:
            e += 0.5 * eri[p, p, q, q]
            if s == t:
                e -= 0.5 * eri[p, q, q, p]
    assert abs(out["e_loc"][0] - e) < 1e-11 * abs(e)
    assert abs(out["ovlp"][0] - np.linalg.det(Ra) * np.linalg.det(Rb)) < 1e-12


def test_slater_condon_limit():
    """phi -> D0 R: E_L -> sum_I c_I <D_I|H|D0> / c_0 (Slater-Condon: only the
    reference, singles and doubles contribute) and O_T -> c_0 det R. The
    numerator and denominator are polynomials in eps; both are extrapolated
    to eps = 0 from eps = +-h, +-2h (error O(h^4))."""
    rng = np.random.default_rng(11)
    M, na, nb = 9, 3, 3
    sys = tiny_system(11, M, na, nb, n_chol=4, n_det=120, max_level=3)
    eri = _eri(sys.L)
    Ra = rng.standard_normal((na, na)) + 1j * rng.standard_normal((na, na))
    Rb = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
    Xa = rng.standard_normal((M, na)) + 1j * rng.standard_normal((M, na))
    Xb = rng.standard_normal((M, nb)) + 1j * rng.standard_normal((M, nb))

    def num_den(eps):
        pa = np.zeros((1, M, na), complex); pa[0, :na] = Ra; pa[0] += eps * Xa
        pb = np.zeros((1, M, nb), complex); pb[0, :nb] = Rb; pb[0] += eps * Xb
        out = oracle.msd(sys, pa, pb, vbias=False)
        return out["e_loc"][0] * out["ovlp"][0], out["ovlp"][0]

    hstep = 1e-3   # O(h^4) truncation ~1e-11; conditioning ~1/h^3 for triples
    vals = {e: num_den(e) for e in (hstep, -hstep, 2 * hstep, -2 * hstep)}
    ext = [(4 * (vals[hstep][k] + vals[-hstep][k]) - (vals[2 * hstep][k] + vals[-2 * hstep][k])) / 6
           for k in (0, 1)]
    detR = np.linalg.det(Ra) * np.linalg.det(Rb)
    sc = sum(c * _slater_condon(M, sys.h1[0], sys.e0, eri, oa, ob, sys.occ_a[0], sys.occ_b[0])
             for c, oa, ob in zip(sys.coeff, sys.occ_a, sys.occ_b))
    assert abs(ext[1] - sys.coeff[0] * detR) < 1e-9 * abs(detR)
    assert abs(ext[0] / ext[1] - sc / sys.coeff[0]) < 1e-9 * abs(sc / sys.coeff[0])


def test_green_function_idempotent_and_trace():
    """G_I^2 = G_I and tr G_I = N_s for every determinant; tr G_T = N_s."""
    sys = tiny_system(5, 10, 4, 3, n_chol=3, n_det=30)
    pa, pb = tiny_walkers(5, 10, 4, 3)
    for I in range(sys.n_det):
        _, _, G = oracle.det_terms(10, sys.occ_a[I], sys.occ_b[I], sys.h1, sys.e0, sys.L,
                                   pa[0], pb[0], want_g=True)
        for s, n in ((0, 4), (1, 3)):
            assert np.max(np.abs(G[s] @ G[s] - G[s])) < 1e-11
            assert abs(np.trace(G[s]) - n) < 1e-12
    GT = oracle.msd(sys, pa, pb, green=True)["G_T"][0]
    assert abs(np.trace(GT[0]) - 4) < 1e-12 and abs(np.trace(GT[1]) - 3) < 1e-12


def test_per_determinant_overlap_is_the_determinant():
    """O_I = det(phi_a[occ_a]) det(phi_b[occ_b]) (numpy's LU as the check)."""
    sys = tiny_system(9, 11, 5, 4, n_chol=2, n_det=50)
    pa, pb = tiny_walkers(9, 11, 5, 4, n_w=2)
    out = oracle.msd(sys, pa, pb, per_det=True, vbias=False)
    for w in range(2):
        for I in range(sys.n_det):
            want = np.linalg.det(pa[w][sys.occ_a[I]]) * np.linalg.det(pb[w][sys.occ_b[I]])
            assert abs(out["det_ovlp"][w, I] - want) < 1e-12 * max(1.0, abs(want))


def test_single_excitation_ratio_closed_form():
    """A single excitation h -> p relative to D0 has ratio
    O_I / O_0 = sign * G0[h, p], sign = (-1)^(number of orbitals of D0
    strictly between h and p)."""
    M, na, nb = 10, 4, 3
    sys = tiny_system(13, M, na, nb, n_chol=2, n_det=1)
    pa, pb = tiny_walkers(13, M, na, nb)
    occ0a, occ0b = list(range(na)), list(range(nb))
    O0, _, G0 = oracle.det_terms(M, occ0a, occ0b, sys.h1, sys.e0, sys.L, pa[0], pb[0], want_g=True)
    for h in range(na):
        for p in range(na, M):
            occ = sorted(set(occ0a) - {h} | {p})
            OI, _ = oracle.det_terms(M, occ, occ0b, sys.h1, sys.e0, sys.L, pa[0], pb[0])
            sign = (-1) ** sum(1 for x in occ0a if h < x < p)
            assert abs(OI / O0 - sign * G0[0, h, p]) < 1e-12


def test_invariance_under_right_rotation():
    """phi -> phi R leaves E_L, the force bias and G_T unchanged and scales
    O_T by det R_a det R_b (a walker is a subspace; Sec. II A)."""
    rng = np.random.default_rng(17)
    M, na, nb = 10, 4, 3
    sys = tiny_system(17, M, na, nb, n_chol=4, n_det=40)
    pa, pb = tiny_walkers(17, M, na, nb)
    Ra = rng.standard_normal((na, na)) + 1j * rng.standard_normal((na, na))
    Rb = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
    a = oracle.msd(sys, pa, pb, green=True)
    b = oracle.msd(sys, pa @ Ra, pb @ Rb, green=True)
    assert abs(b["ovlp"][0] - a["ovlp"][0] * np.linalg.det(Ra) * np.linalg.det(Rb)) \
        < 1e-11 * abs(b["ovlp"][0])
    assert abs(a["e_loc"][0] - b["e_loc"][0]) < 1e-11 * abs(a["e_loc"][0])
    assert _rel(b["vbias"], a["vbias"]) < 1e-11
    assert _rel(b["G_T"], a["G_T"]) < 1e-11


def test_invariance_under_ci_permutation_and_real_walkers():
    """Reordering the CI list changes nothing; real walkers give real
    outputs."""
    M, na, nb = 9, 3, 3
    sys = tiny_system(19, M, na, nb, n_chol=3, n_det=45)
    pa, pb = tiny_walkers(19, M, na, nb, n_w=2)
    a = oracle.msd(sys, pa, pb)
    perm = np.random.default_rng(0).permutation(sys.n_det)
    sys2 = tiny_system(19, M, na, nb, n_chol=3, n_det=45)
    sys2.coeff, sys2.occ_a, sys2.occ_b = sys.coeff[perm], sys.occ_a[perm], sys.occ_b[perm]
    b = oracle.msd(sys2, pa, pb)
    for k in ("ovlp", "e_loc", "vbias"):
        assert _rel(b[k], a[k]) < 1e-12
    ra, rb = tiny_walkers(19, M, na, nb, n_w=2, real=True)
    c = oracle.msd(sys, ra, rb)
    for k in ("ovlp", "e_loc", "vbias"):
        assert np.max(np.abs(c[k].imag)) == 0.0


def test_golden_small_workload():
    """The oracle reproduces its stored outputs on the small workload
    (written by tests/golden/make_golden.py, which calls only the oracle)."""
    import json
    import os
    from paper_2406_08314_gb300 import synth
    doc = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "small_oracle.json")))
    s, w = synth.config_system("small", seed=0)
    out = oracle.msd(s, w.phi_a, w.phi_b)
    c = lambda v: np.array([x[0] + 1j * x[1] for x in v])
    assert _rel(out["ovlp"], c(doc["ovlp"])) < 1e-12
    assert _rel(out["e_loc"], c(doc["e_loc"])) < 1e-12
    assert _rel(out["vbias"][0], c(doc["vbias_w0"])) < 1e-12
