"""Brute-force Fock-space evaluation for tiny systems (pins the oracle).

Independent of the oracle: no determinants, no Green's functions, no Wick
theorem. States are dicts {bit mask: amplitude} over 2M spin orbitals
(alpha orbital p -> bit p, beta orbital p -> bit M + p); the basis state of a
mask is a+_{i1} a+_{i2} ... |0> with i1 < i2 < ..., and operators act with the
usual fermionic sign (-1)^(number of occupied spin orbitals below the index).

  walker  |phi> = prod_j (sum_p phi_a[p, j] a+_{p alpha})
                  prod_j (sum_p phi_b[p, j] a+_{p beta}) |0>
  trial   |D_I> = prod_{p in occ_a, ascending} a+_{p alpha}
                  prod_{p in occ_b, ascending} a+_{p beta} |0>
  H       = e0 + sum_{pq,s} h_pq a+_ps a_qs
            + 1/2 sum_{pqrs,st} (pq|rs) a+_ps a+_rt a_st a_qs,
  (pq|rs) = sum_g L^g_pq L^g_rs,  L_g-hat = sum_{pq,s} L^g_pq a+_ps a_qs.
"""
from __future__ import annotations

import numpy as np


def _annihilate(m, i):
    if not (m >> i) & 1:
        return 0, m
    sign = -1 if bin(m & ((1 << i) - 1)).count("1") & 1 else 1
    return sign, m ^ (1 << i)


def _create(m, i):
    if (m >> i) & 1:
        return 0, m
    sign = -1 if bin(m & ((1 << i) - 1)).count("1") & 1 else 1
    return sign, m | (1 << i)


def _add(out, m, v):
    out[m] = out.get(m, 0.0) + v


def apply_creation_sum(state, coeffs, offset):
    """(sum_p coeffs[p] a+_{offset + p}) |state>."""
    out = {}
    for m, a in state.items():
        for p, c in enumerate(coeffs):
            if c == 0:
                continue
            s, m2 = _create(m, offset + p)
            if s:
                _add(out, m2, s * c * a)
    return out


def walker_state(phi_a, phi_b):
    M = phi_a.shape[0]
    st = {0: 1.0 + 0.0j}
    # the rightmost factor acts first
    for j in reversed(range(phi_b.shape[1])):
        st = apply_creation_sum(st, phi_b[:, j], M)
    for j in reversed(range(phi_a.shape[1])):
        st = apply_creation_sum(st, phi_a[:, j], 0)
    return st


def det_state(M, occ_a, occ_b):
    st = {0: 1.0}
    for p in reversed(sorted(occ_b)):
        e = np.zeros(M); e[p] = 1.0
        st = apply_creation_sum(st, e, M)
    for p in reversed(sorted(occ_a)):
        e = np.zeros(M); e[p] = 1.0
        st = apply_creation_sum(st, e, 0)
    return st


def trial_state(M, coeff, occ_a, occ_b):
    out = {}
    for c, oa, ob in zip(coeff, occ_a, occ_b):
        for m, a in det_state(M, oa, ob).items():
            _add(out, m, c * a)
    return out


def dot(bra, ket):
    """<bra|ket> for a real-coefficient bra."""
    return sum(np.conj(a) * ket.get(m, 0.0) for m, a in bra.items())


def apply_one_body(state, X, M):
    """sum_{pq, s} X_pq a+_ps a_qs |state>."""
    out = {}
    for m, a in state.items():
        for sp in (0, M):
            for q in range(M):
                s1, m1 = _annihilate(m, sp + q)
                if not s1:
                    continue
                for p in range(M):
                    if X[p, q] == 0:
                        continue
                    s2, m2 = _create(m1, sp + p)
                    if s2:
                        _add(out, m2, X[p, q] * s1 * s2 * a)
    return out


def apply_excitation(state, p, q, spin, M):
    """a+_{p s} a_{q s} |state>."""
    off = spin * M
    out = {}
    for m, a in state.items():
        s1, m1 = _annihilate(m, off + q)
        if not s1:
            continue
        s2, m2 = _create(m1, off + p)
        if s2:
            _add(out, m2, s1 * s2 * a)
    return out


def apply_two_body(state, eri, M):
    """1/2 sum_{pqrs, st} (pq|rs) a+_ps a+_rt a_st a_qs |state>."""
    out = {}
    for m, a in state.items():
        for q_so in range(2 * M):
            s1, m1 = _annihilate(m, q_so)
            if not s1:
                continue
            sq, q = divmod(q_so, M)
            for s_so in range(2 * M):
                s2, m2 = _annihilate(m1, s_so)
                if not s2:
                    continue
                ss, s = divmod(s_so, M)
                for r in range(M):
                    s3, m3 = _create(m2, ss * M + r)
                    if not s3:
                        continue
                    for p in range(M):
                        v = eri[p, q, r, s]
                        if v == 0:
                            continue
                        s4, m4 = _create(m3, sq * M + p)
                        if s4:
                            _add(out, m4, 0.5 * v * s1 * s2 * s3 * s4 * a)
    return out


def brute_force(M, h1, e0, L, coeff, occ_a, occ_b, phi_a, phi_b):
    """<Psi_T|X|phi>/<Psi_T|phi> for X = 1 (returned as the overlap itself),
    H, each L_g-hat, and every a+_ps a_qs."""
    psi = trial_state(M, coeff, occ_a, occ_b)
    phi = walker_state(phi_a, phi_b)
    ovlp = dot(psi, phi)
    eri = np.einsum("gpq,grs->pqrs", L, L)
    h = h1[0]
    assert np.allclose(h1[0], h1[1]), "the brute force takes one h for both spins"
    hphi = apply_one_body(phi, h, M)
    vphi = apply_two_body(phi, eri, M)
    energy = (e0 * ovlp + dot(psi, hphi) + dot(psi, vphi)) / ovlp
    vbias = np.array([dot(psi, apply_one_body(phi, Lg, M)) for Lg in L]) / ovlp
    G = np.zeros((2, M, M), complex)
    for spin in range(2):
        for p in range(M):
            for q in range(M):
                G[spin, p, q] = dot(psi, apply_excitation(phi, p, q, spin, M)) / ovlp
    return ovlp, energy, vbias, G
