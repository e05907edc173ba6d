"""Exact rearrangements of the per-determinant energy terms (Sec. III, the
two-body part of the generalized Wick contraction in its Gram form), checked
in numpy on random inputs, independent of the library and the oracle:

* opposite-spin term: the double sum over the alpha and beta minors,
    X_ab = sum_ij sum_kl Ba[i][j] Bb[k][l] K[(h_j, p_i)][(h'_l, p'_k)],
  equals the per-beta-string form sum_ij Ba[i][j] Y_b[(h_j, p_i)] with
    Y_b[x] = sum_kl Bb[k][l] K[x][(h'_l, p'_k)];
* same-spin quadratic part: with K symmetric, each summand
    b_ij b_kl (K[(j,i)][(l,k)] - K[(j,k)][(l,i)])
  is symmetric under (i, j) <-> (k, l), so the full sum equals the diagonal
  pairs plus twice the pairs (k, l) > (i, j);
* same-spin quadratic part, antisymmetrized: with K symmetric,
    Qc - Qx = 2 sum_{i<k} sum_{j<l} (b_ij b_kl - b_il b_kj) A[h_j,h_l;p_i,p_k],
    A[h,h';p,p'] = K[(h,p)][(h',p')] - K[(h,p')][(h',p)].
"""
import numpy as np
import pytest


def _cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("ka,kb,seed", [(1, 1, 0), (2, 3, 1), (4, 4, 2), (3, 6, 3), (6, 5, 4)])
def test_opposite_spin_per_beta_string_form(ka, kb, seed):
    rng = np.random.default_rng(seed)
    nh_a, np_a, nh_b, np_b = 7, 6, 6, 7
    K = _cplx(rng, nh_a * np_a, nh_b * np_b)
    ha = np.sort(rng.choice(nh_a, ka, replace=False))
    pa = np.sort(rng.choice(np_a, ka, replace=False))
    hb = np.sort(rng.choice(nh_b, kb, replace=False))
    pb = np.sort(rng.choice(np_b, kb, replace=False))
    Ba, Bb = _cplx(rng, ka, ka), _cplx(rng, kb, kb)
    direct = 0
    for i in range(ka):
        for j in range(ka):
            for k in range(kb):
                for l in range(kb):
                    direct += Ba[i, j] * Bb[k, l] * K[ha[j] * np_a + pa[i], hb[l] * np_b + pb[k]]
    Y = np.zeros(nh_a * np_a, complex)
    for k in range(kb):
        for l in range(kb):
            Y += Bb[k, l] * K[:, hb[l] * np_b + pb[k]]
    per_beta = sum(Ba[i, j] * Y[ha[j] * np_a + pa[i]] for i in range(ka) for j in range(ka))
    assert abs(direct - per_beta) <= 1e-12 * max(1.0, abs(direct))


def _same_spin_q(b, K, h, p, np_, half):
    k = len(h)
    x = lambda hole, part: h[hole] * np_ + p[part]
    total = 0
    for i in range(k):
        for j in range(k):
            for kk in range(k):
                for l in range(k):
                    n, m = i * k + j, kk * k + l
                    if half and m < n:
                        continue
                    term = b[i, j] * b[kk, l] * (K[x(j, i), x(l, kk)] - K[x(j, kk), x(l, i)])
                    total += term if (not half or m == n) else 2 * term
    return total


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (3, 2), (4, 3), (5, 4)])
def test_same_spin_pair_swap_symmetry(k, seed):
    rng = np.random.default_rng(seed)
    nh, np_ = 8, 6
    A = _cplx(rng, nh * np_, nh * np_)
    K = A + A.T          # symmetric, not Hermitian, as a Gram matrix without conjugation
    h = np.sort(rng.choice(nh, k, replace=False))
    p = np.sort(rng.choice(np_, k, replace=False))
    b = _cplx(rng, k, k)
    full = _same_spin_q(b, K, h, p, np_, half=False)
    half = _same_spin_q(b, K, h, p, np_, half=True)
    assert abs(full - half) <= 1e-12 * max(1.0, abs(full))


def test_pair_swap_needs_symmetric_k():
    """The halving is only valid for symmetric K (a plausible misuse fails)."""
    rng = np.random.default_rng(9)
    nh, np_, k = 8, 6, 3
    K = _cplx(rng, nh * np_, nh * np_)
    h = np.sort(rng.choice(nh, k, replace=False))
    p = np.sort(rng.choice(np_, k, replace=False))
    b = _cplx(rng, k, k)
    full = _same_spin_q(b, K, h, p, np_, half=False)
    half = _same_spin_q(b, K, h, p, np_, half=True)
    assert abs(full - half) > 1e-6 * abs(full)


def _q_direct(B, K, h, p, npp):
    k = len(h)
    x = lambda hh, pp: hh * npp + pp
    qc = qx = 0
    for i in range(k):
        for j in range(k):
            for kk in range(k):
                for l in range(k):
                    qc += B[i, j] * B[kk, l] * K[x(h[j], p[i]), x(h[l], p[kk])]
                    qx += B[i, j] * B[kk, l] * K[x(h[j], p[kk]), x(h[l], p[i])]
    return qc - qx


def _q_antisym(B, K, h, p, npp):
    """2 sum_{i<k} sum_{j<l} (B_ij B_kl - B_il B_kj) A[h_j,h_l;p_i,p_k],
    A[h,h';p,p'] = K[(h,p)][(h',p')] - K[(h,p')][(h',p)]."""
    k = len(h)
    x = lambda hh, pp: hh * npp + pp
    q = 0
    for i in range(k):
        for kk in range(i + 1, k):
            for j in range(k):
                for l in range(j + 1, k):
                    a = K[x(h[j], p[i]), x(h[l], p[kk])] - K[x(h[j], p[kk]), x(h[l], p[i])]
                    q += (B[i, j] * B[kk, l] - B[i, l] * B[kk, j]) * a
    return 2 * q


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (3, 2), (4, 3), (5, 4), (6, 5)])
def test_same_spin_antisymmetrized_pair_form(k, seed):
    """With K symmetric, Qc - Qx is carried by the 2x2 minors of B against the
    pair table A, antisymmetric in the holes and in the particles (the holes
    and particles of a string ascending): C(k,2)^2 terms."""
    rng = np.random.default_rng(seed)
    nh, npp = 8, 7
    Kr = _cplx(rng, nh * npp, nh * npp)
    K = Kr + Kr.T
    h = np.sort(rng.choice(nh, k, replace=False))
    p = np.sort(rng.choice(npp, k, replace=False))
    B = _cplx(rng, k, k)
    want = _q_direct(B, K, h, p, npp)
    got = _q_antisym(B, K, h, p, npp)
    assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


def test_antisymmetrized_form_needs_symmetric_k():
    """For a general (non-symmetric) K the rearrangement does not hold."""
    rng = np.random.default_rng(9)
    nh, npp, k = 6, 6, 3
    K = _cplx(rng, nh * npp, nh * npp)
    h, p = np.array([0, 2, 5]), np.array([1, 3, 4])
    B = _cplx(rng, k, k)
    assert abs(_q_antisym(B, K, h, p, npp) - _q_direct(B, K, h, p, npp)) > 1e-3
