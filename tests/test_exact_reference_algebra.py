"""The exact split of the reference-determinant energy used by the mixed
precision path (Sec. II A: the generalized Wick theorem for the reference
determinant D_0, in the Cholesky form of Eq. 2-3), checked in numpy on
random inputs, independent of the library and the oracle.

With G = D0 D0^T + dG (dG non-zero only in the columns v_r of the orbitals
outside occ0, u_s[(j, r)] = dG_s[occ0_j][v_r]), C_g = sum_s tr(L_g D0_s D0_s^T),
t1_g^s = tr(L_g dG_s), dT_g^s = (dG_s L_g)[occ0][occ0]:

  1/2 sum_g V0_g^2 - 1/2 sum_gs x_g^s
      = 1/2 sum_g C_g^2 - 1/2 sum_s x0^s                  (constants)
      + sum_s u_s . (JJ_s - KK_s)                         (linear in dG)
      + 1/2 sum_g (t1_g^a + t1_g^b)^2 - 1/2 sum_s u_s^T V_s u_s   (quadratic)

with JJ_s[(j, r)] = (sum_g C_g L_g)[v_r][o_j], KK_s[(j, r)] =
(sum_g L_g D0_s D0_s^T L_g)[v_r][o_j], V_s[(j, r)][(l, r')] =
sum_g L_g[v_r][o_l] L_g[v_r'][o_j]; and the exact-integer slice product
(5 slices of 7 bits, chunks of 512 contraction steps) that evaluates the
quadratic forms on the tensor cores.
"""
import numpy as np
import pytest


def _system(rng, M, na, nb, G, occ_a, occ_b):
    L = rng.standard_normal((G, M, M))
    L = 0.5 * (L + L.transpose(0, 2, 1))
    walkers = []
    for occ, n in ((occ_a, na), (occ_b, nb)):
        phi = 0.4 * (rng.standard_normal((M, n)) + 1j * rng.standard_normal((M, n)))
        phi[occ, np.arange(n)] += 1.0
        walkers.append(phi)
    return L, walkers


def _direct(L, occs, phis):
    """1/2 sum_g V0^2 - 1/2 sum_gs tr(L G L G) from the full G rows."""
    V0 = 0
    xs = 0
    for occ, phi in zip(occs, phis):
        Gr = (phi @ np.linalg.inv(phi[occ])).T          # rows occ of G = (Theta D0^dag)^T
        F = np.einsum("jq,gqr->gjr", Gr, L)             # (G L)[occ][:]
        T = F[:, :, occ]
        V0 = V0 + np.einsum("gjj->g", T)
        xs = xs + np.einsum("gjl,glj->g", T, T)
    return 0.5 * np.sum(V0 ** 2) - 0.5 * np.sum(xs)


def _split(L, occs, phis, M):
    G = L.shape[0]
    C = sum(np.einsum("gjj->g", L[:, occ][:, :, occ]) for occ in occs)
    Jm = np.einsum("g,gpq->pq", C, L)
    const = 0.5 * np.sum(C ** 2)
    lin = 0
    t1 = 0
    quad_x = 0
    for occ, phi in zip(occs, phis):
        N = len(occ)
        virt = np.setdiff1d(np.arange(M), occ)
        Gr = (phi @ np.linalg.inv(phi[occ])).T
        u = Gr[:, virt].reshape(-1)                     # (j, r)
        const -= 0.5 * np.sum(L[:, occ][:, :, occ] ** 2)
        P0 = np.zeros((M, M)); P0[occ, occ] = 1.0
        K0 = np.einsum("gpa,ab,gbq->pq", L, P0, L)
        JJ = Jm[np.ix_(virt, occ)].T.reshape(-1)        # [(j, r)] = J[v_r][o_j]
        KK = K0[np.ix_(virt, occ)].T.reshape(-1)
        lin = lin + u @ (JJ - KK)
        X = L[:, virt][:, :, occ]                        # [g][r][l] = L_g[v_r][o_l]
        V = np.einsum("grl,gsj->jrls", X, X).reshape(N * len(virt), N * len(virt))
        W = X.transpose(2, 1, 0).reshape(N * len(virt), G)   # [(j, r)][g] = L_g[v_r][o_j]
        t1 = t1 + W.T @ u
        quad_x = quad_x + u @ V @ u
    return const + lin + 0.5 * np.sum(t1 ** 2) - 0.5 * quad_x


@pytest.mark.parametrize("M,na,nb,G,seed,shuffle", [
    (9, 3, 3, 5, 0, False), (11, 4, 2, 7, 1, True), (8, 1, 5, 4, 2, True)])
def test_reference_energy_split(M, na, nb, G, seed, shuffle):
    rng = np.random.default_rng(seed)
    orb = rng.permutation(M) if shuffle else np.arange(M)
    occ_a, occ_b = np.sort(orb[:na]), np.sort(orb[M - nb:] if shuffle else orb[:nb])
    L, phis = _system(rng, M, na, nb, G, occ_a, occ_b)
    want = _direct(L, (occ_a, occ_b), phis)
    got = _split(L, (occ_a, occ_b), phis, M)
    assert abs(got - want) <= 1e-11 * max(1.0, abs(want)), (got, want)


def test_split_catches_a_dropped_exchange_matrix():
    """Without the KK term (a plausible omission) the split is wrong."""
    rng = np.random.default_rng(3)
    M, n, G = 9, 3, 5
    occ = np.arange(n)
    L, phis = _system(rng, M, n, n, G, occ, occ)
    want = _direct(L, (occ, occ), phis)
    # recompute with K0 = 0
    C = 2 * np.einsum("gjj->g", L[:, occ][:, :, occ])
    Jm = np.einsum("g,gpq->pq", C, L)
    virt = np.arange(n, M)
    bad = 0.5 * np.sum(C ** 2) - np.sum(L[:, occ][:, :, occ] ** 2)
    t1 = 0
    for phi in phis:
        Gr = (phi @ np.linalg.inv(phi[occ])).T
        u = Gr[:, virt].reshape(-1)
        bad += u @ Jm[np.ix_(virt, occ)].T.reshape(-1)
        X = L[:, virt][:, :, occ]
        V = np.einsum("grl,gsj->jrls", X, X).reshape(n * len(virt), n * len(virt))
        t1 = t1 + X.transpose(2, 1, 0).reshape(n * len(virt), G).T @ u
        bad -= 0.5 * (u @ V @ u)
    bad += 0.5 * np.sum(t1 ** 2)
    assert abs(bad - want) > 1e-6 * max(1.0, abs(want))


def _lambda(L, occ, part, hole_pos, phi):
    """Lambda_g[(h, p)] = (G L_g (I - G))[H_h][P_p] from the rows occ of G,
    per vector g (the definition the energy's Gram form uses)."""
    Gr = (phi @ np.linalg.inv(phi[occ])).T
    F = np.einsum("jq,gqr->gjr", Gr, L)
    T, FP, GP = F[:, :, occ], F[:, :, part], Gr[:, part]
    lam = FP - np.einsum("gjl,lp->gjp", T, GP)
    return lam[:, hole_pos, :].reshape(L.shape[0], -1), Gr


@pytest.mark.parametrize("M,n,G,seed", [(9, 3, 5, 4), (12, 5, 8, 5)])
def test_reference_part_of_v0_lambda_sum_is_a_one_body_term(M, n, G, seed):
    """sum_g C_g Lambda_g equals the one-body term (G J (I - G))[H][P] of
    J = sum_g C_g L_g, for any weights C_g: the mixed path forms it in FP64
    with h + J and sums only the walker parts t1_g of V0_g in FP32. A
    version without the -G[occ][P] part of (I - G) fails."""
    rng = np.random.default_rng(seed)
    occ = np.sort(rng.permutation(M)[:n])
    virt = np.setdiff1d(np.arange(M), occ)
    part = virt[: max(1, len(virt) // 2)]
    hole_pos = np.arange(n - min(n, 3), n)
    L, (phi, _) = _system(rng, M, n, n, G, occ, occ)
    C = rng.standard_normal(G) + np.einsum("gjj->g", L[:, occ][:, :, occ])
    lam, Gr = _lambda(L, occ, part, hole_pos, phi)
    want = C @ lam
    J = np.einsum("g,gpq->pq", C, L)
    GJ = Gr @ J                                          # rows occ of G J
    one = (GJ[:, part] - GJ[:, occ] @ Gr[:, part])[hole_pos].reshape(-1)
    assert np.allclose(one, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    bad = GJ[:, part][hole_pos].reshape(-1)
    assert not np.allclose(bad, want, rtol=1e-6, atol=1e-6 * np.abs(want).max())


# ---------------------------------------------------------------- slicing
BETA, S, KCH = 7, 5, 512


def _slices(X):
    """Row-wise: X = 2^e sum_i a_i 2^(-BETA i) + rest, integers a_i."""
    m = np.abs(X).max(axis=1)
    e = np.array([np.frexp(v)[1] if v > 0 else 0 for v in m])
    r = np.ldexp(X, -e[:, None])
    out = []
    for _ in range(S):
        r = r * 2.0 ** BETA
        a = np.rint(r)
        r = r - a
        out.append(a)
    return out, e


def _slice_product(A, B):
    """A B^T from the slices, with every group sum of a chunk checked to be
    an integer below 2^24 (exact in FP32)."""
    As, ea = _slices(A)
    Bs, eb = _slices(B)
    total = np.zeros((A.shape[0], B.shape[0]), dtype=object)
    for k0 in range(0, A.shape[1], KCH):
        sl = slice(k0, k0 + KCH)
        for c in range(2, S + 2):
            acc = sum(As[i - 1][:, sl] @ Bs[c - i - 1][:, sl].T for i in range(1, S + 1) if 1 <= c - i <= S)
            assert np.all(np.abs(acc) < 2 ** 24) and np.all(acc == np.rint(acc))
            total = total + acc.astype(np.int64).astype(object) * (2 ** (BETA * (S + 1 - c)))
    val = np.array([[float(v) for v in row] for row in total])
    return np.ldexp(val, (ea[:, None] + eb[None, :]) - BETA * (S + 1))


def test_slice_integers_and_worst_case_bound():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((6, 1000)) * np.exp(rng.uniform(-20, 20, (6, 1)))
    As, e = _slices(X)
    assert np.abs(As[0]).max() <= 2 ** BETA
    for a in As[1:]:
        assert np.abs(a).max() <= 2 ** (BETA - 1)
    # the largest group (c = S + 1) at its worst case over a whole chunk
    worst = KCH * (2 * 2 ** BETA * 2 ** (BETA - 1) + (S - 2) * 2 ** (2 * (BETA - 1)))
    assert worst < 2 ** 24


@pytest.mark.parametrize("K,seed", [(100, 0), (1300, 1), (3900, 2)])
def test_slice_product_accuracy(K, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((4, K))
    B = rng.standard_normal((5, K)) * 3.0
    got = _slice_product(A, B)
    want = A @ B.T
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :] * K
    assert np.all(np.abs(got - want) <= 2.0 ** -33 * scale)
    # far better than an FP32 product with FP32 accumulation
    f32 = (A.astype(np.float32) @ B.T.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(got - want)) < 1e-3 * np.max(np.abs(f32 - want))


def test_symmetric_tile_schedule():
    """The quadratic form over the symmetric V from column tiles of 96 that
    contract only their diagonal block (once) and the blocks after it
    (twice), with V's rows padded with zeros to a whole number of tiles so
    that no tile mixes V and W columns; a W tile takes the full range."""
    rng = np.random.default_rng(7)
    n, g, tile = 300, 40, 96
    X = rng.standard_normal((n, n))
    V = X + X.T
    W = rng.standard_normal((n, g))
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    npad = -(-n // tile) * tile
    Vp = np.zeros((npad, npad)); Vp[:n, :n] = V
    up = np.zeros(npad, complex); up[:n] = u
    total = 0
    for n0 in range(0, npad, tile):
        cols = slice(n0, n0 + tile)
        diag = up[cols] @ Vp[cols, cols]
        later = up[n0 + tile:] @ Vp[n0 + tile:, cols]
        total += (diag + 2 * later) @ up[cols]
    assert abs(total - u @ V @ u) <= 1e-9 * abs(u @ V @ u)
    t1 = u @ W                          # the W tiles: full range, no doubling
    assert np.allclose(up[:n] @ W, t1)
    # the mistake this layout avoids: a tile holding V and W columns with the
    # full range counts its V columns' earlier rows a third time
    bad = 0
    for n0 in range(0, n, tile):
        cols = slice(n0, min(n, n0 + tile))
        if n0 + tile <= n:
            bad += (u[cols] @ V[cols, cols] + 2 * u[n0 + tile:] @ V[n0 + tile:, cols]) @ u[cols]
        else:
            bad += (u @ V[:, cols]) @ u[cols]
    assert abs(bad - u @ V @ u) > 1e-6 * abs(u @ V @ u)
