"""Pins of the propagation-step oracle (oracle/prop_oracle.py) against what
the mathematics fixes: closed forms, a library matrix exponential, the
Gaussian characteristic function computed by exact quadrature, invariances
and the phaseless weight rule (Sec. II A, Eq. 7-12)."""
import math

import numpy as np
import pytest

import oracle
from oracle import prop_oracle as po
from paper_2406_08314_gb300 import synth

scipy_linalg = pytest.importorskip("scipy.linalg")


def _sym(rng, M, scale=1.0):
    a = rng.standard_normal((M, M)) * scale
    return 0.5 * (a + a.T)


def test_expm_sym_matches_library_expm():
    rng = np.random.default_rng(0)
    A = _sym(rng, 7, 0.4)
    assert np.allclose(po.expm_sym(A), scipy_linalg.expm(A), rtol=1e-13, atol=1e-13)
    assert np.allclose(po.expm_sym(np.zeros((4, 4))), np.eye(4), atol=0)


def test_taylor_apply_within_remainder_bound():
    rng = np.random.default_rng(1)
    M, N = 9, 3
    V = 0.05j * _sym(rng, M) + 0.03 * _sym(rng, M)
    phi = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    exact = scipy_linalg.expm(V) @ phi
    nV = np.linalg.norm(V, 2)
    for n in (1, 2, 4, 6, 8):
        got = po.taylor_apply(V, phi, n)
        bound = nV ** (n + 1) / math.factorial(n + 1) * math.exp(nV) * np.linalg.norm(phi, 2)
        assert np.linalg.norm(got - exact, 2) <= bound * 1.0001 + 1e-15, n
    # order 0 is the identity, order 1 adds exactly V phi
    assert np.array_equal(po.taylor_apply(V, phi, 0), phi)
    assert np.allclose(po.taylor_apply(V, phi, 1), phi + V @ phi, rtol=0, atol=1e-15)


def test_h_prime_rank_one_closed_form():
    rng = np.random.default_rng(2)
    M = 6
    u = rng.standard_normal(M)
    L = np.outer(u, u)[None]          # one Cholesky vector L = u u^T: L L = (u.u) u u^T
    h = np.stack([_sym(rng, M), _sym(rng, M)])
    hp = po.h_prime(h, L)
    for s in range(2):
        assert np.allclose(hp[s], h[s] - 0.5 * (u @ u) * np.outer(u, u), rtol=1e-14, atol=1e-14)


def test_gaussian_average_of_the_field_propagator():
    """E_x[T_n(i sqrt(dt) x L)] over x ~ N(0, 1) is the order-n/2 series of
    exp(-dt L^2 / 2) (odd powers average to zero, E x^2m = (2m-1)!!); Gauss-
    Hermite quadrature with enough nodes is exact for this polynomial in x."""
    rng = np.random.default_rng(3)
    M, N, dt, n = 5, 2, 0.01, 6
    L = _sym(rng, M)
    phi = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    nodes, wts = np.polynomial.hermite_e.hermegauss(n + 2)
    wts = wts / wts.sum()
    avg = sum(w * po.taylor_apply(po.hs_matrix(np.array([x]), np.zeros(1), L[None], dt), phi, n)
              for x, w in zip(nodes, wts))
    L2 = L @ L
    series = sum((-dt / 2) ** m / math.factorial(m) * np.linalg.matrix_power(L2, m) for m in range(n // 2 + 1))
    assert np.allclose(avg, series @ phi, rtol=1e-12, atol=1e-13)
    # and it approaches exp(-dt L^2 / 2) within the series' remainder
    a = np.linalg.norm(0.5 * dt * L2, 2)
    m1 = n // 2 + 1
    bound = a ** m1 / math.factorial(m1) * math.exp(a) * np.linalg.norm(phi, 2)
    assert np.linalg.norm(avg - scipy_linalg.expm(-0.5 * dt * L2) @ phi, 2) <= bound


def test_phaseless_weight_rule():
    for theta, factor in ((0.0, 1.0), (math.pi / 3, 0.5), (2 * math.pi / 3, 0.0), (-math.pi / 4, math.cos(math.pi / 4))):
        S = 2.0 * complex(math.cos(theta), math.sin(theta))
        expo = complex(0.3, -1.1)
        w = po.phaseless_weight(1.5, S, expo)
        assert w == pytest.approx(1.5 * 2.0 * math.exp(0.3) * factor, rel=1e-14, abs=1e-15)


def _one_body_system(M, na, nb, rng):
    eps = np.sort(rng.standard_normal(M))
    h = np.diag(eps)
    L = np.zeros((1, M, M))
    occ_a = np.arange(na)[None].astype(np.int32)
    occ_b = np.arange(nb)[None].astype(np.int32)
    s = synth.System(M, na, nb, np.stack([h, h]), 0.0, L, np.ones(1), occ_a, occ_b, 0, M, {})
    return s, eps


def test_one_body_step_closed_form():
    """L = 0 and a single-determinant trial on the lowest orbitals of a
    diagonal h: B = exp(-dt h) exactly, S = exp(-dt (sum of the occupied
    orbital energies, both spins)), no force bias, w' = w S."""
    rng = np.random.default_rng(4)
    M, na, nb, dt = 7, 3, 2, 0.05
    s, eps = _one_body_system(M, na, nb, rng)
    w = synth.make_walkers(rng, M, na, nb, 3, noise=0.3)
    x = rng.standard_normal((3, 1))
    pa, pb, wn, S = po.step(s, w.phi_a, w.phi_b, np.ones(3), x, dt, order=6)
    E = np.diag(np.exp(-dt * eps))
    assert np.allclose(pa, E[None] @ w.phi_a, rtol=1e-13, atol=1e-14)
    assert np.allclose(pb, E[None] @ w.phi_b, rtol=1e-13, atol=1e-14)
    want = math.exp(-dt * (eps[:na].sum() + eps[:nb].sum()))
    assert np.allclose(S, want, rtol=1e-12)
    assert np.allclose(wn, want, rtol=1e-12)


def test_step_invariant_under_column_mixing_and_qr():
    """phi -> phi R (R invertible per spin) leaves the Green's function, the
    force bias, S and the weights unchanged and maps phi' to phi' R; the QR
    output has orthonormal columns spanning phi'."""
    s, w = synth.config_system("small", seed=5)
    rng = np.random.default_rng(6)
    n = 3
    pa, pb = w.phi_a[:n], w.phi_b[:n]
    x = rng.standard_normal((n, s.n_chol))
    Ra = rng.standard_normal((s.n_alpha, s.n_alpha)) + 1j * rng.standard_normal((s.n_alpha, s.n_alpha))
    Rb = rng.standard_normal((s.n_beta, s.n_beta)) + 1j * rng.standard_normal((s.n_beta, s.n_beta))
    a1, b1, w1, S1 = po.step(s, pa, pb, np.ones(n), x, 0.01)
    a2, b2, w2, S2 = po.step(s, pa @ Ra, pb @ Rb, np.ones(n), x, 0.01)
    assert np.allclose(S2, S1, rtol=1e-10)
    assert np.allclose(w2, w1, rtol=1e-10)
    assert np.allclose(a2, a1 @ Ra, rtol=1e-10, atol=1e-12)
    assert np.allclose(b2, b1 @ Rb, rtol=1e-10, atol=1e-12)
    a3, b3, w3, S3 = po.step(s, pa, pb, np.ones(n), x, 0.01, orthonormalize=True)
    assert np.allclose(w3, w1, rtol=1e-14) and np.allclose(S3, S1, rtol=1e-14)
    for q, p in ((a3, a1), (b3, b1)):
        for i in range(n):
            assert np.allclose(q[i].conj().T @ q[i], np.eye(q.shape[2]), atol=1e-12)
            R = q[i].conj().T @ p[i]
            assert np.allclose(np.tril(R, -1), 0, atol=1e-10)
            assert np.all(np.abs(np.diag(R).imag) < 1e-10) and np.all(np.diag(R).real > 0)
            assert np.allclose(q[i] @ R, p[i], rtol=1e-10, atol=1e-12)


def test_force_bias_enters_the_field_and_the_importance_factor():
    """With xbar from the C oracle's mixed <L_g>: V uses x - xbar with
    xbar = -i sqrt(dt) vbias, and I = S exp(x.xbar - xbar.xbar/2), so
    w' / |S| = exp(Re(x.xbar - xbar.xbar/2)) max(0, cos arg S)."""
    s, w = synth.config_system("small", seed=7)
    rng = np.random.default_rng(8)
    n, dt = 2, 0.02
    pa, pb = w.phi_a[:n], w.phi_b[:n]
    x = rng.standard_normal((n, s.n_chol))
    a1, b1, w1, S1 = po.step(s, pa, pb, np.ones(n), x, dt)
    vb = oracle.msd(s, pa, pb, energy=False, vbias=True)["vbias"]
    for i in range(n):
        xbar = -1j * math.sqrt(dt) * vb[i]
        V = 1j * math.sqrt(dt) * np.tensordot(x[i] - xbar, s.L, axes=(0, 0))
        hp = s.h1[0] - 0.5 * np.einsum("gpr,grq->pq", s.L, s.L)
        half = scipy_linalg.expm(-0.5 * dt * hp)
        ref_a = half @ po.taylor_apply(V, half @ pa[i], 6)
        assert np.allclose(a1[i], ref_a, rtol=1e-12, atol=1e-13)
        ex = np.dot(x[i], xbar) - 0.5 * np.dot(xbar, xbar)
        want = abs(S1[i]) * math.exp(ex.real) * max(0.0, math.cos(np.angle(S1[i])))
        assert w1[i] == pytest.approx(want, rel=1e-13)


def test_force_bias_cancels_the_linear_field_term():
    """The force bias is the shift that removes the O(sqrt(dt)) dependence of
    the importance function on the fields: S = 1 + i sqrt(dt) (x - xbar).vbias
    + O(dt) and exp(x.xbar) = 1 - i sqrt(dt) x.vbias + O(dt), so the odd part
    (I(x) - I(-x)) / 2 is O(dt^3/2). A wrong sign or factor of xbar leaves
    a term of order sqrt(dt) |x.vbias|."""
    s, w = synth.config_system("small", seed=9)
    rng = np.random.default_rng(10)
    n, dt = 2, 1e-8
    pa, pb = w.phi_a[:n], w.phi_b[:n]
    x = rng.standard_normal((n, s.n_chol))
    Ip = po.step(s, pa, pb, np.ones(n), x, dt, return_importance=True)[4]
    Im = po.step(s, pa, pb, np.ones(n), -x, dt, return_importance=True)[4]
    vb = oracle.msd(s, pa, pb, energy=False, vbias=True)["vbias"]
    lin = math.sqrt(dt) * np.abs(np.sum(x * vb, axis=1))     # size of an uncancelled term
    odd = np.abs(Ip - Im) / 2
    assert np.all(lin > 1e-5), lin
    assert np.all(odd < 1e-3 * lin), (odd, lin)
