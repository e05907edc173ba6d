"""CPU oracle for one phaseless AFQMC propagation step (Sec. II A,
Eq. 7-12). TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
benchmark's CPU leg use it; the library never does. It shares no code with
the CUDA path (the trial-level overlaps and force bias come from the C
oracle, msd_oracle.c).

One step, for every walker i with Slater determinants phi^s (s = alpha, beta),
weight w_i and Gaussian fields x (n_chol,):

  h'^s    = h^s - 1/2 sum_g L_g L_g                       (Sec. II A, one-body part)
  vbias_g = <Psi_T| L_g |phi> / <Psi_T|phi>              (mixed estimate, Eq. 7 without
                                                          its prefactor)
  xbar_g  = -i sqrt(dt) vbias_g                           (force bias, Eq. 7; the factor i
                                                          of the Hubbard-Stratonovich
                                                          field, our reading of Eq. 7)
  B(x - xbar) phi^s = e^{-dt h'^s/2} T_n(V) e^{-dt h'^s/2} phi^s,
          V = i sqrt(dt) sum_g (x_g - xbar_g) L_g,        T_n(V) = sum_{k<=n} V^k / k!
  S       = <Psi_T|B phi> / <Psi_T|phi>                   (Eq. 8)
  I       = S exp(x . xbar - xbar . xbar / 2)             (Eq. 10)
  w'      = w |I| max(0, cos(arg S))                      (Eq. 11, phaseless)

optionally followed by a QR orthonormalisation of every phi'^s (the columns
of Q, with the diagonal of R real and positive). Each function below follows
one of these lines.
"""
from __future__ import annotations

import math

import numpy as np

import oracle


def h_prime(h1: np.ndarray, L: np.ndarray) -> np.ndarray:
    """h'^s = h^s - 1/2 sum_g L_g L_g (matrix products), for both spins."""
    corr = np.zeros_like(h1[0])
    for g in range(L.shape[0]):
        corr += L[g] @ L[g]
    return np.stack([h1[s] - 0.5 * corr for s in range(h1.shape[0])])


def expm_sym(A: np.ndarray) -> np.ndarray:
    """exp(A) of a real symmetric matrix from its eigendecomposition."""
    lam, U = np.linalg.eigh(A)
    return (U * np.exp(lam)) @ U.T


def taylor_apply(V: np.ndarray, phi: np.ndarray, order: int) -> np.ndarray:
    """T_n(V) phi = sum_{k=0}^{n} V^k phi / k!, term by term."""
    out = phi.astype(np.complex128).copy()
    term = out.copy()
    for k in range(1, order + 1):
        term = (V @ term) / k
        out = out + term
    return out


def hs_matrix(x: np.ndarray, xbar: np.ndarray, L: np.ndarray, dt: float) -> np.ndarray:
    """V = i sqrt(dt) sum_g (x_g - xbar_g) L_g for one walker."""
    c = 1j * math.sqrt(dt) * (x - xbar)
    return np.tensordot(c, L, axes=(0, 0))


def apply_B(phi: np.ndarray, half: np.ndarray, V: np.ndarray, order: int) -> np.ndarray:
    """e^{-dt h'/2} T_n(V) e^{-dt h'/2} phi for one walker and spin."""
    return half @ taylor_apply(V, half @ phi, order)


def phaseless_weight(w: float, S: complex, exponent: complex) -> float:
    """w' = w |S exp(exponent)| max(0, cos(arg S))."""
    I = S * np.exp(exponent)
    return float(w * abs(I) * max(0.0, math.cos(np.angle(S))))


def qr_positive(phi: np.ndarray) -> np.ndarray:
    """Q of phi = Q R (reduced) with the diagonal of R real and positive."""
    Q, R = np.linalg.qr(phi)
    d = np.diag(R)
    ph = d / np.abs(d)
    return Q * ph[None, :]


def step(system, phi_a, phi_b, weights, x, dt: float, order: int = 6, orthonormalize: bool = False,
         return_importance: bool = False):
    """One propagation step of every walker. Returns (phi_a', phi_b',
    weights', S) with S the overlap ratio of Eq. 8 (before any QR), and the
    importance function I of Eq. 10 as a fifth item when asked."""
    s = system
    phi_a = np.asarray(phi_a, np.complex128)
    phi_b = np.asarray(phi_b, np.complex128)
    n_w = phi_a.shape[0]
    hp = h_prime(s.h1, s.L)
    half = [expm_sym(-0.5 * dt * hp[sp]) for sp in range(2)]
    before = oracle.msd(s, phi_a, phi_b, energy=False, vbias=True)
    new_a = np.empty_like(phi_a)
    new_b = np.empty_like(phi_b)
    expo = np.empty(n_w, np.complex128)
    for i in range(n_w):
        xbar = -1j * math.sqrt(dt) * before["vbias"][i]
        V = hs_matrix(x[i], xbar, s.L, dt)
        new_a[i] = apply_B(phi_a[i], half[0], V, order)
        new_b[i] = apply_B(phi_b[i], half[1], V, order)
        expo[i] = np.dot(x[i], xbar) - 0.5 * np.dot(xbar, xbar)
    after = oracle.msd(s, new_a, new_b, energy=False, vbias=False)
    S = after["ovlp"] / before["ovlp"]
    w_new = np.array([phaseless_weight(weights[i], S[i], expo[i]) for i in range(n_w)])
    if orthonormalize:
        new_a = np.stack([qr_positive(p) for p in new_a])
        new_b = np.stack([qr_positive(p) for p in new_b])
    if return_importance:
        return new_a, new_b, w_new, S, S * np.exp(expo)
    return new_a, new_b, w_new, S
