"""Seeded synthetic inputs for the multi-Slater-determinant AFQMC hot path.

This module only draws random numbers and arranges them into the shapes the
method consumes (Sec. II, "Multi-Slater determinant AFQMC", and Sec. III,
"Benchmark results"): a one-body matrix h, Cholesky vectors L_gamma, a CI trial
(coefficients plus sorted occupation lists per spin, reference determinant
first) and walkers (complex M x N orbital matrices per spin). It computes no
overlap, Green's function or energy; both the CUDA path and the CPU oracle read
what it produces.

Recipe (one numpy Generator per system, draws in the fixed order
h1 -> L -> trial -> walkers):
  * h1: upper triangle N(0, 1), mirrored, divided by M; the same for both
    spins; e0 = 0.
  * L: n_chol random symmetric M x M matrices, orthonormalised in the
    Frobenius inner product (QR of the (M*M, n_chol) stack), multiplied by
    exp(-gamma / decay): the (M*M, n_chol) stack has singular values
    exp(-gamma / decay). Optionally (onsite=x) all vectors are scaled by one
    constant so that the mean on-site Coulomb integral
    (pp|pp) = sum_gamma L_gamma[p, p]^2 is x Ha (a chemical-scale variant).
  * Trial: reference = the first N_sigma orbitals. The active space is
    orbitals [n_core, n_core + n_act_orb); each spin has
    n_o = N_sigma - n_core active occupied and n_v = n_act_orb - n_o active
    virtual orbitals. n_det - 1 distinct (alpha, beta) excitation pairs are
    drawn uniformly over all pairs with 1 <= k_alpha + k_beta <= max_level,
    sorted (stably) by total level; |c_I| = (I + 1)^-power, random signs
    (reference positive), normalised to sum c^2 = 1.
  * Walkers: phi = QR(D0 + noise * (X + iY) / sqrt(2)), X, Y ~ N(0, 1). An
    optional free random walk applies n_steps Gaussian-field one-body
    propagators (Sec. II A, first-order Trotter, no force bias) with a QR
    every 5 steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "System", "Walkers", "make_hamiltonian", "make_trial", "make_walkers",
    "random_walk", "make_system", "CONFIGS", "config_system", "batched_systems",
]


@dataclass
class System:
    """A Hamiltonian plus a CI trial, as the library's set-up calls take them."""
    M: int
    n_alpha: int
    n_beta: int
    h1: np.ndarray          # (2, M, M) float64, symmetric
    e0: float
    L: np.ndarray           # (n_chol, M, M) float64, each symmetric
    coeff: np.ndarray       # (n_det,) float64
    occ_a: np.ndarray       # (n_det, n_alpha) int32, sorted rows; row 0 = reference
    occ_b: np.ndarray       # (n_det, n_beta) int32
    n_core: int = 0
    n_act_orb: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_chol(self) -> int:
        return int(self.L.shape[0])

    @property
    def n_det(self) -> int:
        return int(self.coeff.shape[0])


@dataclass
class Walkers:
    phi_a: np.ndarray       # (n_w, M, n_alpha) complex128
    phi_b: np.ndarray       # (n_w, M, n_beta) complex128

    @property
    def n_w(self) -> int:
        return int(self.phi_a.shape[0])


def make_hamiltonian(rng: np.random.Generator, M: int, n_chol: int,
                     decay: float = 10.0, onsite: float | None = None):
    """h1 (2, M, M) and L (n_chol, M, M) following the module recipe."""
    if n_chol > M * (M + 1) // 2:
        raise ValueError("n_chol exceeds the dimension of symmetric M x M matrices")
    a = rng.standard_normal((M, M))
    h = np.triu(a)
    h = (h + np.triu(h, 1).T) / M
    h1 = np.stack([h, h]).astype(np.float64)
    x = rng.standard_normal((n_chol, M, M))
    x = x + x.transpose(0, 2, 1)
    q, _ = np.linalg.qr(x.reshape(n_chol, M * M).T)      # (M*M, n_chol)
    Q = q.T.reshape(n_chol, M, M)
    Q = 0.5 * (Q + Q.transpose(0, 2, 1))                  # exact symmetry after rounding
    s = np.exp(-np.arange(n_chol) / float(decay))
    L = Q * s[:, None, None]
    if onsite is not None:
        diag = np.einsum("gpp->gp", L)
        L = L * math.sqrt(onsite / float(np.mean(np.sum(diag * diag, axis=0))))
    return h1, np.ascontiguousarray(L)


def _level_counts(n_o: int, n_v: int):
    return [math.comb(n_o, k) * math.comb(n_v, k) for k in range(min(n_o, n_v) + 1)]


def _draw_many(rng, cnt, k, act_occ, act_vir):
    """cnt uniform draws of k holes from act_occ and k particles from act_vir."""
    if k == 0:
        return [((), ())] * cnt
    h = np.sort(np.argsort(rng.random((cnt, len(act_occ))), axis=1)[:, :k], axis=1)
    q = np.sort(np.argsort(rng.random((cnt, len(act_vir))), axis=1)[:, :k], axis=1)
    h = np.asarray(act_occ)[h]
    q = np.asarray(act_vir)[q]
    return [(tuple(int(v) for v in h[i]), tuple(int(v) for v in q[i])) for i in range(cnt)]


def make_trial(rng: np.random.Generator, M: int, n_alpha: int, n_beta: int,
               n_core: int, n_act_orb: int, n_det: int, max_level: int,
               power: float):
    """CI trial: (coeff, occ_a, occ_b), reference determinant first."""
    spins = []
    for n in (n_alpha, n_beta):
        n_o = n - n_core
        n_v = n_act_orb - n_o
        if n_o < 0 or n_v < 0 or n_core + n_act_orb > M:
            raise ValueError("active space does not fit the orbital/electron counts")
        spins.append((np.arange(n_core, n), np.arange(n, n_core + n_act_orb),
                      _level_counts(n_o, n_v)))
    (oa, va, ca), (ob, vb, cb) = spins
    classes, weights = [], []
    for ka in range(len(ca)):
        for kb in range(len(cb)):
            if 1 <= ka + kb <= max_level:
                classes.append((ka, kb))
                weights.append(float(ca[ka]) * float(cb[kb]))
    total = sum(weights)
    if total < n_det - 1:
        raise ValueError("fewer distinct excitations than requested determinants")
    p = np.asarray(weights) / total
    seen = set()
    dets = []
    while len(dets) < n_det - 1:
        need = n_det - 1 - len(dets)
        cls = rng.choice(len(classes), size=need, p=p)
        draws = {}
        for c in np.unique(cls):
            ka, kb = classes[int(c)]
            cnt = int(np.sum(cls == c))
            draws[int(c)] = (_draw_many(rng, cnt, ka, oa, va), _draw_many(rng, cnt, kb, ob, vb))
        used = {c: 0 for c in draws}
        for c in cls:
            c = int(c)
            ka, kb = classes[c]
            i = used[c]
            used[c] += 1
            ea = draws[c][0][i]
            eb = draws[c][1][i]
            key = (ea, eb)
            if key in seen:
                continue
            seen.add(key)
            dets.append((ka + kb, ea, eb))
    order = sorted(range(len(dets)), key=lambda i: dets[i][0])  # stable sort by level
    dets = [dets[i] for i in order]

    def occ_of(n, exc):
        holes, parts = exc
        s = set(range(n)) - set(holes) | set(parts)
        return sorted(s)

    occ_a = np.empty((n_det, n_alpha), np.int32)
    occ_b = np.empty((n_det, n_beta), np.int32)
    occ_a[0] = np.arange(n_alpha)
    occ_b[0] = np.arange(n_beta)
    for i, (_, ea, eb) in enumerate(dets, start=1):
        occ_a[i] = occ_of(n_alpha, ea)
        occ_b[i] = occ_of(n_beta, eb)
    mag = (np.arange(n_det) + 1.0) ** (-float(power))
    sign = rng.choice([-1.0, 1.0], size=n_det)
    sign[0] = 1.0
    coeff = mag * sign
    coeff /= np.sqrt(np.sum(coeff * coeff))
    return coeff.astype(np.float64), occ_a, occ_b


def make_walkers(rng: np.random.Generator, M: int, n_alpha: int, n_beta: int,
                 n_w: int, noise: float = 0.1) -> Walkers:
    out = []
    for n in (n_alpha, n_beta):
        d0 = np.zeros((M, n))
        d0[np.arange(n), np.arange(n)] = 1.0
        x = rng.standard_normal((n_w, M, n)) + 1j * rng.standard_normal((n_w, M, n))
        phi = d0[None] + noise * x / math.sqrt(2.0)
        q, _ = np.linalg.qr(phi)
        out.append(np.ascontiguousarray(q.astype(np.complex128)))
    return Walkers(out[0], out[1])


def _expm_apply(A: np.ndarray, phi: np.ndarray, order: int = 6) -> np.ndarray:
    """exp(A) @ phi by a Taylor series of the given order (batched)."""
    out = phi.copy()
    term = phi
    for n in range(1, order + 1):
        term = A @ term / n
        out = out + term
    return out


def random_walk(rng: np.random.Generator, sys: System, walkers: Walkers,
                n_steps: int, dt: float, qr_every: int = 5) -> Walkers:
    """Free Gaussian-field random walk of the walkers (Sec. II A).

    Each step applies exp(-dt h'/2) exp(i sqrt(dt) sum_g x_g L_g) exp(-dt h'/2)
    with x ~ N(0, 1) per walker and h' = h - 1/2 sum_g L_g L_g. No force bias
    is applied: the inputs must not depend on the hot path they are used to
    test.
    """
    M = sys.M
    L = sys.L.reshape(sys.n_chol, M * M)
    hp = [sys.h1[s] - 0.5 * np.einsum("gpr,grq->pq", sys.L, sys.L) for s in range(2)]
    # both spins share one field per step, as in the spin-summed two-body term
    phis = [walkers.phi_a.copy(), walkers.phi_b.copy()]
    half = [_expm_apply_matrix(-0.5 * dt * hp[s]) for s in range(2)]
    for step in range(n_steps):
        x = rng.standard_normal((walkers.n_w, sys.n_chol))
        vhs = (1j * math.sqrt(dt)) * (x @ L).reshape(walkers.n_w, M, M)
        for s in range(2):
            p = half[s] @ phis[s]
            p = _expm_apply(vhs, p)
            phis[s] = half[s] @ p
        if (step + 1) % qr_every == 0:
            phis = [np.linalg.qr(p)[0] for p in phis]
    return Walkers(np.ascontiguousarray(phis[0]), np.ascontiguousarray(phis[1]))


def _expm_apply_matrix(A: np.ndarray, order: int = 12) -> np.ndarray:
    return _expm_apply(A, np.eye(A.shape[0], dtype=A.dtype), order)


def make_system(seed: int, M: int, n_alpha: int, n_beta: int, n_core: int,
                n_act_orb: int, n_det: int, max_level: int, power: float,
                n_chol: int, decay: float = 10.0, onsite: float | None = None) -> System:
    rng = np.random.default_rng(seed)
    h1, L = make_hamiltonian(rng, M, n_chol, decay, onsite)
    coeff, occ_a, occ_b = make_trial(rng, M, n_alpha, n_beta, n_core, n_act_orb,
                                     n_det, max_level, power)
    sys = System(M, n_alpha, n_beta, h1, 0.0, L, coeff, occ_a, occ_b, n_core,
                 n_act_orb, dict(seed=seed, decay=decay, power=power,
                                 max_level=max_level, onsite=onsite))
    sys.meta["rng"] = rng  # the walker draws continue this stream
    return sys


# The named workloads. Sizes follow the paper's benchmark systems (Sec. III):
# a copper-oxo-dimer-shaped (32e,108o)-class system and an iron-sulfur-dimer
# (30e,20o active) system, plus a small case the oracle finishes in seconds.
CONFIGS = {
    "small": dict(M=20, n_alpha=5, n_beta=5, n_core=0, n_act_orb=10, n_det=100,
                  max_level=4, power=1.5, n_chol=60, n_w=16, walk_steps=0),
    "cu2o2": dict(M=108, n_alpha=16, n_beta=16, n_core=8, n_act_orb=16, n_det=10000,
                  max_level=6, power=1.5, n_chol=400, n_w=640, walk_steps=20),
    "fe2s2": dict(M=160, n_alpha=30, n_beta=30, n_core=15, n_act_orb=20, n_det=120000,
                  max_level=6, power=1.2, n_chol=800, n_w=640, walk_steps=0),
    # the copper-oxo shape at the paper's largest expansion (N_det = 1e6,
    # Sec. III), run with 640 walkers and in the 10-walker regime
    "cu2o2_1e6": dict(M=108, n_alpha=16, n_beta=16, n_core=8, n_act_orb=16, n_det=1000000,
                      max_level=6, power=1.5, n_chol=400, n_w=640, walk_steps=20),
}


def config_system(name: str, seed: int = 0, n_w: int | None = None,
                  n_det: int | None = None, n_chol: int | None = None,
                  decay: float = 10.0, onsite: float | None = None):
    """(System, Walkers) for a named workload; sizes may be overridden."""
    c = dict(CONFIGS[name])
    if n_det is not None:
        c["n_det"] = n_det
    if n_chol is not None:
        c["n_chol"] = n_chol
    if n_w is not None:
        c["n_w"] = n_w
    sys = make_system(seed, c["M"], c["n_alpha"], c["n_beta"], c["n_core"],
                      c["n_act_orb"], c["n_det"], c["max_level"], c["power"],
                      c["n_chol"], decay, onsite)
    rng = sys.meta.pop("rng")
    w = make_walkers(rng, sys.M, sys.n_alpha, sys.n_beta, c["n_w"])
    if c["walk_steps"]:
        w = random_walk(rng, sys, w, c["walk_steps"], 0.005)
    sys.meta["name"] = name
    return sys, w


def batched_systems(n_systems: int = 32, seed0: int = 0, n_w: int = 128,
                    m_range=(40, 160), det_range=(1e3, 1e5), max_level: int = 6,
                    power: float = 1.5):
    """Uneven independent systems: M ~ U[m_range], N = M // 6 per spin,
    n_det log-uniform in det_range, n_chol = 4 M; active space of
    min(N, 8) electrons in twice as many orbitals per spin."""
    out = []
    for i in range(n_systems):
        rng = np.random.default_rng(seed0 + i)
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        n = M // 6
        n_ae = min(n, 8)
        n_det = int(round(math.exp(rng.uniform(math.log(det_range[0]),
                                               math.log(det_range[1])))))
        sys = make_system(seed0 + i, M, n, n, n - n_ae, 2 * n_ae, n_det, max_level,
                          power, 4 * M)
        rng = sys.meta.pop("rng")
        w = make_walkers(rng, M, n, n, n_w)
        sys.meta["name"] = f"batched[{i}]"
        out.append((sys, w))
    return out


def make_walkers_varied(rng: np.random.Generator, M: int, n_alpha: int, n_beta: int,
                        n_w: int, noise_range=(0.05, 0.35)) -> Walkers:
    """Walkers QR(D0 + s_w (X + iY)/sqrt(2)) with a noise level s_w drawn
    uniformly per walker (training and held-out sets of the control
    variate)."""
    s = rng.uniform(noise_range[0], noise_range[1], size=n_w)
    out = []
    for n in (n_alpha, n_beta):
        d0 = np.zeros((M, n))
        d0[np.arange(n), np.arange(n)] = 1.0
        x = rng.standard_normal((n_w, M, n)) + 1j * rng.standard_normal((n_w, M, n))
        q, _ = np.linalg.qr(d0[None] + s[:, None, None] * x / math.sqrt(2.0))
        out.append(np.ascontiguousarray(q.astype(np.complex128)))
    return Walkers(out[0], out[1])
