"""Tiny hand-made systems for the oracle pins and small parity cases."""
import itertools

import numpy as np

from paper_2406_08314_gb300.synth import System


def tiny_system(seed, M, na, nb, n_chol, n_det=None, max_level=None, complex_h=False):
    """Random symmetric h and L (not orthonormalised), and a CI trial whose
    reference is the first N orbitals. n_det=None takes every determinant of
    the space (up to max_level total excitations if given)."""
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((M, M)); h = 0.5 * (h + h.T)
    L = rng.standard_normal((n_chol, M, M)); L = 0.5 * (L + L.transpose(0, 2, 1))
    ref_a, ref_b = tuple(range(na)), tuple(range(nb))
    pairs = []
    for oa in itertools.combinations(range(M), na):
        for ob in itertools.combinations(range(M), nb):
            k = len(set(oa) - set(ref_a)) + len(set(ob) - set(ref_b))
            if (oa, ob) == (ref_a, ref_b):
                continue
            if max_level is None or k <= max_level:
                pairs.append((oa, ob))
    order = rng.permutation(len(pairs))
    if n_det is not None:
        order = order[: n_det - 1]
    pairs = [(ref_a, ref_b)] + [pairs[i] for i in order]
    occ_a = np.array([p[0] for p in pairs], np.int32)
    occ_b = np.array([p[1] for p in pairs], np.int32)
    coeff = rng.standard_normal(len(pairs))
    coeff[0] = 2.0 + abs(coeff[0])
    coeff /= np.linalg.norm(coeff)
    return System(M, na, nb, np.stack([h, h]), float(rng.standard_normal()), L, coeff,
                  occ_a, occ_b)


def tiny_walkers(seed, M, na, nb, n_w=1, noise=0.5, real=False):
    rng = np.random.default_rng(seed + 1000)
    out = []
    for n in (na, nb):
        x = rng.standard_normal((n_w, M, n))
        if not real:
            x = x + 1j * rng.standard_normal((n_w, M, n))
        d0 = np.zeros((M, n)); d0[np.arange(n), np.arange(n)] = 1.0
        out.append(np.ascontiguousarray((d0[None] + noise * x).astype(np.complex128)))
    return out
