"""The seeded generator produces well-formed inputs (CPU only)."""
import numpy as np

from paper_2406_08314_gb300 import synth


def test_small_config_shapes_and_structure():
    s, w = synth.config_system("small", seed=0)
    assert s.h1.shape == (2, 20, 20) and np.allclose(s.h1[0], s.h1[0].T)
    assert s.L.shape == (60, 20, 20) and np.allclose(s.L, s.L.transpose(0, 2, 1))
    assert s.n_det == 100 and abs(np.sum(s.coeff ** 2) - 1) < 1e-12 and s.coeff[0] > 0
    assert (np.diff(s.occ_a, axis=1) > 0).all() and (np.diff(s.occ_b, axis=1) > 0).all()
    assert (s.occ_a[0] == np.arange(5)).all() and (s.occ_b[0] == np.arange(5)).all()
    pairs = {(tuple(a), tuple(b)) for a, b in zip(s.occ_a, s.occ_b)}
    assert len(pairs) == 100                               # distinct determinants
    lv = [len(set(a) - set(range(5))) + len(set(b) - set(range(5)))
          for a, b in zip(s.occ_a, s.occ_b)]
    assert lv[0] == 0 and max(lv) <= 4 and lv == sorted(lv)  # sorted by level
    assert w.phi_a.shape == (16, 20, 5) and w.phi_a.dtype == np.complex128
    for p in (w.phi_a, w.phi_b):                           # orthonormal columns
        assert np.allclose(np.conj(p.transpose(0, 2, 1)) @ p, np.eye(5)[None], atol=1e-12)
    # Frobenius-orthogonal Cholesky vectors with the stated decay
    gram = np.einsum("gpq,hpq->gh", s.L, s.L)
    assert np.allclose(gram - np.diag(np.diag(gram)), 0, atol=1e-10)
    d = np.sqrt(np.diag(gram))
    assert np.allclose(d, np.exp(-0.1 * np.arange(60)))      # singular values exp(-g/10)


def test_chemical_scale_variant():
    s = synth.make_system(0, 20, 5, 5, 0, 10, 50, 4, 1.5, 60, onsite=1.0)
    assert abs(np.mean(np.sum(np.einsum("gpp->gp", s.L) ** 2, axis=0)) - 1.0) < 1e-12


def test_seeded_and_reproducible():
    a, wa = synth.config_system("small", seed=3)
    b, wb = synth.config_system("small", seed=3)
    c, _ = synth.config_system("small", seed=4)
    assert np.array_equal(a.occ_a, b.occ_a) and np.array_equal(wa.phi_b, wb.phi_b)
    assert not np.array_equal(a.L, c.L)


def test_active_space_respected():
    s, _ = synth.config_system("small", seed=1, n_w=1)
    s2 = synth.make_system(5, 30, 8, 8, 4, 8, 300, 6, 1.5, 20)
    for occ, n in ((s2.occ_a, 8), (s2.occ_b, 8)):
        for row in occ:
            holes = set(range(n)) - set(row)
            parts = set(row) - set(range(n))
            assert holes <= set(range(4, 8)) and parts <= set(range(8, 12))
