"""msd_rdm1, the mixed one-body density matrix G_T^s[p][q] =
<Psi_T|a+_ps a_qs|phi>/<Psi_T|phi> (the quantity the force bias contracts
with L_g, Eq. 7), against the oracle's sum over determinants of the full
per-determinant Green's functions (Eq. 14); its trace and its contraction
with the Cholesky vectors tie it to the electron count and to the library's
force bias. Bound: FP64 1e-10, mixed 1e-5, of max |G_T| times the overlap's
cancellation factor sum_I |c_I O_I| / |O_T|."""
import numpy as np
import pytest

import oracle
from paper_2406_08314_gb300 import synth

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("name,n_w,prec,tol", [("small", 16, "fp64", 1e-10), ("cu2o2", 2, "fp64", 1e-10),
                                                ("small", 16, "mixed", 1e-5)])
def test_rdm1_against_oracle(msd, name, n_w, prec, tol):
    s, w = synth.config_system(name, seed=0, n_w=n_w)
    ref = oracle.msd(s, w.phi_a, w.phi_b, energy=False, vbias=True, green=True, per_det=True)
    canc = np.sum(np.abs(s.coeff[None, :] * ref["det_ovlp"]), axis=1) / np.abs(ref["ovlp"])
    ctx = msd.Context(s, prec)
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    g = _np(ctx.rdm1(da, db))
    v = _np(ctx.force_bias(da, db))
    ctx.close()
    want = ref["G_T"]
    scale = tol * canc * np.abs(want).reshape(n_w, -1).max(axis=1)
    err = np.abs(g - want).reshape(n_w, -1).max(axis=1)
    assert np.all(err <= scale), (err / scale).max()
    # trace = electrons per spin
    tr = np.einsum("wspp->ws", g)
    assert np.allclose(tr, [[s.n_alpha, s.n_beta]], rtol=0, atol=tol * 10 * canc.max() * max(s.n_alpha, s.n_beta))
    # sum_s tr(L_g G_T^s) is the force bias the library returns
    vb = np.einsum("gpq,wspq->wg", s.L, g)
    assert np.all(np.abs(vb - v) <= (1e-12 if prec == "fp64" else 1e-4) * np.abs(v).max(axis=1, keepdims=True))


def test_rdm1_host_buffers_and_empty(msd):
    s, w = synth.config_system("small", seed=1, n_w=3)
    ctx = msd.Context(s, "fp64")
    g_host = ctx.rdm1(w.phi_a, w.phi_b)          # numpy in, numpy out
    g_dev = _np(ctx.rdm1(_cuda(w.phi_a), _cuda(w.phi_b)))
    assert isinstance(g_host, np.ndarray) and np.array_equal(g_host, g_dev)
    import torch
    e_a = torch.empty((0, s.M, s.n_alpha), dtype=torch.complex128, device="cuda")
    e_b = torch.empty((0, s.M, s.n_beta), dtype=torch.complex128, device="cuda")
    assert ctx.rdm1(e_a, e_b).shape == (0, 2, s.M, s.M)
    ctx.close()
