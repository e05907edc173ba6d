"""msd_propagate (one phaseless AFQMC step, Sec. II A, Eq. 7-12) against the
propagation oracle: walkers, weights and overlap ratios, with and without
the QR orthonormalisation, over several steps, across walker chunks, in FP64
(1e-10 relative) and with mixed-precision overlaps and force bias (bounded
by the force bias' mixed error)."""
import ctypes

import numpy as np
import pytest

from oracle import prop_oracle as po
from paper_2406_08314_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def msd():
    from paper_2406_08314_gb300 import build
    build.build()
    from paper_2406_08314_gb300 import msd as m
    return m


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _run(msd, s, pa, pb, w, x, dt, order=6, qr=False, prec="fp64", ws=None, fused=True):
    import torch
    ctx = msd.Context(s, prec)
    if ws:
        ctx.set_workspace_limit(ws)
    da, db, dw, dx = _dev(pa), _dev(pb), _dev(w), _dev(x)
    S = ctx.propagate(da, db, dw, dx, dt, order, qr)
    torch.cuda.synchronize()
    out = tuple(t.cpu().numpy() for t in (da, db, dw, S))
    ctx.close()
    return out


@pytest.mark.parametrize("qr", [False, True])
def test_small_one_step_fp64(msd, qr):
    s, w = synth.config_system("small", seed=0)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((w.n_w, s.n_chol))
    wt = rng.uniform(0.5, 1.5, w.n_w)
    a, b, wn, S = _run(msd, s, w.phi_a, w.phi_b, wt, x, 0.01, qr=qr)
    ra, rb, rw, rS = po.step(s, w.phi_a, w.phi_b, wt, x, 0.01, order=6, orthonormalize=qr)
    assert _rel(S, rS) <= TOL
    assert _rel(wn, rw) <= TOL
    assert _rel(a, ra) <= TOL and _rel(b, rb) <= TOL


def test_small_three_steps_with_qr_and_taylor_orders(msd):
    s, w = synth.config_system("small", seed=2)
    rng = np.random.default_rng(3)
    pa, pb, wt = w.phi_a[:5], w.phi_b[:5], np.ones(5)
    ga, gb, gw = pa, pb, wt
    for step, order in enumerate((1, 4, 8)):
        x = rng.standard_normal((5, s.n_chol))
        ga, gb, gw, gS = _run(msd, s, ga, gb, gw, x, 0.02, order=order, qr=(step == 2))
        pa, pb, wt, rS = po.step(s, pa, pb, wt, x, 0.02, order=order, orthonormalize=(step == 2))
        assert _rel(gS, rS) <= TOL, step
        assert _rel(gw, wt) <= TOL, step
        assert _rel(ga, pa) <= TOL and _rel(gb, pb) <= TOL, step


@pytest.mark.parametrize("M,na,nb,n_det,seed", [(12, 5, 4, 60, 0), (14, 7, 3, 40, 1)])
def test_tiny_uneven_spins(msd, M, na, nb, n_det, seed):
    s = synth.make_system(seed, M, na, nb, n_core=1, n_act_orb=M - 2, n_det=n_det, max_level=4,
                          power=1.5, n_chol=9)
    rng = np.random.default_rng(seed + 10)
    w = synth.make_walkers(rng, M, na, nb, 4, noise=0.3)
    x = rng.standard_normal((4, s.n_chol))
    a, b, wn, S = _run(msd, s, w.phi_a, w.phi_b, np.ones(4), x, 0.03, qr=True)
    ra, rb, rw, rS = po.step(s, w.phi_a, w.phi_b, np.ones(4), x, 0.03, orthonormalize=True)
    assert _rel(S, rS) <= TOL and _rel(wn, rw) <= TOL
    assert _rel(a, ra) <= TOL and _rel(b, rb) <= TOL


def test_cu2o2_shaped_two_walkers(msd):
    s, w = synth.config_system("cu2o2", seed=0, n_w=2)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, s.n_chol))
    a, b, wn, S = _run(msd, s, w.phi_a, w.phi_b, np.ones(2), x, 0.005)
    ra, rb, rw, rS = po.step(s, w.phi_a, w.phi_b, np.ones(2), x, 0.005)
    assert _rel(S, rS) <= TOL and _rel(wn, rw) <= TOL
    assert _rel(a, ra) <= TOL and _rel(b, rb) <= TOL


def test_walker_chunks_match(msd):
    """A workspace limit small enough for several walker chunks of the field
    propagator gives the same walkers and weights."""
    s, w = synth.config_system("small", seed=6)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((w.n_w, s.n_chol))
    full = _run(msd, s, w.phi_a, w.phi_b, np.ones(w.n_w), x, 0.01, qr=True)
    chunked = _run(msd, s, w.phi_a, w.phi_b, np.ones(w.n_w), x, 0.01, qr=True, ws=64 * 1024)
    for u, v in zip(full, chunked):
        assert np.allclose(u, v, rtol=1e-13, atol=0)


def test_mixed_precision_context(msd):
    """Mixed contexts take overlaps and force bias from the mixed path; the
    field propagator is FP64 either way. The walkers then differ from the
    FP64 oracle by sqrt(dt) times the force bias' mixed error (<= 1e-4
    relative, see the mixed parity tests), the weights and ratios likewise."""
    s, w = synth.config_system("small", seed=8)
    rng = np.random.default_rng(9)
    x = rng.standard_normal((w.n_w, s.n_chol))
    a, b, wn, S = _run(msd, s, w.phi_a, w.phi_b, np.ones(w.n_w), x, 0.01, prec="mixed")
    ra, rb, rw, rS = po.step(s, w.phi_a, w.phi_b, np.ones(w.n_w), x, 0.01)
    assert _rel(a, ra) <= 1e-5 and _rel(b, rb) <= 1e-5
    assert _rel(wn, rw) <= 1e-5 and _rel(S, rS) <= 1e-5


def test_argument_errors(msd):
    import torch
    s, w = synth.config_system("small", seed=0)
    ctx = msd.Context(s, "fp64")
    lib = msd.lib()
    da, db = _dev(w.phi_a), _dev(w.phi_b)
    wt = torch.ones(w.n_w, dtype=torch.float64, device="cuda")
    x = torch.zeros((w.n_w, s.n_chol), dtype=torch.float64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.msd_propagate(ctx._h, 0, p(da), p(db), p(wt), p(x), 0.01, 6, 0, None, st) == 0
    assert lib.msd_propagate(ctx._h, w.n_w, p(da), p(db), p(wt), p(x), 0.0, 6, 0, None, st) == -1
    assert lib.msd_propagate(ctx._h, w.n_w, p(da), p(db), p(wt), p(x), 0.01, 0, 0, None, st) == -1
    wh = np.ones(w.n_w)
    assert lib.msd_propagate(ctx._h, w.n_w, p(da), p(db), ctypes.c_void_p(wh.ctypes.data), p(x), 0.01, 6, 0,
                             None, st) == -1
    assert b"device pointers" in lib.msd_last_error(ctx._h)
    ctx.close()
