"""Failure detection without a GPU fault: the tensor-core kernels' device
waits (a consumer warp waiting for copies or products) are bounded by a
budget (msd_set_wait_budget). With a budget of 0 every such wait is a single
poll, so the first wait that finds its data not yet there expires: the
kernel stops its pipeline, lets its own copies and products in flight
complete, frees its tensor memory and returns, and the call reports
MSD_ERR_TIMEOUT. The context must then still give the right answers."""
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


@pytest.mark.parametrize("call", ["local_energy", "force_bias"])
def test_expired_wait_reports_timeout_and_context_recovers(msd, call):
    s, w = synth.config_system("small", seed=0)
    ref = oracle.msd(s, w.phi_a, w.phi_b, energy=True, vbias=True)
    ctx = msd.Context(s, "mixed")
    da, db = _cuda(w.phi_a), _cuda(w.phi_b)
    fn = getattr(ctx, call)
    first = fn(da, db).cpu().numpy()
    ctx.set_wait_budget(0)
    codes = []
    for _ in range(3):
        try:
            fn(da, db)
            codes.append("ok")
        except msd.MSDError as e:
            codes.append(e.name)
    assert "MSD_ERR_TIMEOUT" in codes and set(codes) <= {"ok", "MSD_ERR_TIMEOUT"}, codes
    ctx.set_wait_budget(2_000_000_000)
    again = fn(da, db).cpu().numpy()
    ctx.close()
    assert np.array_equal(again, first)
    want = ref["e_loc"] if call == "local_energy" else ref["vbias"]
    assert np.allclose(again, want, rtol=1e-4, atol=1e-6 * np.abs(want).max())
