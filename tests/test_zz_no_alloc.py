"""msd_overlap_noalloc: the overlap entry point for callers that cannot let
the library allocate device memory during a call (a framework that owns all
device allocations, or a loop that must not take cudaMalloc's implicit
synchronisation). It must return what msd_overlap returns, on consecutive
calls, without growing the context's allocated workspace.

Collected last on purpose (file name) so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process."""
import ctypes

import numpy as np
import pytest

from paper_2406_08314_gb300 import synth

pytestmark = pytest.mark.gpu


def test_overlap_noalloc_matches_overlap_on_two_calls():
    import torch

    from paper_2406_08314_gb300 import build
    build.build()
    from paper_2406_08314_gb300 import msd

    # 300 walkers of the copper-oxo-shaped system need several chunks of the
    # 64 MiB static scratch
    s, w = synth.config_system("cu2o2", seed=3, n_w=300)
    da = torch.from_numpy(w.phi_a).cuda()
    db = torch.from_numpy(w.phi_b).cuda()

    ref = msd.Context(s, "fp64")
    ov_ref, rs_ref = ref.overlap(da, db, ratio_sum=True)
    ov_ref, rs_ref = ov_ref.cpu().numpy(), rs_ref.cpu().numpy()
    ref.close()

    ctx = msd.Context(s, "fp64")            # fresh context: no workspace yet
    assert ctx.info("workspace_bytes") == 0
    lib = msd.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        ov = torch.full((w.n_w,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        rs = torch.full((w.n_w,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        rc = lib.msd_overlap_noalloc(ctx._h, w.n_w, ctypes.c_void_p(da.data_ptr()),
                                     ctypes.c_void_p(db.data_ptr()), ctypes.c_void_p(ov.data_ptr()),
                                     ctypes.c_void_p(rs.data_ptr()), stream)
        assert rc == 0, lib.msd_last_error(ctx._h)
        torch.cuda.synchronize()
        ov_n, rs_n = ov.cpu().numpy(), rs.cpu().numpy()
        # same kernels and reduction order as msd_overlap; the FP64 tolerance
        # of the parity tests
        assert np.all(np.abs(ov_n - ov_ref) <= 1e-10 * np.abs(ov_ref)), call
        assert np.all(np.abs(rs_n - rs_ref) <= 1e-10 * np.abs(rs_ref)), call
    assert ctx.info("workspace_bytes") == 0     # nothing was allocated for the calls

    # host buffers are refused (the call cannot stage them)
    ov_h = np.zeros(w.n_w, np.complex128)
    rc = lib.msd_overlap_noalloc(ctx._h, w.n_w, ctypes.c_void_p(da.data_ptr()),
                                 ctypes.c_void_p(db.data_ptr()), ctypes.c_void_p(ov_h.ctypes.data),
                                 None, stream)
    assert rc == -1 and b"device pointers" in lib.msd_last_error(ctx._h)
    ctx.close()
