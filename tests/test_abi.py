"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/msd.h declares (CPU only: no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "msd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(msd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("msd_create", "msd_destroy", "msd_set_hamiltonian", "msd_set_trial",
              "msd_overlap", "msd_force_bias", "msd_local_energy", "msd_det_ratios"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2406_08314_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2406_08314_gb300 import build, msd
    build.build()
    assert sorted(msd.EXPORTS) == _declared()


def test_create_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2406_08314_gb300 import build, msd
    build.build()
    h = ctypes.c_void_p()
    rc = msd.lib().msd_create(ctypes.byref(h), 10, 3, 3, 0, 0)
    assert rc == -3 and h.value is None
    assert b"device" in msd.lib().msd_last_error(None)


def test_switches_reject_a_null_context():
    """Every option setter checks its context on the host before anything
    else (no device is touched), returning MSD_ERR_ARG (-1)."""
    from paper_2406_08314_gb300 import build, msd
    build.build()
    lib = msd.lib()
    for name in ("msd_set_precision", "msd_set_timing", "msd_set_sync", "msd_set_fused",
                 "msd_set_exact_reference", "msd_set_tensor_gram", "msd_set_stream_overlap",
                 "msd_set_pair_form"):
        assert getattr(lib, name)(None, 1) == -1, name
    assert lib.msd_set_workspace_limit(None, ctypes.c_size_t(1 << 20)) == -1
    assert lib.msd_set_wait_budget(None, ctypes.c_ulonglong(1000)) == -1
