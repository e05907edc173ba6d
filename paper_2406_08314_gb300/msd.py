"""Python binding of libmsd (include/msd.h): argument marshalling only.

Every step of the hot path runs in the CUDA library. Importing this module
loads libmsd.so; it raises if the library has not been built (there is no
fallback of any kind). Walkers and outputs are torch tensors (complex128) on
the context's CUDA device, or host arrays (numpy or CPU torch tensors),
which the library stages through device memory.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MSD_FP64 = 0
MSD_MIXED = 1
_ERRORS = {-1: "MSD_ERR_ARG", -2: "MSD_ERR_SHAPE", -3: "MSD_ERR_CUDA", -4: "MSD_ERR_TIMEOUT",
           -5: "MSD_ERR_REF_SINGULAR", -6: "MSD_ERR_STATE", -7: "MSD_ERR_NOMEM"}
EXPORTS = ["msd_create", "msd_destroy", "msd_last_error", "msd_set_hamiltonian", "msd_set_trial",
           "msd_set_precision", "msd_overlap", "msd_det_ratios", "msd_force_bias",
           "msd_local_energy", "msd_evaluate", "msd_det_energies", "msd_rdm1", "msd_info", "msd_set_timing", "msd_reset_stats",
           "msd_kernel_count", "msd_kernel_stat", "msd_set_workspace_limit", "msd_set_sync", "msd_set_fused", "msd_set_pair_form", "msd_set_exact_reference", "msd_set_tensor_gram", "msd_set_stream_overlap", "msd_set_wait_budget", "msd_propagate",
           "msd_launch_count", "msd_overlap_noalloc", "msd_batch_create", "msd_batch_destroy",
           "msd_batch_last_error", "msd_batch_evaluate", "msd_batch_autotune", "msd_batch_config",
           "msd_batch_set_config", "msd_batch_time_persistent", "msd_batch_graph_ready", "msd_batch_graph_kernels", "msd_features", "msd_features_rows",
           "msd_mlp_create", "msd_mlp_destroy", "msd_mlp_last_error", "msd_mlp_param_count",
           "msd_mlp_set_params", "msd_mlp_get_params", "msd_mlp_forward", "msd_mlp_grad", "msd_mlp_adam_step"]
INFO = {"n_det": 1, "n_chol": 2, "n_strings_a": 3, "n_strings_b": 4, "n_holes_a": 5,
        "n_parts_a": 6, "n_holes_b": 7, "n_parts_b": 8, "workspace_bytes": 9, "walker_chunk": 10, "exact_reference": 11}


class MSDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = _ERRORS.get(code, str(code))


def load_library(path: str | None = None) -> ctypes.CDLL:
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmsd.so not found at {path}; build it with "
                           "`python -m paper_2406_08314_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, ci, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    lib.msd_create.argtypes = [ctypes.POINTER(vp), ci, ci, ci, ci, ci]
    lib.msd_destroy.argtypes = [vp]
    lib.msd_destroy.restype = None
    lib.msd_last_error.argtypes = [vp]
    lib.msd_last_error.restype = ctypes.c_char_p
    lib.msd_set_hamiltonian.argtypes = [vp, vp, ctypes.c_double, ci, vp]
    lib.msd_set_trial.argtypes = [vp, ci, vp, vp, vp]
    lib.msd_set_precision.argtypes = [vp, ci]
    for f in ("msd_overlap", "msd_det_ratios", "msd_force_bias", "msd_local_energy",
              "msd_overlap_noalloc"):
        getattr(lib, f).argtypes = [vp, ci, vp, vp, vp, vp, vp]
    lib.msd_evaluate.argtypes = [vp, ci, vp, vp, vp, vp, vp, vp]
    lib.msd_info.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_longlong)]
    lib.msd_set_timing.argtypes = [vp, ci]
    lib.msd_reset_stats.argtypes = [vp]
    lib.msd_kernel_count.argtypes = [vp]
    lib.msd_kernel_stat.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_char_p),
                                    ctypes.POINTER(ctypes.c_longlong), dp]
    lib.msd_set_workspace_limit.argtypes = [vp, ctypes.c_size_t]
    lib.msd_set_sync.argtypes = [vp, ci]
    lib.msd_set_fused.argtypes = [vp, ci]
    lib.msd_set_pair_form.argtypes = [vp, ci]
    lib.msd_set_exact_reference.argtypes = [vp, ci]
    lib.msd_set_tensor_gram.argtypes = [vp, ci]
    lib.msd_set_stream_overlap.argtypes = [vp, ci]
    lib.msd_set_wait_budget.argtypes = [vp, ctypes.c_ulonglong]
    lib.msd_det_energies.argtypes = [vp, ci, vp, vp, ci, vp, vp, vp, vp]
    lib.msd_rdm1.argtypes = [vp, ci, vp, vp, vp, vp]
    lib.msd_propagate.argtypes = [vp, ci, vp, vp, vp, vp, ctypes.c_double, ci, ci, vp, vp]
    lib.msd_launch_count.argtypes = []
    for f in EXPORTS:
        if f not in ("msd_destroy", "msd_last_error"):
            getattr(lib, f).restype = ci
    lib.msd_launch_count.restype = ctypes.c_longlong
    pp = ctypes.POINTER(ctypes.c_void_p)
    lib.msd_batch_create.argtypes = [ctypes.POINTER(vp), pp, ci]
    lib.msd_batch_destroy.argtypes = [vp]
    lib.msd_batch_destroy.restype = None
    lib.msd_batch_last_error.argtypes = [vp]
    lib.msd_batch_last_error.restype = ctypes.c_char_p
    lib.msd_batch_evaluate.argtypes = [vp, ctypes.POINTER(ci), pp, pp, pp, pp, pp, vp]
    lib.msd_batch_autotune.argtypes = [vp, ctypes.POINTER(ci), pp, pp, pp, pp, pp, vp, ctypes.c_char_p]
    lib.msd_batch_config.argtypes = [vp, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(ci)]
    lib.msd_batch_set_config.argtypes = [vp, ci, ci, ci]
    lib.msd_batch_time_persistent.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_double)]
    lib.msd_batch_graph_ready.argtypes = [vp]
    lib.msd_batch_graph_kernels.argtypes = [vp]
    lib.msd_batch_graph_kernels.restype = ctypes.c_longlong
    lib.msd_features.argtypes = [vp, ci, vp, vp, ci, ci, vp, vp]
    lib.msd_features_rows.argtypes = [vp, ci, vp, vp, ci, vp, vp]
    lib.msd_mlp_create.argtypes = [ctypes.POINTER(vp), ci, ci, ci]
    lib.msd_mlp_destroy.argtypes = [vp]
    lib.msd_mlp_destroy.restype = None
    lib.msd_mlp_last_error.argtypes = [vp]
    lib.msd_mlp_last_error.restype = ctypes.c_char_p
    lib.msd_mlp_param_count.argtypes = [vp]
    lib.msd_mlp_param_count.restype = ctypes.c_longlong
    lib.msd_mlp_set_params.argtypes = [vp, vp]
    lib.msd_mlp_get_params.argtypes = [vp, vp]
    lib.msd_mlp_forward.argtypes = [vp, ci, vp, vp, vp]
    lib.msd_mlp_grad.argtypes = [vp, ci, vp, vp, vp, vp, vp]
    lib.msd_mlp_adam_step.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp]
    return lib


_lib = load_library()


def lib() -> ctypes.CDLL:
    return _lib


def launch_count() -> int:
    """Kernel launches made by libmsd in this process so far."""
    return int(_lib.msd_launch_count())


def _torch():
    import torch
    return torch


def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def _ptr(x):
    """Data pointer of a contiguous complex128 torch tensor or numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous and x.dtype == np.complex128
        return ctypes.c_void_p(x.ctypes.data)
    torch = _torch()
    assert x.is_contiguous() and x.dtype == torch.complex128, "expected contiguous complex128"
    return ctypes.c_void_p(x.data_ptr())


class Context:
    """One trial + Hamiltonian on one GPU. Mirrors the C-ABI entry points."""

    def __init__(self, system, precision: str | int = "fp64", device: int = 0):
        prec = {"fp64": MSD_FP64, "mixed": MSD_MIXED}.get(precision, precision)
        h = ctypes.c_void_p()
        rc = _lib.msd_create(ctypes.byref(h), system.M, system.n_alpha, system.n_beta, int(prec),
                             int(device))
        if rc:
            raise MSDError(rc, _lib.msd_last_error(None).decode())
        self._h = h
        self.device = device
        self.M, self.n_alpha, self.n_beta = system.M, system.n_alpha, system.n_beta
        self.n_chol = system.n_chol
        self.n_det = system.n_det
        h1 = np.ascontiguousarray(system.h1, np.float64)
        L = np.ascontiguousarray(system.L, np.float64)
        self._check(_lib.msd_set_hamiltonian(h, h1.ctypes.data_as(ctypes.c_void_p), float(system.e0),
                                             L.shape[0], L.ctypes.data_as(ctypes.c_void_p)))
        self.set_trial(system.coeff, system.occ_a, system.occ_b)

    def _check(self, rc):
        if rc:
            raise MSDError(rc, _lib.msd_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _lib.msd_destroy(self._h)
            self._h = None

    __del__ = close

    def set_trial(self, coeff, occ_a, occ_b):
        c = np.ascontiguousarray(coeff, np.float64)
        a = np.ascontiguousarray(occ_a, np.int32)
        b = np.ascontiguousarray(occ_b, np.int32)
        self._check(_lib.msd_set_trial(self._h, c.shape[0], c.ctypes.data_as(ctypes.c_void_p),
                                       a.ctypes.data_as(ctypes.c_void_p),
                                       b.ctypes.data_as(ctypes.c_void_p)))
        self.n_det = c.shape[0]

    def set_precision(self, precision):
        prec = {"fp64": MSD_FP64, "mixed": MSD_MIXED}.get(precision, precision)
        self._check(_lib.msd_set_precision(self._h, int(prec)))

    def info(self, key: str) -> int:
        v = ctypes.c_longlong()
        self._check(_lib.msd_info(self._h, INFO[key], ctypes.byref(v)))
        return v.value

    # -------------------------------------------------------------- outputs
    def _alloc(self, like, shape):
        if _is_cuda(like):
            torch = _torch()
            return torch.empty(shape, dtype=torch.complex128, device=like.device)
        return np.empty(shape, np.complex128)

    def _stream(self, like, stream):
        if stream is not None:
            return ctypes.c_void_p(int(stream))
        if _is_cuda(like):
            return ctypes.c_void_p(_torch().cuda.current_stream(like.device).cuda_stream)
        return ctypes.c_void_p(0)

    def _walkers(self, phi_a, phi_b):
        n_w = phi_a.shape[0]
        assert tuple(phi_a.shape) == (n_w, self.M, self.n_alpha), phi_a.shape
        assert tuple(phi_b.shape) == (n_w, self.M, self.n_beta), phi_b.shape
        return n_w

    def overlap(self, phi_a, phi_b, stream=None, ratio_sum=False):
        n_w = self._walkers(phi_a, phi_b)
        ov = self._alloc(phi_a, (n_w,))
        rs = self._alloc(phi_a, (n_w,)) if ratio_sum else None
        self._check(_lib.msd_overlap(self._h, n_w, _ptr(phi_a), _ptr(phi_b), _ptr(ov), _ptr(rs),
                                     self._stream(phi_a, stream)))
        return (ov, rs) if ratio_sum else ov

    def overlap_noalloc(self, phi_a, phi_b, ovlp, ratio_sum=None, stream=None):
        """msd_overlap into caller-provided device tensors, with the
        library's static scratch instead of allocated workspace."""
        n_w = self._walkers(phi_a, phi_b)
        self._check(_lib.msd_overlap_noalloc(self._h, n_w, _ptr(phi_a), _ptr(phi_b), _ptr(ovlp),
                                             _ptr(ratio_sum), self._stream(phi_a, stream)))
        return ovlp, ratio_sum

    def features(self, phi_a, phi_b, n_core, n_act, stream=None):
        """Active-space reference Green's function features, FP32
        [n_w][2][n_act][n_act][2] (device)."""
        import torch
        n_w = self._walkers(phi_a, phi_b)
        f = torch.empty((n_w, 2, n_act, n_act, 2), dtype=torch.float32, device=phi_a.device)
        self._check(_lib.msd_features(self._h, n_w, _ptr(phi_a), _ptr(phi_b), int(n_core), int(n_act),
                                      ctypes.c_void_p(f.data_ptr()), self._stream(phi_a, stream)))
        return f

    def features_rows(self, phi_a, phi_b, stream=None):
        """Non-zero rows of the reference Green's function, FP32
        [n_w][ld], ld = 2 (N_a + N_b) M rounded up to a multiple of 64
        (zero padded)."""
        import torch
        n_w = self._walkers(phi_a, phi_b)
        need = 2 * (self.n_alpha + self.n_beta) * self.M
        ld = (need + 63) // 64 * 64
        f = torch.empty((n_w, ld), dtype=torch.float32, device=phi_a.device)
        self._check(_lib.msd_features_rows(self._h, n_w, _ptr(phi_a), _ptr(phi_b), ld,
                                           ctypes.c_void_p(f.data_ptr()), self._stream(phi_a, stream)))
        return f

    def det_ratios(self, phi_a, phi_b, stream=None, ref_ovlp=False):
        n_w = self._walkers(phi_a, phi_b)
        r = self._alloc(phi_a, (n_w, self.n_det))
        o = self._alloc(phi_a, (n_w,)) if ref_ovlp else None
        self._check(_lib.msd_det_ratios(self._h, n_w, _ptr(phi_a), _ptr(phi_b), _ptr(r), _ptr(o),
                                        self._stream(phi_a, stream)))
        return (r, o) if ref_ovlp else r

    def force_bias(self, phi_a, phi_b, stream=None, ovlp=False, out=None):
        n_w = self._walkers(phi_a, phi_b)
        v = out if out is not None else self._alloc(phi_a, (n_w, self.n_chol))
        o = self._alloc(phi_a, (n_w,)) if ovlp else None
        self._check(_lib.msd_force_bias(self._h, n_w, _ptr(phi_a), _ptr(phi_b), _ptr(v), _ptr(o),
                                        self._stream(phi_a, stream)))
        return (v, o) if ovlp else v

    def local_energy(self, phi_a, phi_b, stream=None, ovlp=False, out=None):
        n_w = self._walkers(phi_a, phi_b)
        e = out if out is not None else self._alloc(phi_a, (n_w,))
        o = self._alloc(phi_a, (n_w,)) if ovlp else None
        self._check(_lib.msd_local_energy(self._h, n_w, _ptr(phi_a), _ptr(phi_b), _ptr(e), _ptr(o),
                                          self._stream(phi_a, stream)))
        return (e, o) if ovlp else e

    def evaluate(self, phi_a, phi_b, stream=None, out=None):
        """(ovlp, vbias, e_loc) in one pass; `out` may give the three
        output arrays."""
        n_w = self._walkers(phi_a, phi_b)
        if out is None:
            out = (self._alloc(phi_a, (n_w,)), self._alloc(phi_a, (n_w, self.n_chol)),
                   self._alloc(phi_a, (n_w,)))
        o, v, e = out
        self._check(_lib.msd_evaluate(self._h, n_w, _ptr(phi_a), _ptr(phi_b), _ptr(o), _ptr(v), _ptr(e),
                                      self._stream(phi_a, stream)))
        return o, v, e

    def rdm1(self, phi_a, phi_b, stream=None, out=None):
        """Mixed one-body density matrices G_T [n_w][2][M][M] (complex)."""
        n_w = self._walkers(phi_a, phi_b)
        r = out if out is not None else self._alloc(phi_a, (n_w, 2, self.M, self.M))
        self._check(_lib.msd_rdm1(self._h, n_w, _ptr(phi_a), _ptr(phi_b), _ptr(r), self._stream(phi_a, stream)))
        return r

    def det_energies(self, phi_a, phi_b, w_idx, det_idx, stream=None):
        """E_I of the sampled (walker, determinant) pairs (w_idx[i], det_idx[i])
        from the energy path's own intermediates (complex, like phi_a)."""
        n_w = self._walkers(phi_a, phi_b)
        wi = np.ascontiguousarray(w_idx, np.int32)
        di = np.ascontiguousarray(det_idx, np.int32)
        assert wi.shape == di.shape and wi.ndim == 1
        out = self._alloc(phi_a, (wi.shape[0],))
        self._check(_lib.msd_det_energies(self._h, n_w, _ptr(phi_a), _ptr(phi_b), int(wi.shape[0]),
                                          wi.ctypes.data_as(ctypes.c_void_p), di.ctypes.data_as(ctypes.c_void_p),
                                          _ptr(out), self._stream(phi_a, stream)))
        return out

    def set_tensor_gram(self, on: bool):
        """Mixed precision: Gram matrices on the tensor cores, or by FP32
        FMAs (the default)."""
        self._check(_lib.msd_set_tensor_gram(self._h, int(bool(on))))

    def set_stream_overlap(self, on: bool):
        """Mixed energy: the per-walker sums after the Cholesky contraction,
        then the force bias, on a second stream, concurrent with the strings
        and weights, then with the per-determinant terms (default on;
        identical results either way)."""
        self._check(_lib.msd_set_stream_overlap(self._h, int(bool(on))))

    def set_wait_budget(self, ns: int):
        """Budget (ns) of the tensor-core kernels' device-side waits;
        2_000_000_000 by default, 0 = a single poll."""
        self._check(_lib.msd_set_wait_budget(self._h, int(ns)))

    def set_exact_reference(self, on: bool):
        """Mixed precision: reference-determinant energy to FP64 accuracy
        (default on) or from the FP32 traces."""
        self._check(_lib.msd_set_exact_reference(self._h, int(bool(on))))

    # --------------------------------------------------------------- timing
    def set_timing(self, enable=True):
        self._check(_lib.msd_set_timing(self._h, int(bool(enable))))

    def reset_stats(self):
        self._check(_lib.msd_reset_stats(self._h))

    def kernel_stats(self) -> dict:
        out = {}
        for i in range(_lib.msd_kernel_count(self._h)):
            name = ctypes.c_char_p()
            n = ctypes.c_longlong()
            ms = ctypes.c_double()
            self._check(_lib.msd_kernel_stat(self._h, i, ctypes.byref(name), ctypes.byref(n),
                                             ctypes.byref(ms)))
            out[name.value.decode()] = (n.value, ms.value)
        return out

    def set_workspace_limit(self, nbytes: int):
        self._check(_lib.msd_set_workspace_limit(self._h, int(nbytes)))

    def set_sync(self, sync: bool):
        self._check(_lib.msd_set_sync(self._h, int(bool(sync))))

    def propagate(self, phi_a, phi_b, weights, x, dt: float, order: int = 6, orthonormalize: bool = False):
        """One phaseless AFQMC step (Sec. II A) of device walkers, in place:
        phi_a, phi_b (n_w, M, N) complex128, weights (n_w,) float64, x
        (n_w, n_chol) float64 Gaussian fields. Returns the overlap ratios S
        (n_w,) complex128."""
        import torch
        n_w = phi_a.shape[0]
        for t, dt_ in ((phi_a, torch.complex128), (phi_b, torch.complex128), (weights, torch.float64),
                       (x, torch.float64)):
            if not t.is_cuda or t.dtype != dt_ or not t.is_contiguous():
                raise ValueError("propagate takes contiguous CUDA tensors (complex128 walkers, float64 "
                                 "weights and fields)")
        ratio = torch.empty(n_w, dtype=torch.complex128, device=phi_a.device)
        raw = lambda t: ctypes.c_void_p(t.data_ptr())
        self._check(_lib.msd_propagate(self._h, n_w, raw(phi_a), raw(phi_b), raw(weights), raw(x),
                                       float(dt), int(order), int(bool(orthonormalize)), raw(ratio),
                                       self._stream(phi_a, None)))
        return ratio

    def set_fused(self, fused: bool):
        """Mixed precision: fused tensor-core contraction + epilogue (default)
        or the separate GEMM and epilogue kernels."""
        self._check(_lib.msd_set_fused(self._h, int(bool(fused))))

    def set_pair_form(self, form):
        """Opposite-spin energy term per determinant (False / 0), per beta
        string (True / 1, mixed precision), over runs of determinants sharing
        a string (2) or chosen per trial by the library's cost model ("auto" /
        -1, the default); msd_set_pair_form."""
        f = -1 if form == "auto" else int(form)
        self._check(_lib.msd_set_pair_form(self._h, f))


class Batch:
    """Independent systems evaluated together (msd_batch_*): one persistent
    launch for the per-determinant terms of all systems, recorded as a CUDA
    graph and replayed while the buffers stay the same."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        h = ctypes.c_void_p()
        rc = _lib.msd_batch_create(ctypes.byref(h), arr, len(self.contexts))
        if rc:
            raise MSDError(rc, _lib.msd_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.msd_batch_destroy(self._h)
            self._h = None

    __del__ = close

    def _check(self, rc):
        if rc:
            raise MSDError(rc, _lib.msd_batch_last_error(self._h).decode())

    def _args(self, walkers, outs):
        n = len(self.contexts)
        nw = (ctypes.c_int * n)(*[int(a.shape[0]) for a, _ in walkers])
        P = ctypes.c_void_p * n
        pa = P(*[a.data_ptr() for a, _ in walkers])
        pb = P(*[b.data_ptr() for _, b in walkers])
        ov = P(*[o.data_ptr() for o, _, _ in outs])
        vb = P(*[v.data_ptr() for _, v, _ in outs])
        el = P(*[e.data_ptr() for _, _, e in outs])
        return nw, pa, pb, ov, vb, el

    def outputs(self, walkers):
        import torch
        return [(torch.empty((a.shape[0],), dtype=torch.complex128, device=a.device),
                 torch.empty((a.shape[0], c.n_chol), dtype=torch.complex128, device=a.device),
                 torch.empty((a.shape[0],), dtype=torch.complex128, device=a.device))
                for (a, _), c in zip(walkers, self.contexts)]

    def evaluate(self, walkers, outs=None, stream=None):
        """walkers: [(phi_a, phi_b)] device tensors per system; returns
        [(ovlp, vbias, e_loc)] per system."""
        import torch
        outs = outs if outs is not None else self.outputs(walkers)
        st = ctypes.c_void_p(int(stream) if stream is not None else torch.cuda.current_stream().cuda_stream)
        self._check(_lib.msd_batch_evaluate(self._h, *self._args(walkers, outs), st))
        return outs

    def autotune(self, walkers, outs=None, cache_path=None, stream=None):
        import torch
        outs = outs if outs is not None else self.outputs(walkers)
        st = ctypes.c_void_p(int(stream) if stream is not None else torch.cuda.current_stream().cuda_stream)
        cp = cache_path.encode() if cache_path else None
        self._check(_lib.msd_batch_autotune(self._h, *self._args(walkers, outs), st, cp))
        return self.config()

    def config(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(_lib.msd_batch_config(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"tile_n": a.value, "ctas_per_sm": b.value, "order": c.value}

    def set_config(self, tile_n=0, ctas_per_sm=2, order=0):
        self._check(_lib.msd_batch_set_config(self._h, tile_n, ctas_per_sm, order))

    def time_persistent(self, enable=True):
        """Enable CUDA-event timing of the persistent kernel in the next eager
        run; returns the last such time (ms) or -1."""
        ms = ctypes.c_double()
        self._check(_lib.msd_batch_time_persistent(self._h, int(bool(enable)), ctypes.byref(ms)))
        return ms.value

    def graph_ready(self) -> bool:
        return bool(_lib.msd_batch_graph_ready(self._h))

    def graph_kernels(self) -> int:
        return int(_lib.msd_batch_graph_kernels(self._h))
