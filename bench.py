#!/usr/bin/env python3
"""Throughput of the multi-Slater-determinant AFQMC hot path on GB300.

Metric: walker x determinant overlap + energy evaluations per second on the
iron-sulfur-dimer-shaped workload (M = 160 orbitals, 30 + 30 electrons,
30e/20o active space, N_det = 120000, N_chol = 800, 640 walkers), mixed
precision, with the plain FP64 GPU path and its error measured beside it.

One step = the whole hot path over the 640 walkers: force bias and local
energy, each with the trial overlap (reference inverse, excitation-string
minors, cofactor Green's function, Cholesky contractions, per-determinant
energy, reductions). Inputs are resident in device memory; L2 is flushed
between timed steps. With --gpus N (one process per GPU under torchrun)
every rank evaluates its own 640 walkers (weak scaling, no data exchange).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("walker·det overlap+energy evals/s at N_det=1.2e5; mixed vs FP64 at stated error")


def metric_for(n_det):
    """The headline metric's name; other trial sizes name their own N_det."""
    if n_det == 120000:
        return METRIC
    return METRIC.replace("N_det=1.2e5", "N_det=" + ("%.3g" % n_det).replace("e+0", "e").replace("e+", "e"))
UNIT = "walker*det/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def measure_alu_peaks(dev):
    """FP64, FP32 (SIMT) and TF32 (tensor) rates of this GPU, measured here:
    the best of 5 square cuBLAS GEMMs (torch.matmul, 2 n^3 flops, CUDA events
    on the current stream) at n = 4096 (FP64) and 8192 (FP32 with TF32 off,
    TF32), after a warm-up. Library GEMMs at these sizes run close to the
    respective pipes' peak, as the measured BF16 peak beside them does."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        for key, dtype, n, tf32 in (("fp64_gflops", torch.float64, 4096, False),
                                    ("fp32_gflops", torch.float32, 8192, False),
                                    ("tf32_gflops", torch.float32, 8192, True)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, dtype=dtype, device=dev)
            b = torch.randn(n, n, dtype=dtype, device=dev)
            c = a @ b
            torch.cuda.synchronize(dev)
            best = float("inf")
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[key] = 2.0 * n ** 3 / (best / 1e3) / 1e9
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = "best of 5 cuBLAS GEMMs (torch.matmul): FP64 n=4096, FP32 (TF32 off) and TF32 n=8192"
    return out


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="fe2s2")
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--n-w", type=int, default=None)
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    # library options (alternative implementations of the same step)
    p.add_argument("--no-overlap", action="store_true",
                   help="run every kernel of a step on one stream (msd_set_stream_overlap(0))")
    p.add_argument("--tensor-gram", action="store_true",
                   help="Gram matrices on the tensor cores (msd_set_tensor_gram)")
    p.add_argument("--no-fused", action="store_true",
                   help="mixed: tensor-core GEMM + separate epilogue instead of the fused kernel")
    p.add_argument("--pair-form", default="auto", choices=["auto", "0", "1", "2"],
                   help="opposite-spin term per determinant (0), per beta string (1), over runs sharing a "
                        "string (2) or chosen by the cost model")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("gloo")


def aggregate(ms_total: float, units: float):
    """Max of the timed device milliseconds and sum of the units over ranks
    (gloo on host tensors: timing bookkeeping, not part of the data path)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return ms_total, units
    t = torch.tensor([ms_total], dtype=torch.float64)
    u = torch.tensor([units], dtype=torch.float64)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def load_peaks(dev=None):
    """HBM and BF16 peaks from MEASURED_PEAKS.json (else the fallback), plus
    the FP64, FP32 and TF32 GEMM rates measured on `dev` now."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            peaks, src = json.load(f), "measured"
    else:
        peaks, src = dict(FALLBACK_PEAKS), "fallback"
    if dev is not None:
        alu = measure_alu_peaks(dev)
        peaks.update(alu)
        peaks["alu_how"] = alu["how"]
    return peaks, src


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region (read-only queries)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            import torch
            ident = str(self.dev)
            uuid = getattr(torch.cuda.get_device_properties(self.dev), "uuid", None)
            if uuid is not None:
                ident = "GPU-" + str(uuid)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", ident], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- work accounting
def string_levels(occ, n_det):
    """Distinct excitation strings of one spin (relative to determinant 0)
    and their levels, for work accounting."""
    import numpy as np
    ref = set(occ[0].tolist())
    seen = {}
    for I in range(n_det):
        row = occ[I].tolist()
        holes = tuple(sorted(ref - set(row)))
        parts = tuple(sorted(set(row) - ref))
        seen.setdefault((holes, parts), len(holes))
    lv = np.bincount(np.array(list(seen.values())), minlength=8)
    hole_orbs = set()
    part_orbs = set()
    for (h, p) in seen:
        hole_orbs.update(h)
        part_orbs.update(p)
    return lv, len(hole_orbs), len(part_orbs)


def algorithmic_work(s, n_w):
    """Algorithmic flops per call of each kernel group (one step = one
    force-bias call + one local-energy call). Complex multiply-add = 8 flops,
    complex x real = 4 flops."""
    import numpy as np
    M, G = s.M, s.n_chol
    spins = []
    for occ, N in ((s.occ_a, s.n_alpha), (s.occ_b, s.n_beta)):
        lv, nh, np_ = string_levels(occ, s.n_det)
        spins.append(dict(N=N, lv=lv, nh=nh, np=np_, X=nh * np_, NC=N + np_))
    k = np.arange(8)
    pair_lv = {}
    ref_a, ref_b = set(s.occ_a[0].tolist()), set(s.occ_b[0].tolist())
    for I in range(s.n_det):
        ka = len(ref_a - set(s.occ_a[I].tolist()))
        kb = len(ref_b - set(s.occ_b[I].tolist()))
        pair_lv[(ka, kb)] = pair_lv.get((ka, kb), 0) + 1
    w = {}
    # reference inverse: LU + inverse + Theta product + active block, both spins
    w["k_ref"] = sum(8 * (4 / 3 * sp["N"] ** 3 + M * sp["N"] ** 2 + sp["X"] * sp["N"]) for sp in spins) * n_w
    # string minors: the FP64 part, LU with partial pivoting (k^3/3 complex
    # MACs); the inverse from the factors runs in the working precision
    w["k_strings"] = sum(float(np.sum(sp["lv"] * 8 * k ** 3 / 3)) for sp in spins) * n_w
    w["k_gemm_F"] = sum(4.0 * sp["N"] * M * G * sp["NC"] for sp in spins) * n_w
    w["k_fepi"] = sum(8.0 * (sp["N"] ** 2 + sp["N"] ** 2 * sp["np"] + sp["nh"] * sp["N"] * sp["np"]) * G
                      for sp in spins) * n_w
    w["k_gram"] = 8.0 * G * (spins[0]["X"] ** 2 + spins[1]["X"] ** 2 + spins[0]["X"] * spins[1]["X"]) * n_w
    # the same Gram matrices on the tensor cores (3xTF32; with the transpose
    # of the Lambda rows in the same timed group)
    w["tc_gram"] = w["k_gram"]
    # same-spin string term in its antisymmetrized pair form: per string the
    # linear part (k^2 complex MACs) and, per pair of index pairs, a 2x2
    # minor of B (two complex products and a difference) times the pair
    # table entry: 8 k^2 + 22 C(k,2)^2 flops
    w["k_string_energy"] = sum(float(np.sum(sp["lv"] * (8 * k ** 2 + 22 * (k * (k - 1) // 2) ** 2)))
                               for sp in spins) * n_w
    w["k_pair_cross"] = sum(8.0 * n * (ka * ka * kb * kb + ka * ka) for (ka, kb), n in pair_lv.items()
                            if ka and kb) * n_w
    # the runs form evaluates the same term (the algorithmic work of the
    # per-determinant form is the reference count)
    w["k_pair_run"] = w["k_pair_cross"]
    # the per-beta-string form (mixed precision): Y_b over the alpha block
    # for every excited beta string, then k_a^2 per determinant
    w["k_pair_y"] = (8.0 * spins[0]["X"] * float(np.sum(spins[1]["lv"][1:] * k[1:] ** 2))
                     + sum(8.0 * n * ka * ka for (ka, kb), n in pair_lv.items() if ka and kb)) * n_w
    Kd = sum(sp["NC"] * M for sp in spins)
    w["k_gemm_vbias"] = 4.0 * Kd * G * n_w
    # tensor-core GEMMs: real GEMM flops of the contraction actually needed
    # (rows: walker x electron x re/im; K over the orbitals outside the
    # reference for F), counted once (the 3 TF32 products are the method of
    # the split, not extra algorithmic work)
    w["tc_gemm_F"] = sum(2.0 * (2 * sp["N"]) * (M - sp["N"]) * G * sp["NC"] for sp in spins) * n_w
    # the fused kernel: the same contraction (its epilogue, counted as
    # k_fepi above, runs on the FP32 pipes beside the tensor cores)
    w["tc_fepi"] = w["tc_gemm_F"]
    w["tc_gemm_vbias"] = 2.0 * 2 * Kd * G * n_w
    # CI weights: per string and determinant containing it one complex x real
    # multiply-add (4 flops), then r_s times the sum (6 flops); both spins
    w["k_weights"] = sum(4.0 * s.n_det + 6.0 * float(np.sum(sp["lv"])) for sp in spins) * n_w
    # cofactor accumulation: w_s r_s B_s added into k^2 cofactor entries per
    # string (one complex multiply-add each, 8 flops)
    w["k_cmat"] = sum(8.0 * float(np.sum(sp["lv"] * k ** 2)) for sp in spins) * n_w
    # exact reference sums: the real GEMM of the 2 walker rows per spin with
    # the constant [V | W] (N (M - N) x (N (M - N) + N_chol)), counted once
    w["tc_ozaki"] = sum(2.0 * 2 * (sp["N"] * (M - sp["N"])) * (sp["N"] * (M - sp["N"]) + G) for sp in spins) * n_w
    return w, spins


FP64_KERNELS = {"k_ref", "k_strings", "k_weights", "k_gt", "k_onebody", "k_final", "k_sum_slots"}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a
# kernel, from a one-pass ncu --metrics capture of this bench's default
# workload; reported only while the kernel's source file still hashes to
# the value recorded with the capture (a changed kernel gets null).
NCU_TRAFFIC = {
    # 640 walkers, one spin per launch
    "tc_fepi": {"source": "paper_2406_08314_gb300/csrc/tc_fepi.cu",
                "sha256": "5404f8c55474fc1374c3ea416c64dcc7153923c690cbf55b2d8f3342f0a65f3b",
                "bytes_per_launch": 151910912 + 642991872, "workload": "fe2s2", "n_w": 640},
}


def ncu_traffic(name, workload=None, n_w=None):
    """DRAM bytes per launch of a kernel from its recorded capture, for the
    captured workload and walker count only, while the kernel's source is
    unchanged; None otherwise."""
    import hashlib
    t = NCU_TRAFFIC.get(name)
    if not t or t.get("workload") != workload or t.get("n_w") != n_w:
        return None
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), t["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != t["sha256"]:
                return None
    except OSError:
        return None
    return t["bytes_per_launch"]


def kernel_peak(name, precision, peaks):
    """(bound, peak GFLOP/s, source) for a kernel group, against the rates
    measured on this GPU (measure_alu_peaks, MEASURED_PEAKS.json)."""
    if name == "tc_ozaki":
        return ("tensor", peaks["bf16_tflops"] * 1e3 / 15,
                "measured bf16 burst / 15 BF16 slice products of the exact split")
    if name.startswith("tc_"):
        return ("tensor", peaks["tf32_gflops"] / 3,
                "measured TF32 GEMM / 3 products of the 3xTF32 split")
    if precision == "fp64" or name in FP64_KERNELS:
        return ("alu", peaks["fp64_gflops"], "measured FP64 GEMM")
    return ("alu", peaks["fp32_gflops"], "measured FP32 GEMM (TF32 off)")


# -------------------------------------------------------------- our arm
def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2406_08314_gb300 import build, synth
    if rank == 0:
        build.build()
    barrier()
    from paper_2406_08314_gb300 import msd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s, wk = synth.config_system(args.workload, seed=rank, n_w=args.n_w)
    n_w, n_det = wk.n_w, s.n_det
    units_per_step = n_w * n_det
    da = torch.from_numpy(wk.phi_a).to(dev)
    db = torch.from_numpy(wk.phi_b).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = msd.Context(s, args.precision, device=local)
    ctx.set_sync(False)
    ctx.set_fused(not args.no_fused)
    ctx.set_pair_form(args.pair_form)
    ctx.set_tensor_gram(args.tensor_gram)
    ctx.set_stream_overlap(not args.no_overlap)
    vb = torch.empty((n_w, s.n_chol), dtype=torch.complex128, device=dev)
    el = torch.empty((n_w,), dtype=torch.complex128, device=dev)
    ov = torch.empty((n_w,), dtype=torch.complex128, device=dev)

    def step():
        ctx.evaluate(da, db, out=(ov, vb, el))

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    for _ in range(args.warmup):
        step()
    ctx.set_sync(True)
    step()                                  # surfaces any device-side error
    ctx.set_sync(False)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = msd.launch_count()
    barrier()
    torch.cuda.synchronize(dev)
    ms_total = 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms_total += e0.elapsed_time(e1)
    torch.cuda.synchronize(dev)
    launches = msd.launch_count() - launches0
    clocks = sampler.stop()
    # per-kernel CUDA-event times: the same steps again with every kernel on
    # one stream, where each kernel has the GPU to itself (with two streams
    # the event spans of concurrent kernels overlap and include their waits)
    ctx.set_stream_overlap(False)
    ctx.set_timing(True)
    ctx.reset_stats()
    torch.cuda.synchronize(dev)
    for _ in range(args.steps):
        flush.fill_(1)
        step()
    torch.cuda.synchronize(dev)
    kstats = ctx.kernel_stats()
    ctx.set_timing(False)
    ctx.set_stream_overlap(not args.no_overlap)
    ms_max, units = aggregate(ms_total, float(units_per_step * args.steps))
    ms_per_step = ms_max / args.steps
    value = units / (ms_max / 1e3)

    # plain FP64 GPU path beside it, and the error of this mode against it
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        ctx.set_sync(True)
        o_m, v_m, e_m = ctx.evaluate(da, db)
        ctx.set_precision("fp64")
        ctx.set_sync(False)
        step()                      # warm-up of the FP64 path
        torch.cuda.synchronize(dev)
        t64 = 0.0
        for _ in range(args.fp64_steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            t64 += e0.elapsed_time(e1)
        ctx.set_sync(True)
        o_d, v_d, e_d = ctx.evaluate(da, db)
        de = (e_m - e_d).abs().cpu().numpy()
        dv = (v_m - v_d).abs().max(dim=1).values.cpu().numpy()
        vscale = v_d.abs().max(dim=1).values.cpu().numpy()
        do = ((o_m - o_d).abs() / o_d.abs()).cpu().numpy()
        t64_max, u64 = aggregate(t64, float(units_per_step * args.fp64_steps))
        fp64 = {"value": u64 / (t64_max / 1e3), "ms_per_step": t64_max / args.fp64_steps,
                "steps": args.fp64_steps,
                "error_of_mixed": {
                    "e_loc_abs_max_Ha": float(de.max()), "e_loc_abs_median_Ha": float(np.median(de)),
                    "vbias_rel_max": float(np.max(dv / vscale)),
                    "ovlp_rel_max": float(do.max())}}
        ctx.set_precision(args.precision)
        # the same walkers and trial at a chemical energy scale: the Cholesky
        # vectors scaled so that the mean on-site Coulomb integral
        # sum_g L_g[p][p]^2 is 1 Ha (|E_L| ~ 400 Ha at the Fe2S2 shape)
        import copy
        sc = copy.copy(s)
        diag = np.einsum("gpp->gp", s.L)
        sc.L = s.L * math.sqrt(1.0 / float(np.mean(np.sum(diag * diag, axis=0))))
        got = {}
        for prec in ("mixed", "fp64"):
            cx = msd.Context(sc, prec, device=local)
            cx.set_fused(not args.no_fused)
            cx.set_pair_form(args.pair_form)
            cx.set_tensor_gram(args.tensor_gram)
            got[prec] = cx.local_energy(da, db)
            torch.cuda.synchronize(dev)
            cx.close()
        dc = (got["mixed"] - got["fp64"]).abs().cpu().numpy()
        fp64["error_of_mixed_chemical_scale"] = {
            "e_loc_abs_max_Ha": float(dc.max()), "e_loc_abs_median_Ha": float(np.median(dc)),
            "e_loc_scale_Ha": float(got["fp64"].abs().mean().item()),
            "variant": "Cholesky vectors scaled to mean (pp|pp) = 1 Ha"}

    # end to end through the C-ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        ha = torch.from_numpy(wk.phi_a).pin_memory()
        hb = torch.from_numpy(wk.phi_b).pin_memory()
        # the caller's result buffers, pinned and allocated once like its inputs
        outs_h = tuple(torch.empty(shape, dtype=torch.complex128).pin_memory()
                       for shape in ((n_w,), (n_w, s.n_chol), (n_w,)))
        ctx.set_sync(True)
        ctx.evaluate(ha, hb, out=outs_h)
        barrier()
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 5))
        for _ in range(n_e2e):
            o_h, v_h, e_h = ctx.evaluate(ha, hb, out=outs_h)   # host in, host out (the library stages)
        wall = (time.perf_counter() - t0) * 1e3
        wall_max, u_e2e = aggregate(wall, float(units_per_step * n_e2e))
        phi_bytes = ha.numel() * 16 + hb.numel() * 16
        e2e = {"value": u_e2e / (wall_max / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": phi_bytes,
               "d2h_bytes_per_step": int(v_h.nbytes + e_h.nbytes + o_h.nbytes)}

    work, spins = algorithmic_work(s, n_w)
    peaks, peak_src = load_peaks(dev)
    kernels = {}
    for name, (n_launch, ms) in kstats.items():
        steps = args.steps
        entry = {"launches": n_launch, "ms_per_step": ms / steps,
                 "share": ms / max(1e-9, sum(v[1] for v in kstats.values()))}
        if name in work and ms > 0:
            entry["gflops"] = work[name] * steps / (ms / 1e3) / 1e9
        kernels[name] = entry
    dom = max(kstats.items(), key=lambda kv: kv[1][1])[0] if kstats else None
    for name, entry in kernels.items():
        b, pk, src = kernel_peak(name, args.precision, peaks)
        entry["bound"] = b
        if "gflops" in entry:
            entry["frac"] = entry["gflops"] / pk
    roofline = None
    if dom is not None:
        d = kernels[dom]
        b, pk, src = kernel_peak(dom, args.precision, peaks)
        ach = d.get("gflops")
        roofline = {"kernel": dom, "bound": b, "achieved": ach, "peak": pk, "unit": "GFLOP/s",
                    "frac": (ach / pk) if ach else None, "traffic": ncu_traffic(dom, args.workload, n_w), "peak_source": src}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(s, wk, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": metric_for(s.n_det), "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 minors + f32 contractions" if args.precision == "mixed" else "f64",
            "data": "synthetic (seeded; shapes of the paper's "
                    + ("Fe2S2" if args.workload.startswith("fe2s2") else "Cu2O2") + " system)",
            "config": {"workload": f"{args.workload}: M={s.M}, {s.n_alpha}+{s.n_beta} e, "
                                   f"N_det={n_det}, N_chol={s.n_chol}, {n_w} walkers/GPU",
                       "precision": args.precision, "n_walkers": n_w, "n_det": n_det,
                       "fused": args.precision == "mixed" and not args.no_fused,
                       "gram": "tensor cores" if args.tensor_gram and args.precision == "mixed" else "FMA",
                       "opposite_spin_form": ("per beta string" if "k_pair_y" in kernels else
                                              "runs sharing a string" if "k_pair_run" in kernels else "per determinant"),
                       "n_chol": s.n_chol, "M": s.M,
                       "step": "msd_evaluate: overlap + force bias + local energy",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"walker replicas x{world}",
                       "strings": [int(sp["lv"].sum()) for sp in spins],
                       "streams": ("2: the energy's per-walker sums after the contraction beside the strings "
                                   "and weights, then the force bias beside the per-determinant terms"
                                   if args.precision == "mixed" and not args.no_overlap else "1")},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "fp64": fp64,
            "kernels": kernels,
            "kernels_note": "CUDA-event time of each kernel in a second pass of the timed steps with every "
                            "kernel on one stream (msd_set_stream_overlap(0))"
                            + ("; the timed steps run two streams" if args.precision == "mixed"
                               and not args.no_overlap else ""),
            "peaks_source": peak_src,
            "peaks": {k: peaks[k] for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained", "fp64_gflops",
                                            "fp32_gflops", "tf32_gflops", "alu_how") if k in peaks},
        }
        print(json.dumps(line), flush=True)
    ctx.close()


# ------------------------------------------------------ batched systems
def run_batched(args, rank, world, local):
    """32 independent systems (M uniform in [40, 160], N = M // 6 per spin,
    N_det log-uniform in [1e3, 1e5], N_chol = 4 M, 128 walkers each) in one
    recorded graph with the persistent per-determinant kernel, after the
    autotuner; beside it the same systems evaluated one after another."""
    import torch

    from paper_2406_08314_gb300 import build, synth
    if rank == 0:
        build.build()
    barrier()
    from paper_2406_08314_gb300 import msd
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sysw = synth.batched_systems(n_systems=32, seed0=1000 * rank, n_w=128)
    ctxs = [msd.Context(s, args.precision, device=local) for s, _ in sysw]
    walkers = [(torch.from_numpy(w.phi_a).to(dev), torch.from_numpy(w.phi_b).to(dev)) for _, w in sysw]
    units = float(sum(w.n_w * s.n_det for s, w in sysw))
    batch = msd.Batch(ctxs)
    outs = batch.outputs(walkers)
    import tempfile
    cache = os.path.join(tempfile.gettempdir(), "msd_batch_tune.txt")   # autotuner cache across runs
    t0 = time.perf_counter()
    cfg = batch.autotune(walkers, outs, cache_path=cache)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        batch.evaluate(walkers, outs)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = msd.launch_count()
    ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.evaluate(walkers, outs)       # one graph launch
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    clocks = sampler.stop()
    # kernels launched: host-side launches plus the kernel nodes of every replay
    launches = msd.launch_count() - launches0 + batch.graph_kernels() * args.steps
    ms_max, u = aggregate(ms, units * args.steps)
    # the same systems one after another through msd_evaluate
    for c in ctxs:
        c.set_sync(False)
    for (a, b), c, (o, v, e) in zip(walkers, ctxs, outs):
        c.evaluate(a, b, out=(o, v, e))
    torch.cuda.synchronize(dev)
    ms_seq = 0.0
    for _ in range(max(1, args.steps // 2)):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for (a, b), c, (o, v, e) in zip(walkers, ctxs, outs):
            c.evaluate(a, b, out=(o, v, e))
        e1.record(stream)
        e1.synchronize()
        ms_seq += e0.elapsed_time(e1)
    ms_seq /= max(1, args.steps // 2)
    # the persistent kernel alone (CUDA events around it in one eager run)
    batch.time_persistent(True)
    batch.set_config(cfg["tile_n"], cfg["ctas_per_sm"], cfg["order"])   # next call runs eagerly
    flush.fill_(1)
    batch.evaluate(walkers, outs)
    torch.cuda.synchronize(dev)
    pk_ms = batch.time_persistent(False)
    peaks, _ = load_peaks(dev)
    # its algorithmic work: the per-determinant terms of every system
    pk_work = 0.0
    for (sy, wy) in sysw:
        wk_, _ = algorithmic_work(sy, wy.n_w)
        pk_work += wk_["k_string_energy"] + wk_["k_pair_cross"]
    b_, pk_peak, pk_src = kernel_peak("k_det_batched", args.precision, peaks)
    pk_gflops = pk_work / (pk_ms / 1e3) / 1e9 if pk_ms > 0 else None
    roofline = {"kernel": "k_det_batched", "bound": b_, "achieved": pk_gflops, "peak": pk_peak,
                "unit": "GFLOP/s", "frac": (pk_gflops / pk_peak) if pk_gflops else None, "traffic": None,
                "peak_source": pk_src, "ms": pk_ms}
    # end to end: walkers from pinned host memory into the graph's buffers,
    # one graph launch, the local energies back to the host
    host = [(torch.from_numpy(w.phi_a).pin_memory(), torch.from_numpy(w.phi_b).pin_memory()) for _, w in sysw]
    e_host = [torch.empty(w.n_w, dtype=torch.complex128).pin_memory() for _, w in sysw]
    batch.evaluate(walkers, outs)
    torch.cuda.synchronize(dev)
    n_e2e = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        for (a, b), (ha, hb) in zip(walkers, host):
            a.copy_(ha, non_blocking=True)
            b.copy_(hb, non_blocking=True)
        batch.evaluate(walkers, outs)
        for eh, (o, v, e) in zip(e_host, outs):
            eh.copy_(e, non_blocking=True)
        torch.cuda.synchronize(dev)
    wall = (time.perf_counter() - t0) * 1e3
    wall_max, u_e2e = aggregate(wall, units * n_e2e)
    e2e = {"value": u_e2e / (wall_max / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(sum(ha.numel() * 16 + hb.numel() * 16 for ha, hb in host)),
           "d2h_bytes_per_step": int(sum(eh.numel() * 16 for eh in e_host))}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        big = max(range(len(sysw)), key=lambda i: sysw[i][0].M)
        cpu = cpu_baseline(sysw[big][0], sysw[big][1], args.cpu_seconds)
        cpu["sample"] = f"system {big} of the batch (M={sysw[big][0].M}): " + cpu["sample"]
    if rank == 0:
        print(json.dumps({
            "metric": "walker*det overlap+energy evals/s, 32 batched uneven systems", "value": u / (ms_max / 1e3),
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 minors + f32 contractions" if args.precision == "mixed" else "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": "batched: 32 systems, M~U[40,160], N=M//6+M//6, N_det log-uniform [1e3,1e5], "
                                   "N_chol=4M, 128 walkers each, one recorded graph",
                       "precision": args.precision, "autotuned": cfg, "autotune_s": tune_s,
                       "total_walker_dets": units, "l2": "flushed between timed steps (256 MiB write)"},
            "sequential_ms_per_step": ms_seq, "speedup_vs_sequential": ms_seq / (ms_max / args.steps),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks}), flush=True)
    batch.close()


# ------------------------------------------------- learned control variate
def run_cv(args, rank, world, local):
    """Copper-oxo-shaped system: the network trained on ~1e5 (features,
    E_L) pairs the library computes, then on a held-out population of 640
    walkers the estimate mean(f) + mean over a random 1/8 of (E_L - f)
    against the exact path on the same 1/8 (bias, variance) and against the
    exact path on all 640 (cost)."""
    import numpy as np
    import torch

    from paper_2406_08314_gb300 import build, synth
    if rank == 0:
        build.build()
    barrier()
    from paper_2406_08314_gb300 import cv, msd
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s, w0 = synth.config_system("cu2o2", seed=rank, n_w=640)
    ctx = msd.Context(s, "mixed", device=local)
    rng = np.random.default_rng(100 + rank)

    # training pairs from the method's own runs: 8 seeded phaseless AFQMC
    # runs of 640 walkers (the copper-oxo workload's walkers, dt = 0.005,
    # 20 steps each, propagated on the GPU), one pair per walker and step
    t0 = time.perf_counter()
    xs, es = [], []
    for run in range(8):
        da, db = torch.from_numpy(w0.phi_a).to(dev), torch.from_numpy(w0.phi_b).to(dev)
        x_r, e_r, _ = cv.propagated_pairs(ctx, da, db, 20, dt=0.005, seed=1000 * rank + run)
        xs.append(x_r)
        es.append(e_r)
    x, e = torch.cat(xs), torch.cat(es)          # 102400 training pairs
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    net = cv.MLP(x.shape[1], 256, device=local, seed=1)
    hist = net.fit(x, e, epochs=20, batch=512, lr=1e-3, lr_final=3e-5)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    # held-out population: the 640 walkers of a ninth run after its 20 steps
    da, db = torch.from_numpy(w0.phi_a).to(dev), torch.from_numpy(w0.phi_b).to(dev)
    cv.propagated_pairs(ctx, da, db, 20, dt=0.005, seed=1000 * rank + 99)
    e_all = ctx.local_energy(da, db).real.double().cpu().numpy()
    f_all = net.predict(ctx.features_rows(da, db)).double().cpu().numpy()
    study = cv.estimator_study(e_all, f_all, frac=0.125, draws=4000, seed=3)
    r2 = 1 - np.mean((f_all - e_all) ** 2) / np.var(e_all)
    # cost: exact on all 640 vs surrogate on all + exact on 80
    sub = torch.from_numpy(np.sort(rng.choice(640, 80, replace=False))).to(dev)
    sa, sb = da[sub].contiguous(), db[sub].contiguous()
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_exact = timed(lambda: ctx.local_energy(da, db))
    ms_cv = timed(lambda: (net.predict(ctx.features_rows(da, db)), ctx.local_energy(sa, sb)))
    # variance per unit cost against the exact estimator on all 640 walkers
    var_exact_all = float(np.var(e_all) / 640)
    eff = (var_exact_all * ms_exact) / (study["cv_var"] * ms_cv)
    if rank == 0:
        print(json.dumps({
            "metric": "control-variate local-energy estimate: variance reduction at equal exact cost",
            "value": study["variance_reduction"], "unit": "x", "n_gpus": world, "higher_is_better": True,
            "data": "synthetic (seeded), copper-oxo-shaped system",
            "config": {"workload": "cu2o2: M=108, 16+16 e, N_det=1e4, N_chol=400; network 6912->256x3->1 GELU, "
                                   "BF16 weights, FP32 accumulation; training pairs 102400 from 8 seeded phaseless "
                                   "AFQMC runs (640 walkers x 20 steps, dt 0.005, msd_propagate), 20 epochs; "
                                   "held-out population: a ninth run's 640 walkers after 20 steps, exact on a "
                                   "random 1/8",
                       "features": "non-zero rows of the reference Green's function",
                       "n_train": int(x.shape[0])},
            "r2_heldout": float(r2), "bias": study["cv_bias"], "bias_stderr": study["cv_bias_stderr"],
            "plain_var": study["plain_var"], "cv_var": study["cv_var"],
            "train_s": train_s, "data_generation_s": gen_s, "train_mse_first_last": [hist[0]["train_mse"],
                                                                                     hist[-1]["train_mse"]],
            "ms_exact_640": ms_exact, "ms_surrogate_640_plus_exact_80": ms_cv,
            "variance_per_cost_gain_vs_exact_640": eff}), flush=True)


# -------------------------------------------------------- CPU baseline
def cpu_baseline(s, wk, seconds):
    """The oracle (naive per-determinant FP64, OpenMP over determinants) on a
    bounded sample: walker 0 against random chunks of 32 determinants until
    `seconds` of work; value in walker*det/s."""
    import copy

    import numpy as np

    import oracle
    rng = np.random.default_rng(1234)
    order = rng.permutation(s.n_det)
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds and done < s.n_det:
        idx = np.sort(order[done: done + 32])
        t = copy.copy(s)
        t.coeff, t.occ_a, t.occ_b = s.coeff[idx], s.occ_a[idx], s.occ_b[idx]
        oracle.msd(t, wk.phi_a[:1], wk.phi_b[:1], energy=True, vbias=True)
        done += len(idx)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"1 walker x {done} random determinants (chunks of 32), {dt:.1f} s; "
                      "overlap, mixed Green's function / force bias and energy per determinant"}


# ---------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores: each step evaluates walker 0
    against a bounded random sample of the workload's determinants."""
    if rank != 0:
        return
    import copy

    import numpy as np

    import oracle
    from paper_2406_08314_gb300 import synth
    oracle.build()
    s, wk = synth.config_system(args.workload, seed=0, n_w=args.n_w or 4)
    rng = np.random.default_rng(99)
    per_step = 48

    def step(i):
        idx = np.sort(rng.choice(s.n_det, per_step, replace=False))
        t = copy.copy(s)
        t.coeff, t.occ_a, t.occ_b = s.coeff[idx], s.occ_a[idx], s.occ_b[idx]
        oracle.msd(t, wk.phi_a[:1], wk.phi_b[:1], energy=True, vbias=True)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": metric_for(s.n_det), "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded; shapes of the paper's Fe2S2 system)",
            "config": {"workload": f"{args.workload}: M={s.M}, {s.n_alpha}+{s.n_beta} e, "
                                   f"N_det={s.n_det}, N_chol={s.n_chol}",
                       "sample_per_step": f"1 walker x {per_step} random determinants"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"1 walker x {per_step} random determinants per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_prop(args, rank, world, local):
    """Phaseless propagation of the copper-oxo-shaped system (M = 108, 16+16
    electrons, N_det = 1e4, N_chol = 400, 640 walkers, FP64 as in the plain
    FP64 configuration): each step is one msd_propagate (force bias over all
    determinants, field matrix, Taylor-series propagator of order 6 between
    the exp(-dt h'/2) half steps, overlap ratio and phaseless weights),
    dt = 0.005, QR of the walkers every 5th step."""
    import numpy as np
    import torch

    from paper_2406_08314_gb300 import build, synth
    if rank == 0:
        build.build()
    barrier()
    from paper_2406_08314_gb300 import msd
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s, wk = synth.config_system("cu2o2", seed=rank, n_w=args.n_w)
    n_w, G, dt = wk.n_w, s.n_chol, 0.005
    ctx = msd.Context(s, "fp64", device=local)
    ctx.set_sync(False)
    da = torch.from_numpy(wk.phi_a).to(dev)
    db = torch.from_numpy(wk.phi_b).to(dev)
    wts = torch.ones(n_w, dtype=torch.float64, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000 + rank)
    n_total = args.warmup + 1 + args.steps
    xs = torch.randn((n_total, n_w, G), dtype=torch.float64, device=dev, generator=gen)
    stream = torch.cuda.current_stream(dev)
    counter = [0]

    def step():
        i = counter[0]
        counter[0] += 1
        ctx.propagate(da, db, wts, xs[i % n_total], dt, 6, (i % 5) == 4)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        step()
    ctx.set_sync(True)
    step()
    ctx.set_sync(False)
    torch.cuda.synchronize(dev)
    ctx.set_timing(True)
    ctx.reset_stats()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = msd.launch_count()
    barrier()
    torch.cuda.synchronize(dev)
    ms_total = 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms_total += e0.elapsed_time(e1)
    torch.cuda.synchronize(dev)
    launches = msd.launch_count() - launches0
    clocks = sampler.stop()
    kstats = ctx.kernel_stats()
    ctx.set_timing(False)
    ms_max, units = aggregate(ms_total, float(n_w * args.steps))
    value = units / (ms_max / 1e3)
    w_final = wts.cpu().numpy()

    # end to end: walkers and fields from pinned host memory, walkers and
    # weights back, every step
    e2e = None
    if not args.no_e2e:
        ha = da.cpu().pin_memory()
        hb = db.cpu().pin_memory()
        hw = wts.cpu().pin_memory()
        hx = xs[0].cpu().pin_memory()
        ctx.set_sync(False)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 5))
        for i in range(n_e2e):
            da.copy_(ha, non_blocking=True)
            db.copy_(hb, non_blocking=True)
            wts.copy_(hw, non_blocking=True)
            xs[0].copy_(hx, non_blocking=True)
            ctx.propagate(da, db, wts, xs[0], dt, 6, (i % 5) == 4)
            ha.copy_(da, non_blocking=True)
            hb.copy_(db, non_blocking=True)
            hw.copy_(wts, non_blocking=True)
            torch.cuda.synchronize(dev)
        wall = (time.perf_counter() - t0) * 1e3
        wall_max, u_e2e = aggregate(wall, float(n_w * n_e2e))
        io = ha.numel() * 16 + hb.numel() * 16
        e2e = {"value": u_e2e / (wall_max / 1e3), "unit": "walker*steps/s",
               "h2d_bytes_per_step": io + hw.numel() * 8 + hx.numel() * 8,
               "d2h_bytes_per_step": io + hw.numel() * 8}

    # algorithmic work (flops) per step, FP64
    M = s.M
    work = {"k_gemm_V": 4.0 * M * M * G * n_w,
            "k_apply_rows": sum(2 * 4.0 * M * M * n + 6 * 8.0 * M * M * n for n in (s.n_alpha, s.n_beta)) * n_w}
    peaks, _ = load_peaks(dev)
    fp64_peak = peaks["fp64_gflops"]
    kernels = {}
    for name, (n_launch, ms) in kstats.items():
        entry = {"launches": n_launch, "ms_per_step": ms / args.steps,
                 "share": ms / max(1e-9, sum(v[1] for v in kstats.values()))}
        if name in work and ms > 0:
            entry["gflops"] = work[name] * args.steps / (ms / 1e3) / 1e9
            entry["frac"] = entry["gflops"] / fp64_peak
        kernels[name] = entry
    dom = max(kstats.items(), key=lambda kv: kv[1][1])[0] if kstats else None
    roofline = None
    if dom is not None:
        d = kernels[dom]
        roofline = {"kernel": dom, "bound": "alu", "achieved": d.get("gflops"), "peak": fp64_peak,
                    "unit": "GFLOP/s", "frac": d.get("frac"), "traffic": ncu_traffic(dom, "propagate"),
                    "peak_source": "measured FP64 GEMM (" + peaks["alu_how"] + ")"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import prop_oracle
        import oracle as _o
        _o.build()
        rng = np.random.default_rng(5)
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < args.cpu_seconds and done < 8:
            x = rng.standard_normal((1, G))
            prop_oracle.step(s, wk.phi_a[done:done + 1], wk.phi_b[done:done + 1], np.ones(1), x, dt)
            done += 1
        el = time.perf_counter() - t0
        cpu = {"value": done / el, "unit": "walker*steps/s",
               "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
               "sample": f"{done} walkers x 1 step each (all 1e4 determinants, naive per-determinant overlaps "
                         f"and force bias), {el:.1f} s"}
    if rank == 0:
        print(json.dumps({
            "metric": "phaseless propagation: walker steps/s (force bias + overlap ratio over N_det = 1e4)",
            "value": value, "unit": "walker*steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded; shapes of the paper's copper-oxo system), Gaussian fields N(0, 1)",
            "config": {"workload": f"cu2o2: M={s.M}, {s.n_alpha}+{s.n_beta} e, N_det={s.n_det}, N_chol={G}, "
                                   f"{n_w} walkers/GPU, dt={dt}, Taylor order 6, QR every 5 steps",
                       "walker_det_per_s": value * s.n_det,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"walker replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "kernels": kernels,
            "weights_after": {"mean": float(w_final.mean()), "min": float(w_final.min()),
                              "max": float(w_final.max())}}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    dist_init(world)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        run_batched(args, rank, world, local)
    elif args.workload == "cv":
        run_cv(args, rank, world, local)
    elif args.workload == "propagate":
        run_prop(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    barrier()


if __name__ == "__main__":
    main()
