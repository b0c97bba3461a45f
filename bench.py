"""Benchmark of the GB300 domain-wall operator: Dhop throughput against the HBM roofline, and
plain vs mixed-precision CG time to a 1e-10 true residual.

Workload (one "step"): one DhopEO + one DhopOE (a full-lattice hopping application, 1320 flops
per 5D output site) on a 16^4 x Ls=16 lattice with weakly disordered links exp(0.3 i H),
Gaussian spinors, M5 = 1.8, m = 0.01, antiperiodic in time. The headline `value` is the FP32
variant; FP64, FP16- and BF16-storage variants are reported under "variants". Inputs are seeded
synthetic fields (the paper's production gauge ensembles are not available here).

L2 hygiene: each step works on one of three independent sets (operator with its own links,
input and output fields; 3 x 221 MB in FP32), used round-robin, so every step's inputs were last
touched two steps earlier and have been evicted from the 126 MiB L2 by the other sets' traffic.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--no-cg] [--no-cg32] [--no-sweep]
Under torchrun each rank runs the same workload on its own GPU (replicas: the operator has no
data-path collective); rank 0 prints one JSON line with the aggregate over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2203_06777_gb300 import synth  # noqa: E402

WORKLOAD = "dwf_16x16x16x16_ls16_exp0.3"
CG_WORKLOAD = "dwf_24x24x24x24_ls12_exp0.4"
FLOPS_PER_SITE = 1320
METRIC = "DWF Dhop GFlop/s (1320 flop per 5D site) and HBM GB/s vs roofline; mixed vs FP64 CG time-to-1e-10"
BC = (1, 1, 1, -1)
L2_BYTES = 135_528_448


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def pipe_peaks(dwf):
    """FMA throughput of this GPU measured by the library's own loop kernels (grid_dwf_pipe_peak):
    the FP64 ceiling is the roofline of the IEEE FP64 hopping term, which this part's FP64 pipe
    bounds (no FP64 tensor path is used); FP32 scalar / packed FP32x2 for context."""
    names = (("fp64_fma_gflops", dwf.PEAK_FP64_FMA), ("fp32_fma_gflops", dwf.PEAK_FP32_FMA),
             ("fp32x2_fma_gflops", dwf.PEAK_FP32X2_FMA))
    out = {k: round(dwf.pipe_peak(v), 1) for k, v in names}
    out["method"] = ("grid_dwf_pipe_peak: 8 independent FMA chains x 4096 trips per thread, 8 CTAs x 256 threads "
                     "per SM, best of 3 CUDA-event timings after a warm-up; 2 flops per FMA, 4 per packed FMA")
    return out


KERNEL_SOURCES = ["paper_2203_06777_gb300/csrc/dhop_kernel.cuh", "paper_2203_06777_gb300/csrc/dhop_inst.cuh",
                  "paper_2203_06777_gb300/csrc/dwf_common.cuh", "paper_2203_06777_gb300/csrc/dhop_p32.cu"]
TRAFFIC_PROFILE = "profiles/dhop_fp32_16x16x16x16_ls16.md"
TRAFFIC_PROFILE_32 = "profiles/dhop_fp32_32x32x32x32_ls16.md"


def kernel_source_hash() -> str:
    """Hash of the FP32 hop's sources with their comments removed (a capture stays valid while the
    code it measured is unchanged)."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(re.sub(r"[ \t]+\n", "\n", text).encode())
    return h.hexdigest()[:16]


def measured_traffic(profile=TRAFFIC_PROFILE):
    """DRAM bytes per launch of the FP32 Dhop kernel from a committed ncu summary, if that
    capture was taken of the kernel sources as they are now; otherwise None."""
    try:
        text = open(os.path.join(ROOT, profile)).read()
    except OSError:
        return None
    fields = dict(line.split(":", 1) for line in text.splitlines() if line.startswith(("traffic_bytes_per_launch:",
                                                                                       "source_hash:")))
    if fields.get("source_hash", "").strip() != kernel_source_hash():
        return None
    try:
        return float(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def algorithmic_bytes_per_site(real_bytes: int, Ls: int, link_reals: int = 18) -> float:
    """Each input spinor read once, each output written once, 8 links per 4D site amortised over Ls
    (18 reals each, or 12 with compressed links)."""
    return real_bytes * (24 + 24) + 8 * link_reals * real_bytes / Ls


# ---------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first_sample(self, timeout=3.0):
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)

    def wait_next_sample(self, timeout=1.0):
        n = len(self.lines)
        t0 = time.time()
        while self.proc and len(self.lines) == n and time.time() - t0 < timeout:
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- distributed plumbing


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, world: int) -> float:
    """Max over ranks (the job's time is its slowest rank's); a no-op at world size 1."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job rate: the units every rank processed, divided by the slowest rank's time."""
    return units_per_rank * world / seconds_max


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ---------------------------------------------------------------- GPU arm


def make_sets(dwf, torch, spec, prec, nsets, seed0, fp64_arith=0, compress12=False):
    dims, Ls = spec["dims"], spec["Ls"]
    sets = []
    for k in range(nsets):
        U = synth.random_gauge(dims, seed=1000 * spec["case"] + seed0 + 10 * k, eps=spec["eps"])
        op = dwf.GridDWF(dims, Ls, spec["M5"], spec["mass"], bc=BC, fp64_arith=fp64_arith, compress12=compress12)
        op.set_gauge(torch.from_numpy(U).cuda())
        psi = synth.random_spinor(dims, Ls, seed=1000 * spec["case"] + seed0 + 10 * k + 1)
        src = op.pack(torch.from_numpy(psi).cuda(), prec, dwf.FULL)
        dst = op.field(prec, dwf.FULL, zero=True)
        op.dhop(src, dwf.FULL, out=dst)  # converts and caches the links of this precision
        sets.append((op, src, dst))
    torch.cuda.synchronize()
    return sets


def launches_per_step(op, prec, dwf) -> int:
    """Kernel launches of one full-lattice Dhop: the packed precisions run both halves in one
    launch (plus one tail launch when sites-per-CTA does not divide the half lattice); FP64 one
    launch per half."""
    if prec == dwf.FP64:
        return 2
    lsh = (op.Ls + 1) // 2
    spc = 128 // lsh
    if lsh == 8:
        spc = 8
    else:  # the largest CTA of whole warps made of whole 4-site blocks, where one exists
        spc = next((s for s in range(spc - spc % 4, 3, -4) if (s * lsh) % 32 == 0), spc)
    spc = min(max(1, spc), op.half_sites)
    return 1 if op.half_sites % spc == 0 else 2


def soak(dwf, torch, sets, seconds):
    """Run the step untimed for about `seconds` (clock sampling; not part of any timing)."""
    t0 = time.perf_counter()
    i = 0
    while time.perf_counter() - t0 < seconds:
        for _ in range(20):
            op, src, dst = sets[i % len(sets)]
            op.dhop(src, dwf.FULL, out=dst)
            i += 1
        torch.cuda.synchronize()


def hold_stream(torch, stream, us=150):
    """Keep `stream` busy for about `us` microseconds (torch's bounded clock-spin kernel) so that the
    host has queued the first timed launches when the start event is reached: the timed region
    then holds the K steps back to back, not the host's latency to issue the first one."""
    if hasattr(torch.cuda, "_sleep"):
        with torch.cuda.stream(stream):
            torch.cuda._sleep(int(us * 2000))  # ~2 GHz SM clock


def time_dhop(dwf, torch, sets, steps, warmup, world):
    """Time `steps` full-lattice Dhop applications (DhopEO + DhopOE, one call each) with CUDA events."""
    stream = torch.cuda.current_stream()

    def step(i):
        op, src, dst = sets[i % len(sets)]
        op.dhop(src, dwf.FULL, out=dst)

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hold_stream(torch, stream)
    e0.record(stream)
    for i in range(steps):
        step(warmup + i)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    return e0.elapsed_time(e1) / 1e3


def time_dhop_e2e(dwf, torch, sets, steps, warmup, world):
    """The same Dhop through the public API with host buffers, as a streaming user runs it: each
    step copies its input from pinned host memory to the device, applies the two half-lattice
    hops and copies the result back to pinned host memory. Copies run on their own streams and
    two device buffer sets alternate, so step i's transfers overlap step i-1's and i+1's
    compute; events order every buffer reuse. Timed from the first copy to the last result."""
    op, src, dst = sets[0]
    nbuf = 2
    host_in = [torch.empty(src.shape, dtype=src.dtype, pin_memory=True) for _ in range(nbuf)]
    host_out = [torch.empty(dst.shape, dtype=dst.dtype, pin_memory=True) for _ in range(nbuf)]
    for h in host_in:
        h.copy_(src)
    dev_in = [torch.empty_like(src) for _ in range(nbuf)]
    dev_out = [torch.empty_like(dst) for _ in range(nbuf)]
    s_h2d, s_cmp, s_d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(nbuf)]     # input copied
    ev_done = [torch.cuda.Event() for _ in range(nbuf)]   # compute finished
    ev_out = [torch.cuda.Event() for _ in range(nbuf)]    # result copied back
    for b in range(nbuf):
        ev_out[b].record(s_d2h)

    def step(i):
        b = i % nbuf
        with torch.cuda.stream(s_h2d):
            s_h2d.wait_event(ev_done[b])  # the compute that last read dev_in[b] is done
            dev_in[b].copy_(host_in[b], non_blocking=True)
            ev_in[b].record(s_h2d)
        with torch.cuda.stream(s_cmp):
            s_cmp.wait_event(ev_in[b])
            s_cmp.wait_event(ev_out[b])  # dev_out[b] has been copied back
            op.dhop(dev_in[b], dwf.FULL, out=dev_out[b])
            ev_done[b].record(s_cmp)
        with torch.cuda.stream(s_d2h):
            s_d2h.wait_event(ev_done[b])
            host_out[b].copy_(dev_out[b], non_blocking=True)
            ev_out[b].record(s_d2h)

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_h2d)
    s_cmp.wait_event(e0)
    s_d2h.wait_event(e0)
    for i in range(steps):
        step(warmup + i)
    s_h2d.wait_stream(s_d2h)
    e1.record(s_h2d)
    torch.cuda.synchronize()
    barrier(world)
    nbytes = src.numel() * src.element_size()
    return e0.elapsed_time(e1) / 1e3, nbytes, dst.numel() * dst.element_size()


def run_cg(dwf, torch, spec, maxiter=20000):
    dims, Ls = spec["dims"], spec["Ls"]
    U = synth.random_gauge(dims, seed=1000 * spec["case"] + 1, eps=spec["eps"])
    op = dwf.GridDWF(dims, Ls, spec["M5"], spec["mass"], bc=BC)
    op.set_gauge(torch.from_numpy(U).cuda())
    b = op.pack(torch.from_numpy(synth.random_spinor(dims, Ls, seed=1000 * spec["case"] + 2)).cuda(), dwf.FP64,
                dwf.FULL)
    out = {}
    x64 = None
    # *_ff: the FP64 operator applications (the whole FP64 CG; the mixed CG's true residuals) in
    # float-float arithmetic
    for name, mode, arith in (("fp64", dwf.CG_FP64, 0), ("mixed_fp32", dwf.CG_MIXED_FP32, 0),
                              ("mixed_fp16", dwf.CG_MIXED_FP16, 0), ("mixed_bf16", dwf.CG_MIXED_BF16, 0),
                              ("fp64_ff", dwf.CG_FP64, 1), ("mixed_fp32_ff", dwf.CG_MIXED_FP32, 1),
                              ("mixed_fp16_ff", dwf.CG_MIXED_FP16, 1)):
        op.set_fp64_arith(arith)
        torch.cuda.synchronize()
        x, st = op.cg(b, tol=1e-10, maxiter=maxiter, mode=mode, raise_on_fail=False)
        torch.cuda.synchronize()
        rec = {"seconds": round(st.seconds, 4), "iterations": st.iterations, "reliable_updates": st.reliable_updates,
               "true_residual": st.true_residual, "converged": st.converged,
               "dhop_gflops": round(st.flops / st.seconds / 1e9, 1)}
        if x64 is None:
            x64 = x
        else:
            d = x - x64
            rec["rel_err_vs_fp64_solution"] = float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(x64))
        out[name] = rec
    out["speedup_mixed_fp32_vs_fp64"] = round(out["fp64"]["seconds"] / out["mixed_fp32"]["seconds"], 2)
    out["speedup_mixed_fp16_vs_fp64"] = round(out["fp64"]["seconds"] / out["mixed_fp16"]["seconds"], 2)
    out["workload"] = CG_WORKLOAD
    out["tol"] = 1e-10
    op.close()
    return out


def run_force(dwf, torch, spec, reps=20):
    """Action and force (FP32 fields, FP64 accumulation) on the 16^4 x 16 derivative-timing
    workload: S = |M psi|^2, the su(3) force and the ambient gradient, per call."""
    dims, Ls = spec["dims"], spec["Ls"]
    U = synth.random_gauge(dims, seed=1000 * spec["case"], eps=spec["eps"])
    op = dwf.GridDWF(dims, Ls, spec["M5"], spec["mass"], bc=BC)
    op.set_gauge(torch.from_numpy(U).cuda())
    f = op.pack(torch.from_numpy(synth.random_spinor(dims, Ls, seed=1000 * spec["case"] + 1)).cuda(), dwf.FP32,
                dwf.FULL)
    shape = (dims[3], dims[2], dims[1], dims[0], 4, 3, 3)
    F = torch.empty(shape, dtype=torch.complex128, device="cuda")
    G = torch.empty(shape, dtype=torch.complex128, device="cuda")
    chi = op.field(dwf.FP32, dwf.FULL)
    for _ in range(3):
        op.force(f, chi=chi)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        op.lib.grid_dwf_set_stream(op._h, dwf._ptr(torch.cuda.current_stream().cuda_stream))
        rc = op.lib.grid_dwf_force(op._h, dwf.FP32, dwf._ptr(f), dwf._ptr(chi), dwf._ptr(F), dwf._ptr(G), None)
        assert rc == 0
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # the same with FP64 fields (FP64 throughout; bound by the FP64 pipe)
    f64 = op.pack(torch.from_numpy(synth.random_spinor(dims, Ls, seed=1000 * spec["case"] + 1)).cuda(), dwf.FP64,
                  dwf.FULL)
    chi64 = op.field(dwf.FP64, dwf.FULL)
    op.force(f64, chi=chi64)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(max(2, reps // 4)):
        rc = op.lib.grid_dwf_force(op._h, dwf.FP64, dwf._ptr(f64), dwf._ptr(chi64), dwf._ptr(F), dwf._ptr(G), None)
        assert rc == 0
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / max(2, reps // 4)
    # FP64 fields with the float-float arithmetic (M psi and the force kernel)
    op.set_fp64_arith(dwf.FP64_ARITH_FLOAT_FLOAT)
    op.force(f64, chi=chi64)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        rc = op.lib.grid_dwf_force(op._h, dwf.FP64, dwf._ptr(f64), dwf._ptr(chi64), dwf._ptr(F), dwf._ptr(G), None)
        assert rc == 0
    e1.record()
    torch.cuda.synchronize()
    ms64ff = e0.elapsed_time(e1) / reps
    op.close()
    return {"workload": "dwf_16x16x16x16_ls16_haar", "ms_per_force": round(ms, 4), "reps": reps,
            "precision": "fp32 fields, fp64 accumulation across blocks of 8 slice pairs",
            "ms_per_force_fp64": round(ms64, 4), "ms_per_force_fp64_float_float": round(ms64ff, 4),
            "includes": "M psi with |M psi|^2 summed in the same launch (Dhop with the fused Mooee term and norm, both halves), a one-CTA sum of the partials, force and ambient-gradient kernel"}


def run_pf_force(dwf, torch, spec):
    """Pseudofermion action phi^+ (Mpc^+ Mpc)^-1 phi and its force on the 16^4 x 16 exp(0.3 i H)
    workload: mixed-precision solve to a 1e-10 true residual, then the force contraction, per call
    (FP64 plain solve for comparison)."""
    dims, Ls = spec["dims"], spec["Ls"]
    U = synth.random_gauge(dims, seed=1000 * spec["case"], eps=spec["eps"])
    op = dwf.GridDWF(dims, Ls, spec["M5"], spec["mass"], bc=BC)
    op.set_gauge(torch.from_numpy(U).cuda())
    phi_c = synth.random_spinor(dims, Ls, seed=1000 * spec["case"] + 7)
    phi = op.pack(torch.from_numpy(phi_c).cuda(), dwf.FP64, dwf.ODD)
    out = {"workload": WORKLOAD, "tol": 1e-10}
    for name, mode, prec in (("mixed_fp32_solve_fp32_force", dwf.CG_MIXED_FP32, dwf.FP32),
                             ("fp64_solve_fp64_force", dwf.CG_FP64, dwf.FP64)):
        op.pf_force(phi, tol=1e-6, mode=mode, precision=prec, raise_on_fail=False)  # warm-up: workspaces, links
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S, F, G, X, st = op.pf_force(phi, tol=1e-10, mode=mode, precision=prec, raise_on_fail=False)
        torch.cuda.synchronize()
        out[name] = {"seconds": round(time.perf_counter() - t0, 4), "iterations": st.iterations,
                     "reliable_updates": st.reliable_updates, "true_residual": st.true_residual,
                     "converged": st.converged, "S": S}
    op.close()
    return out


def run_sweep32(dwf, torch, steps=20, warmup=3, fp64_peak=None):
    """Roofline sweep of DhopEO + DhopOE at 32^4 x 16 (exp(0.5 i H) links, m = 0.005): FP32, FP16,
    BF16 and FP64 storage. One operand set: a 32^4 x 16 half field (805 MB in FP32) is larger than
    L2, so no rotation is needed. Fields are drawn on the device by the seeded generators."""
    spec = synth.WORKLOADS["dwf_32x32x32x32_ls16_exp0.5"]
    dims, Ls = spec["dims"], spec["Ls"]
    n5 = int(np.prod(dims)) // 2 * Ls
    hbm_peak, _ = peaks()
    dev = torch.device("cuda")
    U = synth.random_gauge_device(dims, 1000 * spec["case"], spec["eps"], dev)
    psi = synth.random_spinor_device(dims, Ls, 1000 * spec["case"] + 1, dev)
    op = dwf.GridDWF(dims, Ls, spec["M5"], spec["mass"], bc=BC)
    op.set_gauge(U)
    del U
    out = {"workload": "dwf_32x32x32x32_ls16_exp0.5", "steps": steps, "l2": "one set, half field > L2"}
    stream = torch.cuda.current_stream()
    for name, prec, rb in (("f32", dwf.FP32, 4), ("f16", dwf.FP16, 2), ("bf16", dwf.BF16, 2), ("f64", dwf.FP64, 8)):
        src = op.pack(psi, prec, dwf.FULL)
        dst = op.field(prec, dwf.FULL, zero=True)
        half = op.half_reals
        n = steps
        for _ in range(warmup):
            op.dhop(src, dwf.FULL, out=dst)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        hold_stream(torch, stream)
        e0.record(stream)
        for _ in range(n):
            op.dhop(src, dwf.FULL, out=dst)
        e1.record(stream)
        torch.cuda.synchronize()
        per_half = e0.elapsed_time(e1) / 1e3 / (2 * n)  # per half-lattice application
        gbs = algorithmic_bytes_per_site(rb, Ls) * n5 / per_half / 1e9
        rec = {"us_per_half_lattice": round(per_half * 1e6, 2), "gflops": round(FLOPS_PER_SITE * n5 / per_half / 1e9, 1),
               "algorithmic_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4)}
        if name == "f64" and fp64_peak:
            rec["alu_frac"] = round(rec["gflops"] / fp64_peak, 4)
        out[name] = rec
        del src, dst
    op.close()
    torch.cuda.empty_cache()
    return out


def run_cg32(dwf, torch):
    """Mixed-precision vs FP64 CG at 32^4 x 16, m = 0.005, exp(0.5 i H) links, one Gaussian source,
    to a 1e-10 true residual (on by default; --no-cg32 skips it: the IEEE FP64 solve takes about 14 s)."""
    spec = synth.WORKLOADS["dwf_32x32x32x32_ls16_exp0.5"]
    dims, Ls = spec["dims"], spec["Ls"]
    dev = torch.device("cuda")
    op = dwf.GridDWF(dims, Ls, spec["M5"], spec["mass"], bc=BC)
    op.set_gauge(synth.random_gauge_device(dims, 1000 * spec["case"], spec["eps"], dev))
    b = op.pack(synth.random_spinor_device(dims, Ls, 1000 * spec["case"] + 2, dev), dwf.FP64, dwf.FULL)
    out = {"workload": "dwf_32x32x32x32_ls16_exp0.5", "tol": 1e-10}
    x64 = None
    # *_ff: FP64 operator applications in float-float arithmetic
    for name, mode, arith in (("mixed_fp32", dwf.CG_MIXED_FP32, 0), ("mixed_fp16", dwf.CG_MIXED_FP16, 0),
                              ("fp64", dwf.CG_FP64, 0), ("mixed_fp16_ff", dwf.CG_MIXED_FP16, 1),
                              ("fp64_ff", dwf.CG_FP64, 1)):
        op.set_fp64_arith(arith)
        x, st = op.cg(b, tol=1e-10, maxiter=20000, mode=mode, raise_on_fail=False)
        out[name] = {"seconds": round(st.seconds, 3), "iterations": st.iterations,
                     "reliable_updates": st.reliable_updates, "true_residual": st.true_residual,
                     "converged": st.converged}
        if name == "mixed_fp32":
            x64 = x.clone()
        elif x64 is not None:
            out[name]["rel_diff_vs_mixed_fp32_solution"] = float(torch.linalg.vector_norm(x - x64) /
                                                                 torch.linalg.vector_norm(x64))
    out["speedup_mixed_fp32_vs_fp64"] = round(out["fp64"]["seconds"] / out["mixed_fp32"]["seconds"], 2)
    out["speedup_mixed_fp16_vs_fp64"] = round(out["fp64"]["seconds"] / out["mixed_fp16"]["seconds"], 2)
    op.close()
    return out


def profile_case(args):
    """A fixed, short launch sequence for a profiler (ncu), fields drawn on the device:
    --profile-kernel dhop: the full-lattice Dhop of one precision on the named workload, 3 warm-up
    calls then 3 more; force: the action and force (FP32 fields) likewise; cg: one mixed solve
    (mode from --variants: f32, f16, bf16) to 1e-10; mpc: a half-lattice DhopEO three times, then
    Mpc (its two launches, with the fused fifth-dimension epilogues) three times. Prints one line
    with the CUDA-event time (a number taken under a profiler is not a result)."""
    import torch

    from paper_2203_06777_gb300 import dwf

    torch.cuda.set_device(0)
    spec = synth.WORKLOADS[args.profile]
    dims, Ls = spec["dims"], spec["Ls"]
    if args.profile_kernel in ("force", "cg"):
        dev = torch.device("cuda")
        op = dwf.GridDWF(dims, Ls, spec["M5"], spec["mass"], bc=BC)
        op.set_gauge(synth.random_gauge_device(dims, 1000 * spec["case"], spec["eps"] or 0.3, dev))
        psi = synth.random_spinor_device(dims, Ls, 1000 * spec["case"] + 1, dev)
        if args.profile_kernel == "force":
            f = op.pack(psi, dwf.FP32, dwf.FULL)
            chi = op.field(dwf.FP32, dwf.FULL)
            for _ in range(3):
                op.force(f, chi=chi)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                op.force(f, chi=chi)
            torch.cuda.synchronize()
            print(json.dumps({"profile_case": args.profile, "kernel": "force",
                              "ms_per_call": round((time.perf_counter() - t0) * 1e3 / 3, 3)}), flush=True)
        else:
            mode = {"f32": dwf.CG_MIXED_FP32, "f16": dwf.CG_MIXED_FP16, "bf16": dwf.CG_MIXED_BF16}[
                args.variants.split(",")[0]]
            b = op.pack(psi, dwf.FP64, dwf.FULL)
            x, st = op.cg(b, tol=1e-10, maxiter=20000, mode=mode, raise_on_fail=False)
            print(json.dumps({"profile_case": args.profile, "kernel": "cg", "seconds": round(st.seconds, 4),
                              "iterations": st.iterations, "reliable_updates": st.reliable_updates,
                              "true_residual": st.true_residual}), flush=True)
        op.close()
        return
    prec = {"f32": dwf.FP32, "f16": dwf.FP16, "bf16": dwf.BF16, "f64": dwf.FP64, "f64ff": dwf.FP64}[args.variants.split(",")[0]]
    dev = torch.device("cuda")
    if args.profile_kernel == "mpc":
        op = dwf.GridDWF(dims, Ls, spec["M5"], spec["mass"], bc=BC)
        op.set_gauge(synth.random_gauge_device(dims, 1000 * spec["case"], spec["eps"] or 0.3, dev))
        half = op.pack(synth.random_spinor_device(dims, Ls, 1000 * spec["case"] + 1, dev), prec, dwf.ODD)
        out, te = torch.empty_like(half), torch.empty_like(half)
        torch.cuda.empty_cache()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        for _ in range(3):
            op.dhop(half, dwf.EVEN, out=out)
        e1.record()
        for _ in range(3):
            op.mpc(half, out=out, tmp_even=te)
        e2.record()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": args.profile, "kernel": "mpc", "variant": args.variants.split(",")[0],
                          "us_per_dhop_half": round(e0.elapsed_time(e1) * 1e3 / 3, 2),
                          "us_per_mpc": round(e1.elapsed_time(e2) * 1e3 / 3, 2)}), flush=True)
        op.close()
        return
    op = dwf.GridDWF(dims, Ls, spec["M5"], spec["mass"], bc=BC,
                     fp64_arith=dwf.FP64_ARITH_FLOAT_FLOAT if args.variants.startswith("f64ff") else 0)
    op.set_gauge(synth.random_gauge_device(dims, 1000 * spec["case"], spec["eps"] or 0.3, dev))
    src = op.pack(synth.random_spinor_device(dims, Ls, 1000 * spec["case"] + 1, dev), prec, dwf.FULL)
    dst = op.field(prec, dwf.FULL, zero=True)
    torch.cuda.empty_cache()  # only the fields, links and workspaces stay on the device
    for _ in range(3):
        op.dhop(src, dwf.FULL, out=dst)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        op.dhop(src, dwf.FULL, out=dst)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile, "variant": args.variants.split(",")[0],
                      "us_per_call": round(e0.elapsed_time(e1) * 1e3 / 3, 2),
                      "launches_per_call": launches_per_step(op, prec, dwf)}), flush=True)
    op.close()


def cpu_baseline_sample(spec, target_seconds=10.0):
    """The FP64 oracle as it stands, DhopEO + DhopOE on the full lattice, on all host cores."""
    import oracle

    dims, Ls = spec["dims"], spec["Ls"]
    U = synth.random_gauge(dims, seed=1000 * spec["case"], eps=spec["eps"])
    psi = synth.random_spinor(dims, Ls, seed=1000 * spec["case"] + 1)
    threads = oracle.default_threads()
    n5 = int(np.prod(dims)) // 2 * Ls
    t0 = time.perf_counter()
    oracle.dhop(dims, Ls, BC, U, psi, out_parity=0, nthreads=threads)
    oracle.dhop(dims, Ls, BC, U, psi, out_parity=1, nthreads=threads)
    first = time.perf_counter() - t0
    reps = max(1, int(target_seconds / max(first, 1e-3)))
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.dhop(dims, Ls, BC, U, psi, out_parity=0, nthreads=threads)
        oracle.dhop(dims, Ls, BC, U, psi, out_parity=1, nthreads=threads)
    dt = time.perf_counter() - t0
    gflops = FLOPS_PER_SITE * 2 * n5 * reps / dt / 1e9
    return {"value": round(gflops, 3), "unit": "GFlop/s", "cores": threads, "kind": "oracle",
            "sample": f"{reps} x (DhopEO + DhopOE) FP64 on the full {WORKLOAD} lattice, {dt:.1f} s"}


def gpu_arm(args):
    import torch

    from paper_2203_06777_gb300 import dwf

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    spec = synth.WORKLOADS[WORKLOAD]
    dims, Ls = spec["dims"], spec["Ls"]
    n5 = int(np.prod(dims)) // 2 * Ls
    hbm_peak, peak_kind = peaks()
    peaks_alu = pipe_peaks(dwf)
    variants = {}
    results = {}
    clocks = None
    e2e = None
    wanted = args.variants.split(",")
    for name, prec, rb in (("f32", dwf.FP32, 4), ("f32c12", dwf.FP32, 4), ("f64", dwf.FP64, 8), ("f64ff", dwf.FP64, 8),
                           ("f16", dwf.FP16, 2), ("bf16", dwf.BF16, 2)):
        if name not in wanted:
            continue
        arith = dwf.FP64_ARITH_FLOAT_FLOAT if name == "f64ff" else dwf.FP64_ARITH_NATIVE
        c12 = name == "f32c12"
        sets = make_sets(dwf, torch, spec, prec, 3, seed0=0, fp64_arith=arith, compress12=c12)
        steps = args.steps
        if name == "f32":
            with ClockSampler(torch.cuda.current_device()) as cs:
                # The sampler reads nvidia-smi every 50 ms; a short timed region (20 steps take about
                # 1 ms) would see no sample, so the same step runs untimed for ~0.3 s first (clocks at
                # their loaded value) and the sampler's window brackets that soak and the timed region.
                cs.wait_first_sample()
                if not args.no_clock_soak:
                    soak(dwf, torch, sets, 0.3)
                secs = time_dhop(dwf, torch, sets, steps, args.warmup, world)
                cs.wait_next_sample()
            clocks = cs.summary()
            clocks["window"] = "0.3 s untimed soak of the same step, the warm-up and the timed region"
        else:
            secs = time_dhop(dwf, torch, sets, steps, args.warmup, world)
        secs = reduce_max(secs, world)
        launches = steps * launches_per_step(sets[0][0], prec, dwf)
        per_step = secs / steps
        bytes_site = algorithmic_bytes_per_site(rb, Ls, 12 if c12 else 18)
        gbs = bytes_site * 2 * n5 / per_step / 1e9
        gflops = FLOPS_PER_SITE * 2 * n5 / per_step / 1e9
        rec = {"gflops": round(gflops, 1), "algorithmic_gbs": round(gbs, 1),
               "hbm_frac": round(gbs / hbm_peak, 4), "us_per_step": round(per_step * 1e6, 2),
               "us_per_half_lattice": round(per_step / 2 * 1e6, 2), "launches_per_step": launches // steps,
               "bytes_per_site": bytes_site, "steps": steps}
        if name == "f64":
            rec["alu_frac"] = round(gflops / peaks_alu["fp64_fma_gflops"], 4)
            rec["bound"] = "alu"
            rec["alu_peak_gflops"] = peaks_alu["fp64_fma_gflops"]
            rec["alu_peak_kind"] = "measured (grid_dwf_pipe_peak, FP64 FMA)"
        if c12:
            rec["links"] = "12 reals per link (third row rebuilt as the conjugated cross product)"
            rec["speedup_vs_f32"] = round(variants["f32"]["us_per_step"] / rec["us_per_step"], 3) if "f32" in variants else None
        if name == "f64ff":
            rec["arithmetic"] = "float-float (FP64 storage, pairs of FP32 numbers, ~46 significant bits)"
            rec["bound"] = "instruction issue (FP32, integer and FP64 pipes)"
            if "f64" in variants:
                rec["speedup_vs_f64"] = round(variants["f64"]["us_per_step"] / rec["us_per_step"], 2)
        results[name] = (secs, steps, launches, per_step, gbs, gflops)
        variants[name] = rec
        if name == "f32":
            e2e_steps = args.steps
            e2e_secs, hb, db = time_dhop_e2e(dwf, torch, sets, e2e_steps, args.warmup, world)
            e2e_secs = reduce_max(e2e_secs, world)
            e2e = {"value": round(world * FLOPS_PER_SITE * 2 * n5 * e2e_steps / e2e_secs / 1e9, 1), "unit": "GFlop/s",
                   "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db, "steps": e2e_steps}
        for st in sets:
            st[0].close()
        del sets
        torch.cuda.empty_cache()
    if "f32" not in results:
        if rank == 0:
            print(json.dumps({"variants": variants}), flush=True)
        return
    secs, steps, launches, per_step, gbs, gflops = results["f32"]
    value = job_throughput(FLOPS_PER_SITE * 2 * n5 * steps, world, secs) / 1e9
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "GFlop/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": round(secs / steps * 1e3, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded exp(0.3 i H) links, Gaussian spinors)",
        "config": {"workload": WORKLOAD, "lattice": list(dims), "Ls": Ls, "M5": spec["M5"], "mass": spec["mass"],
                   "bc": list(BC), "step": "DhopEO + DhopOE (one full-lattice launch)", "parallelism": f"replicas x{world}",
                   "l2": "3 rotating operator+field sets (663 MB FP32) > L2"},
        "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(gbs / hbm_peak, 4), "traffic": measured_traffic(), "peak_kind": peak_kind,
                     "kernel": "dhop_kernel<FP32> (DhopEO + DhopOE in one launch)",
                     "bytes_per_launch": algorithmic_bytes_per_site(4, Ls) * 2 * n5,
                     "source_hash": kernel_source_hash()},
        "variants": variants,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_cg and rank == 0:
        line["cg"] = run_cg(dwf, torch, synth.WORKLOADS[CG_WORKLOAD])
    line["pipe_peaks"] = peaks_alu
    if not args.no_sweep and rank == 0:
        sw = run_sweep32(dwf, torch, fp64_peak=peaks_alu["fp64_fma_gflops"])
        line["sweep_32x32x32x32_ls16"] = sw
        # the largest single-GPU workload's headline: the same kernel on the 32^4 x 16 lattice
        # (half field 805 MB in FP32, larger than L2: one operand set)
        f32 = sw["f32"]
        line["roofline_32x32x32x32_ls16"] = {
            "bound": "hbm", "achieved": f32["algorithmic_gbs"], "peak": hbm_peak, "unit": "GB/s",
            "frac": f32["hbm_frac"], "traffic": measured_traffic(TRAFFIC_PROFILE_32), "peak_kind": peak_kind,
            "kernel": "dhop_kernel<FP32> (DhopEO + DhopOE in one launch)", "gflops": f32["gflops"],
            "bytes_per_launch": algorithmic_bytes_per_site(4, 16) * 2 * (32 ** 4 // 2) * 16,
            "us_per_launch": round(2 * f32["us_per_half_lattice"], 2), "steps": sw["steps"]}
    if not args.no_cg32 and rank == 0:
        line["cg_32x32x32x32_ls16"] = run_cg32(dwf, torch)
    if not args.no_force and rank == 0:
        line["force"] = run_force(dwf, torch, synth.WORKLOADS["dwf_16x16x16x16_ls16_haar"])
        line["pf_force"] = run_pf_force(dwf, torch, spec)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_sample(spec)
    barrier(world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ---------------------------------------------------------------- reference arm (the oracle)


def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    spec = synth.WORKLOADS[WORKLOAD]
    dims, Ls = spec["dims"], spec["Ls"]
    U = synth.random_gauge(dims, seed=1000 * spec["case"], eps=spec["eps"])
    psi = synth.random_spinor(dims, Ls, seed=1000 * spec["case"] + 1)
    threads = oracle.default_threads()
    n5 = int(np.prod(dims)) // 2 * Ls

    def step():
        oracle.dhop(dims, Ls, BC, U, psi, out_parity=0, nthreads=threads)
        oracle.dhop(dims, Ls, BC, U, psi, out_parity=1, nthreads=threads)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = FLOPS_PER_SITE * 2 * n5 * args.steps / dt / 1e9
    line = {"metric": METRIC, "value": round(value, 3), "unit": "GFlop/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "lattice": list(dims), "Ls": Ls, "step": "DhopEO + DhopOE"},
            "cpu_baseline": {"value": round(value, 3), "unit": "GFlop/s", "cores": threads, "kind": "oracle",
                             "sample": f"each step one DhopEO + DhopOE FP64 on the full {WORKLOAD} lattice"},
            "e2e": {"value": round(value, 3), "unit": "GFlop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--variants", default="f32,f32c12,f64,f64ff,f16,bf16",
                    help="comma list of f32,f32c12 (FP32 with 12-real links),f64,f64ff,f16,bf16")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cg", action="store_true", help="skip the CG time-to-solution comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 32^4 x 16 Dhop roofline sweep")
    ap.add_argument("--no-cg32", action="store_true", help="skip the 32^4 x 16 mixed vs FP64 CG (about 25 s)")
    ap.add_argument("--no-clock-soak", action="store_true",
                    help="skip the untimed 0.3 s run of the step before the FP32 timing (a fixed launch count, for ncu)")
    ap.add_argument("--no-force", action="store_true", help="skip the action/force and pseudofermion force timing")
    ap.add_argument("--profile", default=None, help="run only a short launch sequence of this workload "
                    "(a synth.WORKLOADS name) for a profiler, in the first precision of --variants")
    ap.add_argument("--profile-kernel", default="dhop", choices=["dhop", "force", "cg", "mpc"],
                    help="what --profile runs: the hopping term, the action and force, one mixed CG solve, "
                    "or a half-lattice hop and Mpc")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.profile:
        profile_case(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
