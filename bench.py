#!/usr/bin/env python3
"""Throughput of the Viana-Bray bit-packed Metropolis sweep on GB300, in spin updates per ns.

Workload (one "step" = one sweep of both temperature instances, measurements included when the
schedule falls inside the timed window):
  Poissonian random graph, N = 2^22, mean degree c = 4, J = +-1, 64 disorder samples packed per
  uint64 lane word, two replicas, temperatures T = 1.0 and T = 0.6 (two instances on the same
  graph and couplings), snapshots at t_w = 2^4..2^15 and measurements of C(t_w, t_w + 2^k), q, E
  on the log schedule up to 2^16 sweeps.  Spin updates per step = 2 * N * 64 * 2.

Under torchrun (N > 1 GPUs) every rank runs its own independent instance (its own graph seed):
weak scaling with no collective on the data path; rank 0 prints the one JSON line.

Beside the headline, the same line carries one object per other configuration of the metric
(one GPU only): "sk" (SK, N = 8192, 256 replicas sharing J, T = 0.4, B = 128), "vb_batch" (512
uneven Poissonian graphs, N in [2^10, 2^20]) and "sk_batch" (32 uneven SK samples, N in
[2^9, 2^14], 128 replicas), each with its own value, ms_per_step, roofline, e2e, clocks and CPU
baseline.  --skip-extra leaves them out.

--impl reference times the plain CPU oracle (single thread) on a bounded sample of the same
workload instead (the test oracle as it stands).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sg_inputs  # noqa: E402

N_VERTS = 1 << 22
MEAN_DEGREE = 4.0
LANES = 64
REPLICAS = 2
TEMPS = (1.0, 0.6)
T_MAX = 1 << 16
TW = [1 << k for k in range(4, 16)]
WORKLOAD = "vb_packed_poisson_c4_N4194304_lanes64_R2_T1.0+0.6"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def graph_seed(rank: int) -> int:
    """Each rank simulates its own independent instance (weak scaling, no data exchange)."""
    return 2 + 1000 * rank


def instance(rank: int, n: int = N_VERTS):
    rp, col, eid = sg_inputs.poisson_graph(n, MEAN_DEGREE, graph_seed(rank))
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, graph_seed(rank))
    return rp, col, jb


def max_over_ranks(ms: float, device=None) -> float:
    """The job time is the slowest rank's (all ranks started after the same barrier)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(updates_per_rank_step: int, steps: int, world: int, ms: float) -> float:
    """Whole-job throughput: all ranks' spin updates over the slowest rank's time (per ns)."""
    return world * updates_per_rank_step * steps / (ms * 1e6)


def algorithmic_bytes_per_sweep(n, n_entries_directed, R):
    """vinfo 4 B/vertex + (col 4 B + J 8 B) per directed entry + own R words read and written."""
    return 4 * n + 12 * n_entries_directed + 16 * n * R


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the colour kernel's code (comments and layout removed, so a comment edit does
    not invalidate the recorded traffic, while any code change does)."""
    import re
    h = hashlib.sha256()
    for f in ("vb_colour.cuh", "sg_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1906_11195_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per sweep of the colour kernel from the committed ncu summary, if it was
    taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "vb_packed_colour_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_sha") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_sweep"])


class _Nvml:
    """The few NVML queries the clock record needs (SM clock, its maximum, the active clock
    event reasons), called through ctypes on NVML (libnvidia-ml.so.1, part of the GPU's display
    driver install).  Reads only."""
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        found = False
        try:  # the CUDA device by its PCI address (NVML numbers every GPU of the host)
            import torch
            p = torch.cuda.get_device_properties(index)
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
            found = self.lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(self.h)) == 0
        except Exception:
            found = False
        if not found and self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        try:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        v = ctypes.c_uint()
        if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(v)) != 0:
            raise RuntimeError("no max clock")
        self.max_mhz = float(v.value)

    def sample(self):
        ct = self.ct
        v, r = ct.c_uint(), ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(v)) != 0:
            return None
        if self.reasons_fn(self.h, ct.byref(r)) != 0:
            return None
        return float(v.value), int(r.value)


class ClockSampler:
    """SM clock and throttle reasons sampled every millisecond from a thread, from enqueued()
    (the timed work is queued and the GPU runs it) to stop(), so that even a timed region of a
    few milliseconds holds several samples while the queries cannot delay the launches (NVML
    through ctypes; nvidia-smi at 200 ms from start() where NVML cannot be loaded)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.thread = None
        self.path = None
        self.go = None

    def enqueued(self):
        if self.go is not None:
            self.go.set()

    def start(self):
        import threading
        try:
            self.nvml = _Nvml(self.index)
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            self.samples = []
            self.stop_ev = threading.Event()
            self.go = threading.Event()

            def loop():
                while not self.go.wait(0.001):
                    if self.stop_ev.is_set():
                        return
                while True:
                    s = self.nvml.sample()
                    if s is not None:
                        self.samples.append(s)
                    if self.stop_ev.is_set():
                        return
                    time.sleep(0.001)

            self.thread = threading.Thread(target=loop, daemon=True)
            self.thread.start()
            return
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.go.set()
            self.stop_ev.set()
            self.thread.join(timeout=5)
            self.thread = None
            if not self.samples:
                return None
            reasons = set()
            for _, r in self.samples:
                for bit, nm in _Nvml.REASONS.items():
                    if r & bit:
                        reasons.add(nm)
            return {"sm_mhz": statistics.median(m for m, _ in self.samples),
                    "sm_max_mhz": self.nvml.max_mhz, "reasons": sorted(reasons),
                    "samples": len(self.samples), "source": "nvml, 1 ms"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 200 ms"}


def cpu_baseline_sample(rp, col, jb, budget_lanes=16):
    """The CPU oracle (single thread) on one sweep of the same graph at T = 1.0, R = 2."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.vb_run(rp, col, jb, budget_lanes, [TEMPS[0]] * REPLICAS, 1, 1)
    dt = time.perf_counter() - t0
    updates = N_VERTS * budget_lanes * REPLICAS
    return {"value": updates / (dt * 1e9), "unit": "spin updates/ns", "cores": 1, "kind": "oracle",
            "sample": f"1 sweep of the N=2^22 graph at T=1.0, {budget_lanes} lanes x {REPLICAS} "
                      f"replicas ({updates} spin updates, {dt:.1f} s, initial draw included)"}


def _oracle_worker(args):
    """One process of the all-core CPU sample: the oracle as it stands on its own copy of the
    graph (regenerated from the seed), timed around the sweep only."""
    lanes, seed, n_verts = args
    import oracle
    rp, col, eid = sg_inputs.poisson_graph(n_verts, MEAN_DEGREE, seed)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, seed)
    t0 = time.perf_counter()
    oracle.vb_run(rp, col, jb, lanes, [TEMPS[0]] * REPLICAS, 1, 1)
    return n_verts * lanes * REPLICAS, time.perf_counter() - t0


def cpu_baseline_all_cores(budget_lanes=16, n_verts=N_VERTS):
    """The same oracle sweep in one process per host core at once (independent disorder
    samples, as the paper's CPU runs were), started with spawn after the GPU work: the aggregate
    rate over the slowest process's time."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    n = max(1, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_worker, [(budget_lanes, graph_seed(0), n_verts)] * n)
    updates = sum(u for u, _ in res)
    dt = max(t for _, t in res)
    return {"value": updates / (dt * 1e9), "unit": "spin updates/ns", "cores": n, "kind": "oracle",
            "sample": f"{n} processes, each 1 sweep of an N={n_verts} graph at T=1.0, {budget_lanes} "
                      f"lanes x {REPLICAS} replicas ({dt:.1f} s for the slowest)"}


def reference_sample(steps, warmup):
    """Size of one reference step: the oracle (single thread, about 0.0115 spin updates/ns on
    one Grace core) sweeps a graph of the same ensemble (Poissonian, c = 4, R = 2, T = 1.0) whose
    size keeps warm-up + timed steps within about three minutes: the full N = 2^22 graph with as
    many lanes as fit, else one lane of a smaller graph N = 2^k (k >= 10)."""
    per_update_ns = 1.0 / 0.0115
    budget_s = min(4.0, 170.0 / max(1, steps + warmup))
    fit = budget_s * 1e9 / per_update_ns / REPLICAS  # spin updates of one replica per step
    if fit >= N_VERTS:
        return N_VERTS, int(min(64, fit // N_VERTS))
    k = max(10, int(np.floor(np.log2(max(1.0, fit)))))
    return 1 << k, 1


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n, lanes = reference_sample(args.steps, args.warmup)
    rp, col, jb = instance(0, n=n)
    temps = [TEMPS[0]] * REPLICAS
    for _ in range(args.warmup):
        oracle.vb_run(rp, col, jb, lanes, temps, 1, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.vb_run(rp, col, jb, lanes, temps, 1, 1)
    dt = time.perf_counter() - t0
    updates = args.steps * n * lanes * REPLICAS
    value = updates / (dt * 1e9)
    sample = (f"per step: 1 oracle sweep (initial draw included) of a Poissonian c=4 graph with "
              f"N={n}, {lanes} lane(s) x {REPLICAS} replicas, T=1.0")
    line = {
        "impl": "reference", "metric": "spin updates/ns", "value": value, "unit": "spin updates/ns",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "spin updates/ns", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "spin updates/ns", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(args):
    """One T = 1.0 instance of the full-size graph with no measurement schedule: W + K sweeps.
    This is the small case used for detailed ncu captures of the colour kernel (about 0.3 GB on
    the device, inputs larger than L2).  With --workload sk: the SK workload's handle (N = 8192,
    256 replicas, T = 0.4, B = 128, about 0.4 GB on the device), W sweeps and then K sweeps in
    one call (one persistent launch per replayed graph).  Prints timing only; not a bench line."""
    import torch
    if args.workload == "sk":
        import paper_1906_11195_gb300 as sg
        from paper_1906_11195_gb300 import _build
        _build.build()
        torch.cuda.set_device(0)
        J = sg_inputs.sk_couplings(SK_N, 3)
        run = sg.SKRun(J, [SK_T] * SK_R, 1, kernel=sg.SG_SK_BLOCKED, block=SK_B)
        run.sweep(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run.sweep(args.steps)
        e1.record()
        torch.cuda.synchronize()
        run.synchronize()
        ms = e0.elapsed_time(e1) / max(1, args.steps)
        print(json.dumps({"mode": "profile", "workload": SK_WORKLOAD, "ms_per_sweep": ms,
                          "sweeps": args.steps, "launches": run.launches}), flush=True)
        run.close()
        return 0

    import paper_1906_11195_gb300 as sg
    from paper_1906_11195_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    rp, col, jb = instance(0, n=1 << args.profile_log2n)
    temps = [TEMPS[0]] * REPLICAS if args.profile_replicas == 2 else \
        [T for T in TEMPS for _ in range(args.profile_replicas // len(TEMPS))]
    g = dict(row_ptr=rp, col=col, jbits=jb, seed=1, temps=temps)
    run = sg.VBRun([g], n_lanes=LANES, n_replicas=len(temps), kernel=sg.SG_VB_PACKED)
    run.sweep(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run.sweep(args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    print(json.dumps({"mode": "profile", "ms_per_sweep": ms, "sweeps": args.steps,
                      "launches": run.launches}), flush=True)
    run.close()
    return 0


SK_N, SK_R, SK_T, SK_B = 8192, 256, 0.4, 128
SK_WORKLOAD = f"sk_blocked_N{SK_N}_R{SK_R}_T{SK_T}_B{SK_B}"
VB_BATCH_WORKLOAD = "vb_batch_512_graphs_N2^10..2^20_c4_lanes64_R2_T1.0"
SK_BATCH_WORKLOAD = "sk_batch_32_samples_N2^9..2^14_R128_T0.4+0.6_autotuned_B"
L2_FLUSH_BYTES = 256 << 20  # twice the 129 MB L2


def e4m3_peak():
    """e4m3 dense tensor peak: the measured bf16 burst rate x 2 (the nominal e4m3/bf16 ratio)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return 2.0 * float(json.load(f)["bf16_tflops"]), "measured bf16 burst x 2 (nominal e4m3/bf16 ratio)"
    return 2.0 * 1900.0, "fallback bf16 1.9 PFLOP/s x 2 (nominal e4m3/bf16 ratio)"


SK_TIMED_CHUNK = 64  # sweeps per timed iteration of a workload whose inputs fit in L2: the
                    # largest replayed graph, one persistent SK launch


def _timed_region(run, steps, stream, flush=None, sampler=None):
    """CUDA-event time (ms) of `steps` sweeps of `run` on `stream`.  With a flush buffer, the
    sweeps are timed in iterations of SK_TIMED_CHUNK consecutive sweeps (one replayed graph, one
    persistent launch for SK) and the buffer (larger than L2) is rewritten between iterations,
    outside the timed intervals; otherwise one interval covers all sweeps."""
    import torch
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nvtx_push("timed_region")
        e0.record(stream)
        run.sweep(steps)
        e1.record(stream)
        nvtx_pop()
        if sampler is not None:
            sampler.enqueued()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)
    chunks = [min(SK_TIMED_CHUNK, steps - c) for c in range(0, steps, SK_TIMED_CHUNK)]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in chunks]
    nvtx_push("timed_region")
    for k, ((a, b), n) in enumerate(zip(evs, chunks)):
        a.record(stream)
        run.sweep(n)
        b.record(stream)
        with torch.cuda.stream(stream):
            flush.fill_(k & 0x7F)
    nvtx_pop()
    if sampler is not None:
        sampler.enqueued()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def _e2e(create, steps, updates_per_step, dev, stream, sg):
    """The same metric end to end through the C ABI from host buffers: attach (H2D of the
    handle's device image) + `steps` sweeps + D2H of every count, around one host clock; the
    host-side instance preparation (validation, layout) precedes the timed region."""
    import torch
    h = create()
    nb = sg.sg_workspace_bytes(h)
    buf = torch.empty(nb, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sg.sg_attach(h, buf.data_ptr(), nb, stream.cuda_stream)
    sg.sg_sweep(h, steps)
    C, q, E = sg.sg_read_results(h)
    dt = time.perf_counter() - t0
    h2d, d2h = sg.sg_transfer_bytes(h)
    sg.sg_destroy(h)
    del buf
    return {"value": updates_per_step * steps / (dt * 1e9), "unit": "spin updates/ns",
            "h2d_bytes_per_step": h2d // steps, "d2h_bytes_per_step": d2h // steps,
            "note": f"attach (H2D of the {h2d} B instance image into a {nb} B workspace) + {steps} "
                    f"sweeps + D2H of all counts ({d2h} B), counted by the library"}


def measure_sk(args, dev, stream, steps, warmup, cpu=True):
    """SK, N = 8192, +-1 couplings, 256 replicas sharing J, T = 0.4, block B = 128 as configured
    (one step = one sweep of all replicas).  The working set (about 90 MB) fits in L2, so the
    sweeps are timed in iterations of SK_TIMED_CHUNK with L2 flushed before each.  Beside it:
    the autotuner's choice."""
    import torch

    import paper_1906_11195_gb300 as sg
    J = sg_inputs.sk_couplings(SK_N, 3)
    R = SK_R
    tw, tm = sg_inputs.log_schedule([1 << k for k in range(0, 12)], 1 << 12)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def timed(block):
        run = sg.SKRun(J, [SK_T] * R, 1, kernel=sg.SG_SK_BLOCKED, block=block, tw=tw, tm=tm,
                       device=dev, stream=stream)
        run.sweep(warmup)
        torch.cuda.synchronize()
        l0 = run.launches
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        ms = _timed_region(run, steps, stream, flush, sampler)
        clocks = sampler.stop()
        run.synchronize()
        launches = run.launches - l0
        run.close()
        return ms / steps, launches, clocks

    ms, launches, clocks = timed(SK_B)
    a_ms, _, _ = timed(0)
    flops = 2.0 * SK_N * (SK_N - SK_B) * R  # off-block field update of one sweep
    peak, peak_src = e4m3_peak()
    achieved = flops / (ms * 1e-3) / 1e12
    out = {"metric": "spin updates/ns", "unit": "spin updates/ns", "value": SK_N * R / (ms * 1e6),
           "ms_per_step": ms, "steps": steps, "warmup": warmup, "gpu_launches": launches,
           "config": {"workload": SK_WORKLOAD, "N": SK_N, "replicas": R, "T": SK_T, "block": SK_B,
                      "schedule": "tw = 2^0..2^11, log-spaced measurements",
                      "l2": f"working set ~90 MB < L2: timed in iterations of up to {SK_TIMED_CHUNK} "
                            "sweeps (the largest replayed graph: one persistent launch), a "
                            "256 MB L2 flush before each"},
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                        "kernel": "field update on the tensor cores (e4m3 tcgen05), one unit = one sweep",
                        "algorithmic_flops_per_sweep": flops,
                        "note": "achieved = 2 N (N - B) R flops per sweep over the whole sweep's "
                                "event time (every kernel of the sweep): a lower bound of the "
                                "field kernel's own rate"},
           "autotuned": {"value": SK_N * R / (a_ms * 1e6), "ms_per_step": a_ms},
           "clocks": clocks}
    out["e2e"] = _e2e(lambda: sg.sg_create_sk(J, R, [SK_T] * R, 1, sg.SG_SK_BLOCKED, SK_B, tw, tm),
                      warmup + steps, SK_N * R, dev, stream, sg)
    if cpu:
        import oracle
        oracle.build()
        rs, sw = 4, 3
        t0 = time.perf_counter()
        oracle.sk_run(J, [SK_T] * rs, 1, sw)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": SK_N * rs * sw / (dt * 1e9), "unit": "spin updates/ns",
                               "cores": 1, "kind": "oracle",
                               "sample": f"{sw} sweeps of N={SK_N} from the quench, {rs} replicas, "
                                         f"T={SK_T} ({dt:.1f} s, initial fields included)"}
    del flush
    return out


def _gen_vb_graph(args):
    k, n = args
    rp, col, eid = sg_inputs.poisson_graph(int(n), MEAN_DEGREE, (4 << 20) + k)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, (4 << 20) + k)
    return rp, col, jb


def vb_batch_graphs(count=512):
    """The uneven batch: count Poissonian c = 4 graphs, N = round(2^U), U ~ Uniform[10, 20],
    drawn in parallel host processes (spawned, so safe after CUDA initialisation)."""
    import multiprocessing as mp
    sizes = sg_inputs.log_uniform_sizes(count, 10, 20, 4)
    jobs = list(enumerate(int(n) for n in sizes))
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        res = pool.map(_gen_vb_graph, jobs, chunksize=4)
    graphs = [dict(row_ptr=rp, col=col, jbits=jb, seed=(4 << 20) + k, temps=[1.0] * REPLICAS)
              for k, (rp, col, jb) in enumerate(res)]
    return sizes, graphs


def measure_vb_batch(args, dev, stream, steps, warmup, cpu=True, count=512):
    """Batched uneven VB: 512 Poissonian c = 4 graphs, N log-uniform in [2^10, 2^20], 64 lanes,
    R = 2, T = 1.0, all graphs in lock-step (one fused launch per sweep for the whole batch,
    replayed from CUDA graphs).  One step = one sweep of the whole batch."""
    import torch

    import paper_1906_11195_gb300 as sg
    t0 = time.perf_counter()
    sizes, graphs = vb_batch_graphs(count)
    log(f"vb_batch: generated {len(graphs)} graphs, sum N = {int(sizes.sum())} in {time.perf_counter() - t0:.1f} s")
    tw, tm = sg_inputs.log_schedule([1 << k for k in range(4, 14)], 1 << 14)
    t0 = time.perf_counter()
    run = sg.VBRun(graphs, n_lanes=LANES, n_replicas=REPLICAS, kernel=sg.SG_VB_PACKED, tw=tw, tm=tm,
                   device=dev, stream=stream)
    log(f"vb_batch: created and attached in {time.perf_counter() - t0:.1f} s")
    run.sweep(warmup)
    torch.cuda.synchronize()
    l0 = run.launches
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms = _timed_region(run, steps, stream, sampler=sampler) / steps
    clocks = sampler.stop()
    run.synchronize()
    launches = run.launches - l0
    run.close()
    n_sum = int(sizes.sum())
    updates = n_sum * LANES * REPLICAS
    n_entries = sum(int(g["row_ptr"][-1]) for g in graphs)
    bytes_sweep = algorithmic_bytes_per_sweep(n_sum, n_entries, REPLICAS)
    peak, peak_kind = peaks()
    achieved = bytes_sweep / (ms * 1e-3) / 1e9
    out = {"metric": "spin updates/ns", "unit": "spin updates/ns", "value": updates / (ms * 1e6),
           "ms_per_step": ms, "steps": steps, "warmup": warmup, "gpu_launches": launches,
           "config": {"workload": VB_BATCH_WORKLOAD, "graphs": len(graphs), "sum_N": n_sum,
                      "schedule": "tw = 2^4..2^13, log-spaced measurements",
                      "l2": f"inputs larger than L2: {bytes_sweep / 1e9:.2f} GB streamed per sweep"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                        "kernel": "k_vb_packed_colour over the whole batch, one unit = one sweep",
                        "algorithmic_bytes_per_sweep": bytes_sweep,
                        "note": "achieved over the timed region (measurements included)"},
           "clocks": clocks}
    out["e2e"] = _e2e(lambda: sg.sg_create_vb(graphs, LANES, REPLICAS, sg.SG_VB_PACKED, tw, tm),
                      warmup + steps, updates, dev, stream, sg)
    if cpu:
        import oracle
        oracle.build()
        k = int(np.argmin(np.abs(sizes - (1 << 16))))
        g = graphs[k]
        lanes = 16
        t0 = time.perf_counter()
        oracle.vb_run(g["row_ptr"], g["col"], g["jbits"], lanes, g["temps"], g["seed"], 4)
        dt = time.perf_counter() - t0
        n = int(sizes[k])
        out["cpu_baseline"] = {"value": n * lanes * REPLICAS * 4 / (dt * 1e9), "unit": "spin updates/ns",
                               "cores": 1, "kind": "oracle",
                               "sample": f"4 sweeps of batch graph {k} (N={n}), {lanes} lanes x "
                                         f"{REPLICAS} replicas ({dt:.2f} s, initial draw included)"}
    return out


def sk_batch_samples():
    sizes = [int(x) for x in sg_inputs.log_uniform_sizes(32, 9, 14, 5)]
    R = 128
    samples = [dict(J=sg_inputs.sk_couplings(n, (5 << 20) + k), seed=(5 << 20) + k,
                    temps=[0.4] * (R // 2) + [0.6] * (R // 2)) for k, n in enumerate(sizes)]
    return sizes, R, samples


def measure_sk_batch(args, dev, stream, steps, warmup, cpu=True):
    """Batched uneven SK: 32 samples, N = round(2^U), U ~ Uniform[9, 14], +-1 couplings,
    R = 128 replicas (64 at T = 0.4, 64 at T = 0.6), block chosen per sample by the autotuner;
    all samples advance in lock-step, one CUDA graph branch per sample.  One step = one sweep of
    every sample."""
    import torch

    import paper_1906_11195_gb300 as sg
    t0 = time.perf_counter()
    sizes, R, samples = sk_batch_samples()
    log(f"sk_batch: generated {len(samples)} samples, sum N = {sum(sizes)} in {time.perf_counter() - t0:.1f} s")
    tw, tm = sg_inputs.log_schedule([3, 12, 48], 1 << 14)
    t0 = time.perf_counter()
    run = sg.SKBatchRun(samples, R, kernel=sg.SG_SK_BLOCKED, block=0, tw=tw, tm=tm, device=dev,
                        stream=stream)
    log(f"sk_batch: created, attached and tuned in {time.perf_counter() - t0:.1f} s")
    run.sweep(warmup)
    torch.cuda.synchronize()
    l0 = run.launches
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms = _timed_region(run, steps, stream, sampler=sampler) / steps
    clocks = sampler.stop()
    run.synchronize()
    launches = run.launches - l0
    run.close()
    updates = sum(sizes) * R
    flops = sum(2.0 * n * n * R for n in sizes)
    peak, peak_src = e4m3_peak()
    achieved = flops / (ms * 1e-3) / 1e12
    j_bytes = sum(n * n for n in sizes)
    out = {"metric": "spin updates/ns", "unit": "spin updates/ns", "value": updates / (ms * 1e6),
           "ms_per_step": ms, "steps": steps, "warmup": warmup, "gpu_launches": launches,
           "config": {"workload": SK_BATCH_WORKLOAD, "sizes": sizes, "replicas": R,
                      "schedule": "tw = 3, 12, 48, log-spaced measurements",
                      "l2": f"inputs larger than L2: {j_bytes / 1e9:.2f} GB of e4m3 couplings"},
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                        "kernel": "field update on the tensor cores (e4m3 tcgen05), one unit = one sweep of every sample",
                        "algorithmic_flops_per_sweep": flops,
                        "note": "2 N^2 R flops per sample per sweep over the whole sweep's event time"},
           "clocks": clocks}
    out["e2e"] = _e2e(lambda: sg.sg_create_sk_batch(samples, R, sg.SG_SK_BLOCKED, 0, tw, tm),
                      warmup + steps, updates, dev, stream, sg)
    if cpu:
        import oracle
        oracle.build()
        k = int(np.argmin(np.abs(np.array(sizes) - 2048)))
        x = samples[k]
        rs, sw = 4, 3
        t0 = time.perf_counter()
        oracle.sk_run(x["J"], x["temps"][:rs], x["seed"], sw)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": sizes[k] * rs * sw / (dt * 1e9), "unit": "spin updates/ns",
                               "cores": 1, "kind": "oracle",
                               "sample": f"{sw} sweeps of batch sample {k} (N={sizes[k]}), {rs} "
                                         f"replicas at T=0.4 ({dt:.2f} s)"}
    return out


def _single_gpu():
    import torch

    from paper_1906_11195_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    return dev, torch.cuda.current_stream(dev)


def run_vb_batch(args):
    """The batched uneven VB workload on its own (the same object as the default run's vb_batch
    key); --batch sets the number of graphs."""
    dev, stream = _single_gpu()
    out = measure_vb_batch(args, dev, stream, args.steps, args.warmup, cpu=not args.skip_cpu,
                           count=args.batch)
    print(json.dumps(out), flush=True)
    return 0


T_08_TC = 0.8 / float(np.arctanh(1.0 / np.sqrt(3.0)))  # 0.8 T_c of the z = 4 model, 1.21492
PAPER_P100_UPDATES_PER_NS = 1000.0 / 15.0  # the paper's ~15 ps per spin update (one P100)


def run_rrbg(args):
    """The paper's own GPU ensemble (not the headline line): a random regular bipartite graph
    of degree 4, N = 2^22, 64 coupling sets per word, R = 2, T = 0.8 T_c; the greedy colouring
    is exactly the two halves, so a sweep is the paper's two half-updates.  Snapshots at
    t_w = 2^2 .. 2^12, measurements on the log schedule; one step = one sweep."""
    import torch

    import paper_1906_11195_gb300 as sg
    from paper_1906_11195_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    n = N_VERTS
    rp, col, eid = sg_inputs.random_regular_graph(n, 4, 6, bipartite=True)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 6)
    tw, tm = sg_inputs.log_schedule([1 << k for k in range(2, 13)], args.warmup + args.steps)
    g = dict(row_ptr=rp, col=col, jbits=jb, seed=1, temps=[T_08_TC] * REPLICAS)
    run = sg.VBRun([g], n_lanes=LANES, n_replicas=REPLICAS, kernel=sg.SG_VB_PACKED, tw=tw, tm=tm)
    stream = torch.cuda.current_stream()
    run.sweep(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = run.launches
    nvtx_push("timed_region")
    e0.record(stream)
    run.sweep(args.steps)
    e1.record(stream)
    nvtx_pop()
    torch.cuda.synchronize()
    run.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    bytes_sweep = algorithmic_bytes_per_sweep(n, int(rp[-1]), REPLICAS)
    peak, _ = peaks()
    value = n * LANES * REPLICAS / (ms * 1e6)
    out = {"metric": "spin updates/ns", "unit": "spin updates/ns",
           "value": value, "ms_per_step": ms, "steps": args.steps,
           "warmup": args.warmup, "gpu_launches": run.launches - l0,
           "vs_baseline": None,
           # the paper's own figure for this ensemble, another machine: context, not a baseline
           "context": {"paper_p100_updates_per_ns": PAPER_P100_UPDATES_PER_NS,
                       "ratio_to_paper_p100": value / PAPER_P100_UPDATES_PER_NS,
                       "note": "paper: ~15 ps per spin update on one P100, bipartite random "
                               "regular graph z = 4, T = 0.8 T_c"},
           "config": {"workload": f"vb_packed_rrbg_z4_N{n}_lanes64_R2_T{T_08_TC:.5f}",
                      "colour_classes": 2},
           "roofline": {"bound": "hbm", "achieved": bytes_sweep / (ms * 1e-3) / 1e9,
                        "peak": peak, "unit": "GB/s",
                        "frac": bytes_sweep / (ms * 1e-3) / 1e9 / peak}}
    run.close()
    print(json.dumps(out), flush=True)
    return 0


def run_vb_windows(args):
    """The headline VB workload with the main text's estimator (not the headline line): every
    sweep from tau = 2^4 on is measured (C against every snapshot taken, q, E) and added into
    geometric windows of ratio 2^(1/4), on top of the point schedule; one step = one sweep of
    each temperature instance.  Shows what the per-sweep measurement costs."""
    import torch

    import paper_1906_11195_gb300 as sg
    from paper_1906_11195_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    rp, col, jb = instance(0)
    tw, tm = sg_inputs.log_schedule(TW, T_MAX)
    bounds = sg_inputs.geometric_windows(16, args.warmup + args.steps + 1)
    runs = [sg.VBRun([dict(row_ptr=rp, col=col, jbits=jb, seed=1, temps=[T] * REPLICAS)],
                     n_lanes=LANES, n_replicas=REPLICAS, kernel=sg.SG_VB_PACKED, tw=tw, tm=tm,
                     windows=bounds) for T in TEMPS]
    stream = torch.cuda.current_stream()
    for r in runs:
        r.sweep(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sum(r.launches for r in runs)
    nvtx_push("timed_region")
    e0.record(stream)
    for r in runs:
        r.sweep(args.steps)
    e1.record(stream)
    nvtx_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    launches = sum(r.launches for r in runs) - l0
    for r in runs:
        r.synchronize()
        r.close()
    updates = len(TEMPS) * N_VERTS * LANES * REPLICAS
    print(json.dumps({"metric": "spin updates/ns", "unit": "spin updates/ns",
                      "value": updates / (ms * 1e6), "ms_per_step": ms, "steps": args.steps,
                      "warmup": args.warmup, "gpu_launches": launches,
                      "config": {"workload": WORKLOAD + "_windowed",
                                 "windows": f"{len(bounds) - 1} geometric windows, ratio 2^(1/4), "
                                            f"from tau = 16, every sweep measured"}}), flush=True)
    return 0


def run_aging(args):
    """The paper's analysis chain at small scale (not a throughput line): bipartite random
    regular graphs of degree 4 at T = 0.8 T_c, N = 2^12 .. 2^18 (2^21 vertices per size in one
    batch, 64 coupling sets x 2 replicas per graph), t_w = 4, C(t_w + t, t_w) averaged over
    geometric windows of ratio 2^(1/4) up to t_w + t = --aging-tmax; then the extrapolation to
    infinite size (quadratic in N^(-2/3)) per window and the inverse Frechet and M = 1..3
    polynomial fits of C_inf(t) on the last window of 8 octaves."""
    import math

    import torch

    import paper_1906_11195_gb300 as sg
    from paper_1906_11195_gb300 import _build, analysis
    _build.build()
    torch.cuda.set_device(0)
    tw0 = 4
    bounds = sg_inputs.geometric_windows(8, args.aging_tmax)
    sizes = [1 << k for k in (12, 14, 16, 18)]
    curves = []
    t0 = time.perf_counter()
    for n in sizes:
        ng = max(1, (1 << 21) // n)
        graphs = []
        for i in range(ng):
            sd = (n << 8) + i
            rp, col, eid = sg_inputs.random_regular_graph(n, 4, sd, bipartite=True)
            jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, sd)
            graphs.append(dict(row_ptr=rp, col=col, jbits=jb, seed=sd, temps=[T_08_TC] * REPLICAS))
        run = sg.VBRun(graphs, n_lanes=LANES, n_replicas=REPLICAS, kernel=sg.SG_VB_PACKED,
                       tw=[tw0], tm=[], windows=bounds)
        run.sweep(int(bounds[-1]))
        run.synchronize()
        C, _, _, cnt = run.windows()
        run.close()
        avg, t_mean = analysis.window_averages(bounds, C[:, :, :, 0, :].sum(axis=(0, 1, 2)),
                                               cnt[0] * ng * LANES * REPLICAS)
        curves.append(avg / n)
        log(f"N = {n}: {ng} graphs, {time.perf_counter() - t0:.1f} s")
    curves = np.array(curves)  # [size][window]
    ok = ~np.isnan(curves).any(axis=0)
    c_inf, coef, _ = analysis.finite_size_extrapolation(np.array(sizes), curves[:, ok],
                                                        nu=2.0 / 3.0, order=2)
    t = t_mean[ok] - tw0
    keep = t >= 1
    t, ci = t[keep], c_inf[keep]
    n_last = int(math.floor(math.log2(t.max())))
    win = (t >= 2.0 ** (n_last - 8)) & (t <= 2.0 ** n_last)
    fits = {}
    if win.sum() >= 4 and np.all(ci[win] > 0):
        a, b, g, r = analysis.frechet_fit(t[win], ci[win])
        fits["frechet"] = {"A": a, "B": b, "gamma": g, "ssr": r}
        for M in (1, 2, 3):
            a, b, g, r = analysis.polynomial_fit(t[win], ci[win], M)
            fits[f"poly_M{M}"] = {"A": a, "B": b, "gamma": g, "ssr": r}
    out = {"workload": "aging_rrbg_z4_T0.8Tc_tw4", "T": T_08_TC, "sizes": sizes,
           "t": t.round(2).tolist(), "C_by_size": curves[:, ok][:, keep].round(6).tolist(),
           "C_inf": ci.round(6).tolist(), "leading_coef_N^-2/3": coef[0][keep].round(4).tolist(),
           "fit_window": [float(2.0 ** (n_last - 8)), float(2.0 ** n_last)], "fits": fits}
    print(json.dumps(out), flush=True)
    return 0


def run_e6(args):
    """The paper's bipartite vs non-bipartite comparison (not a throughput line): C(t_w + t, t_w)
    at t_w = 4 on random regular graphs of degree 4, bipartite and plain, T = 0.8 T_c, for
    N = 2^14 (32 graphs per ensemble) and N = 2^22 (2 graphs), 64 coupling sets x 2 replicas per
    graph, t = 2^0 .. 2^k with 4 + 2^k <= --e6-tmax; prints both mean curves, their standard
    errors (from per-graph means) and the z-scores of the differences.  A third ensemble, the
    bipartite graphs under a random vertex labelling (same graphs, several colour classes),
    separates the effect of the graph from that of the update order."""
    import math

    import torch

    import paper_1906_11195_gb300 as sg
    from paper_1906_11195_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    out = {"workload": "e6_bipartite_vs_plain_rrg_z4_tw4", "T": T_08_TC, "sizes": {}}
    for n, ng in ((1 << 14, 32), (1 << 22, 2)):
        kmax = int(math.log2(max(1, args.e6_tmax - 4)))
        tm = np.array([4 + 2 ** k for k in range(kmax + 1)], dtype=np.int64)
        res = {}
        for kind in ("bipartite", "plain", "bipartite_relabelled"):
            bip = kind != "plain"
            graphs = []
            for i in range(ng):
                sd = 7000 + i + 100 * bip + n
                rp, col, eid = sg_inputs.random_regular_graph(n, 4, sd, bipartite=bip)
                if kind == "bipartite_relabelled":
                    # the same bipartite graph under a random vertex labelling: greedy colouring
                    # then gives several classes, so only the update order differs
                    rng = np.random.default_rng(sd)
                    perm = rng.permutation(n)
                    src = np.repeat(np.arange(n), np.diff(rp))
                    keep = src < col
                    rp, col, e2 = sg_inputs.csr_from_edges(n, perm[src[keep]], perm[col[keep]])
                    eid = e2
                jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, sd)
                graphs.append(dict(row_ptr=rp, col=col, jbits=jb, seed=sd,
                                   temps=[T_08_TC] * REPLICAS))
            run = sg.VBRun(graphs, n_lanes=LANES, n_replicas=REPLICAS, kernel=sg.SG_VB_PACKED,
                           tw=[4], tm=tm)
            run.sweep(int(tm[-1]))
            run.synchronize()
            C, _, _ = run.results()
            run.close()
            pg = C[:, :, :, 0, :].astype(np.float64).mean(axis=(1, 2)) / n
            se = pg.std(axis=0, ddof=1) / math.sqrt(ng) if ng > 1 else np.zeros(pg.shape[1])
            res[kind] = (pg.mean(axis=0), se)
        entry = {"graphs_per_ensemble": ng, "t": (tm - 4).tolist()}
        for kind, (m, e) in res.items():
            entry["C_" + kind] = m.round(6).tolist()
            entry["se_" + kind] = e.round(6).tolist()
        for a, b in (("bipartite", "plain"), ("bipartite_relabelled", "plain")):
            (m1, e1), (m2, e2) = res[a], res[b]
            z = np.abs(m1 - m2) / np.maximum(np.sqrt(e1 ** 2 + e2 ** 2), 1e-12)
            entry[f"z_{a}_vs_{b}"] = z.round(2).tolist()
        out["sizes"][str(n)] = entry
    print(json.dumps(out), flush=True)
    return 0


def run_sk(args):
    """The SK workload on its own (the default run's sk key), plus every other block size on
    fresh handles (B never changes the trajectory) and the plain kernel; --sk-replicas and
    --sk-block vary the replicas sharing J and the block of the extra comparison."""
    import torch

    import paper_1906_11195_gb300 as sg
    dev, stream = _single_gpu()
    out = measure_sk(args, dev, stream, args.steps, args.warmup, cpu=not args.skip_cpu)
    J = sg_inputs.sk_couplings(SK_N, 3)
    R = args.sk_replicas
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    others = {}
    for b in (64, 128, 256, 512):
        run = sg.SKRun(J, [SK_T] * R, 1, kernel=sg.SG_SK_BLOCKED, block=b)
        run.sweep(args.warmup)
        torch.cuda.synchronize()
        e0.record(stream)
        run.sweep(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1) / args.steps
        run.close()
        others[f"B{b}_R{R}"] = {"value": SK_N * R / (bms * 1e6), "ms_per_step": bms}
    out["other_blocks"] = others
    if not args.skip_plain:
        pr = sg.SKRun(J, [SK_T] * SK_R, 1, kernel=sg.SG_SK_PLAIN)
        pr.sweep(1)
        torch.cuda.synchronize()
        e0.record(stream)
        pr.sweep(2)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / 2
        pr.close()
        out["plain_kernel"] = {"value": SK_N * SK_R / (pms * 1e6), "ms_per_sweep": pms}
    print(json.dumps(out), flush=True)
    return 0


def run_sk_batch(args):
    """The batched uneven SK workload on its own (the default run's sk_batch key)."""
    dev, stream = _single_gpu()
    out = measure_sk_batch(args, dev, stream, args.steps, args.warmup, cpu=not args.skip_cpu)
    print(json.dumps(out), flush=True)
    return 0


def run_gpu(args):
    import torch

    import paper_1906_11195_gb300 as sg
    from paper_1906_11195_gb300 import _build

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        _build.build()
    if ws > 1:
        dist.barrier()
    _build.build()

    rp, col, jb = instance(rank)
    tw, tm = sg_inputs.log_schedule(TW, T_MAX)
    graphs = [dict(row_ptr=rp, col=col, jbits=jb, seed=1 + rank, temps=[T] * REPLICAS) for T in TEMPS]
    stream = torch.cuda.current_stream(dev)

    runs = [sg.VBRun([g], n_lanes=LANES, n_replicas=REPLICAS, kernel=sg.SG_VB_PACKED, tw=tw, tm=tm,
                     device=dev, stream=stream) for g in graphs]
    for r in runs:
        r.sweep(args.warmup)
    torch.cuda.synchronize()
    launches0 = sum(r.launches for r in runs)

    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nvtx_push("timed_region")  # lets a profiler capture exactly the timed launches
    ev0.record(stream)
    for r in runs:
        r.sweep(args.steps)
    ev1.record(stream)
    nvtx_pop()
    sampler.enqueued()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    launches = sum(r.launches for r in runs) - launches0
    for r in runs:
        r.synchronize()
    ms = max_over_ranks(ms, dev)
    updates_per_step = len(TEMPS) * N_VERTS * LANES * REPLICAS
    value = job_value(updates_per_step, args.steps, ws, ms)
    for r in runs:
        r.close()

    # roofline of the colour kernel: a handle with no measurement schedule times pure sweeps
    kr = max(20, min(args.steps, 200))
    rl = sg.VBRun([graphs[0]], n_lanes=LANES, n_replicas=REPLICAS, kernel=sg.SG_VB_PACKED,
                  device=dev, stream=stream)
    rl.sweep(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rl.sweep(kr)
    e1.record(stream)
    torch.cuda.synchronize()
    sweep_ms = e0.elapsed_time(e1) / kr
    rl.close()
    bytes_sweep = algorithmic_bytes_per_sweep(N_VERTS, int(rp[-1]), REPLICAS)
    peak, peak_kind = peaks()
    # achieved: the colour kernel's algorithmic bytes of every sweep in the timed region over the
    # whole timed region (the few snapshot/measurement launches in it count against the kernel,
    # so this is a lower bound); achieved_isolated: the same over sweeps timed alone
    sweep_ms_timed = ms / (args.steps * len(TEMPS))
    achieved = bytes_sweep / (sweep_ms_timed * 1e-3) / 1e9
    traffic = recorded_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                "kernel": "k_vb_packed_colour<2>, one unit = one sweep (all colour classes)",
                "algorithmic_bytes_per_sweep": bytes_sweep, "ms_per_sweep": sweep_ms_timed,
                "achieved_isolated": bytes_sweep / (sweep_ms * 1e-3) / 1e9,
                "ms_per_sweep_isolated": sweep_ms,
                "frac_kernel": bytes_sweep / (sweep_ms * 1e-3) / 1e9 / peak,
                "note": "frac: the colour kernel's algorithmic bytes over the whole timed step "
                        "(snapshot and measurement launches included); frac_kernel: the same "
                        "over sweeps timed alone (no schedule), the kernel's own fraction; "
                        "traffic: DRAM bytes per sweep from the committed ncu summary of this "
                        "kernel source (not measured in this run), null if the source changed"}

    # the plain one-thread-per-(vertex, lane, replica) kernel on the same graph, T = 1.0
    plain = None
    if not args.skip_plain:
        pr = sg.VBRun([graphs[0]], n_lanes=LANES, n_replicas=REPLICAS, kernel=sg.SG_VB_PLAIN,
                      device=dev, stream=stream)
        pr.sweep(1)
        torch.cuda.synchronize()
        kp = 3
        e0.record(stream)
        pr.sweep(kp)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / kp
        pr.close()
        plain = {"value": N_VERTS * LANES * REPLICAS / (pms * 1e6), "unit": "spin updates/ns",
                 "ms_per_sweep": pms, "sweeps": kp}

    # end to end through the public API: H2D of the prepared instances, K sweeps each, D2H of
    # the measurement counts; host-side instance preparation (validation, colouring, layout)
    # happens before the timed region
    handles, bufs = [], []
    for g in graphs:
        h = sg.sg_create_vb([g], LANES, REPLICAS, sg.SG_VB_PACKED, tw, tm)
        nb = sg.sg_workspace_bytes(h)
        handles.append((h, nb))
        bufs.append(torch.empty(nb, dtype=torch.uint8, device=dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    each = []
    for (h, nb), buf in zip(handles, bufs):
        ta = time.perf_counter()
        sg.sg_attach(h, buf.data_ptr(), nb, stream.cuda_stream)
        each.append((time.perf_counter() - ta) * 1e3)
    t1 = time.perf_counter()
    for h, _ in handles:
        sg.sg_sweep(h, args.warmup + args.steps)
    t2 = time.perf_counter()
    for h, _ in handles:
        C, q, E = sg.sg_read_results(h)
    e2e_s = time.perf_counter() - t0
    phases = {"attach_ms": (t1 - t0) * 1e3, "attach_ms_each": each, "sweep_calls_ms": (t2 - t1) * 1e3,
              "read_ms": (time.perf_counter() - t2) * 1e3}
    h2d = d2h = 0
    for h, _ in handles:
        a, b = sg.sg_transfer_bytes(h)
        h2d += a
        d2h += b
        sg.sg_destroy(h)
    e2e_steps = args.warmup + args.steps
    e2e = {"value": ws * updates_per_step * e2e_steps / (e2e_s * 1e9), "unit": "spin updates/ns",
           "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps,
           "phases": phases,
           "note": "H2D of both instances' images at attach + sweeps + D2H of all counts (bytes "
                   "counted by the library), spread over the steps; phases: host time of the "
                   "attach calls (copies, autotuner), the sweep calls (queued) and the reads "
                   "(which wait for the sweeps)"}

    # the other configurations of the metric, each with its own value, roofline, e2e, clocks
    # and CPU baseline (one GPU only; each is a separate JSON object inside the line)
    extra = {}
    if ws == 1 and not args.skip_extra:
        es = max(1, min(args.steps, args.extra_steps))
        ew = max(3, min(args.warmup, 8))
        for key, fn in (("sk", measure_sk), ("vb_batch", measure_vb_batch),
                        ("sk_batch", measure_sk_batch)):
            t0 = time.perf_counter()
            try:
                extra[key] = fn(args, dev, stream, es, ew, cpu=not args.skip_cpu)
            except Exception as e:  # a failing extra leaves the headline line intact
                extra[key] = {"error": f"{type(e).__name__}: {e}"}
            log(f"{key}: {time.perf_counter() - t0:.1f} s")
            torch.cuda.empty_cache()

    cpu = cpu_all = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        cpu = cpu_baseline_sample(rp, col, jb)
        try:
            cpu_all = cpu_baseline_all_cores()
        except Exception as e:  # the single-core figure stands on its own
            log(f"all-core CPU sample skipped: {e}")

    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": "spin updates/ns", "value": value, "unit": "spin updates/ns", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N_VERTS, "mean_degree": MEAN_DEGREE, "lanes": LANES,
                   "replicas": REPLICAS, "temps": list(TEMPS), "step": "1 sweep of each temperature",
                   "schedule": f"tw=2^4..2^15, log-spaced measurements to 2^16 ({len(tm)} times)",
                   "l2": "inputs larger than L2: 201 MB of graph streamed per sweep (spins, 64 MiB, "
                         "are meant to stay in L2)",
                   "parallelism": f"replicas only, {ws} independent instance(s)"},
        "roofline": roofline,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "plain_kernel": plain,
        "speedup_vs_plain": (value / ws) / plain["value"] if plain else None,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=T_MAX - 3,
                    help="timed sweeps (default: with 3 warm-up sweeps the run ends at tau = 2^16, "
                         "covering the whole measurement schedule)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-extra", action="store_true",
                    help="headline VB line only (no sk, vb_batch, sk_batch keys)")
    ap.add_argument("--extra-steps", type=int, default=256,
                    help="timed steps of each extra configuration (at most --steps)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run only the single-instance sweep case used for ncu captures")
    ap.add_argument("--profile-log2n", type=int, default=22, help="log2 N of the profile case")
    ap.add_argument("--profile-replicas", type=int, default=2, choices=[2, 4],
                    help="replicas of the profile case (4: two per temperature)")
    ap.add_argument("--workload", default="vb",
                    choices=["vb", "sk", "vb_batch", "sk_batch", "rrbg", "e6", "vb_windows",
                             "aging"],
                    help="vb: the headline bit-packed Viana-Bray line; sk: the SK blocked line; "
                         "vb_batch: the uneven batch of Viana-Bray graphs; sk_batch: the uneven "
                         "batch of SK samples; rrbg: the paper's bipartite regular graph; e6: "
                         "bipartite vs plain regular graphs, C(t_w + t, t_w) at t_w = 4; "
                         "vb_windows: the headline workload measured every sweep into "
                         "geometric windows; aging: the paper's extrapolations at small scale")
    ap.add_argument("--aging-tmax", type=int, default=2 ** 14, help="last time of the aging run")
    ap.add_argument("--e6-tmax", type=int, default=4 + 2 ** 16, help="last time of the e6 curves")
    ap.add_argument("--batch", type=int, default=512, help="graphs in the vb_batch workload")
    ap.add_argument("--sk-block", type=int, default=SK_B)
    ap.add_argument("--sk-replicas", type=int, default=SK_R,
                    help="replicas sharing J in the sk workload (a multiple of 128 above 128)")
    args = ap.parse_args()
    if args.warmup < 3:
        log("warning: fewer than 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args)
    if args.workload == "sk":
        return run_sk(args)
    if args.workload == "vb_batch":
        return run_vb_batch(args)
    if args.workload == "sk_batch":
        return run_sk_batch(args)
    if args.workload == "rrbg":
        return run_rrbg(args)
    if args.workload == "e6":
        return run_e6(args)
    if args.workload == "vb_windows":
        return run_vb_windows(args)
    if args.workload == "aging":
        return run_aging(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
