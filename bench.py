#!/usr/bin/env python3
"""Benchmark of the SPH cell-pair offload pipeline on one B300.

Workload: the Gresho-vortex shaped set of 256^3 particles (jittered lattice,
55/73/64/64 particles per cell, the paper's "Gresho256", Sec. 3.4).  One
step = density -> ghost -> gradient -> force over the whole set.  Metric:
pair interactions per second of the whole step, plus pack+unpack GB/s per
loop, for a split (sAoS) store against AoS (Sec. 3.1).  The headline is the
list pipeline on the pack-force-type layout; the paper's per-task cycle
(pipeline "plain") is timed beside it.

Output: the study sections (measured peaks, link rate, per-layout stage
times, list-build work counts, host-staged breakdown, precision, ...) as
one JSON line each, {"section": name, "data": ...}; then, as the LAST line,
the compact headline (metric, value, e2e, roofline, cpu_baseline, clocks,
per-loop rates), kept under a few KB.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-interactions/s and pack+unpack GB/s per loop, sAoS vs AoS, 1 B300"
UNIT = "pair-interactions/s"
BENCH_LAYOUT = "pack_force_type"
BUNDLE_SLOTS = 1 << 25
N_SIDE = 256
ALL_LAYOUTS = ("aos", "aos_random", "pack_grad", "pack_force", "pack_shared",
               "pack_grad_type", "pack_force_type", "pack_shared_type", "soa",
               "pack_force_repl", "fused")
LOOP_NAMES = ("density", "gradient", "force")
# algorithmic bytes: view read + written per slot (pack), result read per slot
# plus output fields read + written per particle (unpack)
VIEW_IN = (44, 52, 69)
VIEW_OUT = (32, 8, 24)
# FP32 operations (FADD, FMUL = 1, FFMA = 2) of the implemented formulas.
# List build, fixed-point plans (the Gresho plan): per staged candidate the
# three fixed-point separations (1 FMUL each), H_j + delta, two squares and
# the box distance (6 FADD, r^2 with 1 FMUL + 2 FFMA) = 17; per prefiltered
# (particle, candidate) pair 3 FADD + r^2 = 8; per exact test the same 8.
# Two-float plans: per staged candidate the shift (TwoSum, 3 x 8 FADD) and
# the rest as above = 38; per exact test the two-float separation
# (3 x 3 FADD) + r^2 = 14.
FLOPS_STAGE = {True: 17, False: 38}
FLOPS_CANDIDATE = 8
FLOPS_EXACT = {True: 8, False: 14}
FLOPS_PAIR = (73, 52, 113)
# derived FP32 CUDA-core peak (148 SMs x 128 lanes x 2 flop x 2.032 GHz):
# only a fallback when the measured one is missing
FP32_PEAK_DERIVED = 148 * 128 * 2 * 2.032e9 / 1e12
# the headline line is kept below this size (the driver keeps the tail of
# stdout; study sections go on earlier lines)
HEADLINE_MAX_BYTES = 2800
# DRAM bytes per slot of the interaction kernels from an ncu capture of a
# smaller case (traffic grows with the slots a launch processes), valid only
# for the kernel source with this digest (else reported as null)
NCU_TRAFFIC = {
    # DRAM bytes per unit (slot for the per-task kernels, particle otherwise)
    # from one ncu capture, valid while the kernel's source file is unchanged
    ("plain", "kernel", 2): {"bytes_per_unit": 92.1, "src": "e4b699e728bdf76e",
                             "file": "physics_kernels.cuh"},
    # the symmetric list build's two passes together (128^3 capture:
    # 1197.0 MB + 829.5 MB DRAM over 2,097,152 particles)
    ("list", "list", 0): {"bytes_per_unit": 966.3, "src": "59da718261f29ae0",
                          "file": "list_kernels.cuh"},
}
# bytes per particle of the batched pack records (nf float4 + index lanes)
# (the density pack also writes the list loop's two fixed-point lanes; the
# list pipeline's packs write compact records, for density on plans with the
# fixed-point list build only those two lanes, as at Gresho256)
BATCH_REC = (5 * 16 + 4, 4 * 16 + 4, 5 * 16 + 9)
LIST_REC = (2 * 16 + 4, 3 * 16 + 4, 4 * 16 + 9)
CSRC = os.path.join(ROOT, "paper_2606_23891_b300", "csrc")


def src_digest(name: str = "physics_kernels.cuh") -> str:
    with open(os.path.join(CSRC, name), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ---------------------------------------------------------------- clocks --
_SAMPLER = r"""
import ctypes as C, sys, time
ids, period = sys.argv[1:-1], float(sys.argv[-1])
nv = C.CDLL("libnvidia-ml.so.1")
if nv.nvmlInit_v2() != 0:
    sys.exit("nvmlInit failed")
h = C.c_void_p()
ok = False
for i in ids:
    if i.startswith("pci:"):
        ok = nv.nvmlDeviceGetHandleByPciBusId_v2(i[4:].encode(), C.byref(h)) == 0
    else:
        ok = nv.nvmlDeviceGetHandleByUUID(i.encode(), C.byref(h)) == 0
    if ok:
        break
if not ok:
    sys.exit("no NVML handle for %s" % ids)
SM = 1
mx = C.c_uint()
nv.nvmlDeviceGetMaxClockInfo(h, SM, C.byref(mx))
reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
    nv.nvmlDeviceGetCurrentClocksThrottleReasons
print("max %d" % mx.value, flush=True)
clk, rs = C.c_uint(), C.c_ulonglong()
while True:
    t = time.time()
    nv.nvmlDeviceGetClockInfo(h, SM, C.byref(clk))
    reasons(h, C.byref(rs))
    print("%.6f %d %d" % (t, clk.value, rs.value), flush=True)
    time.sleep(period)
"""


class ClockSampler:
    """SM clock and throttle reasons of one GPU, sampled every `period`
    seconds by a separate process (NVML, read-only queries) that runs for the
    whole benchmark; start() and stop() mark a timed region on the wall clock
    and stop() summarises the samples taken inside it."""
    REASONS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40,
               "sw_thermal_slowdown": 0x20, "sw_power_cap": 0x4}
    _shared = {}

    def __init__(self, index: int, period: float = 0.01):
        self.index = index
        key = (index, period)
        if key not in ClockSampler._shared:
            ClockSampler._shared[key] = self._launch(index, period)
        self.proc, self.samples, self.info = ClockSampler._shared[key]
        self.t0 = None

    @staticmethod
    def _ids(index):
        """NVML names of the CUDA device: its UUID (with and without the GPU-
        prefix) and its PCI bus id (CUDA and NVML number devices differently)."""
        import torch
        pr = torch.cuda.get_device_properties(index)
        ids = []
        u = getattr(pr, "uuid", None)
        if u is not None:
            u = str(u)
            ids += [u if u.startswith("GPU-") else "GPU-" + u, u]
        try:
            ids.append("pci:%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id))
        except AttributeError:
            pass
        return ids

    @staticmethod
    def _launch(index, period):
        import threading
        samples, info = [], {"max": 0.0, "source": "nvml"}
        ids = ClockSampler._ids(index)
        try:
            proc = subprocess.Popen([sys.executable, "-c", _SAMPLER] + ids + [str(period)],
                                    stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
        except OSError:
            return None, samples, info

        def reader(p, parse):
            for line in p.stdout:
                try:
                    parse(line)
                except (ValueError, IndexError):
                    continue

        def parse_nvml(line):
            parts = line.split()
            if parts[0] == "max":
                info["max"] = float(parts[1])
            else:
                samples.append((float(parts[0]), float(parts[1]), int(parts[2])))
        threading.Thread(target=reader, args=(proc, parse_nvml), daemon=True).start()
        t_end = time.time() + 20.0            # sampling before the first region
        while not samples and time.time() < t_end and proc.poll() is None:
            time.sleep(0.05)
        if samples:
            return proc, samples, info
        # NVML unavailable: nvidia-smi at its shortest loop, with timestamps
        info["error"] = (proc.stderr.read() if proc.poll() is not None else "no sample")[-200:]
        info["source"] = "nvidia-smi"
        try:
            smi = subprocess.Popen(
                ["nvidia-smi", "-i", ids[0] if ids else str(index),
                 "--query-gpu=timestamp,clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return None, samples, info
        import datetime

        def parse_smi(line):
            parts = [q.strip() for q in line.split(",")]
            t = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            info["max"] = max(info["max"], float(parts[2]))
            samples.append((t, float(parts[1]), int(parts[3], 16)))
        threading.Thread(target=reader, args=(smi, parse_smi), daemon=True).start()
        t_end = time.time() + 20.0
        while not samples and time.time() < t_end and smi.poll() is None:
            time.sleep(0.05)
        return smi, samples, info

    def start(self):
        self.t0 = time.time()

    def stop(self):
        if self.proc is None or self.t0 is None:
            return None
        t1 = time.time()
        time.sleep(0.05)                      # samples of the region's end are read
        inside = [(m, r) for t, m, r in list(self.samples) if self.t0 <= t <= t1]
        if not inside:
            return None
        reasons = sorted(nm for nm, bit in self.REASONS.items()
                         if any(r & bit for _, r in inside))
        return {"sm_mhz": statistics.median(m for m, _ in inside),
                "sm_max_mhz": self.info["max"], "reasons": reasons, "samples": len(inside),
                "region_s": round(t1 - self.t0, 3), "source": self.info["source"]}

    @classmethod
    def close_all(cls):
        for proc, _, _ in cls._shared.values():
            if proc is not None:
                proc.terminate()
        cls._shared.clear()


# ------------------------------------------------------ measured peaks --
def _event_ms(fn, reps: int = 1) -> float:
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_peaks(index: int, target_ms: float = 150.0) -> dict:
    """FP32 FMA, FP64 FMA and FP64 add peaks of this GPU from the library's
    microbenchmark (sph_peak_run), each the best of 3 launches of about
    target_ms, with the SM clock sampled during them."""
    import torch
    from paper_2606_23891_b300 import sph
    sink = torch.zeros(256, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    clocks = ClockSampler(index)
    clocks.start()
    out = {}
    for kind, name in ((sph.PEAK_FP32_FMA, "fp32_tflops"), (sph.PEAK_FP64_FMA, "fp64_fma_tflops"),
                       (sph.PEAK_FP64_ADD, "fp64_add_tflops")):
        iters = 16
        ms = _event_ms(lambda: sph.sph_peak_run(kind, iters, sink.data_ptr(), st))
        iters = max(16, int(iters * target_ms / max(ms, 1e-3)))
        best = 0.0
        for _ in range(3):
            fl = [0.0]

            def run():
                fl[0] = sph.sph_peak_run(kind, iters, sink.data_ptr(), st)
            ms = _event_ms(run)
            best = max(best, fl[0] / (ms * 1e-3) / 1e12)
        out[name] = best
    out["clocks"] = clocks.stop()
    out["how"] = ("sph_peak_run: 8 x 256 threads per SM, 8 independent chains of FMA "
                  "(2 flops) or add; best of 3 launches of ~%d ms, CUDA events" % target_ms)
    return out


def measure_link(nbytes: int = 1 << 30, reps: int = 5) -> dict:
    """Pinned host <-> device copy rate: one cudaMemcpyAsync of nbytes per
    direction (torch copy_ of a page-locked tensor), best of reps."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h2d = min(_event_ms(lambda: d.copy_(h, non_blocking=True)) for _ in range(reps))
    d2h = min(_event_ms(lambda: h.copy_(d, non_blocking=True)) for _ in range(reps))
    del h, d
    torch.cuda.empty_cache()
    return {"h2d_GBps": nbytes / (h2d * 1e-3) / 1e9, "d2h_GBps": nbytes / (d2h * 1e-3) / 1e9,
            "bytes": nbytes, "how": "one pinned cudaMemcpyAsync per direction, best of %d" % reps}


def list_build_counts(off) -> dict:
    """The list build's work per step, counted by its measurement variant
    (sph_batch_list_count) over every bundle: candidates staged, pairs past
    the warp-box cull (each prefiltered), prefilter hits, exact tests and
    entries written."""
    import torch
    from paper_2606_23891_b300 import sph
    cnt = torch.zeros(5, dtype=torch.int64, device=off.device)
    for b in range(off.binfo["nbundles"]):
        sph.sph_batch_pack_list(off.store, off.bplan, 0, b, off.bbuf_in.data_ptr(), off.params,
                                off.stream)
        sph.sph_batch_list_count(off.store, off.bplan, b, off.bbuf_in.data_ptr(),
                                 off.blist.data_ptr(), off.blist_bytes, off.params,
                                 cnt.data_ptr(), off.stream)
    sph.sph_sync(off.stream)
    keys = ("staged", "culled_in", "prefilter_hits", "exact_tests", "entries")
    return dict(zip(keys, (int(v) for v in cnt.cpu().tolist())))


def sig(x, n: int = 4):
    """x rounded to n significant digits (compact JSON)."""
    if isinstance(x, float) and x != 0.0 and np.isfinite(x):
        return float("%.*g" % (n, x))
    return x


def compact_line(line: dict, limit: int = HEADLINE_MAX_BYTES) -> str:
    """The headline JSON, dropping the optional keys (last first) until it
    fits in `limit` bytes."""
    optional = ["staged", "peaks", "per_loop"]
    out = json.dumps(line, separators=(",", ":"))
    while len(out) > limit and optional:
        line.pop(optional.pop(), None)
        out = json.dumps(line, separators=(",", ":"))
    return out


# ---------------------------------------------------------- distributed --
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier_max(value: float, ws: int) -> float:
    """The maximum of `value` over the ranks (every rank gets it)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ms_max: float, ws: int) -> float:
    """Whole-job throughput: the units all ranks processed (each rank a full
    replica) over the slowest rank's time."""
    return units_per_rank * ws / (ms_max * 1e-3)


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------- CPU arms --
def oracle_sample(f, nsample: int, seed: int):
    """Time the oracle's full chain on `nsample` particles of the workload."""
    import oracle
    rng = np.random.Generator(np.random.PCG64(seed))
    sel = np.sort(rng.choice(f["x"].shape[0], nsample, replace=False)).astype(np.int64)
    t = time.perf_counter()
    out = oracle.chain(f, oracle.params(), sel)
    dt = time.perf_counter() - t
    pairs = sum(out["pairs"].values())
    oracle_sample.last = (sel, out)
    return pairs, dt


def precision_study(off, f, sel, ref, steps, mixed_step, x64_step=None):
    """Per-loop error of the mixed-precision path (FP32, two-float and
    fixed-point separations), of the FP64-separation arm (FP32 fields, FP64
    pair separations; list pipeline) and of the all-FP64 batched path against
    the oracle on the sampled particles, with the step times of the last two."""
    import torch
    import oracle
    from oracle import compare
    sc = oracle.dh_scales(f, oracle.params(), sel)
    res = {"sample": int(len(sel))}
    mixed_step()
    got = off.export()
    e = compare.errors({k: v[sel] for k, v in got.items()}, ref, sc)
    res["mixed"] = {"per_loop": compare.per_loop(e), "fields": e,
                    "rho_dh": compare.relative_distribution(got["rho_dh"][sel], ref["rho_dh"],
                                                            sc[0])}
    if x64_step is not None:
        x64_step()                                    # warm-up (allocates the lanes)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            x64_step()
        e1.record()
        torch.cuda.synchronize()
        res["fp64_separation_ms_per_step"] = e0.elapsed_time(e1) / steps
        got = off.export()
        e = compare.errors({k: v[sel] for k, v in got.items()}, ref, sc)
        res["fp64_separation"] = {"per_loop": compare.per_loop(e), "fields": e}
        off.x64 = None
        torch.cuda.empty_cache()
    off.fp64_step()                                   # warm-up (allocates buffers)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        off.fp64_step()
    e1.record()
    torch.cuda.synchronize()
    res["fp64_ms_per_step"] = e0.elapsed_time(e1) / steps
    got = off.export()
    e = compare.errors({k: v[sel] for k, v in got.items()}, ref, sc)
    res["fp64"] = {"per_loop": compare.per_loop(e), "fields": e}
    res["metrics"] = ("relative error for rho, wcount, f_gradh, pressure, soundspeed, "
                      "v_sig; err / (sum of the terms' magnitudes) for the h-derivatives; "
                      "max err / rms for div v, curl v, laplace u, a, du/dt, dh/dt; "
                      "absolute error for the Balsara switch")
    off.f64_in = off.f64_out = None
    torch.cuda.empty_cache()
    return res


def cpu_cores() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    from paper_2606_23891_b300 import ics
    f = ics.gresho(n_side=args.n_side)
    for _ in range(args.warmup):
        oracle_sample(f, 1, 1)
    tot_pairs, tot_t = 0, 0.0
    for k in range(args.steps):
        p, t = oracle_sample(f, args.ref_sample, 100 + k)
        tot_pairs += p
        tot_t += t
    value = tot_pairs / tot_t
    sample = ("%d steps x %d particles of the %d^3 Gresho set; each particle's full "
              "density->ghost->gradient->force chain by brute-force O(N) scans "
              "(neighbour densities included)" % (args.steps, args.ref_sample, args.n_side))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "gresho256", "particles": int(f["x"].shape[0])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- GPU arm --
def candidates(off) -> int:
    ci, cj, sh, cs, bs = off.task_list()
    cnt = np.diff(cs).astype(np.int64)
    ni = cnt[ci]
    nj = np.where(cj >= 0, cnt[np.maximum(cj, 0)], 0)
    return int(np.where(cj >= 0, 2 * ni * nj, ni * (ni - 1)).sum())


class StepTimer:
    """Run one step with CUDA events around every stage on the launch stream.
    pipeline "plain": per-task bundles (pack -> kernel -> unpack per bundle);
    "batched": cell-dedup bundles (one persistent launch per bundle)."""

    def __init__(self, off, pipeline: str = "plain"):
        import torch
        self.torch = torch
        self.off = off
        self.pipeline = pipeline
        self.recs = []
        self.launches = 0

    def ev(self):
        e = self.torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    def step(self, record: bool):
        """The stages of one step.  The batched and list pipelines write each
        particle's result in their unpack (no init pass; the density unpack
        applies the ghost); the list pipeline builds each bundle's lists from
        the density loop's pack."""
        from paper_2606_23891_b300 import sph
        off = self.off
        lists = self.pipeline == "list"
        batched = self.pipeline in ("batched", "list")
        nb = off.binfo["nbundles"] if batched else off.nbundles()
        st = off.stream
        if lists and getattr(off, "blist", None) is None:
            off.list_build()            # sizes the list pool (first step only)
        for loop in range(3):
            if not batched:
                sph.sph_init(off.store, loop, off.params, st)
                self.launches += 1
            for b in range(nb):
                e0 = self.ev() if record else None
                if lists:
                    sph.sph_batch_pack_list(off.store, off.bplan, loop, b,
                                            off.bbuf_in.data_ptr(), off.params, st)
                elif batched:
                    sph.sph_batch_pack(off.store, off.bplan, loop, b, off.bbuf_in.data_ptr(),
                                       off.params, st)
                else:
                    off.pack(loop, b)
                e1 = self.ev() if record else None
                e1b = e1
                if lists and loop == 0:
                    sph.sph_batch_list_build_bundle(off.store, off.bplan, b,
                                                    off.bbuf_in.data_ptr(), off.blist.data_ptr(),
                                                    off.blist_bytes, off.params, st)
                    self.launches += 1
                    e1b = self.ev() if record else None
                if lists:
                    sph.sph_batch_list_interact(off.bplan, loop, b, off.bbuf_in.data_ptr(),
                                                off.bbuf_out.data_ptr(), off.blist.data_ptr(),
                                                off.blist_bytes, off.params, st)
                elif batched:
                    sph.sph_batch_interact(off.bplan, loop, b, off.bbuf_in.data_ptr(),
                                           off.bbuf_out.data_ptr(), off.params, st)
                else:
                    off.interact(loop, b)
                e2 = self.ev() if record else None
                if batched:     # the density unpack applies the ghost too
                    sph.sph_batch_unpack_write(off.store, off.bplan, loop, b,
                                               off.bbuf_out.data_ptr(), off.bbuf_in.data_ptr(),
                                               off.params, int(loop == 0), st)
                else:
                    off.unpack(loop, b)
                e3 = self.ev() if record else None
                self.launches += 3
                if record:
                    self.recs.append((loop, e0, e1, e1b, e2, e3))
            if loop == 0 and not batched:
                sph.sph_ghost(off.store, 0, off.params, st)
                self.launches += 1

    def stage_ms(self):
        out = {(s, l): 0.0 for s in ("pack", "kernel", "unpack") for l in range(3)}
        cnt = {l: 0 for l in range(3)}
        for loop, e0, e1, e1b, e2, e3 in self.recs:
            out[("pack", loop)] += e0.elapsed_time(e1)
            if e1b is not e1:   # the bundle's list build, from the density pack
                out[("list", 0)] = out.get(("list", 0), 0.0) + e1.elapsed_time(e1b)
            out[("kernel", loop)] += e1b.elapsed_time(e2)
            out[("unpack", loop)] += e2.elapsed_time(e3)
            cnt[loop] += 1
        return out, cnt


def run_layout(off, steps, warmup, ws, clocks=None, pipeline="plain"):
    import torch
    timer = StepTimer(off, pipeline)
    for _ in range(warmup):
        timer.step(record=False)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    timer.launches = 0
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(steps):
        timer.step(record=True)
    end.record()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    cl = clocks.stop() if clocks else None
    total_ms = start.elapsed_time(end)
    return total_ms, timer, cl


def run_e2e(off, f, steps, warmup, pipeline="plain"):
    """The same step from pinned host inputs to pinned host results, every
    byte through the library: per step sph_hostio_begin (H2D of the step's
    inputs, import), the step's library calls, sph_hostio_end (export, D2H
    of its results); the copies of neighbouring steps overlap the current
    step's kernels on the library's two copy streams."""
    import torch
    from paper_2606_23891_b300 import sph
    from paper_2606_23891_b300.pipeline import STEP_INPUTS, STEP_RESULTS, StreamingSteps
    timer = StepTimer(off, pipeline)
    ss = StreamingSteps(off, lambda: timer.step(record=False), STEP_INPUTS, STEP_RESULTS)
    pin_in, pin_out = ss.pinned_in(), ss.pinned_out()
    for name, t in pin_in.items():
        t.numpy()[...] = np.asarray(f[name], t.numpy().dtype).reshape(t.shape)
    h2d, d2h = ss.bytes_per_step()
    for _ in range(warmup):
        ss.step(pin_in, pin_out)
    ss.drain()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record()
    ss.s_in.wait_event(start)              # the first copy starts inside the region
    for _ in range(steps):
        ss.step(pin_in, pin_out)
    ss.drain()
    end.record()
    torch.cuda.synchronize()
    sph.sph_sync(off.stream)
    ss.close()
    return start.elapsed_time(end) / steps, h2d, d2h


def run_host_staged(f, layouts, steps, bundle_slots, link, fission_bundles=2):
    """The paper's own setting: store in pinned host memory, host pack and
    unpack (all host cores), double-buffered H2D / kernel / D2H on two
    streams.  Per layout: wall-clock per step, and a step with every stage
    timed (sph_offload_loop_host_stats), giving the offload-time breakdown
    of the paper's Fig. 1 and the copies' rate against the measured link."""
    import torch
    from paper_2606_23891_b300 import sph
    from paper_2606_23891_b300.pipeline import HostOffload
    out = {}
    host = None
    for lname in layouts:
        if host is not None:
            host.close()
            del host
        host = HostOffload(f, layout=lname, bundle_max_slots=bundle_slots)
        host.step()                                   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            host.step()
        torch.cuda.synchronize()
        step_s = (time.perf_counter() - t0) / steps
        stats = host.step_stats()
        tot = {k: sum(st[k] for st in stats) for k in stats[0]}
        stage_ms = {"host_pack": 1e3 * tot["host_pack_s"], "h2d": tot["h2d_ms"],
                    "kernel": tot["kernel_ms"], "d2h": tot["d2h_ms"],
                    "host_unpack": 1e3 * tot["host_unpack_s"]}
        serial = sum(stage_ms.values())
        wall = 1e3 * tot["wall_s"]
        h2d_gbps = tot["h2d_bytes"] / (tot["h2d_ms"] * 1e-3) / 1e9
        d2h_gbps = tot["d2h_bytes"] / (tot["d2h_ms"] * 1e-3) / 1e9
        loops = {}
        for l, st in enumerate(stats):
            loops[LOOP_NAMES[l]] = {
                "wall_ms": 1e3 * st["wall_s"], "host_pack_ms": 1e3 * st["host_pack_s"],
                "h2d_ms": st["h2d_ms"], "kernel_ms": st["kernel_ms"], "d2h_ms": st["d2h_ms"],
                "host_unpack_ms": 1e3 * st["host_unpack_s"],
                "host_wait_ms": 1e3 * st["host_wait_s"], "h2d_bytes": st["h2d_bytes"],
                "d2h_bytes": st["d2h_bytes"], "bundles": st["bundles"]}
        # loop-fission variants (Sec. 3.3, Fig. 4) on the first bundles of
        # each loop; the isolated unpacks fold result buffers into the store,
        # which is not read again
        fission = {}
        nb = host.info["nbundles"]
        nbf = min(nb, fission_bundles)
        for name, fv in sph.FISSION.items():
            tp = tu = 0.0
            for l in range(3):
                for b in range(nbf):
                    t1 = time.perf_counter()
                    sph.sph_pack_host_fission(host.store, host.tasks, l, b,
                                              host.host_in[0][0].ctypes.data, fv)
                    t2 = time.perf_counter()
                    sph.sph_unpack_host_fission(host.store, host.tasks, l, b,
                                                host.host_out[0][0].ctypes.data, fv)
                    tu += time.perf_counter() - t2
                    tp += t2 - t1
            fission[name] = {"pack_ms": 1e3 * tp, "unpack_ms": 1e3 * tu}
        base_ms = fission["none"]["pack_ms"] + fission["none"]["unpack_ms"]
        for v in fission.values():
            v["relative_to_none"] = (v["pack_ms"] + v["unpack_ms"]) / base_ms
        out[lname] = {
            "ms_per_step": 1e3 * step_s, "timed_step_ms": wall, "stage_ms": stage_ms,
            "stage_share": {k: v / serial for k, v in stage_ms.items()},
            "pack_unpack_share": (stage_ms["host_pack"] + stage_ms["host_unpack"]) / serial,
            "launch_share": (stage_ms["h2d"] + stage_ms["kernel"] + stage_ms["d2h"]) / serial,
            "overlap": 1.0 - wall / serial,
            "h2d_GBps": h2d_gbps, "d2h_GBps": d2h_gbps,
            "h2d_link_frac": h2d_gbps / link["h2d_GBps"],
            "d2h_link_frac": d2h_gbps / link["d2h_GBps"],
            "h2d_bytes_per_step": tot["h2d_bytes"], "d2h_bytes_per_step": tot["d2h_bytes"],
            "loops": loops,
            "loop_fission": {"bundles_per_loop": nbf, "variants": fission}}
    if host is not None:
        host.close()
    return {"bundle_max_slots": bundle_slots, "threads": cpu_cores(), "link": link,
            "h2d_link": "pinned host memory, cudaMemcpyAsync on 2 streams",
            "stage_times": "host stages on the host clock; copies and kernels with CUDA "
                           "events, summed over bundles (they overlap)",
            "layouts": out}


def layout_phase_study(per_layout: dict, convert_ms: dict, base: str) -> dict:
    """Kernel-dependent layouts (one layout per algorithmic phase): per
    pipeline, the fixed layout with the least pack + unpack time over the
    three loops against the best layout of each loop plus the conversions
    between consecutive phases (density -> gradient -> force -> density).  A
    conversion X -> Y is estimated from the measured X -> base and
    base -> Y conversions (each a full store pass) as their mean."""
    out = {"convert_ms": {k: {"to_base": v[0], "from_base": v[1]} for k, v in convert_ms.items()}}

    def conv(a, b):
        if a == b:
            return 0.0
        ta = 0.0 if a == base else convert_ms[a][0]
        tb = 0.0 if b == base else convert_ms[b][1]
        return 0.5 * (ta + tb) if a != base and b != base else ta + tb
    pipelines = next(iter(per_layout.values())).keys()
    for pl in pipelines:
        pu = {l: [v[pl]["loops"][n]["pack_ms"] + v[pl]["loops"][n]["unpack_ms"]
                  for n in LOOP_NAMES] for l, v in per_layout.items()}
        fixed = min(pu, key=lambda l: sum(pu[l]))
        best = [min(pu, key=lambda l: pu[l][k]) for k in range(3)]
        phase = sum(pu[best[k]][k] for k in range(3)) + sum(
            conv(best[k], best[(k + 1) % 3]) for k in range(3))
        out[pl] = {"fixed_best": {"layout": fixed, "pack_unpack_ms": sum(pu[fixed])},
                   "best_per_loop": {LOOP_NAMES[k]: {"layout": best[k], "pack_unpack_ms": pu[best[k]][k]}
                                     for k in range(3)},
                   "phase_dependent_ms": phase}
    return out


def plan_candidates(f, leaf_max: int = 128) -> dict:
    """Candidate pairs per loop under the uniform grid of the per-task cycle
    (cell pairs: 2 n_i n_j, self n_i (n_i - 1)) and under the octree-leaf
    plan (each leaf's particles x those of its neighbour entries); host-only
    plan builds, nothing runs on the GPU."""
    from paper_2606_23891_b300 import sph
    x = np.ascontiguousarray(f["x"], np.float64)
    h = np.ascontiguousarray(f["h"], np.float32)
    n = x.shape[0]
    out = {}
    try:
        perm = np.empty(n, np.int64)
        t = sph.sph_tasks_build(n, x.ctypes.data, h.ctypes.data, sph.grid_params(),
                                perm.ctypes.data)
        info = sph.sph_tasks_info(t)
        ncell = info["ncell_x"] * info["ncell_y"] * info["ncell_z"]
        ci = np.empty(info["ntasks"], np.int32)
        cj = np.empty(info["ntasks"], np.int32)
        cs = np.empty(ncell + 1, np.int64)
        sph.sph_tasks_get(t, ci.ctypes.data, cj.ctypes.data, 0, cs.ctypes.data, 0)
        sph.sph_tasks_destroy(t)
        cnt = np.diff(cs).astype(np.float64)
        ni, nj = cnt[ci], np.where(cj >= 0, cnt[np.maximum(cj, 0)], 0.0)
        out["grid"] = {"ncell": [info["ncell_" + a] for a in "xyz"],
                       "max_cell": info["max_cell"],
                       "candidates": float(np.where(cj >= 0, 2 * ni * nj, ni * (ni - 1)).sum())}
    except sph.SphError as e:
        out["grid"] = {"unsupported": str(e)}
    def occupancy(c):
        return {"min": int(c.min()), "max": int(c.max()), "mean": float(c.mean()),
                "median": float(np.median(c))}

    perm, ls, nbs, nb = sph.sph_tree_plan(x, h, leaf_max=leaf_max)
    cnt = np.diff(ls).astype(np.float64)
    owner = np.repeat(np.arange(cnt.size), np.diff(nbs))
    out["tree"] = {"leaf_max": leaf_max, "leaves": int(cnt.size), "occupancy": occupancy(cnt),
                   "candidates": float((cnt[owner] * cnt[nb >> 6]).sum())}
    # the cell tree's own rule (split while half the edge covers the largest
    # support inside): occupancy to set beside the paper's cosmological trace
    perm, ls, nbs, nb = sph.sph_tree_plan(x, h, leaf_max=8, rule=1)
    cnt = np.diff(ls).astype(np.float64)
    owner = np.repeat(np.arange(cnt.size), np.diff(nbs))
    out["octree_rule"] = {"leaves": int(cnt.size), "occupancy": occupancy(cnt),
                          "candidates": float((cnt[owner] * cnt[nb >> 6]).sum())}
    return out


def run_cosmology(args, ws, fp32_peak):
    """Clustered set (lognormal, sigma(ln rho) = 2): the batched pipeline on the
    octree-leaf plan, autotuned, per layout, with CUDA-graph replay."""
    import torch
    from paper_2606_23891_b300 import ics, sph
    from paper_2606_23891_b300.autotune import GraphStep, tune_tree
    from paper_2606_23891_b300.pipeline import Offload
    t = time.perf_counter()
    f = ics.lognormal(n_side=args.cosmo_n_side)
    t_gen = time.perf_counter() - t
    n = f["x"].shape[0]
    H = 1.825742 * f["h"].astype(np.float64)
    t = time.perf_counter()
    off = Offload(f, layout=args.cosmo_layouts[0], plan="tree", leaf_max=128)
    t_build = time.perf_counter() - t
    pairs = [off.count_pairs(l) for l in range(3)]
    tuning = tune_tree(off, reps=1, step="list") if args.autotune else None
    grid = plan_candidates(f, off.leaf_max)
    res = {"workload": "lognormal%d: %d^3 particles from a lognormal density field, "
                       "sigma(ln rho) = 2, octree-leaf plan" % (args.cosmo_n_side, args.cosmo_n_side),
           "particles": n, "support_range": [float(H.min()), float(H.max())],
           "generate_s": t_gen, "plan_build_s": t_build, "candidates_per_loop": grid,
           "pairs": dict(zip(LOOP_NAMES, pairs)),
           "pairs_per_particle": [p / n for p in pairs], "autotune": tuning,
           "plan": {k: off.binfo[k] for k in ("cells", "max_cell", "nbrs", "threads",
                                              "nbundles", "max_slots")},
           "layouts": {}}
    res["plan"]["leaf_max"] = off.leaf_max
    head = None
    for lname in args.cosmo_layouts:
        o = off if lname == args.cosmo_layouts[0] else Offload(f, layout=lname, share=off)
        res["layouts"][lname] = {}
        for pipeline in (["list", "batched"] if o is off else ["list"]):
            total_ms, timer, _ = run_layout(o, args.steps, args.warmup, ws, None, pipeline)
            total_ms = barrier_max(total_ms, ws)
            st, cnt = timer.stage_ms()
            ms = total_ms / args.steps
            loops = {}
            for l in range(3):
                pk, kr, up = (st[(s_, l)] / args.steps for s_ in ("pack", "kernel", "unpack"))
                loops[LOOP_NAMES[l]] = {"pack_ms": pk, "kernel_ms": kr, "unpack_ms": up,
                                        "kernel_useful_fp32_TFLOPs":
                                            pairs[l] * FLOPS_PAIR[l] / (kr * 1e-3) / 1e12}
            r = {"ms_per_step": ms, "pair_interactions_per_s": job_rate(sum(pairs), ms, ws),
                 "loops": loops}
            if ("list", 0) in st:
                r["list_build_ms"] = st[("list", 0)] / args.steps
            res["layouts"][lname][pipeline] = r
            if head is None:
                head = (st, cnt, ms, timer.launches)
        if o is not off:
            o.close()
            del o
            torch.cuda.empty_cache()
    gs = GraphStep(off, step=off.list_step)
    for _ in range(args.warmup):
        gs.replay()
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record()
    for _ in range(args.steps):
        gs.replay()
    g1.record()
    torch.cuda.synchronize()
    gms = barrier_max(g0.elapsed_time(g1), ws) / args.steps
    res["cuda_graph"] = {"ms_per_step": gms,
                         "pair_interactions_per_s": job_rate(sum(pairs), gms, ws)}
    del gs
    st, cnt, ms, launches = head
    top = max(st, key=lambda k: st[k])
    stage, loop = top
    ncand = grid["tree"]["candidates"]
    if stage == "list":
        nbl = off.binfo["nbundles"]
        dur = st[top] / (args.steps * nbl)
        c = list_build_counts(off)
        fixed = sph.sph_batch_list_fixed(off.bplan)
        ach = (c["staged"] * FLOPS_STAGE[fixed] + c["culled_in"] * FLOPS_CANDIDATE +
               c["exact_tests"] * FLOPS_EXACT[fixed]) / nbl / (dur * 1e-3) / 1e12
        res["list_build_counts"] = c
        name = "neighbour-list build (tree plan)"
    else:
        dur = st[top] / cnt[loop]
        ach = pairs[loop] * FLOPS_PAIR[loop] / cnt[loop] * args.steps / (dur * 1e-3) / 1e12
        name = "list interaction/%s (tree plan)" % LOOP_NAMES[loop]
    res["roofline"] = {"kernel": name, "bound": "alu", "achieved": ach,
                       "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak}
    res["gpu_launches_per_step"] = launches / args.steps
    off.close()
    del off
    torch.cuda.empty_cache()
    return res


def run_precision_clustered(args):
    """The precision study on the clustered recipe (lognormal, tree plan):
    per-loop error of the mixed-precision list step and of the all-FP64
    step against the oracle on sampled particles, and both step times."""
    import torch
    from paper_2606_23891_b300 import ics
    from paper_2606_23891_b300.pipeline import Offload
    f = ics.lognormal(n_side=args.precision_clustered_n_side)
    off = Offload(f, layout="pack_force_type", plan="tree", leaf_max=128)
    for _ in range(2):
        off.list_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    off.list_step()
    e1.record()
    torch.cuda.synchronize()
    mixed_ms = e0.elapsed_time(e1)
    t = time.perf_counter()
    oracle_sample(f, args.precision_clustered_sample, 17)
    sel, ref = oracle_sample.last
    t = time.perf_counter() - t
    res = precision_study(off, f, sel, ref, 1, off.list_step)
    res.update({"workload": "lognormal%d (tree plan)" % args.precision_clustered_n_side,
                "mixed_ms_per_step": mixed_ms, "oracle_s": t})
    # the same set kept in pinned host memory and staged through the plan's
    # bundles (host pack, H2D, batched kernel, D2H, host unpack, 2 streams)
    if args.host_steps > 0:
        from paper_2606_23891_b300.pipeline import HostOffload
        off.batch_step()
        want = off.export()
        nleaf = off.binfo["cells"]
        off.close()
        del off
        torch.cuda.empty_cache()
        host = HostOffload(f, layout="pack_force_type", plan="tree", leaf_max=128,
                           max_target_cells=max(1, nleaf // 8))
        host.batch_step()                              # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.host_steps):
            host.batch_step()
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0) / args.host_steps
        got = host.export()
        err = max(float(np.max(np.abs(got[k].astype(np.float64) - want[k])) /
                        max(float(np.sqrt(np.mean(want[k].astype(np.float64) ** 2))), 1e-30))
                  for k in ("rho", "a", "u_dt"))
        res["host_staged"] = {"ms_per_step": ms, "bundles": host.info["nbundles"],
                              "threads": cpu_cores(),
                              "max_rms_rel_diff_vs_device": err}
        host.close()
    else:
        off.close()
        del off
    torch.cuda.empty_cache()
    return res


def run_adjoint(args, ws):
    """Differentiation workload: gradient of sum |a|^2 + sum (du/dt)^2 with
    respect to x, m, u through density -> ghost -> force, on the Gresho
    recipe at each requested size (forward list step and adjoint timed), with
    a central-difference check of the gradient on a few particles of the
    smallest size (FP64 C oracle on local subsets)."""
    import torch
    import oracle
    from paper_2606_23891_b300 import ics
    from paper_2606_23891_b300.pipeline import Offload
    res = {"loss": "sum_i |a_i|^2 + sum_i (du_i/dt)^2", "wrt": ["x", "m", "u"], "sizes": {}}
    for ns in args.adjoint_n_side:
        f = ics.gresho(n_side=ns)
        off = Offload(f, layout="pack_force_type")
        off.batch(threads=args.batch_threads)
        dev = off.device
        off.list_step()
        ab = off.export_device(("a", "u_dt"))
        abar, ebar = 2 * ab["a"], 2 * ab["u_dt"]

        def timed(fn, reps):
            fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps
        fwd = timed(off.list_step, args.steps)
        bwd = timed(lambda: off.adjoint(abar, ebar), args.steps)
        pairs = off.count_pairs(2)
        r = {"particles": off.n, "forward_ms": fwd, "adjoint_ms": bwd,
             "force_pairs": pairs,
             "adjoint_pair_visits_per_s": 2 * pairs / (bwd * 1e-3)}
        if ns == min(args.adjoint_n_side) and args.adjoint_fd > 0:
            gx, gm, gu = (t.cpu().numpy() for t in off.adjoint(abar, ebar))
            r["fd_check"] = adjoint_fd(f, gx, gm, gu, args.adjoint_fd)
        res["sizes"]["gresho%d" % ns] = r
        off.close()
        del off
        torch.cuda.empty_cache()
    return res


def adjoint_fd(f, gx, gm, gu, npick: int) -> dict:
    """Central differences of the FP64 oracle loss for npick particles: each
    on the subset within 4.5 H_max of the particle, the loss restricted to
    the outputs within 2 H_max of it (all that move with it)."""
    import oracle
    n = f["x"].shape[0]
    Hmax = oracle.KERNEL_GAMMA * float(f["h"].max())
    rng = np.random.Generator(np.random.PCG64(4))

    def local(g, k, sub):
        s = {key: np.ascontiguousarray(v[sub]) for key, v in g.items()}
        kk = int(np.nonzero(sub == k)[0][0])
        d = s["x"] - s["x"][kk]
        d -= np.rint(d)
        near = np.nonzero(np.sqrt((d * d).sum(axis=1)) < 2.05 * Hmax)[0].astype(np.int64)
        out = oracle.chain(s, oracle.params(), near)
        return float(((out["a"] ** 2).sum(axis=1) + out["u_dt"] ** 2).sum())
    got = {"x": [], "m": [], "u": []}
    ref = {"x": [], "m": [], "u": []}
    t = time.perf_counter()
    for k in rng.choice(n, npick, replace=False):
        d = f["x"] - f["x"][k]
        d -= np.rint(d)
        sub = np.nonzero(np.sqrt((d * d).sum(axis=1)) < 4.5 * Hmax)[0]
        for c in range(3):
            g = {key: v.copy() for key, v in f.items()}
            eps = 1e-6 * Hmax
            g["x"][k, c] += eps
            lp = local(g, k, sub)
            g["x"][k, c] -= 2 * eps
            lm = local(g, k, sub)
            ref["x"].append((lp - lm) / (2 * eps))
            got["x"].append(gx[k, c])
        for name, key, gv in (("mass", "m", gm), ("u", "u", gu)):
            g = {kk: v.copy() for kk, v in f.items()}
            v0 = np.float32(f[name][k])
            up, dn = np.float32(v0 * np.float32(1.001)), np.float32(v0 * np.float32(0.999))
            g[name][k] = up
            lp = local(g, k, sub)
            g[name][k] = dn
            lm = local(g, k, sub)
            ref[key].append((lp - lm) / (float(up) - float(dn)))
            got[key].append(gv[k])
    err = {key: float(np.linalg.norm(np.subtract(got[key], ref[key])) / np.linalg.norm(ref[key]))
           for key in got}
    return {"particles": npick, "rel_err_norm": err, "seconds": time.perf_counter() - t}


def run_ours(args, ws, rank, local):
    import torch
    from paper_2606_23891_b300 import ics, sph
    from paper_2606_23891_b300.pipeline import Offload

    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    ClockSampler(local)                       # the sampling process, started early
    mpeaks = measured_peaks()
    peaks = measure_peaks(local) if args.peaks else {}
    link = measure_link() if args.host_steps > 0 else None
    f = ics.gresho(n_side=args.n_side)
    t_build = time.perf_counter()
    base = Offload(f, layout=args.layouts[0], bundle_max_slots=args.bundle_slots)
    t_build = time.perf_counter() - t_build
    pairs = [base.count_pairs(l) for l in range(3)]
    ncand = candidates(base)
    slots = base.info["slots"]
    n = base.n
    per_layout = {}
    head = None
    tuning = None
    if ("batched" in args.pipelines or "list" in args.pipelines) and args.autotune:
        from paper_2606_23891_b300.autotune import tune
        tuning = tune(base, reps=1, step="list" if args.head_pipeline == "list" else "batched")
        args.batch_threads = tuning["threads"]
    else:
        base.batch(threads=args.batch_threads)
    bslots = base.binfo["max_slots"]

    def loop_stats(st, ms_step, pipeline):
        loops = {}
        for l in range(3):
            pk, kr, up = (st[(s_, l)] / args.steps for s_ in ("pack", "kernel", "unpack"))
            if pipeline == "plain":
                pack_b = slots * 2 * VIEW_IN[l]
                unpack_b = slots * VIEW_OUT[l] + n * 2 * VIEW_OUT[l]
            else:  # each particle packed once; one result per particle
                rec = LIST_REC if pipeline == "list" else BATCH_REC
                pack_b = bslots * (VIEW_IN[l] + rec[l])
                unpack_b = n * VIEW_OUT[l] + n * 2 * VIEW_OUT[l]
            loops[LOOP_NAMES[l]] = {
                "pack_ms": pk, "kernel_ms": kr, "unpack_ms": up,
                "pack_unpack_GBps": (pack_b + unpack_b) / ((pk + up) * 1e-3) / 1e9,
                "pack_GBps": pack_b / (pk * 1e-3) / 1e9,
                "unpack_GBps": unpack_b / (up * 1e-3) / 1e9,
                "pair_interactions_per_s": pairs[l] / ((pk + kr + up) * 1e-3),
                "kernel_useful_fp32_TFLOPs": pairs[l] * FLOPS_PAIR[l] / (kr * 1e-3) / 1e12,
            }
        res = {"ms_per_step": ms_step,
               "pair_interactions_per_s": job_rate(sum(pairs), ms_step, ws), "loops": loops}
        if ("list", 0) in st:
            res["list_build_ms"] = st[("list", 0)] / args.steps
        return res

    convert_ms = {}

    def time_convert(dst, src, reps=3):
        sph.sph_store_convert(dst.store, src.store, dst.stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            sph.sph_store_convert(dst.store, src.store, dst.stream)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for lname in args.layouts:
        off = base if lname == args.layouts[0] else Offload(
            f, layout=lname, share=base)
        if off is not base:
            off.use_batch_of(base)
        per_layout[lname] = {}
        for pipeline in args.pipelines:
            is_head = lname == args.headline and pipeline == args.head_pipeline
            clocks = ClockSampler(local) if is_head else None
            total_ms, timer, cl = run_layout(off, args.steps, args.warmup, ws, clocks, pipeline)
            total_ms = barrier_max(total_ms, ws)
            st, cnt = timer.stage_ms()
            per_layout[lname][pipeline] = loop_stats(st, total_ms / args.steps, pipeline)
            if is_head:
                head = (off, total_ms, timer, cl, st, cnt)
        if off is not base:
            convert_ms[lname] = (time_convert(off, base), time_convert(base, off))
        if head is None or head[0] is not off:
            if off is not base:
                off.close()
                del off
                torch.cuda.empty_cache()
    off, total_ms, timer, cl, st, cnt = head
    ms_step = total_ms / args.steps
    kernel_dependent = layout_phase_study(per_layout, convert_ms, args.layouts[0]) \
        if convert_ms else None
    value = job_rate(sum(pairs), ms_step, ws)
    graph = None
    if args.head_pipeline in ("batched", "list"):
        # the same step recorded once into a CUDA graph and replayed
        from paper_2606_23891_b300.autotune import GraphStep
        gs = GraphStep(off, step=off.list_step if args.head_pipeline == "list" else None)
        for _ in range(args.warmup):
            gs.replay()
        gms = barrier_max(_event_ms(gs.replay, args.steps), ws)
        graph = {"ms_per_step": gms, "pair_interactions_per_s": job_rate(sum(pairs), gms, ws)}
        del gs
    # dominant kernel of the headline layout
    top = max(st, key=lambda k: st[k])
    stage, loop = top
    per_step = cnt[loop] / args.steps             # launches per step (bundles)
    dur = st[top] / cnt[loop]                     # ms per launch
    # the measured FP32 peak, at the median SM clock of the headline's timed
    # region (the FMA microbenchmark may run at a power-capped clock)
    fp32_peak, fp32_src = FP32_PEAK_DERIVED, "derived: 148 SMs x 128 FP32 lanes x 2 x 2.032 GHz"
    if peaks.get("fp32_tflops"):
        fp32_peak, fp32_src = peaks["fp32_tflops"], "measured (sph_peak_run FP32 FMA)"
        pc = peaks.get("clocks") or {}
        if pc.get("sm_mhz") and cl and cl.get("sm_mhz"):
            fp32_peak = peaks["fp32_tflops"] * cl["sm_mhz"] / pc["sm_mhz"]
            fp32_src = ("measured (sph_peak_run FP32 FMA, %.4g TFLOP/s at %.0f MHz), scaled to "
                        "the timed region's %.0f MHz" % (peaks["fp32_tflops"], pc["sm_mhz"],
                                                         cl["sm_mhz"]))
    build_counts = None
    if args.head_pipeline == "list":
        build_counts = list_build_counts(off)
    if stage == "list":
        # the neighbour-list build: its work counted by the measurement
        # variant (staged candidates, prefiltered pairs, exact tests) times
        # the FP32 operations of the implemented formulas
        fixed = sph.sph_batch_list_fixed(off.bplan)
        per_step = off.binfo["nbundles"]
        dur = st[top] / (args.steps * per_step)
        flops = (build_counts["staged"] * FLOPS_STAGE[fixed] +
                 build_counts["culled_in"] * FLOPS_CANDIDATE +
                 build_counts["exact_tests"] * FLOPS_EXACT[fixed]) / per_step
        achieved = flops / (dur * 1e-3) / 1e12
        tr = NCU_TRAFFIC.get(("list", "list", 0))
        traffic = (tr["bytes_per_unit"] * n / per_step
                   if tr and tr["src"] == src_digest(tr["file"]) else None)
        roof = {"kernel": "k_blist + k_blist_rev (neighbour-list build)", "bound": "alu",
                "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic, "peak_source": fp32_src,
                "ms": dur}
    elif stage == "kernel":
        flops = pairs[loop] * FLOPS_PAIR[loop] / per_step
        achieved = flops / (dur * 1e-3) / 1e12
        tr = NCU_TRAFFIC.get((args.head_pipeline, stage, loop))
        units = slots if args.head_pipeline == "plain" else n
        traffic = (tr["bytes_per_unit"] * units / per_step
                   if tr and tr["src"] == src_digest(tr["file"]) else None)
        roof = {"kernel": "%s interaction/%s" % (args.head_pipeline, LOOP_NAMES[loop]),
                "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic, "peak_source": fp32_src,
                "ms": dur}
    else:
        if args.head_pipeline == "plain":
            bpl = (slots * 2 * VIEW_IN[loop] if stage == "pack"
                   else slots * VIEW_OUT[loop] + n * 2 * VIEW_OUT[loop]) / per_step
        else:
            rec = LIST_REC if args.head_pipeline == "list" else BATCH_REC
            bpl = (bslots * (VIEW_IN[loop] + rec[loop]) if stage == "pack"
                   else n * 3 * VIEW_OUT[loop]) / per_step
        achieved = bpl / (dur * 1e-3) / 1e9
        peak = mpeaks.get("hbm_gbs", 6400.0)
        roof = {"kernel": "%s/%s" % (stage, LOOP_NAMES[loop]), "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_source": "measured" if mpeaks else "fallback", "ms": dur}
    head_loops = per_layout[args.headline][args.head_pipeline]["loops"]
    loop_fracs = {LOOP_NAMES[l]: head_loops[LOOP_NAMES[l]]["kernel_useful_fp32_TFLOPs"] / fp32_peak
                  for l in range(3)}
    e2e_ms, h2d, d2h = run_e2e(off, f, args.steps, 2, args.head_pipeline)
    e2e_ms = barrier_max(e2e_ms, ws)
    cpu = None
    if rank == 0 and ws == 1 and args.cpu_sample > 0:
        p, t = oracle_sample(f, args.cpu_sample, 7)
        cpu = {"value": p / t, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": "%d particles of gresho%d, full density-ghost-gradient-force chain "
                         "each, brute-force O(N) scans, %.1f s"
                         % (args.cpu_sample, args.n_side, t)}
    precision = None
    if cpu is not None and args.precision_steps > 0 and args.head_pipeline in ("batched", "list"):
        sel, ref = oracle_sample.last
        precision = precision_study(off, f, sel, ref, args.precision_steps,
                                    off.list_step if args.head_pipeline == "list"
                                    else off.batch_step,
                                    off.list_step_x64 if args.head_pipeline == "list" else None)
        precision["mixed_ms_per_step"] = ms_step
    cfg_vals = {"tasks": base.info["ntasks"], "bundles": base.info["nbundles"],
                "bbundles": base.binfo["nbundles"],
                "store_gb": off.nbytes / 1e9, "buf_gb": base.buf_in.numel() / 1e9}
    # the Gresho stores and buffers are not needed by the remaining sections
    off.close()
    base.close()
    del off, base
    torch.cuda.empty_cache()
    staged = None
    if args.host_steps > 0:
        staged = run_host_staged(f, args.host_layouts, args.host_steps, args.host_bundle_slots,
                                 link)
        for lname, v in staged["layouts"].items():
            v["pair_interactions_per_s"] = sum(pairs) / (v["ms_per_step"] * 1e-3)
    del f
    adj = run_adjoint(args, ws) if args.adjoint_n_side else None
    prec_cl = (run_precision_clustered(args)
               if args.precision_clustered_n_side > 0 and rank == 0 and ws == 1 else None)
    cosmo = run_cosmology(args, ws, fp32_peak) if args.cosmo_n_side > 0 else None
    sections = {
        "config_detail": {
            "batch_threads": args.batch_threads, "batch_bundles": cfg_vals["bbundles"],
            "tasks": cfg_vals["tasks"], "bundles": cfg_vals["bundles"],
            "bundle_max_slots": args.bundle_slots, "slots_per_loop": slots,
            "cell_pair_candidates_per_loop": ncand, "pairs": dict(zip(LOOP_NAMES, pairs)),
            "task_build_s": t_build},
        "peaks": peaks, "link": link, "layouts": per_layout, "cuda_graph": graph,
        "autotune": tuning, "list_build_counts": build_counts, "roofline": roof,
        "loop_fp32_frac": loop_fracs, "host_staged": staged, "precision": precision,
        "precision_clustered": prec_cl, "kernel_dependent_layout": kernel_dependent,
        "cosmology": cosmo, "adjoint": adj,
    }
    if rank == 0:
        for name, body in sections.items():
            if body is not None:
                print(json.dumps({"section": name, "data": body}))
    per_loop = {"fields": ["pair-interactions/s", "pack+unpack GB/s"]}
    for lname, v in per_layout.items():
        for pl, r in v.items():
            per_loop["%s/%s" % (lname, pl)] = [
                [sig(r["loops"][nm]["pair_interactions_per_s"], 3),
                 sig(r["loops"][nm]["pack_unpack_GBps"], 4)] for nm in LOOP_NAMES]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "gresho256", "particles": n, "layout": args.headline,
                   "pipeline": args.head_pipeline,
                   "l2": "inputs larger than L2 (store %.2f GB)" % cfg_vals["store_gb"],
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "e2e": {"value": job_rate(sum(pairs), e2e_ms, ws), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": sig(e2e_ms),
                "api": "sph_hostio_begin/end around sph_batch_* calls, pinned host arrays"},
        "gpu_launches": timer.launches,
        "roofline": {k: sig(v) for k, v in roof.items()},
        "cpu_baseline": cpu,
        "clocks": cl,
        "per_loop": per_loop,
        "peaks": {"fp32_tflops": sig(peaks.get("fp32_tflops")),
                  "fp64_fma_tflops": sig(peaks.get("fp64_fma_tflops")),
                  "fp64_add_tflops": sig(peaks.get("fp64_add_tflops")),
                  "hbm_gbs": mpeaks.get("hbm_gbs")},
    }
    if link is not None:
        line["peaks"].update(h2d_gbs=sig(link["h2d_GBps"]), d2h_gbs=sig(link["d2h_GBps"]))
    if staged is not None:
        line["staged"] = {
            lname: {"ms": sig(v["ms_per_step"]),
                    "share": {k: sig(x, 3) for k, x in v["stage_share"].items()},
                    "h2d_frac": sig(v["h2d_link_frac"], 3),
                    "overlap": sig(v["overlap"], 3)}
            for lname, v in staged["layouts"].items()}
    ClockSampler.close_all()
    if rank == 0:
        print(compact_line(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--layouts", default="pack_force_type,aos",
                    help="store layouts to time ('all': the 11 layouts)")
    ap.add_argument("--headline", default=BENCH_LAYOUT)
    ap.add_argument("--bundle-slots", type=int, default=BUNDLE_SLOTS)
    ap.add_argument("--n-side", type=int, default=N_SIDE)
    ap.add_argument("--cpu-sample", type=int, default=16)
    ap.add_argument("--ref-sample", type=int, default=2)
    ap.add_argument("--cosmo-n-side", type=int, default=0,
                    help="clustered (lognormal) set on the tree plan; 0: skip")
    ap.add_argument("--cosmo-layouts", type=lambda s: s.split(","),
                    default=["pack_force_type", "aos"])
    ap.add_argument("--adjoint-n-side", type=lambda s: [int(v) for v in s.split(",") if v],
                    default=[], help="Gresho sizes of the adjoint timing ('' skips)")
    ap.add_argument("--adjoint-fd", type=int, default=8,
                    help="particles of the central-difference check of the adjoint")
    ap.add_argument("--precision-clustered-n-side", type=int, default=0,
                    help="lognormal set of the clustered precision study (0: skip)")
    ap.add_argument("--precision-clustered-sample", type=int, default=8)
    ap.add_argument("--precision-steps", type=int, default=2,
                    help="timed steps of the all-FP64 path (0: skip the precision study)")
    ap.add_argument("--pipelines", default="plain,list")
    ap.add_argument("--peaks", type=int, default=1, help="measure the FP32/FP64 peaks")
    ap.add_argument("--head-pipeline", default="list")
    ap.add_argument("--batch-threads", type=int, default=128)
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--host-steps", type=int, default=2)
    ap.add_argument("--host-layouts", default="aos,pack_force_type,soa")
    ap.add_argument("--host-bundle-slots", type=int, default=1 << 24)
    args = ap.parse_args(argv)
    args.layouts = list(ALL_LAYOUTS) if args.layouts == "all" else \
        [s for s in args.layouts.split(",") if s]
    args.host_layouts = [s for s in args.host_layouts.split(",") if s]
    args.pipelines = [s for s in args.pipelines.split(",") if s]
    if args.head_pipeline not in args.pipelines:
        args.pipelines.append(args.head_pipeline)
    if args.headline not in args.layouts:
        args.layouts.append(args.headline)
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
