"""Throughput benchmark: bulk CG-D detection + CG-P precoding on GB300.

Workload (one step): S slots of the 128-antenna, 16-user, 64-QAM uplink and
downlink, each slot 1200 subcarriers x 14 OFDM symbols with the channel
constant over the 14 symbols (one instance = one subcarrier, 14 right-hand
sides), i.i.d. CN(0,1) channels, SNR 10 dB, K = 3 CG iterations; by default
the matched filter, Gram and q = H v run on the tensor cores with hi+lo split
FP16 operands and FP32 accumulation, the CG recursion in FP32. A step is one
cg_detect over all S*1200 instances (matched filter, Gram, CG,
approximate SINR tracker, max-log LLRs) and one cg_precode over the same
channels (Gram, CG, q = H v). Inputs are drawn once, resident in HBM and
larger than L2.

Prints one JSON line (rank 0) on stdout with the headline figures, and the
full record of every side measurement on stderr ("detail: {...}").
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload instead.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

B, U, QAM, R, NSC = 128, 16, 6, 14, 1200
SNR_DB = 10.0
KITER = 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--slots", type=int, default=32, help="1200x14 slots per step")
    ap.add_argument("--B", type=int, default=B, help="antennas (profiling runs of other shapes)")
    ap.add_argument("--U", type=int, default=U)
    ap.add_argument("--qam", type=int, default=QAM, help="bits per QAM symbol")
    ap.add_argument("--K", type=int, default=KITER)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--precision", default="fp16x3", choices=list(PRECISIONS))
    ap.add_argument("--no-plain", action="store_true", help="skip timing the FP32 plain path")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 256x32 workload")
    ap.add_argument("--no-neumann", action="store_true", help="skip the Neumann comparator")
    ap.add_argument("--no-cgls", action="store_true", help="skip the CGLS comparator")
    ap.add_argument("--no-sweep", action="store_true", help="skip the K / U / A p sweep")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    return ap.parse_args()


PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2, "bf16x3": 3, "fp16x3": 4}
# arithmetic of each precision mode: tensor-core operands (x3 = hi+lo split,
# three products) with FP32 accumulation, the CG recursion and LLRs in FP32
DTYPES = {"fp32": "f32", "bf16": "bf16+f32", "fp16": "f16+f32", "bf16x3": "bf16x3+f32",
          "fp16x3": "f16x3+f32"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (read-only queries)
    every millisecond on a thread, so a timed region of a few milliseconds
    still gets samples under load."""
    # NVML clock-event reason bits (nvmlClocksEventReason*)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int):
        import ctypes
        import threading
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)):
            raise OSError("no NVML handle")
        self.get_reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.samples = []
        self.stop_flag = threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        ct = self.ct
        clk, rs = ct.c_uint(), ct.c_ulonglong()
        while not self.stop_flag.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(clk)) == 0 and \
                    self.get_reasons(self.h, ct.byref(rs)) == 0:
                self.samples.append((clk.value, rs.value))
            time.sleep(0.001)

    def start(self):
        self.thread.start()

    def stop(self) -> dict:
        self.stop_flag.set()
        self.thread.join(timeout=5)
        mx = self.ct.c_uint()
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, self.ct.byref(mx))
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": mx.value, "reasons": ["no samples"]}
        reasons = sorted({nm for _, r in self.samples for bit, nm in self.REASONS.items()
                          if r & bit})
        return {"sm_mhz": statistics.median(c for c, _ in self.samples),
                "sm_max_mhz": mx.value, "reasons": reasons, "samples": len(self.samples),
                "source": "nvml, 1 ms"}


def clock_sampler(index: int):
    """NVML sampler when the library loads, else nvidia-smi at 200 ms."""
    try:
        return NvmlClockSampler(index)
    except (OSError, AttributeError):
        return ClockSampler(index)


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------

def detect_bytes_per_instance(Bn, Un, Rn, q):
    """Algorithmic HBM bytes of one CG-D instance: H and Y read once; x_hat,
    mu, rho, LLRs and the status word written once."""
    return (Bn * Un + Rn * Bn) * 8 + Rn * Un * (8 + 4 + 4 + 4 * q) + 4


def precode_bytes_per_instance(Bn, Un, Rn):
    """Algorithmic HBM bytes of one CG-P instance: H and T read, q, ||q|| and
    the status word written."""
    return (Bn * Un + Rn * Un) * 8 + Rn * Bn * 8 + Rn * 4 + 4


def detect_kernel_name(precision: str, Un: int) -> str:
    """The detection kernel the C ABI dispatches to for this precision."""
    if precision == "fp32":
        return f"detect_kernel<{Un}>"
    el = "BF16" if precision.startswith("bf16") else "FP16"
    x3 = "true" if precision.endswith("x3") else "false"
    ut = 8 if Un <= 8 else 16 if Un <= 16 else 32
    return f"detect_warp_kernel<{ut}, {el}, {x3}>"


# Sources that define the timed tensor-core kernels (detect_warp_kernel,
# precode_warp_kernel) and their launcher: a profile's traffic counts only
# while these are unchanged.
KERNEL_SOURCES = ("cg_common.cuh", "cg_kernels.cuh", "cg_tc.cuh", "cg_warp.cuh", "warp.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1404_0424_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(name: str):
    """dram bytes per launch recorded in profiles/<name>.md, if the kernel
    sources have not changed since that capture."""
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    mh = re.search(r"kernel_source_hash:\s*(\w+)", txt)
    mt = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    if not mh or not mt or mh.group(1) != kernel_source_hash():
        return None
    return float(mt.group(1))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing (reported baseline and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_worker(job):
    """One host worker: FP64 oracle detect + precode on subcarriers of a seeded
    batch (B=128, 64-QAM, 14 symbols) until `seconds` have passed."""
    seed, Un, K, seconds = job
    import oracle
    from paper_1404_0424_gb300 import workload as wl
    d = wl.uplink(B, Un, QAM, n=16, R=R, snr_db=SNR_DB, seed=seed)
    t0 = time.perf_counter()
    inst = 0
    while True:
        i = inst % 16
        oracle.cg_detect(d["H"][i:i + 1], d["Y"][i:i + 1], d["N0"], 1.0, K, QAM)
        oracle.cg_precode(d["H"][i:i + 1], d["x"][i:i + 1], d["N0"], 1.0, K)
        inst += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return inst, time.perf_counter() - t0


def time_oracle(seconds: float, Un: int, K: int, cores: int = 0):
    """The FP64 oracle as it stands, one single-threaded worker per host core
    (processes started with spawn), each for `seconds`. Returns (solves/s,
    subcarriers done, wall seconds, workers)."""
    import multiprocessing as mp
    cores = cores or (os.cpu_count() or 1)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    jobs = [(7 + w, Un, K, seconds) for w in range(cores)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    inst = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return inst * 2 * R / busy, inst, wall, cores


# ---------------------------------------------------------------------------
# uneven batch (4096 problems) and serving (Poisson arrivals)
# ---------------------------------------------------------------------------

def run_batched(cabi, torch, dev, n_prob=4096, seed=2, reps=10):
    """4096 detection problems, (B, U) uniform over {64x8, 128x16, 128x32,
    256x32}, 16/64/256-QAM, 1-14 symbols, SNR uniform 5-25 dB, K = min(U/4, 8),
    one instance each; one plan (CG_PREC_AUTO), one graph launch per run."""
    import numpy as np
    from paper_1404_0424_gb300 import workload as wl
    rng = np.random.default_rng(seed)
    shapes = [(64, 8), (128, 16), (128, 32), (256, 32)]
    keep, descs, solves, nbytes = [], [], 0, 0
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    for _ in range(n_prob):
        B, U = shapes[rng.integers(4)]
        R = int(rng.integers(1, 15))
        q = int(rng.choice([4, 6, 8]))
        K = max(1, min(U // 4, 8))
        N0 = wl.snr_to_n0(float(rng.uniform(5, 25)), U)
        H = torch.randn((1, B, U), dtype=torch.complex64, device=dev, generator=g)
        Y = torch.randn((1, R, B), dtype=torch.complex64, device=dev, generator=g)
        o = [torch.empty((1, R, U), dtype=torch.complex64, device=dev),
             torch.empty((1, R, U), device=dev), torch.empty((1, R, U), device=dev),
             torch.empty((1, R, U, q), device=dev), torch.empty((1,), dtype=torch.int32,
                                                                device=dev)]
        keep.append((H, Y, o, B, U, R, K, q, N0))
        descs.append(cabi.desc(0, B, U, R, K, N0, H, Y, o[0], qam_bits=q, mu=o[1], rho=o[2],
                               aux=o[3], status=o[4]))
        solves += R
        nbytes += detect_bytes_per_instance(B, U, R, q)
    stream = torch.cuda.current_stream(dev)
    rc, plan, bad = cabi.cg_plan_create(descs, -1, stream)
    if rc:
        return {"error": cabi.cg_strerror(rc)}
    _, prec, nbins = cabi.cg_plan_info(plan)
    _, sched = cabi.cg_plan_schedule(plan)
    for _ in range(3):
        cabi.cg_plan_run(plan, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        cabi.cg_plan_run(plan, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    cabi.cg_plan_destroy(plan)
    # one FP32 launch per problem (the plain form of the same batch)
    e0.record(stream)
    for H, Y, o, B, U, R, K, q, N0 in keep:
        p = cabi.params(B, U, q, K, R, N0, precision=0)
        cabi.cg_detect(p, 1, H, Y, o[0], o[1], o[2], o[3], o[4], stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    ok = all(int(o[4][0]) == 0 for _, _, o, *_ in keep)
    peaks, kind = measured_peaks()
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"workload": "4096 uneven detection problems: (B,U) in {64x8,128x16,128x32,256x32}, "
                        "16/64/256-QAM, 1-14 symbols, SNR 5-25 dB, K=min(U/4,8)",
            "precision": {3: "bf16x3", 4: "fp16x3"}.get(prec, prec), "bins": nbins,
            "ms_per_run": round(ms, 4), "solves_per_s": round(solves / (ms / 1e3), 1),
            "gb_per_s": round(gbs, 1), "frac_hbm": round(gbs / peaks["hbm_gbs"], 4),
            "peak_kind": kind,
            "schedule": {"order": ("given", "longest_first")[sched["order"]],
                         "bins": ("sequential", "concurrent")[sched["concurrent"]],
                         "grid_pct": sched["grid_pct"],
                         "source": ("fixed", "timed", "cached")[sched["source"]],
                         "tuned_ms": round(sched["ms"], 4)},
            "plain_one_launch_per_problem": {"ms": round(ms_plain, 3),
                                             "solves_per_s": round(solves / (ms_plain / 1e3), 1)},
            "status_ok": ok}


def run_large(cabi, torch, dev, precision):
    """The 256-antenna, 32-user workload: 256-QAM, 16384 subcarriers x 14
    symbols, K = 8, detection and precoding timed apart with CUDA events."""
    from paper_1404_0424_gb300 import workload as wl
    Bl, Ul, ql, Rl, Kl, nl = 256, 32, 8, 14, 8, 16384
    up = wl.uplink_torch(Bl, Ul, ql, n=nl, R=Rl, snr_db=15.0, seed=77, device=dev)
    H, Y, N0 = up["H"], up["Y"], up["N0"]
    T = up["x"].contiguous()
    del up
    xhat = torch.empty((nl, Rl, Ul), dtype=torch.complex64, device=dev)
    mu = torch.empty((nl, Rl, Ul), dtype=torch.float32, device=dev)
    rho = torch.empty_like(mu)
    llr = torch.empty((nl, Rl, Ul, ql), dtype=torch.float32, device=dev)
    st = torch.empty((nl,), dtype=torch.int32, device=dev)
    q = torch.empty((nl, Rl, Bl), dtype=torch.complex64, device=dev)
    qn = torch.empty((nl, Rl), dtype=torch.float32, device=dev)
    stp = torch.empty((nl,), dtype=torch.int32, device=dev)
    p = cabi.params(Bl, Ul, ql, Kl, Rl, N0, precision=PRECISIONS[precision])
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        rc = cabi.cg_detect(p, nl, H, Y, xhat, mu, rho, llr, st, stream)
        rc |= cabi.cg_precode(p, nl, H, T, q, qn, 0, stp, stream)
        if rc:
            raise RuntimeError(cabi.cg_strerror(rc))
    torch.cuda.synchronize()
    ok = int(st.abs().sum()) == 0 and int(stp.abs().sum()) == 0
    reps = 5
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    for _ in range(reps):
        cabi.cg_detect(p, nl, H, Y, xhat, mu, rho, llr, st, stream)
    e[1].record(stream)
    for _ in range(reps):
        cabi.cg_precode(p, nl, H, T, q, qn, 0, stp, stream)
    e[2].record(stream)
    torch.cuda.synchronize()
    dms, pms = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
    # the exact tracker (Eq. 10) on the tensor cores against the FP32
    # CUDA-core kernel, the latter on a quarter of the batch (x4 reported)
    pe = cabi.params(Bl, Ul, ql, Kl, Rl, N0, sinr_mode=1, precision=PRECISIONS[precision])
    pf = cabi.params(Bl, Ul, ql, Kl, Rl, N0, sinr_mode=1, precision=0)
    nq = nl // 4
    cabi.cg_detect(pe, nl, H, Y, xhat, mu, rho, llr, st, stream)
    cabi.cg_detect(pf, nq, H, Y, xhat, mu, rho, llr, st, stream)
    e[0].record(stream)
    for _ in range(2):
        cabi.cg_detect(pe, nl, H, Y, xhat, mu, rho, llr, st, stream)
    e[1].record(stream)
    cabi.cg_detect(pf, nq, H, Y, xhat, mu, rho, llr, st, stream)
    e[2].record(stream)
    torch.cuda.synchronize()
    exact_ms, exact_fp32_ms = e[0].elapsed_time(e[1]) / 2, e[1].elapsed_time(e[2]) * 4
    peaks, kind = measured_peaks()
    db = detect_bytes_per_instance(Bl, Ul, Rl, ql) * nl
    pb = precode_bytes_per_instance(Bl, Ul, Rl) * nl
    out = {"workload": "B=256, U=32, 256-QAM, 16384 subcarriers x 14 symbols, K=8, SNR 15 dB, "
                       "i.i.d. channels", "precision": precision,
           "detect_ms": round(dms, 4), "precode_ms": round(pms, 4),
           "solves_per_s": round(2 * nl * Rl / ((dms + pms) / 1e3), 1),
           "detect_gbs": round(db / dms / 1e6, 1), "precode_gbs": round(pb / pms / 1e6, 1),
           "detect_frac_hbm": round(db / dms / 1e6 / peaks["hbm_gbs"], 4),
           "precode_frac_hbm": round(pb / pms / 1e6 / peaks["hbm_gbs"], 4),
           "peak_kind": kind, "status_ok": ok,
           "exact_tracker_detect_ms": round(exact_ms, 4),
           "exact_tracker_fp32_detect_ms": round(exact_fp32_ms, 3)}
    del H, Y, T, xhat, mu, rho, llr, st, q, qn, stp
    torch.cuda.empty_cache()
    return out


def run_serving(seconds):
    """Poisson arrivals at 20k requests/s (the load generator's mix), served
    (cg_serve_*, FP16X3) and plain (one FP32 launch per request); then the
    same mix at 500 and 5000 requests/s, where latency rather than
    throughput is what a serving path has to show."""
    from paper_1404_0424_gb300 import build as bld

    def one(mode, rate):
        cmd = [bld.LOADGEN, "--mode", mode, "--rate", str(rate), "--seconds", str(seconds),
               "--capacity", "64", "--precision", "4", "--seed", "1"]
        try:
            res = subprocess.run(cmd, capture_output=True, text=True, timeout=seconds + 120)
            line = res.stdout.strip().splitlines()[-1] if res.stdout.strip() else "{}"
            return json.loads(line)
        except Exception as exc:  # noqa: BLE001
            return {"error": repr(exc)}

    out = {mode: one(mode, 20000) for mode in ("served", "plain")}
    out["low_load"] = {}
    for rate in (500, 5000):
        for mode in ("served", "plain"):
            r = one(mode, rate)
            out["low_load"][f"{mode}_{rate}"] = {k: r.get(k) for k in
                                                 ("lat_p50_ms", "lat_p99_ms",
                                                  "device_service_p50_p99_ms",
                                                  "per_class_count_p50_p99_ms", "completed",
                                                  "error") if k in r}
    out["workload"] = ("Poisson 20k req/s (and 500, 5000 req/s), 50/50 detect/precode, "
                       "B in {64,128,256}, U in {8,16,32}, 16/64/256-QAM, 12-1200 subcarriers, "
                       "1-14 symbols, SNR 5-25 dB, K=min(U/4,8); latency from scheduled "
                       "arrival")
    return out


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    from paper_1404_0424_gb300 import build, cabi, shard, workload as wl

    B, QAM = args.B, args.qam  # the workload's shape (defaults: the headline configuration)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cabi.library(build.build())

    Un, K = args.U, args.K
    n = args.slots * NSC
    up = wl.uplink_torch(B, Un, QAM, n=n, R=R, snr_db=SNR_DB, seed=1000 + rank, device=dev)
    H, Y, N0 = up["H"], up["Y"], up["N0"]
    T = up["x"].contiguous()          # downlink symbols on the same channels
    del up
    xhat = torch.empty((n, R, Un), dtype=torch.complex64, device=dev)
    mu = torch.empty((n, R, Un), dtype=torch.float32, device=dev)
    rho = torch.empty_like(mu)
    llr = torch.empty((n, R, Un, QAM), dtype=torch.float32, device=dev)
    st = torch.empty((n,), dtype=torch.int32, device=dev)
    q = torch.empty((n, R, B), dtype=torch.complex64, device=dev)
    qn = torch.empty((n, R), dtype=torch.float32, device=dev)
    stp = torch.empty((n,), dtype=torch.int32, device=dev)
    prec = PRECISIONS[args.precision]
    p = cabi.params(B, Un, QAM, K, R, N0, precision=prec)
    stream = torch.cuda.current_stream(dev)

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        rc = cabi.cg_detect(p, n, H, Y, xhat, mu, rho, llr, st, stream)
        if evs is not None:
            evs[1].record(stream)
        rc |= cabi.cg_precode(p, n, H, T, q, qn, 0, stp, stream)
        if evs is not None:
            evs[2].record(stream)
        if rc:
            raise RuntimeError(cabi.cg_strerror(rc))

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0 and int(stp.abs().sum()) == 0
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = clock_sampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        step(evs[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    det_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    pre_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    elapsed_ms = shard.max_over_ranks(elapsed_ms, dist, dev)   # timing only

    ms_step = elapsed_ms / args.steps
    solves_step = 2 * n * R * world
    value = solves_step / (ms_step / 1e3)
    llrs = n * R * Un * QAM * world / (ms_step / 1e3)

    # the plain FP32 CUDA-core path on the same batch, for comparison
    plain = None
    if not args.no_plain and prec != 0:
        pp = cabi.params(B, Un, QAM, K, R, N0, precision=0)
        for _ in range(2):
            cabi.cg_detect(pp, n, H, Y, xhat, mu, rho, llr, st, stream)
            cabi.cg_precode(pp, n, H, T, q, qn, 0, stp, stream)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        reps = 5
        e[0].record(stream)
        for _ in range(reps):
            cabi.cg_detect(pp, n, H, Y, xhat, mu, rho, llr, st, stream)
        e[1].record(stream)
        for _ in range(reps):
            cabi.cg_precode(pp, n, H, T, q, qn, 0, stp, stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        pd, pq = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
        plain = {"what": "same batch, precision fp32 (CUDA-core Gram, matched filter, CG)",
                 "value": round(2 * n * R / ((pd + pq) / 1e3), 1), "unit": "solves/s",
                 "detect_ms": round(pd, 4), "precode_ms": round(pq, 4)}

    # the Neumann-series comparator (Sec. III-F) on the same batch, K = 3 terms
    neumann = None
    if not args.no_neumann and prec != 0:
        pn = cabi.params(B, Un, QAM, K, R, N0, precision=prec)
        for _ in range(2):
            cabi.cg_neumann_detect(pn, n, H, Y, xhat, st, stream)
            cabi.cg_neumann_precode(pn, n, H, T, q, qn, 0, stp, stream)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        reps = 5
        e[0].record(stream)
        for _ in range(reps):
            rc = cabi.cg_neumann_detect(pn, n, H, Y, xhat, st, stream)
        e[1].record(stream)
        for _ in range(reps):
            rc |= cabi.cg_neumann_precode(pn, n, H, T, q, qn, 0, stp, stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        if rc:
            raise RuntimeError(cabi.cg_strerror(rc))
        nd, nq = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
        nbytes = n * ((B * Un + R * B) * 8 + R * Un * 8 + 4)
        neumann = {"what": f"truncated Neumann series, {K} terms (Sec. III-F): x_hat only "
                           "(detection) and q, ||q|| (precoding), same batch and precision",
                   "detect_ms": round(nd, 4), "precode_ms": round(nq, 4),
                   "solves_per_s": round(2 * n * R / ((nd + nq) / 1e3), 1),
                   "detect_gbs": round(nbytes / nd / 1e6, 1),
                   "precode_gbs": round(precode_bytes_per_instance(B, Un, R) * n / nq / 1e6, 1)}

    # the rest of the 128-antenna configuration on the same batch: K in {2, 3, 4},
    # U = 8 (the first 8 users' columns would change the data, so U = 8 draws its
    # own channels), and the implicit product against the explicit Gram
    sweep = None
    if not args.no_sweep and prec != 0:
        def pair_ms(pp, Hh, Yy, Tt, nn, xo, mo, ro, lo, so, qo, qno, spo, reps=3):
            for _ in range(2):
                cabi.cg_detect(pp, nn, Hh, Yy, xo, mo, ro, lo, so, stream)
                cabi.cg_precode(pp, nn, Hh, Tt, qo, qno, 0, spo, stream)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            rcs = 0
            for _ in range(reps):
                rcs |= cabi.cg_detect(pp, nn, Hh, Yy, xo, mo, ro, lo, so, stream)
                rcs |= cabi.cg_precode(pp, nn, Hh, Tt, qo, qno, 0, spo, stream)
            ev[1].record(stream)
            torch.cuda.synchronize()
            if rcs:
                raise RuntimeError(cabi.cg_strerror(rcs))
            return ev[0].elapsed_time(ev[1]) / reps
        sweep = {"what": "detect + precode per step, ms, same batch of 38,400 instances"}
        for kk in (2, 3, 4):
            sweep[f"U16_K{kk}_{args.precision}"] = round(pair_ms(
                cabi.params(B, Un, QAM, kk, R, N0, precision=prec), H, Y, T, n, xhat, mu, rho,
                llr, st, q, qn, stp), 4)
        sweep[f"U16_K3_{args.precision}_exact_tracker"] = round(pair_ms(
            cabi.params(B, Un, QAM, K, R, N0, sinr_mode=1, precision=prec), H, Y, T, n, xhat,
            mu, rho, llr, st, q, qn, stp), 4)
        sweep["U16_K3_fp32_exact_tracker"] = round(pair_ms(
            cabi.params(B, Un, QAM, K, R, N0, sinr_mode=1, precision=0), H, Y, T, n, xhat,
            mu, rho, llr, st, q, qn, stp), 4)
        sweep["U16_K3_fp32_explicit"] = round(pair_ms(
            cabi.params(B, Un, QAM, K, R, N0, precision=0, amul_mode=1), H, Y, T, n, xhat, mu,
            rho, llr, st, q, qn, stp), 4)
        sweep["U16_K3_fp32_implicit"] = round(pair_ms(
            cabi.params(B, Un, QAM, K, R, N0, precision=0, amul_mode=2), H, Y, T, n, xhat, mu,
            rho, llr, st, q, qn, stp), 4)
        u8 = wl.uplink_torch(B, 8, QAM, n=n, R=R, snr_db=SNR_DB, seed=3000 + rank, device=dev)
        H8, Y8, T8 = u8["H"], u8["Y"], u8["x"].contiguous()
        x8 = torch.empty((n, R, 8), dtype=torch.complex64, device=dev)
        m8 = torch.empty((n, R, 8), dtype=torch.float32, device=dev)
        r8 = torch.empty_like(m8)
        l8 = torch.empty((n, R, 8, QAM), dtype=torch.float32, device=dev)
        for kk in (2, 3, 4):
            sweep[f"U8_K{kk}_{args.precision}"] = round(pair_ms(
                cabi.params(B, 8, QAM, kk, R, u8["N0"], precision=prec), H8, Y8, T8, n, x8, m8,
                r8, l8, st, q, qn, stp), 4)
        del u8, H8, Y8, T8, x8, m8, r8, l8
        sweep["solves_per_step"] = 2 * n * R

    # CG least squares (Sec. III-E, no Gram, FP32 CUDA cores) on the same batch
    cgls = None
    if not args.no_cgls:
        pc = cabi.params(B, Un, QAM, K, R, N0, amul_mode=3)
        for _ in range(2):
            cabi.cg_detect(pc, n, H, Y, xhat, mu, rho, llr, st, stream)
            cabi.cg_precode(pc, n, H, T, q, qn, 0, stp, stream)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        reps = 3
        e[0].record(stream)
        for _ in range(reps):
            rc = cabi.cg_detect(pc, n, H, Y, xhat, mu, rho, llr, st, stream)
        e[1].record(stream)
        for _ in range(reps):
            rc |= cabi.cg_precode(pc, n, H, T, q, qn, 0, stp, stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        if rc:
            raise RuntimeError(cabi.cg_strerror(rc))
        cd, cq = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
        cgls = {"what": f"CG least squares, {K} iterations (Sec. III-E): no Gram, FP32 CUDA "
                        "cores, all outputs, same batch",
                "detect_ms": round(cd, 4), "precode_ms": round(cq, 4),
                "solves_per_s": round(2 * n * R / ((cd + cq) / 1e3), 1)}

    # plain per-call latency: one 1200 x 14 slot (detect + precode) per call
    lat = []
    Hs, Ys, Ts = H[:NSC], Y[:NSC], T[:NSC]
    for i in range(60):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cabi.cg_detect(p, NSC, Hs, Ys, xhat, mu, rho, llr, st, stream)
        cabi.cg_precode(p, NSC, Hs, Ts, q, qn, 0, stp, stream)
        e1.record(stream)
        e1.synchronize()
        if i >= 10:
            lat.append(e0.elapsed_time(e1))
    lat.sort()

    # end-to-end through the host-memory ABI (pinned buffers, copies timed)
    e2e = None
    if not args.no_e2e:
        ne = n
        Hh = H[:ne].cpu().pin_memory()
        Yh = Y[:ne].cpu().pin_memory()
        Th = T[:ne].cpu().pin_memory()
        ox = torch.empty((ne, R, Un), dtype=torch.complex64).pin_memory()
        om = torch.empty((ne, R, Un), dtype=torch.float32).pin_memory()
        orh = torch.empty_like(om).pin_memory()
        ol = torch.empty((ne, R, Un, QAM), dtype=torch.float32).pin_memory()
        os_ = torch.empty((ne,), dtype=torch.int32).pin_memory()
        oq = torch.empty((ne, R, B), dtype=torch.complex64).pin_memory()
        oqn = torch.empty((ne, R), dtype=torch.float32).pin_memory()
        osp = torch.empty((ne,), dtype=torch.int32).pin_memory()

        def e2e_step():
            rc = cabi.cg_detect_host(p, ne, Hh, Yh, ox, om, orh, ol, os_, stream)
            rc |= cabi.cg_precode_host(p, ne, Hh, Th, oq, oqn, 0, osp, stream)
            if rc:
                raise RuntimeError(cabi.cg_strerror(rc))

        for _ in range(2):
            e2e_step()
        ke = max(3, args.steps // 4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        dt = (time.perf_counter() - t0) / ke
        h2d = ne * (B * Un + R * B) * 8 + ne * (B * Un + R * Un) * 8
        d2h = ne * (detect_bytes_per_instance(B, Un, R, QAM) - (B * Un + R * B) * 8) + \
            ne * (R * B * 8 + R * 4 + 4)
        e2e = {"value": 2 * ne * R / dt, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "instances_per_step": ne}
        # the host link itself: one large pinned copy each way, then both at once
        # on two streams; the step's bytes over its time set against them
        big = 512 << 20
        hsrc = torch.empty(big, dtype=torch.uint8).pin_memory()
        hdst = torch.empty(big, dtype=torch.uint8).pin_memory()
        dbuf = torch.empty(big, dtype=torch.uint8, device=dev)
        dbuf2 = torch.empty(big, dtype=torch.uint8, device=dev)
        s2 = torch.cuda.Stream(dev)

        def copy_gbs(fn, nbytes, reps=5):
            fn()
            torch.cuda.synchronize()
            t0c = time.perf_counter()
            for _ in range(reps):
                fn()
            torch.cuda.synchronize()
            return nbytes * reps / (time.perf_counter() - t0c) / 1e9

        def both():
            dbuf.copy_(hsrc, non_blocking=True)
            with torch.cuda.stream(s2):
                hdst.copy_(dbuf2, non_blocking=True)
        h2d_gbs = copy_gbs(lambda: dbuf.copy_(hsrc, non_blocking=True), big)
        d2h_gbs = copy_gbs(lambda: hdst.copy_(dbuf, non_blocking=True), big)
        both_gbs = copy_gbs(both, 2 * big)
        e2e["host_link"] = {"h2d_gbs": round(h2d_gbs, 1), "d2h_gbs": round(d2h_gbs, 1),
                            "both_directions_gbs": round(both_gbs, 1),
                            "step_gbs": round((h2d + d2h) / dt / 1e9, 1),
                            "what": "pinned copies of 512 MiB; step_gbs = the e2e step's "
                                    "host<->device bytes over its time"}
        del hsrc, hdst, dbuf, dbuf2
        cabi.cg_release_workspace()

    peaks, peak_kind = measured_peaks()
    det_bytes = detect_bytes_per_instance(B, Un, R, QAM) * n
    achieved = det_bytes / (det_ms / 1e3) / 1e9
    traffic = profiled_traffic(f"detect_{args.precision}_{B}x{Un}")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "traffic": traffic, "kernel": detect_kernel_name(args.precision, Un),
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": det_bytes}
    pre_bytes = precode_bytes_per_instance(B, Un, R) * n
    pre_gbs = pre_bytes / (pre_ms / 1e3) / 1e9

    batched = None
    if rank == 0 and not args.no_batched:
        batched = run_batched(cabi, torch, dev)
    large = None
    if rank == 0 and not args.no_large and prec != 0:
        large = run_large(cabi, torch, dev, args.precision)
    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        serving = run_serving(args.serve_seconds)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, ninst, dt, cores = time_oracle(args.cpu_seconds, Un, K)
        cpu = {"value": round(rate, 2), "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": f"{ninst} subcarriers x {R} symbols (B={B}, U={Un}, 64-QAM, K={K}), "
                         f"detect + precode, FP64 numpy, {cores} spawned single-threaded "
                         f"workers for {args.cpu_seconds:.0f} s each"}

    if rank == 0:
        step_gbs = (det_bytes + pre_bytes) * world / (ms_step / 1e3) / 1e9
        detail = {
            "detect_solves_per_s": round(n * R * world / (det_ms / 1e3), 1),
            "precode_solves_per_s": round(n * R * world / (pre_ms / 1e3), 1),
            "llrs_per_s": round(llrs, 1),
            "latency_ms": {"slot_p50": round(lat[len(lat) // 2], 4),
                           "slot_p99": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 4),
                           "slot_what": "one 1200x14 slot, detect + precode, one launch each"},
            "batched": batched, "large_256x32": large, "neumann": neumann, "cgls": cgls,
            "sweep_128": sweep, "serving": serving, "plain_fp32": plain,
        }
        srv = serving or {}
        low = srv.get("low_load", {})
        line = {
            "metric": f"CG solves/s (detect + precode) at B={B}, U={Un}, {1 << QAM}-QAM, R={R}, "
                      f"K={K}",
            "value": round(value, 1), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic (seeded i.i.d. CN(0,1) channels, Gray 64-QAM, AWGN at 10 dB)",
            "config": {"workload": f"uplink CG-D + downlink CG-P, B={B}, U={Un}, {1 << QAM}-QAM, "
                                   f"{NSC} subcarriers x {R} symbols per slot, K={K}, "
                                   f"SNR {SNR_DB} dB",
                       "precision": args.precision,
                       "slots_per_step": args.slots, "instances_per_step": n,
                       "l2": "inputs larger than L2 (%.2f GB read per step)" %
                             ((det_bytes + pre_bytes) / 1e9),
                       "parallelism": f"replicas x{world}"},
            "detect_ms": round(det_ms, 4), "precode_ms": round(pre_ms, 4),
            "step_frac": round(step_gbs / peaks["hbm_gbs"], 4),
            "precode_frac": round(pre_gbs / peaks["hbm_gbs"], 4),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 2 * args.steps,
            "clocks": ck,
            "latency_ms": {"slot_p50": detail["latency_ms"]["slot_p50"],
                           "served_p50": srv.get("served", {}).get("lat_p50_ms"),
                           "served_p99": srv.get("served", {}).get("lat_p99_ms"),
                           "plain_p50": srv.get("plain", {}).get("lat_p50_ms"),
                           "served_500_p50": low.get("served_500", {}).get("lat_p50_ms"),
                           "plain_500_p50": low.get("plain_500", {}).get("lat_p50_ms")},
        }
        if batched and "error" not in batched:
            line["batched"] = {k: batched.get(k) for k in ("ms_per_run", "gb_per_s", "frac_hbm",
                                                           "precision", "schedule")}
            line["batched"]["plain_ms"] = batched["plain_one_launch_per_problem"]["ms"]
        if large:
            line["large_256x32"] = {k: large.get(k) for k in (
                "detect_ms", "precode_ms", "detect_frac_hbm", "precode_frac_hbm",
                "exact_tracker_detect_ms", "exact_tracker_fp32_detect_ms")}
        print("detail: " + json.dumps(detail), file=sys.stderr)
        sys.stderr.flush()
        print(json.dumps(line))
        sys.stdout.flush()
    if dist:
        dist.destroy_process_group()
    _ = np, math


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    Un, K = args.U, args.K
    per = []
    warm = max(args.warmup, 3)
    budget = max(1.0, 120.0 / (args.steps + warm))
    cores = 0
    for s in range(args.steps + warm):
        rate, ninst, dt, cores = time_oracle(budget, Un, K)
        if s >= warm:
            per.append((rate, ninst, budget))
    rate = sum(r[1] for r in per) * 2 * R / sum(r[2] for r in per)
    line = {
        "impl": "reference",
        "metric": "CG solves/s (detect + precode) at B=128, U=16, 64-QAM, R=14, K=3",
        "value": round(rate, 2), "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": warm, "ms_per_step": round(1e3 * sum(r[2] for r in per) / len(per), 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded i.i.d. CN(0,1) channels, Gray 64-QAM, AWGN at 10 dB)",
        "config": {"workload": f"uplink CG-D + downlink CG-P, B={B}, U={Un}, 64-QAM, "
                               f"{NSC} subcarriers x {R} symbols per slot, K={K}, "
                               f"SNR {SNR_DB} dB", "parallelism": f"host, {cores} processes"},
        "cpu_baseline": {"value": round(rate, 2), "unit": "solves/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"each step: {cores} single-threaded FP64 numpy workers, "
                                   f"subcarriers for {budget:.1f} s each"},
        "e2e": {"value": round(rate, 2), "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
