#!/usr/bin/env python3
"""Benchmark: negacyclic RNS NTT, N = 2^16, L = 45 limbs, forward + inverse.

One step = the forward then the inverse transform of one RNS polynomial of 45
limbs (the 45 largest primes < 2^60 with q = 1 mod 2^17), uint64 residues,
seeded uniform inputs.  Steps are independent polynomials; step i runs on
stream i mod --streams (one plan per stream), so one step's tail overlaps the
next step's start.  The roofline figure uses per-launch CUDA-event durations
from a separate single-stream pass.  Metric: limb-NTT/s (each limb forward or inverse
counts as one), with the fraction of the HBM roofline for one read plus one
write of the data per transform.

Arms:
  default            the CUDA library through its C ABI (device buffers);
  --impl reference   the CPU oracle, timed on the host cores.
Multi-GPU (torchrun): every rank transforms its own polynomials on its own GPU
(replicas, no collective); value = all ranks' limb-NTTs / max rank time.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ntt_inputs as I  # noqa: E402

L2_BYTES = 129 * 1024 * 1024
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic_c2_n65536_l45.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--twiddle", default="auto", choices=["auto", "table", "ot1", "ot2"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "fused", "per_pass"])
    ap.add_argument("--geometry", type=int, default=0, choices=[0, 1, 2],
                    help="pass geometry of the C2 plans when not autotuned (NTT_GEOMETRY_*)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--streams", type=int, default=3,
                    help="independent steps spread over this many streams (one plan each)")
    ap.add_argument("--ctas-per-sm", type=int, default=1,
                    help="persistent CTAs per SM of the timed steps' fused launches (0: as many as fit); "
                         "with one, launches on different streams share every SM")
    ap.add_argument("--no-batch-compare", action="store_true",
                    help="skip the per-limb C2 path and the uneven 96-job batch")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving workload")
    ap.add_argument("--no-peak-measure", action="store_true",
                    help="skip the live butterfly-rate measurement (for profiling runs)")
    ap.add_argument("--no-ablation", action="store_true", help="skip the N sweep of kernel organisations")
    ap.add_argument("--ablation-only", action="store_true",
                    help="run only the kernel-organisation sweep and print it (for profiling its launches)")
    ap.add_argument("--ablation-reps", type=int, default=40)
    ap.add_argument("--word-size-only", action="store_true",
                    help="run only the word-size comparison and print it (for profiling its launches)")
    ap.add_argument("--no-select", action="store_true",
                    help="build the C2 plans from the autotuner's choice instead of timing the candidate "
                         "configurations (organisation, twiddles, geometry, streams) in the timed setting")
    ap.add_argument("--no-tune", action="store_true",
                    help="plans with the fixed default options instead of the autotuner's choice")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--launch-steps", type=int, default=500,
                    help="steps of the single-stream pass that times each launch")
    ap.add_argument("--l2-twiddles", action="store_true",
                    help="plans with NTT_PLAN_L2_TWIDDLES (twiddle tables kept in L2 by a persisting window)")
    ap.add_argument("--traffic-json", default=None,
                    help="write the DRAM-traffic summary of the C2 kernels from ncu CSV files (--traffic-csv) "
                         "to this JSON file and exit")
    ap.add_argument("--traffic-csv", nargs="*", default=[],
                    help="ncu --csv logs of dram__bytes_read.sum, dram__bytes_write.sum, gpu__time_duration.sum")
    ap.add_argument("--traffic-command", default="",
                    help="the command line that produced the CSV files (recorded in the JSON)")
    ap.add_argument("--int8-probe", action="store_true",
                    help="time the library int8 GEMM (torch._int_mm) against bf16 and print it (tensor-core check)")
    ap.add_argument("--only", default=None, choices=["c1", "c4"],
                    help="run one secondary leg alone and print its JSON (for profiling its kernels): "
                         "c1 = the N=2^12 single-limb latency leg, c4 = the uneven 96-job batch, default plans")
    ap.add_argument("--prequeue-ms", type=float, default=3.0,
                    help="device-side delay queued before the start event of the C2 timings, so that the "
                         "host has queued the first steps when timing starts (0: none)")
    ap.add_argument("--split-calls", action="store_true",
                    help="each step as two calls (ntt_forward, ntt_inverse) instead of one ntt_execute")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


KERNEL_SOURCES = ("arith.cuh", "device_types.cuh", "ntt_pass.cuh", "tma.cuh", "ntt_fused.cuh",
                  "launch.cuh", "k_n16.cu", "k_n16_g1.cu", "k_n16_g2.cu")


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def agree_on_rank0(obj, dist):
    """Rank 0's value of a picklable object on every rank (itself alone)."""
    if dist is None:
        return obj
    box = [obj]
    dist.broadcast_object_list(box, src=0)
    return box[0]


def whole_job_value(limbs_per_step: int, steps: int, ranks: int, total_ms: float) -> float:
    """limb-NTT/s of the whole job: every rank transforms its own polynomials
    (replicas), each step one forward and one inverse of limbs_per_step limbs."""
    return 2 * limbs_per_step * steps * ranks / (total_ms / 1e3)


def kernel_source_hash() -> str:
    """Hash of the sources the N = 2^16 transform kernels are built from, with
    comments and blank space removed (a comment edit keeps a profile valid)."""
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2012_01968_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f)) as fh:
            txt = fh.read()
        txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", " ", txt)
        h.update(f.encode())
        h.update(" ".join(txt.split()).encode())
    return h.hexdigest()[:16]


def profile_traffic(kind: str, geometry: int, twiddle: str, direction: str):
    """DRAM traffic of one steady-state call of the C2 transform (the fused
    launch, or the per-pass call's column and row launches together; ncu
    counters, committed under profiles/), for the plan's organisation,
    geometry, twiddle supply and direction, if it was taken on the current
    kernel sources (else None)."""
    try:
        with open(TRAFFIC_JSON) as f:
            entries = json.load(f)["entries"]
    except (OSError, KeyError, ValueError):
        return None
    h = kernel_source_hash()
    for e in entries:
        if (e.get("kind", "fused"), e.get("geometry"), e.get("twiddle"), e.get("direction"),
                e.get("source_hash")) == (kind, geometry, twiddle, direction, h):
            return e
    return None


def int8_probe(torch):
    """Dense int8 GEMM rate of the library path (torch._int_mm, cuBLASLt)
    against bf16 (torch.matmul) on square-ish shapes: whether an exact
    integer tensor-core pass could pay on this GPU."""
    out = {"unit": "TOPS (int8) / TFLOP/s (bf16)", "shapes": []}
    for m, k, n in ((8192, 8192, 8192), (16384, 8192, 8192)):
        a8 = torch.randint(-128, 127, (m, k), dtype=torch.int8, device="cuda")
        b8 = torch.randint(-128, 127, (k, n), dtype=torch.int8, device="cuda")
        ab = a8.to(torch.bfloat16)
        bb = b8.to(torch.bfloat16)
        res = {"m": m, "k": k, "n": n}
        for name, fn in (("int8", lambda: torch._int_mm(a8, b8)), ("bf16", lambda: ab @ bb)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            reps = 20
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            res[name] = 2.0 * m * k * n * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
        out["shapes"].append(res)
    return out


def write_traffic_json(out, csvs, command):
    """Mean DRAM traffic per launch of each C2 fused kernel in ncu CSV logs
    (steady-state launches taken with --cache-control none, so a launch's
    writes include the write-back of dirty lines it evicts), keyed by
    geometry, twiddle supply, direction and the current kernel source hash."""
    import csv as _csv
    import re
    N, L = 1 << 16, 45
    geoms = {(8, 4): 0, (8, 3): 1, (7, 3): 2}
    per = {}
    pass_sets = []           # per CSV file (one per-pass configuration each): direction -> launches
    for path in csvs:
        passes = {}
        pass_sets.append(passes)
        hdr = None
        for r in _csv.reader(open(path)):
            if r and r[0] == "ID":
                hdr = r
                continue
            if not hdr or len(r) != len(hdr):
                continue
            d = dict(zip(hdr, r))
            name = d["Kernel Name"]
            v = float(d["Metric Value"].replace(",", ""))
            metric = {"dram__bytes_read.sum": "read", "dram__bytes_write.sum": "write",
                      "gpu__time_duration.sum": "t"}[d["Metric Name"]]
            if "ntt_pass_kernel" in name:
                # P, LOGC, KMAX, ROWS, FWD, XIN, FINAL, HAS_S0, OTS, TW_SMEM, W, TBL_LAST
                pa = [x.strip() for x in re.search(r"ntt_pass_kernel<([^>]*)>", name).group(1).split(",")]
                P, logc, rows, fwd, ots = int(pa[0]), int(pa[1]), int(pa[3]) == 1, int(pa[4]), int(pa[8])
                if len(pa) >= 12 and pa[11] in ("1", "true"):
                    ots = 0          # table plan: the last stage reads the table, not OT factors
                direction = "forward" if fwd else "inverse"
                e = passes.setdefault(direction, {"col": {"read": [], "write": [], "t": []},
                                                  "row": {"read": [], "write": [], "t": []}})
                part = e["row" if rows else "col"]
                part[metric].append(v)
                if rows:
                    e["p1"], e["logc"], e["ots"] = 16 - P, logc, ots
                continue
            if "ntt_fused_kernel" not in name:
                continue
            args = [x.strip() for x in re.search(r"ntt_fused_kernel<([^>]*)>", name).group(1).split(",")]
            p1, p2, lc, fwd, ots = int(args[0]), int(args[1]), int(args[2]), int(args[4]), int(args[5])
            chain = len(args) >= 10 and int(args[9]) == 1
            if p1 + p2 != 16:
                continue
            key = (geoms.get((p1, lc), -1), "table" if ots == 0 else f"ot{ots}",
                   "forward+inverse" if chain else ("forward" if fwd else "inverse"))
            e = per.setdefault(key, {"kernel": name.split("(")[0].replace("void ", ""), "read": [], "write": [], "t": []})
            e[metric].append(v)
    entries = []
    h = kernel_source_hash()
    for (g, tw, direction), e in sorted(per.items()):
        rd, wr = float(np.mean(e["read"])), float(np.mean(e["write"]))
        transforms = 2 if direction == "forward+inverse" else 1
        data = 8 * N * L                    # one read of the array
        entries.append({"kind": "fused", "kernel": e["kernel"], "geometry": g, "twiddle": tw, "direction": direction,
                        "source_hash": h, "launches": len(e["read"]),
                        "dram_read_bytes": rd, "dram_write_bytes": wr, "dram_bytes": rd + wr,
                        "alg_bytes": 16 * N * L * transforms,
                        "data_read_bytes": min(rd, data), "twiddle_read_bytes": max(0.0, rd - data),
                        "duration_us_mean_under_ncu": float(np.mean(e["t"])) / 1e3,
                        "how": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                               "--cache-control none on steady-state launches of the bench's timed loop; writes "
                               "include write-back of lines evicted during the launch; data_read_bytes = one read "
                               "of the array (8 N L), the rest of the reads counted as twiddle reads"})
    for direction, e in [(d, ps[d]) for ps in pass_sets for d in sorted(ps)]:
        if "p1" not in e or not e["col"]["read"]:
            continue
        rd = float(np.mean(e["col"]["read"])) + float(np.mean(e["row"]["read"]))
        wr = float(np.mean(e["col"]["write"])) + float(np.mean(e["row"]["write"]))
        entries.append({"kind": "per_pass", "kernel": "ntt_pass_kernel (column pass) + ntt_pass_kernel (row pass)",
                        "geometry": geoms.get((e["p1"], e["logc"]), -1),
                        "twiddle": "table" if e["ots"] == 0 else f"ot{e['ots']}", "direction": direction,
                        "source_hash": h, "launches": len(e["col"]["read"]) + len(e["row"]["read"]),
                        "dram_read_bytes": rd, "dram_write_bytes": wr, "dram_bytes": rd + wr,
                        "alg_bytes": 16 * N * L, "data_read_bytes": min(rd, 8 * N * L),
                        "twiddle_read_bytes": max(0.0, rd - 8 * N * L),
                        "duration_us_mean_under_ncu": (float(np.mean(e["col"]["t"])) + float(np.mean(e["row"]["t"]))) / 1e3,
                        "how": "per call: the mean column-pass launch plus the mean row-pass launch, same counters "
                               "and cache control as the fused entries; the second pass re-reads the first pass's "
                               "output, mostly from L2"})
    with open(out, "w") as f:
        json.dump({"workload": "c2_n65536_l45", "command": command, "entries": entries}, f, indent=1)
        f.write("\n")
    print(json.dumps({"traffic_json": out, "entries": len(entries)}))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# Integer-multiply roofline of the butterfly (secondary bound).  Measured on
# this GPU with a register-only micro-benchmark: a warp's IMAD occupies the
# FMA-heavy pipe of its SM sub-partition for 2 cycles, IMAD.WIDE and IMAD.HI
# for 4.  Shoup's lazy product (arith.cuh) issues 2 IMAD.HI, 3 IMAD.WIDE and
# 4 IMAD per butterfly: 28 pipe cycles per warp butterfly, i.e. 4 x 32 / 28
# butterflies per SM and clock.
SMS, SM_MHZ_MAX = 152, 2070.0
BFLY_PER_SM_CLK = 4 * 32 / (2 * 4 + 3 * 4 + 4 * 2)


def alu_peak_gbfly(sm_mhz=SM_MHZ_MAX):
    return SMS * BFLY_PER_SM_CLK * sm_mhz * 1e6 / 1e9


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# CPU oracle leg
# ----------------------------------------------------------------------------
def oracle_time(primes, N, seconds_target: float, threads: int | None = None, batch: int = 1):
    """Oracle forward + inverse over all limbs of `batch` polynomials, repeated
    until ~seconds_target elapse, limb-parallel on `threads` host threads (all
    cores by default); returns (limb-NTT/s, threads, sample text)."""
    import oracle
    orc = oracle.get()
    cores = threads or os.cpu_count() or 1
    data = I.batch_uniform(2, batch, primes, N)
    reps = 0
    t0 = time.perf_counter()
    while True:
        f = orc.ntt_batch(data, primes, +1, cores)
        b = orc.ntt_batch(f, primes, -1, cores)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds_target:
            break
    if not np.array_equal(b, data):
        raise RuntimeError("oracle round trip failed")
    v = reps * 2 * batch * len(primes) / el
    return v, cores, f"{reps} x (forward + inverse of all {batch * len(primes)} limbs), N={N}, {el:.1f} s"


def run_reference(args, metric, unit, w):
    """The reference arm: the CPU oracle on the host cores, on this arm's
    workload.  One step = the forward then the inverse of the whole C2
    polynomial (all 45 limbs), limb-parallel on every host core.  The timed
    sample is `--steps` steps, extended by whole steps until it lasts at least
    5 s, so that the rate does not hang on one short sample."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    orc = oracle.get()
    cores = os.cpu_count() or 1
    N, primes = w.N, w.primes
    data = I.batch_uniform(w.seed, 1, primes, N)

    def one_step():
        f = orc.ntt_batch(data, primes, +1, cores)
        return orc.ntt_batch(f, primes, -1, cores)

    for _ in range(max(0, args.warmup)):
        one_step()
    steps = 0
    t0 = time.perf_counter()
    while True:
        back = one_step()
        steps += 1
        el = time.perf_counter() - t0
        if steps >= args.steps and el >= 5.0:
            break
    if not np.array_equal(back, data):
        raise RuntimeError("oracle round trip failed")
    L = len(primes)
    value = 2.0 * L * steps / el
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "steps_timed": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": config_dict(w, args, ws),
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                         "sample": f"{steps} steps x (forward + inverse of all {L} limbs of the N={N} "
                                   f"polynomial), limb-parallel on {cores} host threads, {el:.1f} s"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


KERNEL_NAMES = {0: "auto", 1: "fused", 2: "per_pass", 3: "radix2", 4: "high_radix"}


def opts_summary(o):
    return {"kernel": KERNEL_NAMES[int(o.kernel)],
            "twiddle": "table" if o.twiddle_mode == 1 else f"ot{o.ot_stages}" if o.twiddle_mode == 2 else "auto",
            "geometry": int(o.geometry)}


def autotune(G, N, primes, batch, reps=10):
    """The library's autotuner for (N, primes, batch): the chosen options and
    a short report (the five fastest candidates, forward + inverse µs)."""
    best, entries = G.ntt_autotune(N, primes, batch, reps=reps)
    ranked = sorted((e for e in entries if e.status == 0), key=lambda e: e.forward_us + e.inverse_us)
    rep = {"chosen": opts_summary(best), "candidates": len(entries),
           "fastest_us": [dict(opts_summary(e.opts), us=round(e.forward_us + e.inverse_us, 2)) for e in ranked[:5]]}
    return best, rep


def _ok(G, st, what):
    """Raise on a failed library call (the timing loops call the C ABI directly)."""
    if st:
        raise RuntimeError(f"{what}: {G.ntt_status_string(st)} ({G.ntt_last_cuda_error()})")


def host_link_rates(torch, hin, hout, reps=20):
    """Pinned host <-> device copy rates of this machine's link (GB/s): one
    direction at a time, and both at once on two streams, for the buffers
    the end-to-end call moves; and each direction split into 2, 4 and 8
    chunks copied concurrently on as many streams (whether more copy engines
    raise the rate)."""
    d = torch.empty_like(hin, device="cuda")
    d2 = torch.empty_like(hin, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    nbytes = hin.numel() * hin.element_size()
    many = [torch.cuda.Stream() for _ in range(8)]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    def h2d():
        with torch.cuda.stream(s1):
            d.copy_(hin, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            hout.copy_(d2, non_blocking=True)

    def both():
        h2d()
        d2h()

    def split(k, to_device):
        n = hin.numel() // k

        def fn():
            for i in range(k):
                lo, hi = i * n, (hin.numel() if i == k - 1 else (i + 1) * n)
                with torch.cuda.stream(many[i]):
                    if to_device:
                        d[lo:hi].copy_(hin[lo:hi], non_blocking=True)
                    else:
                        hout[lo:hi].copy_(d2[lo:hi], non_blocking=True)
        return fn
    return {"h2d_gbs": nbytes / timed(h2d) / 1e9, "d2h_gbs": nbytes / timed(d2h) / 1e9,
            "both_gbs": 2 * nbytes / timed(both) / 1e9,
            "h2d_gbs_by_streams": {k: nbytes / timed(split(k, True)) / 1e9 for k in (2, 4, 8)},
            "d2h_gbs_by_streams": {k: nbytes / timed(split(k, False)) / 1e9 for k in (2, 4, 8)}}


def per_limb_c2(G, torch, w, host, steps):
    """The plain per-limb path on the C2 polynomial: one single-prime plan per
    limb and one launch per limb and direction (45 x 2 launches per step)."""
    L = len(w.primes)
    plans = [G.Plan(w.N, [q]) for q in w.primes]
    lib = G.lib()
    try:
        bufs = [torch.from_numpy(host[0, l].view(np.int64).copy()).cuda() for l in range(L)]
        ref = [b.clone() for b in bufs]
        s = torch.cuda.Stream()

        def step():
            for l in range(L):
                _ok(G, lib.ntt_forward(plans[l].handle, bufs[l].data_ptr(), 1, s.cuda_stream), "per-limb forward")
                _ok(G, lib.ntt_inverse(plans[l].handle, bufs[l].data_ptr(), 1, s.cuda_stream), "per-limb inverse")

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            step()
        e1.record(s)
        torch.cuda.synchronize()
        if not all(torch.equal(a, b) for a, b in zip(bufs, ref)):
            raise RuntimeError("per-limb round trip mismatch")
        ms = e0.elapsed_time(e1)
        return {"value": 2 * L * steps / (ms / 1e3), "unit": "limb-NTT/s", "steps": steps,
                "launches_per_step": 2 * L, "ms_per_step": ms / steps}
    finally:
        for p in plans:
            p.close()


def batched_c4(G, torch, reps, tuned=None, plan_kw=None):
    """The uneven 96-job workload (N in 2^14..2^17, L in [1, 60], mixed
    directions): one ntt_batch_submit, its CUDA-graph replay, and the same
    jobs as 96 single calls on one stream.  `tuned` maps log2 N to plan
    options (the autotuner's); `plan_kw`: the same plan options for every
    size; neither: the default options (one mixed-size launch per
    submission)."""
    w = I.workload_c4()
    chain = I.chain_2_18_60()
    plans = {n: (G.Plan.from_opts(1 << n, chain, tuned[n]) if tuned else G.Plan(1 << n, chain, **(plan_kw or {})))
             for n in range(14, 18)}
    lib = G.lib()
    try:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(w.seed)
        # residues below 2^59 < every prime of the chain (timing input; parity is tested elsewhere)
        bufs = [torch.randint(0, 1 << 59, (j.L * j.N,), generator=gen, dtype=torch.int64, device="cuda")
                for j in w.jobs]
        spec = [(plans[I.log2_exact(j.N)].handle, b, 1, j.L, G.NTT_OP_FORWARD if j.dir > 0 else G.NTT_OP_INVERSE)
                for j, b in zip(w.jobs, bufs)]
        jobs = G.make_jobs(spec)
        limbs = sum(j.L for j in w.jobs)
        s = torch.cuda.Stream()
        out = {"jobs": len(w.jobs), "limb_ntts_per_submission": limbs,
               "bytes_per_submission": sum(16 * j.L * j.N for j in w.jobs)}

        def timed(fn):
            # everything on stream s: graph replays run on torch's current stream
            with torch.cuda.stream(s):
                for _ in range(2):
                    fn()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                for _ in range(reps):
                    fn()
                e1.record(s)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            return {"value": limbs / (ms / 1e3), "unit": "limb-NTT/s", "ms_per_submission": ms}

        with G.Batch() as b:
            out["batched"] = timed(lambda: b.submit(jobs, s))
            out["launches_per_submission"] = batch_last_launches(G, b)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                b.submit(jobs, s)
            out["graph"] = timed(g.replay)
            if b.device_status() != 0:
                raise RuntimeError("batch device status reports a failed bounded wait")

        def singles():
            for h, buf, bt, lv, op in spec:
                _ok(G, (lib.ntt_forward_levels if op == G.NTT_OP_FORWARD else lib.ntt_inverse_levels)(
                    h, buf.data_ptr(), bt, lv, s.cuda_stream), "single call")
        out["per_job_calls"] = timed(singles)
        return out
    finally:
        for p in plans.values():
            p.close()


def PER_PASS_KW(G):
    """Plan options of the per-pass variants of the batch and serving legs:
    the per-pass organisation, OT on the last two stages, row tiles of half
    height (measured fastest for the C4 mix in that organisation)."""
    return {"twiddle_mode": G.NTT_TWIDDLE_OT, "ot_stages": 2, "kernel": G.NTT_KERNEL_PER_PASS,
            "geometry": G.NTT_GEOMETRY_SMALL_ROW_TILE}


def batch_last_launches(G, b):
    """Kernel launches the batch's last submission made (library test hook)."""
    import ctypes
    f = G.lib().ntt_internal_batch_last_launches
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]
    n = ctypes.c_uint32()
    return int(n.value) if f(b.handle, ctypes.byref(n)) == 0 else None


def serve_c5(G, torch, count, budget_gb=64, ring_gb=80, tuned=None, max_batch_jobs=64, slots=3,
             loads=(0.5, 0.8, 0.95), repeats=5, plan_kw=None):
    """The serving workload: `count` requests (N in 2^15..2^17, L in [4, 60],
    mixed directions) on device-resident data, admitted by an HBM budget.
    A capacity run (every request submitted at once), then Poisson arrivals at
    50 / 80 / 95% of that capacity; latency = submission to completion.  At
    each Poisson load the first tenth of the requests is a warm-up, left out
    of the statistics; the three loads run `repeats` times in a row, and each
    load reports its median run with the p99 of every run."""
    import collections
    chain = I.chain_2_18_60()
    plans = {n: (G.Plan.from_opts(1 << n, chain, tuned[n]) if tuned else G.Plan(1 << n, chain, **(plan_kw or {})))
             for n in (15, 16, 17)}
    word = 8
    ring_words = (ring_gb << 30) // word
    ring = torch.empty(ring_words, dtype=torch.int64, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    ring.random_(0, 1 << 59, generator=gen)         # residues below every prime of the chain
    base = I.serving_requests(count, 1.0, seed=5)   # sizes and directions; gaps rescaled per rate
    sizes = [r.L * r.N for r in base]
    warm = count // 10                         # warm-up requests of each Poisson run
    try:
        def run(rate):
            # the load generator must not pause: no Python garbage collection
            # while requests arrive (a collection would release a burst late)
            gc.collect()
            gc.disable()
            try:
                return run_load(rate)
            finally:
                gc.enable()

        def run_load(rate):
            with G.Server(budget_gb << 30, max_batch_jobs=max_batch_jobs, slots=slots) as srv:
                inflight = collections.deque()          # (ticket, start, end) in ring order
                tickets = []
                off = 0
                gaps = [r.t_arrival for r in base]
                t0 = time.perf_counter()
                for i, r in enumerate(base):
                    n = r.N.bit_length() - 1
                    if off + sizes[i] > ring_words:
                        off = 0
                    lo, hi = off, off + sizes[i]
                    # recycle: wait for older requests whose bytes this one overwrites
                    while inflight and inflight[0][1] < hi and inflight[0][2] > lo:
                        srv.wait(inflight.popleft()[0])
                    if rate is not None:
                        due = t0 + gaps[i] / rate
                        while time.perf_counter() < due:
                            pass
                    t = srv.submit(plans[n].handle, ring[lo:hi], 1, r.L,
                                   G.NTT_OP_FORWARD if r.dir > 0 else G.NTT_OP_INVERSE)
                    inflight.append((t, lo, hi))
                    tickets.append(t)
                    off = hi + ((-hi) % 2)              # 16-byte aligned starts
                for t in tickets:
                    srv.wait(t)
                times = [srv.times(t) for t in tickets]
                for t in tickets:
                    srv.release(t)
                sched = srv.stats()
            # at a Poisson load the first `warm` requests bring host and device
            # to that load's steady state and are left out of the statistics
            first = warm if rate is not None else 0
            sub = np.array([x[0] for x in times[first:]], dtype=np.float64)
            done = np.array([x[2] for x in times[first:]], dtype=np.float64)
            lat = (done - sub) / 1e3
            dev_us = np.array([x[3] for x in times[first:]], dtype=np.float64) / 1e3
            admit = np.array([x[1] for x in times[first:]], dtype=np.float64)
            queue_us = (admit - sub) / 1e3                  # submission to the batch's start
            turn_us = (done - admit) / 1e3                  # batch start to completion seen
            span = (done.max() - sub.min()) / 1e9
            limbs = sum(r.L for r in base[first:])
            return {"limb_ntt_per_s": limbs / span, "requests_per_s": (count - first) / span,
                    "gb_per_s": 16 * sum(sizes[first:]) / span / 1e9, "measured_requests": count - first,
                    "latency_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                   "mean": float(lat.mean())},
                    "batch_device_us": {"p50": float(np.percentile(dev_us, 50)),
                                        "p99": float(np.percentile(dev_us, 99))},
                    "max_gap_between_completions_us": float(np.max(np.diff(np.sort(done)))) / 1e3,
                    "timeline_us": {"queue_p50": float(np.percentile(queue_us, 50)),
                                    "queue_p99": float(np.percentile(queue_us, 99)),
                                    "batch_p50": float(np.percentile(turn_us, 50)),
                                    "batch_p99": float(np.percentile(turn_us, 99))},
                    "scheduler": {(k[:-3] + "_us" if k.endswith("_ns") else k): (v / 1e3 if k.endswith("_ns") else v)
                                  for k, v in sched.items()}}

        cap = run(None)
        if tuned:
            plans_used = ("the autotuner's choice per N for 60 limbs x 6 polynomials per launch; the loads "
                          "are fractions of the capacity these plans reach with full 64-request batches, "
                          "which the smaller batches formed at 80% load run less efficiently")
        elif plan_kw:
            plans_used = "plans with the options " + json.dumps(plan_kw) + " (per-pass organisation)"
        else:
            plans_used = "library default plans (fused, default split: one mixed-size launch per batch)"
        out = {"requests": count, "budget_gb": budget_gb, "data": "device-resident, in place",
               "plans": plans_used, "capacity": cap}
        out["max_batch_jobs"], out["slots"] = max_batch_jobs, slots
        # the three loads, `repeats` times in a row: the p99 of every run, to show
        # whether a run's tail is an outlier
        runs = {frac: [] for frac in loads}
        for _ in range(repeats):
            for frac in loads:
                runs[frac].append(run(frac * cap["requests_per_s"]))
        for frac in loads:
            p99 = [r["latency_us"]["p99"] for r in runs[frac]]
            med = float(np.median(p99))
            out[f"poisson_{int(frac * 100)}pct"] = dict(
                runs[frac][int(np.argsort(p99)[len(p99) // 2])], offered_requests_per_s=frac * cap["requests_per_s"],
                p99_us_runs=p99, p50_us_runs=[r["latency_us"]["p50"] for r in runs[frac]],
                requests_per_batch_runs=[r["scheduler"]["requests"] / max(1, r["scheduler"]["batches"])
                                         for r in runs[frac]],
                max_completion_gap_us_runs=[r["scheduler"]["max_completion_gap_us"] for r in runs[frac]],
                max_launch_us_runs=[r["scheduler"]["max_launch_us"] for r in runs[frac]],
                max_loop_gap_us_runs=[r["scheduler"]["max_loop_gap_us"] for r in runs[frac]],
                max_device_us_runs=[r["scheduler"]["max_device_us"] for r in runs[frac]],
                queue_p99_us_runs=[r["timeline_us"]["queue_p99"] for r in runs[frac]],
                p99_max_over_median=max(p99) / med if med > 0 else None)
        out["scheduler_units"] = "_us keys in microseconds; batches and requests are counts"
        return out
    finally:
        for p in plans.values():
            p.close()
        del ring


def paper_ablation(G, torch, reps=40, sizes=(14, 15, 16, 17)):
    """The structure of the paper's N sweep (21 limbs, forward transform,
    log N = 14..17) on this GPU: the radix-2 launch-per-stage organisation
    the paper starts from, its register-based high-radix step (radix 2^2 ..
    2^5 per launch), the launch-per-pass organisation (the paper's two-kernel
    shared-memory design), and the one-launch fused kernel, each with table
    and OT twiddles.  Buffers rotate over more than 2x L2."""
    chain = I.prime_chain(21, 1 << 18)          # 21 largest primes < 2^60 = 1 mod 2^18
    configs = (("radix2", G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_RADIX2),
               ("high_radix4", G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_HIGH_RADIX, 2),
               ("high_radix8", G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_HIGH_RADIX, 3),
               ("high_radix16", G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_HIGH_RADIX, 4),
               ("high_radix32", G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_HIGH_RADIX, 5),
               ("per_pass_table", G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_PER_PASS),
               ("per_pass_ot1", G.NTT_TWIDDLE_OT, 1, G.NTT_KERNEL_PER_PASS),
               ("fused_table", G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_FUSED),
               ("fused_ot1", G.NTT_TWIDDLE_OT, 1, G.NTT_KERNEL_FUSED))
    lib = G.lib()
    s = torch.cuda.Stream()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(21)
    out = {"limbs": 21, "unit": "us per forward transform of all 21 limbs (one stream, events)"}
    for n in sizes:
        N = 1 << n
        words = 21 * N
        nbuf = max(2, -(-2 * L2_BYTES // (words * 8)) + 1)
        pool = torch.empty(nbuf * words, dtype=torch.int64, device="cuda")
        pool.random_(0, 1 << 59, generator=gen)
        row = {}
        for name, mode, ots, kern, *radix in configs:
            with G.Plan(N, chain, mode, ots, kern, radix_log2=radix[0] if radix else 0) as p:
                ptr = [pool[i * words:(i + 1) * words].data_ptr() for i in range(nbuf)]
                for i in range(min(5, reps)):
                    _ok(G, lib.ntt_forward(p.handle, ptr[i % nbuf], 1, s.cuda_stream), name)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                for i in range(reps):
                    _ok(G, lib.ntt_forward(p.handle, ptr[i % nbuf], 1, s.cuda_stream), name)
                e1.record(s)
                torch.cuda.synchronize()
                row[name] = e0.elapsed_time(e1) * 1e3 / reps
        row["speedup_fused_ot1_vs_radix2"] = row["radix2"] / row["fused_ot1"]
        row["speedup_high_radix16_vs_radix2"] = row["radix2"] / row["high_radix16"]
        row["speedup_per_pass_ot1_vs_radix2"] = row["radix2"] / row["per_pass_ot1"]
        out[f"logN{n}"] = row
        del pool
    return out


def large_ring_c3(G, torch, reps=50, opts=None):
    """The large ring: N = 2^17, L = 60, one ciphertext (batch 2), forward
    then inverse per step on one stream; and the negacyclic product of two
    polynomials (two forwards in one launch, element-wise product, inverse)."""
    w = I.workload_c3()
    N, primes, L = w.N, w.primes, len(w.primes)
    host = I.batch_uniform(w.seed, 2, primes, N)
    src = torch.from_numpy(host.view(np.int64).copy()).cuda()
    words = src.numel()
    nbuf = max(2, -(-2 * L2_BYTES // (words * 8)) + 1)
    bufs = [src.clone() for _ in range(nbuf)]
    s = torch.cuda.Stream()
    lib = G.lib()
    with (G.Plan.from_opts(N, primes, opts) if opts is not None else G.Plan(N, primes)) as p:
        def timed(fn, k):
            with torch.cuda.stream(s):
                for i in range(3):
                    fn(i)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                for i in range(k):
                    fn(i)
                e1.record(s)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / k

        def step(i):
            b = bufs[i % nbuf].data_ptr()
            _ok(G, lib.ntt_forward(p.handle, b, 2, s.cuda_stream), "C3 forward")
            _ok(G, lib.ntt_inverse(p.handle, b, 2, s.cuda_stream), "C3 inverse")
        ms = timed(step, reps)
        if not all(torch.equal(b, src) for b in bufs):
            raise RuntimeError("C3 round trip mismatch")
        # independent ciphertexts on two streams (a clone of the plan each),
        # as the C2 timed steps run: buffer i on stream i mod 2
        streams2 = [s, torch.cuda.Stream()]
        nb2 = nbuf + (nbuf % 2)
        while len(bufs) < nb2:
            bufs.append(src.clone())
        with p.clone() as p2:
            hs = [p.handle, p2.handle]

            def step2(i):
                b, j = bufs[i % nb2].data_ptr(), i % 2
                _ok(G, lib.ntt_forward(hs[j], b, 2, streams2[j].cuda_stream), "C3 forward")
                _ok(G, lib.ntt_inverse(hs[j], b, 2, streams2[j].cuda_stream), "C3 inverse")
            for i in range(4):
                step2(i)
            torch.cuda.synchronize()
            cur = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            for st in streams2:
                st.wait_event(e0)
            for i in range(2 * reps):
                step2(i)
            for st in streams2:
                e = torch.cuda.Event()
                e.record(st)
                cur.wait_event(e)
            e1.record(cur)
            torch.cuda.synchronize()
            ms2 = e0.elapsed_time(e1) / (2 * reps)
            if not all(torch.equal(b, src) for b in bufs) or p2.device_status() != 0:
                raise RuntimeError("C3 two-stream round trip mismatch")
        c = torch.empty(L * N, dtype=torch.int64, device="cuda")

        def product(i):
            b = bufs[i % nbuf].view(-1)     # its two polynomials a = b[:LN], b = b[LN:] (left transformed)
            st = lib.ntt_mul_negacyclic(p.handle, b[:L * N].data_ptr(), b[L * N:].data_ptr(), c.data_ptr(), 1,
                                        s.cuda_stream)
            _ok(G, st, "ntt_mul_negacyclic")
        ms_mul = timed(product, reps)

        def product_in_place(i):
            b = bufs[i % nbuf].view(-1)     # c = a: the inverse's first pass applies the product
            st = lib.ntt_mul_negacyclic(p.handle, b[:L * N].data_ptr(), b[L * N:].data_ptr(), b[:L * N].data_ptr(),
                                        1, s.cuda_stream)
            _ok(G, st, "ntt_mul_negacyclic")
        ms_mul_ip = timed(product_in_place, reps)
        if p.device_status() != 0:
            raise RuntimeError("C3 device status reports a failed bounded wait")
    return {"workload": "N=2^17, L=60, batch 2 (one ciphertext), forward + inverse, one stream",
            "value": 2 * 2 * L / (ms / 1e3), "unit": "limb-NTT/s", "ms_per_step": ms,
            "alg_bytes_per_step": 2 * 2 * 16 * L * N,
            "two_streams": {"value": 2 * 2 * L / (ms2 / 1e3), "unit": "limb-NTT/s", "ms_per_step": ms2,
                            "how": "independent ciphertexts, step i on stream i mod 2 (a plan clone each), "
                                   "CUDA events around all steps"},
            "negacyclic_product_us": ms_mul * 1e3,
            "negacyclic_product": "c = a * b mod (X^N + 1), 60 limbs: 2 forwards in one launch, product, inverse",
            "negacyclic_product_in_place_us": ms_mul_ip * 1e3,
            "negacyclic_product_in_place": "the same with c = a: with a fused plan the inverse's first pass "
                                           "multiplies each tile by b (no separate element-wise pass)"}


def twiddle_modes_c2(G, torch, w, bufs, nbuf, reps=200):
    """C2 per-launch times under each twiddle supply (table, OT of the last
    one or two stages): one stream, CUDA events around the loop."""
    out = {}
    lib = G.lib()
    s = torch.cuda.Stream()
    for name, mode, ots in (("table", G.NTT_TWIDDLE_TABLE, 0), ("ot1", G.NTT_TWIDDLE_OT, 1),
                            ("ot2", G.NTT_TWIDDLE_OT, 2)):
        with G.Plan(w.N, w.primes, mode, ots) as p:
            for fwd in (True, False):
                fn = lib.ntt_forward if fwd else lib.ntt_inverse
                for i in range(5):
                    _ok(G, fn(p.handle, bufs[i % nbuf].data_ptr(), 1, s.cuda_stream), name)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                for i in range(reps):
                    _ok(G, fn(p.handle, bufs[i % nbuf].data_ptr(), 1, s.cuda_stream), name)
                e1.record(s)
                torch.cuda.synchronize()
                out[f"{name}_{'forward' if fwd else 'inverse'}_us"] = e0.elapsed_time(e1) * 1e3 / reps
            # each buffer went through as many inverses as forwards: unchanged
    torch.cuda.synchronize()
    return out


def word_size(G, torch, N, primes64, seed, reps=100):
    """Sec. IV's word-size question: one modulus built from primes below 2^60
    in 64-bit words, or from 28-bit primes in 32-bit words (about twice as
    many limbs, at least as many bits), forward + inverse per step on one
    stream.  Each word size with one launch per pass (table twiddles) and with
    the fused kernel (OT1, the default of both; 32-bit also with the table)."""
    import math
    bits64 = sum(math.log2(q) for q in primes64)
    cand = I.prime_chain(4 * len(primes64), 2 * N, below=1 << 28)
    L32, acc = 0, 0.0
    while acc < bits64:
        acc += math.log2(cand[L32])
        L32 += 1
    p32 = cand[:L32]
    lib = G.lib()
    s = torch.cuda.Stream()

    def timed(step):
        for i in range(3):
            step(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for i in range(reps):
            step(i)
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps

    out = {"workload": f"N=2^{N.bit_length() - 1}, modulus {bits64:.0f} bits, forward + inverse, one stream",
           "limbs_64": len(primes64), "limbs_32": L32, "bits_32": acc}
    h64 = I.batch_uniform(seed, 1, primes64, N)
    src64 = torch.from_numpy(h64.view(np.int64).copy()).cuda()
    nb64 = max(2, -(-2 * L2_BYTES // (src64.numel() * 8)) + 1)
    b64 = [src64.clone() for _ in range(nb64)]
    for name, kern in (("u64_per_pass_us", G.NTT_KERNEL_PER_PASS), ("u64_fused_us", G.NTT_KERNEL_AUTO)):
        mode = G.NTT_TWIDDLE_TABLE if kern == G.NTT_KERNEL_PER_PASS else G.NTT_TWIDDLE_AUTO
        with G.Plan(N, primes64, mode, 0, kern) as p:
            def step(i):
                b = b64[i % nb64].data_ptr()
                _ok(G, lib.ntt_forward(p.handle, b, 1, s.cuda_stream), "u64 forward")
                _ok(G, lib.ntt_inverse(p.handle, b, 1, s.cuda_stream), "u64 inverse")
            out[name] = timed(step)
    if not all(torch.equal(b, src64) for b in b64):
        raise RuntimeError("64-bit word-size round trip mismatch")
    h32 = I.batch_uniform(seed, 1, p32, N)
    src32 = torch.from_numpy(h32.astype(np.uint32).view(np.int32).copy()).cuda()
    nb32 = max(2, -(-2 * L2_BYTES // (src32.numel() * 4)) + 1)
    b32 = [src32.clone() for _ in range(nb32)]
    for name, kern, mode in (("u32_per_pass_us", G.NTT_KERNEL_PER_PASS, G.NTT_TWIDDLE_TABLE),
                             ("u32_fused_table_us", G.NTT_KERNEL_FUSED, G.NTT_TWIDDLE_TABLE),
                             ("u32_fused_us", G.NTT_KERNEL_FUSED, G.NTT_TWIDDLE_OT)):
        with G.Plan32(N, p32, kern, mode) as p:
            def step32(i):
                b = b32[i % nb32].data_ptr()
                _ok(G, lib.ntt_forward32(p.handle, b, 1, s.cuda_stream), "u32 forward")
                _ok(G, lib.ntt_inverse32(p.handle, b, 1, s.cuda_stream), "u32 inverse")
            out[name] = timed(step32)
            if p.device_status() != 0:
                raise RuntimeError("32-bit plan device status reports a failed bounded wait")
    if not all(torch.equal(b, src32) for b in b32):
        raise RuntimeError("32-bit word-size round trip mismatch")
    out["u32_vs_u64_per_pass"] = out["u64_per_pass_us"] / out["u32_per_pass_us"]
    out["u32_fused_vs_u64_fused"] = out["u64_fused_us"] / out["u32_fused_us"]
    return out


def word_sizes(G, torch):
    """The word-size comparison on the C2 ring (N = 2^16, 45 x 60-bit primes)
    and on the paper's own case (N = 2^17, Q about 2^1200: 20 x 60-bit primes)."""
    w = I.workload_c2()
    return {"c2_n65536": word_size(G, torch, w.N, w.primes, w.seed),
            "paper_n131072_q1200": word_size(G, torch, 1 << 17, I.chain_for(1 << 17, 20), 7)}


def single_limb_c1(G, torch, reps=500):
    """C1: one limb of N = 2^12, forward then inverse, one stream: the latency
    of the default one-pass kernel (one CTA per limb) and of the cluster kernel
    (one limb over a cluster of 8 CTAs), each as two calls and as one
    ntt_execute call (forward + inverse in one launch for the cluster plan)."""
    w = I.workload_c1()
    host = I.batch_uniform(w.seed, 1, w.primes, w.N)
    d = torch.from_numpy(host.view(np.int64).copy()).cuda()
    ref = d.clone()
    lib = G.lib()
    s = torch.cuda.Stream()
    both = G.NTT_OP_FORWARD | G.NTT_OP_INVERSE

    def timed(p, one_call):
        def step():
            if one_call:
                _ok(G, lib.ntt_execute(p.handle, d.data_ptr(), 1, both, s.cuda_stream), "C1 execute")
            else:
                _ok(G, lib.ntt_forward(p.handle, d.data_ptr(), 1, s.cuda_stream), "C1 forward")
                _ok(G, lib.ntt_inverse(p.handle, d.data_ptr(), 1, s.cuda_stream), "C1 inverse")
        for _ in range(10):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            step()
        e1.record(s)
        torch.cuda.synchronize()
        if not torch.equal(d, ref):
            raise RuntimeError("C1 round trip mismatch")
        return e0.elapsed_time(e1) * 1e3 / reps

    with G.Plan(w.N, w.primes) as p:
        one_pass = timed(p, False)
        one_pass_exec = timed(p, True)
    with G.Plan(w.N, w.primes, G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_CLUSTER) as p:
        clus = timed(p, False)
        clus_exec = timed(p, True)
        # the same one-launch steps replayed from a CUDA graph (no per-launch
        # submission gaps on the device)
        K = 100
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(K):
                _ok(G, lib.ntt_execute(p.handle, d.data_ptr(), 1, both, s.cuda_stream), "C1 execute (capture)")
        with torch.cuda.stream(s):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        with torch.cuda.stream(s):
            for _ in range(10):
                g.replay()
        e1.record(s)
        torch.cuda.synchronize()
        clus_graph = e0.elapsed_time(e1) * 1e3 / (10 * K)
        if not torch.equal(d, ref):
            raise RuntimeError("C1 round trip mismatch (graph)")
    return {"workload": "N=2^12, L=1, forward + inverse, one stream", "us_per_step": one_pass,
            "value": 2 / (one_pass / 1e6), "unit": "limb-NTT/s",
            "us_per_step_execute": one_pass_exec,
            "cluster": {"kernel": "one limb per cluster of 8 CTAs (NTT_KERNEL_CLUSTER)",
                        "us_per_step": clus, "us_per_step_execute_one_launch": clus_exec,
                        "us_per_step_execute_graph": clus_graph,
                        "value": 2 / (min(clus, clus_exec) / 1e6), "unit": "limb-NTT/s"},
            "timing": f"CUDA events around {reps} back-to-back steps on one stream"}


# Configurations the C2 leg times in its own setting (steps on several streams,
# plan clones) before the timed region: (organisation, twiddle supply, geometry,
# persistent CTAs per SM, streams).  The autotuner ranks configurations by one
# call at a time on one stream; with several streams the ranking changes (the
# per-pass launches of different streams interleave on the SMs).
C2_CANDIDATES = (
    ("fused", "ot1", 0, 1, 3), ("fused", "table", 0, 1, 3), ("fused", "ot1", 0, 0, 2),
    ("per_pass", "ot1", 1, 0, 2), ("per_pass", "ot2", 1, 0, 2), ("per_pass", "ot2", 1, 0, 3),
    ("per_pass", "ot1", 0, 0, 2), ("per_pass", "ot2", 0, 0, 2),
    ("per_pass", "table", 1, 0, 2), ("per_pass", "table", 1, 0, 3),
)
TWIDDLES = {"auto": (0, 0), "table": (1, 0), "ot1": (2, 1), "ot2": (2, 2)}


def prequeue(torch, ms):
    """Queue a device-side delay of about `ms` milliseconds on the current
    stream, before the start event of a timed region: the steps the host
    queues behind it are then waiting on the device when timing starts, so
    the timed region measures the device's throughput and not how fast the
    host issues the first launches.  Nothing of the method runs in it."""
    if ms > 0:
        torch.cuda._sleep(int(ms * 1e-3 * 2.0e9))


def select_c2(G, torch, N, primes, bufs, steps=400, warmup=20, prequeue_ms=0.0):
    """Time each C2 candidate configuration as the timed region runs it (the
    forward + inverse of one polynomial per step, steps spread over the
    candidate's streams, CUDA events around all steps) and return the fastest
    with the table of all."""
    kernels = {"fused": G.NTT_KERNEL_FUSED, "per_pass": G.NTT_KERNEL_PER_PASS}
    both = G.NTT_OP_FORWARD | G.NTT_OP_INVERSE
    lib = G.lib()
    L = len(primes)
    rows = []
    for kname, tw, geom, ctas, S in C2_CANDIDATES:
        if len(bufs) % S:
            raise ValueError("buffers must be a multiple of the streams (each buffer on one stream)")
        base = G.Plan(N, primes, *TWIDDLES[tw], kernels[kname], geom, ctas_per_sm=ctas)
        plans = [base] + [base.clone() for _ in range(S - 1)]
        ss = [torch.cuda.Stream() for _ in range(S)]
        hs = [p.handle for p in plans]

        def step(i):
            j = i % S
            _ok(G, lib.ntt_execute(hs[j], bufs[i % len(bufs)].data_ptr(), 1, both, ss[j].cuda_stream),
                "candidate step")
        for i in range(warmup):
            step(i)
        torch.cuda.synchronize()
        cur = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        prequeue(torch, prequeue_ms)
        e0.record(cur)
        for st in ss:
            st.wait_event(e0)
        for i in range(steps):
            step(i)
        for st in ss:
            e = torch.cuda.Event()
            e.record(st)
            cur.wait_event(e)
        e1.record(cur)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / (2 * steps)
        ok = all(p.device_status() == 0 for p in plans)
        for p in reversed(plans):
            p.close()
        rows.append({"kernel": kname, "twiddle": tw, "geometry": geom, "ctas_per_sm": ctas, "streams": S,
                     "us_per_transform": round(us, 2), "value": L / us * 1e6, "ok": ok})
    best = max((r for r in rows if r["ok"]), key=lambda r: r["value"])
    return best, {"how": f"{steps} steps of each candidate in the timed region's setting, CUDA events",
                  "candidates": rows}


def config_dict(w, args, ws):
    return {"workload": "c2_n65536_l45_fwd_inv", "N": w.N, "L": len(w.primes), "polys_per_step": 1,
            "primes": "45 largest primes < 2^60 with q = 1 mod 2^17", "seed": w.seed,
            "twiddle": args.twiddle, "parallelism": f"replicas{ws}",
            "streams": args.streams,
            "ctas_per_sm": args.ctas_per_sm,
            "overlap": "step i runs on stream i mod streams with its own plan (clones sharing one set of tables); "
                       "steps are independent polynomials; with one persistent CTA per SM per launch, "
                       "launches on different streams share the SMs",
            "l2": "inputs rotate over buffers totalling > 2x L2 (129 MB)",
            "prequeue_ms": getattr(args, "prequeue_ms", 0.0)}


# ----------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------
def main():
    args = parse()
    metric = "limb-NTT/s, N=2^16 L=45 forward+inverse (bit-exact)"
    unit = "limb-NTT/s"
    w = I.workload_c2()
    if args.traffic_json:
        write_traffic_json(args.traffic_json, args.traffic_csv, args.traffic_command)
        return
    if args.impl == "reference":
        run_reference(args, metric, unit, w)
        return

    import torch
    import paper_2012_01968_gb300 as G

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()
    G.lib()
    if args.only:
        leg = single_limb_c1(G, torch) if args.only == "c1" else batched_c4(G, torch, 10)
        if rank == 0:
            print(json.dumps({args.only: leg}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.int8_probe:
        if rank == 0:
            print(json.dumps({"int8_probe": int8_probe(torch)}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.ablation_only or args.word_size_only:
        if rank == 0:
            if args.ablation_only:
                out = {"paper_ablation": paper_ablation(G, torch, args.ablation_reps, (16, 17))}
            else:
                w2 = I.workload_c2()
                out = {"word_size": {"c2_n65536": word_size(G, torch, w2.N, w2.primes, w2.seed, args.ablation_reps)}}
            print(json.dumps(out), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    N, primes, L = w.N, w.primes, len(w.primes)
    mode = {"auto": (G.NTT_TWIDDLE_AUTO, 0), "table": (G.NTT_TWIDDLE_TABLE, 0),
            "ot1": (G.NTT_TWIDDLE_OT, 1), "ot2": (G.NTT_TWIDDLE_OT, 2)}[args.twiddle]
    kern = {"auto": G.NTT_KERNEL_AUTO, "fused": G.NTT_KERNEL_FUSED, "per_pass": G.NTT_KERNEL_PER_PASS}[args.kernel]
    S = max(1, args.streams)
    # one plan (tables + work area) per stream: steps on different streams are
    # independent polynomials and may overlap on the device
    c2_tune = c2_select = None
    l2f = G.NTT_PLAN_L2_TWIDDLES if args.l2_twiddles else 0
    poly_bytes = N * L * 8
    nbuf = max(2 * max(S, 3), -(-2 * L2_BYTES // poly_bytes) + 1)
    # step i uses buffer i mod nbuf on stream i mod S: with nbuf a multiple of
    # every stream count in use (S, and the 2 and 3 of the selection's
    # candidates), each buffer stays on one stream, so no two steps in flight
    # on different streams share an array
    m = math.lcm(6, S)
    nbuf = -(-nbuf // m) * m
    host = I.batch_uniform(w.seed, 1, primes, N)
    src = torch.from_numpy(host.view(np.int64).copy()).cuda()
    bufs = [src.clone() for _ in range(nbuf)]
    tuned_run = not args.no_tune and args.twiddle == "auto" and args.kernel == "auto" and args.geometry == 0
    if tuned_run:
        best, c2_tune = autotune(G, N, primes, 1, reps=20)
    if tuned_run and not args.no_select:
        chosen, c2_select = select_c2(G, torch, N, primes, bufs, prequeue_ms=args.prequeue_ms)
        # replicas: every rank times the candidates on its own GPU, and all
        # run rank 0's choice, so that the ranks' steps are the same work
        chosen = agree_on_rank0(chosen, dist)
        args.streams = S = chosen["streams"]
        args.ctas_per_sm = chosen["ctas_per_sm"]
        kern = {"fused": G.NTT_KERNEL_FUSED, "per_pass": G.NTT_KERNEL_PER_PASS}[chosen["kernel"]]
        plans = [G.Plan(N, primes, *TWIDDLES[chosen["twiddle"]], kern, chosen["geometry"], flags=l2f,
                        ctas_per_sm=args.ctas_per_sm)]
        for b in bufs:
            if not torch.equal(b, src):
                raise RuntimeError("round trip mismatch in the configuration selection")
    elif tuned_run:
        plans = [G.Plan.from_opts(N, primes, best, flags=l2f or None, ctas_per_sm=args.ctas_per_sm)]
    else:
        plans = [G.Plan(N, primes, *mode, kern, args.geometry, flags=l2f, ctas_per_sm=args.ctas_per_sm)]
    # the other streams' plans share the first plan's tables (ntt_plan_clone)
    plans += [plans[0].clone() for _ in range(S - 1)]
    plan = plans[0]
    info = plan.info()
    streams = [torch.cuda.Stream() for _ in range(S)]
    lib = G.lib()
    handles = [p.handle for p in plans]

    both = G.NTT_OP_FORWARD | G.NTT_OP_INVERSE

    def step(i):
        j = i % S
        b = bufs[i % nbuf].data_ptr()
        sh = streams[j].cuda_stream
        if args.split_calls:
            bad = lib.ntt_forward(handles[j], b, 1, sh) or lib.ntt_inverse(handles[j], b, 1, sh)
        else:
            bad = lib.ntt_execute(handles[j], b, 1, both, sh)
        if bad:
            raise RuntimeError("launch failed: " + G.ntt_last_cuda_error())

    for i in range(max(args.warmup, S)):
        step(i)
    torch.cuda.synchronize()
    # correctness of the timed path: forward + inverse restores the input
    for b in bufs:
        if not torch.equal(b, src):
            raise RuntimeError("round trip mismatch before timing")

    K = args.steps
    cur = torch.cuda.current_stream()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(dev_index)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.15)
    prequeue(torch, args.prequeue_ms)
    e_start.record(cur)
    for st in streams:
        st.wait_event(e_start)
    for i in range(K):
        step(i)
    for st in streams:
        e = torch.cuda.Event()
        e.record(st)
        cur.wait_event(e)
    e_end.record(cur)
    torch.cuda.synchronize()
    clocks = clk.stop()
    if dist is not None:
        dist.barrier()
    total_ms = max_over_ranks(e_start.elapsed_time(e_end), dist, "cuda")
    for b in bufs:
        if not torch.equal(b, src):
            raise RuntimeError("round trip mismatch after timing")
    for p in plans:
        if p.device_status() != 0:
            raise RuntimeError("device status reports a failed bounded wait")
    value = whole_job_value(L, K, ws, total_ms)

    # per-launch durations, one stream, CUDA events around every call
    # (launches do not overlap here): the separate forward and inverse calls,
    # and the one-launch forward + inverse call.  A clone of the timed plan
    # with as many CTAs per SM as fit: the launch configuration for a stream
    # that runs alone (the same kernel as the timed steps)
    Kp = min(K, args.launch_steps)
    s0 = streams[0]
    solo = plans[0].clone()
    solo.set_ctas_per_sm(0)
    handles = [solo.handle] + handles[1:]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * Kp + 1)]
    evc = [torch.cuda.Event(enable_timing=True) for _ in range(Kp + 1)]
    torch.cuda.synchronize()
    with torch.cuda.stream(s0):
        ev[0].record(s0)
        for i in range(Kp):
            b = bufs[i % nbuf].data_ptr()
            _ok(G, lib.ntt_forward(handles[0], b, 1, s0.cuda_stream), "forward")
            ev[2 * i + 1].record(s0)
            _ok(G, lib.ntt_inverse(handles[0], b, 1, s0.cuda_stream), "inverse")
            ev[2 * i + 2].record(s0)
        evc[0].record(s0)
        for i in range(Kp):
            _ok(G, lib.ntt_execute(handles[0], bufs[i % nbuf].data_ptr(), 1, both, s0.cuda_stream), "execute")
            evc[i + 1].record(s0)
    torch.cuda.synchronize()
    fwd_ms = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(Kp)]
    inv_ms = [ev[2 * i + 1].elapsed_time(ev[2 * i + 2]) for i in range(Kp)]
    chain_ms = [evc[i].elapsed_time(evc[i + 1]) for i in range(Kp)]
    single_ms = ev[0].elapsed_time(ev[2 * Kp]) / Kp

    peak, peak_src = measured_peak_hbm()
    fwd_avg = float(np.mean(fwd_ms))
    inv_avg = float(np.mean(inv_ms))
    chain_avg = float(np.mean(chain_ms))
    chained = info.kernel == G.NTT_KERNEL_FUSED and info.passes == 2
    bfly_per_transform = L * (N // 2) * (N.bit_length() - 1)      # (N/2) log2 N butterflies per limb
    per_pass_step = info.kernel == G.NTT_KERNEL_PER_PASS and info.passes == 2 and not args.split_calls
    if chained and not args.split_calls:
        # the timed steps' launch: forward + inverse of the polynomial
        dom_name, dom_ms, per_launch = "ntt_execute (forward + inverse, 1 fused launch)", chain_avg, 2
    elif per_pass_step:
        # the timed steps' call: forward + inverse as four pass launches (the
        # inverse's passes read the forward's output, mostly from L2, so the
        # unit is the whole call)
        dom_name, dom_ms, per_launch = "ntt_execute (forward + inverse, 4 pass launches)", chain_avg, 2
    else:
        dom_name, dom_ms = ("ntt_forward", fwd_avg) if fwd_avg >= inv_avg else ("ntt_inverse", inv_avg)
        per_launch = 1
    alg_bytes = 2 * poly_bytes * per_launch          # one read + one write per transform
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9
    bfly_per_launch = bfly_per_transform * per_launch
    bfly_achieved = bfly_per_launch / (dom_ms / 1e3) / 1e9
    step_bytes = 4 * poly_bytes                      # forward + inverse, each one read + one write
    frac_step = (step_bytes * K / (total_ms / 1e3) / 1e9) / peak

    # end to end through the host-buffer C ABI call (pinned host memory)
    e2e = None
    if True:
        hin = torch.from_numpy(host.view(np.int64).copy()).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        ops = G.NTT_OP_FORWARD | G.NTT_OP_INVERSE
        for _ in range(3):
            G.ntt_execute_host(handles[0], hin, hout, 1, ops, streams[0])
        E = args.e2e_steps
        # the asynchronous call on two alternating streams: consecutive steps
        # overlap (one step's copy-in with the previous step's transforms and
        # copy-out); every step still copies its input in and its result out
        alt = [torch.cuda.Stream(), torch.cuda.Stream()]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(E):
            G.ntt_execute_host_async(handles[0], hin, hout, 1, ops, alt[k % 2])
        for a_s in alt:
            a_s.synchronize()
        el = time.perf_counter() - t0
        if not torch.equal(hout, hin):
            raise RuntimeError("e2e round trip mismatch")
        # the synchronous call, each step waiting for its result
        t0 = time.perf_counter()
        for _ in range(E):
            G.ntt_execute_host(handles[0], hin, hout, 1, ops, streams[0])
        el_sync = time.perf_counter() - t0
        if not torch.equal(hout, hin):
            raise RuntimeError("e2e round trip mismatch")
        e2e = {"value": 2 * L * E / el, "unit": unit, "h2d_bytes_per_step": poly_bytes,
               "d2h_bytes_per_step": poly_bytes, "steps": E, "call": "ntt_execute_host_async on two alternating streams, then one sync",
               "synchronous_call_value": 2 * L * E / el_sync}
        link = host_link_rates(torch, hin, hout)
        # a step needs its input in and its result out: with both directions
        # overlapped at best, the link alone takes max(in, out, both) per step
        t_link = max(poly_bytes / link["h2d_gbs"], poly_bytes / link["d2h_gbs"],
                     2 * poly_bytes / link["both_gbs"]) / 1e9
        e2e["host_link"] = dict(link, step_floor_us=t_link * 1e6, value_bound=2 * L / t_link,
                                frac_of_bound=(2 * L * E / el) / (2 * L / t_link))

    per_limb = batched = None
    chain = I.chain_2_18_60()
    tuned = {}
    if ws == 1 and not (args.no_batch_compare and args.no_serve) and not args.no_tune:
        # the uneven-batch and serving sizes, tuned at 60 limbs x a few polynomials per launch
        tuned = {n: autotune(G, 1 << n, chain, 6) for n in range(14, 18)}
    if ws == 1 and not args.no_batch_compare:
        per_limb = per_limb_c2(G, torch, w, host, 100)
        batched = batched_c4(G, torch, 10)
        if tuned:
            batched["autotuned"] = batched_c4(G, torch, 10, {n: t[0] for n, t in tuned.items()})
            batched["autotune"] = {f"N=2^{n}": t[1] for n, t in tuned.items()}
        # every size on the per-pass organisation (OT2, smaller row tiles): the
        # jobs' pass launches interleave on the batch's internal streams
        batched["per_pass_plans"] = batched_c4(G, torch, 10, plan_kw=PER_PASS_KW(G))
    large = modes = c1 = words = None
    if ws == 1 and not args.no_batch_compare:
        w3 = I.workload_c3()
        large = large_ring_c3(G, torch)
        if not args.no_tune:
            o3, r3 = autotune(G, w3.N, w3.primes, 2)
            large["autotuned"] = large_ring_c3(G, torch, opts=o3)
            large["autotune"] = r3
        modes = twiddle_modes_c2(G, torch, w, bufs, nbuf)
        c1 = single_limb_c1(G, torch)
        words = word_sizes(G, torch)
    ablation = None
    if ws == 1 and not args.no_ablation:
        ablation = paper_ablation(G, torch)
    served = None
    if ws == 1 and not args.no_serve:
        served = serve_c5(G, torch, args.serve_requests)
        if tuned:
            served["autotuned"] = serve_c5(G, torch, args.serve_requests,
                                           tuned={n: t[0] for n, t in tuned.items()})
        # every size on per-pass plans: a served batch's jobs then run as pass
        # launches interleaved on the batch's internal streams (capacity, and
        # the three loads three times)
        served["per_pass_plans"] = serve_c5(G, torch, args.serve_requests, repeats=3, plan_kw=PER_PASS_KW(G))

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        v, cores, sample = oracle_time(primes, N, 10.0)
        cpu = {"value": v, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample}
        # the other views of the same baseline: one host thread, and the large ring (C3)
        v1, _, s1 = oracle_time(primes, N, 5.0, threads=1)
        w3 = I.workload_c3()
        v3, c3, s3 = oracle_time(w3.primes, w3.N, 5.0, batch=2)
        cpu["single_thread"] = {"value": v1, "unit": unit, "cores": 1, "sample": s1}
        cpu["large_ring_c3"] = {"value": v3, "unit": unit, "cores": c3, "sample": s3}
    twname = "table" if info.twiddle_mode == G.NTT_TWIDDLE_TABLE else f"ot{int(info.ot_stages)}"
    kname = dom_name if per_launch == 2 else \
        f"{dom_name} ({'1 fused launch' if info.kernel == G.NTT_KERNEL_FUSED else str(info.passes) + ' pass launches'})"
    direction = "forward+inverse" if per_launch == 2 else ("forward" if dom_name == "ntt_forward" else "inverse")
    kind = {G.NTT_KERNEL_FUSED: "fused", G.NTT_KERNEL_PER_PASS: "per_pass"}.get(int(info.kernel))
    if per_pass_step:
        # the forward call's and the inverse call's entries together
        pf = profile_traffic(kind, int(info.geometry), twname, "forward")
        pv = profile_traffic(kind, int(info.geometry), twname, "inverse")
        prof = None if not (pf and pv) else {
            k: pf[k] + pv[k] for k in ("dram_read_bytes", "dram_write_bytes", "dram_bytes", "twiddle_read_bytes")}
        if prof:
            prof["data_read_bytes"] = prof["dram_read_bytes"] - prof["twiddle_read_bytes"]
            prof["how"] = pf["how"] + "; the step's forward call and inverse call summed"
    else:
        prof = profile_traffic(kind, int(info.geometry), twname, direction) if kind else None
    traffic = prof["dram_bytes"] if prof else None
    line = {
        "metric": metric, "value": value, "unit": unit, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": config_dict(w, args, ws),
        "hbm_roofline_frac_step": frac_step,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_split": None if not prof else {
                         k: prof[k] for k in ("dram_read_bytes", "dram_write_bytes", "data_read_bytes",
                                              "twiddle_read_bytes", "how") if k in prof},
                     "kernel": kname,
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_us": dom_ms * 1e3,
                     "units_per_launch": f"{per_launch * L} limb-NTTs of N={N} (16 N bytes each: one read, one write)"
                                         + ("" if info.kernel == G.NTT_KERNEL_FUSED else
                                            "; one ntt_execute call of 4 pass launches" if per_pass_step else
                                            f"; per call of {int(info.passes)} pass launches"),
                     "launch_timing": f"CUDA events around each of {Kp} calls on one stream (a clone of the timed plan"
                                      " with as many CTAs per SM as fit)",
                     "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src},
        "roofline_alu": {"bound": "alu", "achieved": bfly_achieved, "peak": alu_peak_gbfly(),
                         "unit": "G butterfly/s", "frac": bfly_achieved / alu_peak_gbfly(),
                         "kernel": kname,
                         "units_per_launch": f"{bfly_per_launch} butterflies ({per_launch * L} limb-NTTs x (N/2) log2 N)",
                         "avg_launch_us": dom_ms * 1e3,
                         "peak_source": "152 SMs x 2070 MHz x 4.57 butterflies per SM-clock (FMA-heavy pipe: "
                                        "2 IMAD.HI + 3 IMAD.WIDE at 4 cycles and 4 IMAD at 2 cycles per warp butterfly)",
                         "peak_measured": None if args.no_peak_measure else G.ntt_measure_butterfly_rate(),
                         "peak_measured_source": "ntt_measure_butterfly_rate: register-only butterfly loop, live",
                         "timed_region_frac": bfly_per_transform * 2 * K / (total_ms / 1e3) / 1e9 / alu_peak_gbfly()},
        "per_transform_us": {"forward": fwd_avg * 1e3, "inverse": inv_avg * 1e3,
                             "forward_plus_inverse_one_launch": chain_avg * 1e3,
                             "timed_region_per_transform": total_ms * 1e3 / (2 * K),
                             "single_stream_per_transform": single_ms * 1e3 / 2,
                             "single_stream_per_transform_one_launch": chain_avg * 1e3 / 2},
        "step_call": "ntt_forward + ntt_inverse" if args.split_calls else "ntt_execute(FORWARD | INVERSE)",
        "plan": {"twiddle_mode": int(info.twiddle_mode), "ot_stages": int(info.ot_stages),
                 "passes": int(info.passes), "pass1_log2": int(info.pass1_log2),
                 "row_tile_log2": int(info.row_tile_log2), "geometry": int(info.geometry),
                 "kernel": KERNEL_NAMES[int(info.kernel)],
                 "chosen_by": ("timed candidates in the timed setting (select_c2)" if c2_select else
                               "ntt_autotune" if c2_tune else "fixed options")},
        "autotune_c2": c2_tune,
        "select_c2": c2_select,
        "e2e": e2e,
        "per_limb_path": per_limb,
        "batched_uneven_c4": batched,
        "served_c5": served,
        "paper_ablation": ablation,
        "large_ring_c3": large,
        "twiddle_modes_c2": modes,
        "single_limb_c1": c1,
        "word_size": words,
        "gpu_launches": K * (1 if chained and not args.split_calls else
                             2 * (1 if info.kernel == G.NTT_KERNEL_FUSED else int(info.passes))),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    for p in plans:
        p.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
