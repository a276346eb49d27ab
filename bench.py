"""Throughput of the two-stage JSON parse on GB300 (one JSON line on stdout).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload config2|config1|config0]

A step is one whole parse (setup, stage 1, stage 2, finalize kernels and the
result header copy) of one synthetic document that already sits in HBM.  The
default workload is the 1 GiB single document (records in a root array, ~26%
non-ASCII bytes in string values, escape runs across block and tile edges, 1%
of records nested to depth 1024): larger than L2, so no flush is needed between steps.

`value` is whole-job input GB/s over K steps timed with CUDA events on the
launching stream (max over ranks); a step is one run as sj_parse performs it
(the captured graph).  `stage_ms` comes from K more steps with CUDA events
recorded between the stages (direct launches, one stage at a time).  `e2e` is the same metric through sj_parse
with a pinned host buffer (host-to-device copy inside every step, result
header read back; the median of three repetitions of up to 10 steps, all
three listed); a document larger than the parser's largest chunk is copied
in chunks on a second stream while the kernels parse the chunks that have
landed.  `roofline` reports the algorithmic bytes of the whole parse (input,
indices, tape, string buffer) over the step time against the measured HBM
copy bandwidth, with each kernel's share under `roofline.kernels`; `cpu_baseline` times the CPU oracle on a bounded
sample of the same workload on this host's cores.

Two more objects ride on the same line: `batch` (the 100,000-document batch
of config3 in one graph-launched run, against the same documents parsed one
per launch) and `serving` (the config4 arrival trace replayed against the
continuous-batching server: docs/s, GB/s, p50/p99 latency).

--impl reference times the CPU oracle itself (the only reference that exists
for this workload) on a bounded sample per step.

N > 1 (torchrun): every rank parses its own document of the same size
(independent replicas, weak scaling); only the timing uses the process group.
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

WORKLOADS = {
    "config2": ("1 GiB single document: root array of config-0 style records, ~26% non-ASCII "
                "bytes in string values (14% of all string bytes), \\u surrogate pairs, escape runs on 64 B / 2 KiB / 128 KiB edges, "
                "1% of records nested to depth 1024", 1 << 30),
    "config1": ("2.5 MB number-heavy single document (polygons of [lon,lat] pairs, 15-17 "
                "significant digits, minimal white space)", 2_500_000),
    "config0": ("64 KB record document, 2-space pretty printing", 65536),
}


def make_doc(workload: str, seed: int, size: int | None = None) -> np.ndarray:
    import gen
    if workload == "config2":
        return gen.config2(seed, size=size or (1 << 30))
    if workload == "config1":
        return gen.config1(seed)
    return gen.config0(seed)


def record_prefix(doc: np.ndarray, nbytes: int) -> bytes:
    """The first whole records of a config-2 document, closed into a valid array."""
    b = doc[: nbytes].tobytes()
    cut = b.rfind(b"\n  },\n  {")
    if cut < 0:
        return doc.tobytes()
    return b[: cut + 4] + b"\n]\n"


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# The files that define each profiled kernel; host-side code (api.cu,
# server.cpp, the query and the allocation-free entry) does not change their
# DRAM traffic, and neither does a change to another stage's kernel.
_S1 = ("s1.cu", "s1_common.cuh", "sj_internal.cuh")
_S2 = ("s2.cu", "strings.cuh", "number.cuh", "pow5_table.h", "sj_internal.cuh")
KERNEL_SOURCES = {"s1_blocks": _S1, "s1_flatten": _S1, "s2_reduce": _S2, "s2_numbers": _S2,
                  "s2_build": _S2}


def source_hash(kernel: str, read=None) -> str:
    """Hash of the sources of one kernel (`read(name)` gives a file's bytes;
    by default the working tree)."""
    csrc = os.path.join(ROOT, "paper_1902_08318_gb300", "csrc")
    if read is None:
        def read(name):
            with open(os.path.join(csrc, name), "rb") as f:
                return f.read()
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        h.update(name.encode() + read(name))
    return h.hexdigest()[:16]


# Every source that defines a kernel of the parse (for the whole-parse figure).
_ALL = ("s1.cu", "s1_common.cuh", "scan.cu", "s2.cu", "strings.cuh", "number.cuh", "pow5_table.h",
        "sj_internal.cuh")
KERNEL_SOURCES["whole_parse"] = _ALL
NCU_DOC_BYTES = 1073742825  # the document the committed capture was taken on


def ncu_traffic(kernel: str):
    """DRAM bytes per launch (or per whole parse) of the 1 GiB benchmark
    document from the committed ncu capture, if it was taken on the current
    sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p) or kernel not in KERNEL_SOURCES:
        return None
    with open(p) as f:
        d = json.load(f)
    ent = d.get("whole_parse") if kernel == "whole_parse" else d.get("kernels", {}).get(kernel)
    if not ent or "bytes" not in ent or ent.get("source_hash") != source_hash(kernel):
        return None
    return ent["bytes"]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self, gpu_index: int = 0) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != gpu_index:
                    continue
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def lexeme_bytes(doc_dev, idx_dev) -> tuple[int, int]:
    """Input bytes of the string, number and atom lexemes (read by stage 2),
    and the number of number tokens."""
    import torch
    x = doc_dev
    n = idx_dev.numel()
    pos = idx_dev.to(torch.int64)
    first = x[pos]
    is_val = (first == ord('"')) | (first == ord("t")) | (first == ord("f")) | (first == ord("n")) | \
        (first == ord("-")) | ((first >= ord("0")) & (first <= ord("9")))
    nxt = torch.empty_like(pos)
    nxt[:-1] = pos[1:]
    nxt[-1] = x.numel()
    q = (nxt - 1)[is_val]
    p0 = pos[is_val]
    for _ in range(64):  # step back over white space before the next token
        c = x[q]
        ws = (c == 32) | (c == 9) | (c == 10) | (c == 13)
        if not bool(ws.any()):
            break
        q = q - ws.to(torch.int64)
    del n
    nums = (first == ord("-")) | ((first >= ord("0")) & (first <= ord("9")))
    return int((q - p0 + 1).sum().item()), int(nums.sum().item())


def run_ours(args, rank: int, world: int, dist) -> dict | None:
    import torch

    import paper_1902_08318_gb300 as sj

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    desc, size = WORKLOADS[args.workload]
    doc = make_doc(args.workload, 2000 + rank, size=(args.doc_mb << 20) if args.doc_mb else None)
    if args.doc_mb and args.workload == "config2":  # a smaller document of the same recipe
        desc = desc.replace("1 GiB single document", f"{args.doc_mb} MiB single document")
    B = int(doc.size)
    doc_dev = torch.from_numpy(doc).to(dev)
    parser = sj.Parser(max_bytes=B + 64)
    stream = torch.cuda.current_stream()

    # correctness gate on the benchmarked input (error code only; the
    # element-by-element parity lives in the gpu tests)
    r = parser.parse(doc_dev, stream=stream)
    if r.error != 0:
        raise SystemExit(f"benchmark document rejected: {r.error_name}")
    S, T, SB = r.n_indices, r.tape_words, r.string_bytes
    lex, nnum = lexeme_bytes(doc_dev, r.indices()[: S])
    # launch shapes: the autotuner times each main kernel at every allowed
    # shape on this document (outside the timed region)
    tuned = None if args.no_autotune else parser.autotune(doc_dev, stream=stream)
    launch = parser.launch()

    # ---- device-timed region: the captured graph of a run, as sj_parse runs it
    for _ in range(args.warmup):
        parser.parse_async(doc_dev, stream=stream)
    parser.parse_wait()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        parser.parse_async(doc_dev, stream=stream)
    parser.parse_wait()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)

    # ---- per-stage durations: the same steps again with CUDA events between
    # the stages (direct launches, each stage alone; the numbers kernel then
    # runs after the frontier instead of beside it)
    parser.set_profiling(True)
    parser.parse_async(doc_dev, stream=stream)
    parser.parse_wait()
    stage_sum = {k: 0.0 for k in sj.STAGES}
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        parser.parse_async(doc_dev, stream=stream)
        for k, v in parser.stage_times().items():  # waits for this step
            stage_sum[k] += v
    p1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop(dev.index)
    ms_profiled = p0.elapsed_time(p1) / args.steps
    if dist:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    stage_ms = {k: v / args.steps for k, v in stage_sum.items()}

    # ---- end to end through sj_parse from pinned host memory ------------------
    parser.set_profiling(False)
    e2e_reps = []
    if args.no_e2e:
        ms_e2e, e2e_steps = float("nan"), 1
    else:
        ms_e2e, e2e_steps, e2e_reps = e2e_leg(parser, doc, stream, args, dev, dist)
    if rank != 0:
        return None
    out = report(args, world, desc, B, S, T, SB, lex, nnum, ms_step, stage_ms, ms_e2e, e2e_steps,
                 clk, parser.kernels_per_run())
    out["ms_per_step_profiled"] = round(ms_profiled, 4)
    if e2e_reps:
        out["e2e"]["ms_per_step_repetitions"] = e2e_reps
    out["launch"] = {"blocks_per_sm": {k: c for k, (c, _) in launch.items()},
                     "max_blocks_per_sm": {k: m for k, (_, m) in launch.items()},
                     "autotuned": tuned is not None}
    return out


def e2e_leg(parser, doc, stream, args, dev, dist):
    """The same parse through sj_parse from pinned host memory: three
    repetitions of up to 10 synchronous steps; the median repetition is
    reported and all three are listed (a host stall while the launches of a
    chunked run are queued shows up in one repetition, not in the others)."""
    import torch
    host = torch.from_numpy(doc).pin_memory()
    for _ in range(max(1, args.warmup // 2)):
        parser.parse(host, stream=stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_steps = max(1, min(args.steps, 10))
    reps = []
    for _ in range(3):
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(e2e_steps):
            rr = parser.parse(host, stream=stream)
            assert rr.error == 0
        f1.record(stream)
        torch.cuda.synchronize()
        ms = f0.elapsed_time(f1)
        if dist:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        reps.append(ms)
    return sorted(reps)[1], e2e_steps, [round(r / e2e_steps, 4) for r in reps]


def report(args, world, desc, B, S, T, SB, lex, nnum, ms_step, stage_ms, ms_e2e, e2e_steps, clk,
           kernels_per_run):
    peaks = load_peaks()
    gbs = world * B / (ms_step * 1e-3) / 1e9
    e2e = world * B / (ms_e2e / e2e_steps * 1e-3) / 1e9
    # algorithmic bytes of the parse: the input read once and the outputs the
    # method must produce -- indices, tape, string buffer.  Each kernel's
    # share is what it must read or write of that (re-reads of the input or
    # of the indices, and intermediate arrays, are overhead).
    algo_path = B + 4 * S + 8 * T + SB
    algo = {"setup": 0, "s1_blocks": B, "s1_scan": 0, "s1_flatten": 4 * S, "s2_reduce": 0,
            "s2_scan_frontier": 0, "s2_numbers": 16 * nnum, "s2_build": 8 * (T - 2 * nnum) + SB,
            "finalize": 0}
    dom = max(stage_ms, key=lambda k: stage_ms[k])
    kernels = {}
    for k, ms in stage_ms.items():
        ent = {"ms": round(ms, 4), "algorithmic_bytes": algo.get(k, 0)}
        if ms > 0 and algo.get(k, 0):
            ach = algo[k] / (ms * 1e-3) / 1e9
            ent["achieved"] = round(ach, 1)
            ent["frac"] = round(ach / peaks["hbm_gbs"], 4)
        if k in KERNEL_SOURCES:
            tr = ncu_traffic(k)
            ent["traffic"] = None if tr is None else int(tr * B / NCU_DOC_BYTES)
        kernels[k] = ent
    whole = ncu_traffic("whole_parse")
    traffic = None if whole is None else int(whole * B / NCU_DOC_BYTES)
    achieved = algo_path / (ms_step * 1e-3) / 1e9
    out = {
        "metric": "parse GB/s (input bytes, device-timed)",
        "value": round(gbs, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "bytes_per_doc": B,
                   "indices": S, "tape_words": T, "string_bytes": SB, "number_tokens": nnum,
                   "lexeme_bytes": lex,
                   "l2": "inputs larger than L2 (no flush)" if B > 129e6 else "L2 not flushed",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm",
                     "kernel": "whole parse: algorithmic bytes B + 4S + 8T + SB over the step time",
                     "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": round(achieved / peaks["hbm_gbs"], 4),
                     "traffic": traffic,
                     "traffic_note": "DRAM bytes (read + write) of all 20 launches of one parse, "
                                     "from the committed one-pass ncu capture on this 1 GiB "
                                     "document (profiles/ncu_traffic.json; scaled by input bytes "
                                     "for another size); null when a kernel source changed since",
                     "algorithmic_bytes": algo_path,
                     "input_frac": round(B / (ms_step * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                     "dominant": dom, "kernels": kernels,
                     "peak_source": peaks["source"]},
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "e2e": {"value": round(e2e, 3) if e2e == e2e else None, "unit": "GB/s",
                "h2d_bytes_per_step": B, "d2h_bytes_per_step": 56,
                "path": ("pinned host document copied in chunks (first 32 MiB, growing by 7/4 up to "
                         "512 MiB) on a copy stream; stage 1 of each landed chunk on a second "
                         "stream, stage 2 on the run's stream as far as the landed chunks allow"
                         if B > (512 << 20) else
                         "pinned host document read by stage 1 over the host link")},
        "gpu_launches": kernels_per_run * args.steps,
        "clocks": clk,
    }
    return out


def pct(x, q) -> float:
    return float(np.percentile(np.asarray(x), q))


def batch_leg(args, dev) -> dict:
    """Batched: the 100,000-document batch (config3) in one graph-launched run,
    against the same documents parsed one per launch."""
    import torch

    import gen
    import paper_1902_08318_gb300 as sj
    buf, off = gen.config3()
    n = off.size - 1
    total = int(off[-1])
    buf_dev = torch.from_numpy(np.require(buf, requirements=["W"])).to(dev)
    p = sj.Parser(max_bytes=total + 64, max_docs=n)
    res, _ = p.parse_batch(buf_dev, off)
    for _ in range(args.warmup):
        p.parse_batch(buf_dev, off)
    torch.cuda.synchronize()
    k = max(3, min(args.steps, 10))
    lat = []
    for _ in range(k):
        t0 = time.perf_counter()
        p.parse_batch(buf_dev, off)  # waits for the run and its result copy
        lat.append(time.perf_counter() - t0)
    dt = sum(lat)
    # one document per launch (sj_parse), on the first documents of the batch
    single = sj.Parser(max_bytes=(1 << 20) + 64)
    m = min(n, 5000)
    for i in range(50):
        single.parse(buf_dev[int(off[i]): int(off[i + 1])])
    torch.cuda.synchronize()
    one = []
    t_all = time.perf_counter()
    for i in range(m):
        t0 = time.perf_counter()
        single.parse(buf_dev[int(off[i]): int(off[i + 1])])
        one.append(time.perf_counter() - t0)
    t_all = time.perf_counter() - t_all
    return {
        "workload": "config3: 100,000 documents of the config-0 generator, log-normal sizes "
                    "(median 2 KB, sigma 1.5, 100 B - 1 MB), 1% with one defect",
        "docs": n, "bytes": total, "invalid_docs": int(np.count_nonzero(res["error"])),
        "batched": {"docs_per_s": round(n * k / dt, 1), "GB_per_s": round(total * k / dt / 1e9, 2),
                    "ms_per_batch": round(dt / k * 1e3, 3),
                    "latency_ms_p50": round(pct(lat, 50) * 1e3, 3),
                    "latency_ms_p99": round(pct(lat, 99) * 1e3, 3),
                    "launches_per_batch": p.kernels_per_run(), "steps": k},
        "one_per_launch": {"docs": m, "docs_per_s": round(m / t_all, 1),
                           "GB_per_s": round(int(off[m]) / t_all / 1e9, 3),
                           "latency_ms_p50": round(pct(one, 50) * 1e3, 4),
                           "latency_ms_p99": round(pct(one, 99) * 1e3, 4)},
        "timing": "host clock around each synchronous call (batch: all 100,000 results ready)",
    }


def small_doc_leg(args, dev) -> dict:
    """The 2.5 MB number-heavy document (config1) and the 64 KB record document
    (config0), parsed from HBM through sj_parse (the captured graph, waited
    for): per-parse latency on the host clock, and the input bytes per second
    that one parse after another achieves."""
    import torch

    import gen
    import paper_1902_08318_gb300 as sj
    out = {}
    for name, doc in (("config1", gen.config1(1000)), ("config0", gen.config0(0))):
        d = torch.from_numpy(np.require(doc, requirements=["W"])).to(dev)
        p = sj.Parser(max_bytes=int(doc.size) + 64)
        stream = torch.cuda.current_stream()
        for _ in range(20):
            r = p.parse(d, stream=stream)
        assert r.error == 0, r.error_name
        lat = []
        for _ in range(300):
            t0 = time.perf_counter()
            p.parse(d, stream=stream)
            lat.append(time.perf_counter() - t0)
        out[name] = {"bytes": int(doc.size), "latency_ms_p50": round(pct(lat, 50) * 1e3, 4),
                     "latency_ms_p99": round(pct(lat, 99) * 1e3, 4),
                     "GB_per_s_at_p50": round(doc.size / pct(lat, 50) / 1e9, 2), "parses": len(lat),
                     "kernels_per_parse": p.kernels_per_run()}
    out["timing"] = "host clock around each synchronous sj_parse (graph launch, result header read back)"
    return out


def query_leg(args, dev) -> dict:
    """The paper's tape query (Table "tab:userid"): parse a twitter-like
    document and select the distinct user.id values from its device tape."""
    import torch

    import gen
    import paper_1902_08318_gb300 as sj
    doc = gen.tweets(4100, 256 << 20, 200_000)
    B = int(doc.size)
    d = torch.from_numpy(np.require(doc, requirements=["W"])).to(dev)
    p = sj.Parser(max_bytes=B + 64)
    q = sj.Query(1 << 20)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        r = p.parse(d, stream=stream)
        vals = q.distinct(r, ("user", "id"), stream=stream)
    torch.cuda.synchronize()
    k = max(3, min(args.steps, 10))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_parse = t_query = 0.0
    for _ in range(k):
        ev[0].record(stream)
        r = p.parse(d, stream=stream)
        ev[1].record(stream)
        vals = q.distinct(r, ("user", "id"), stream=stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
        t_parse += ev[0].elapsed_time(ev[1])
        t_query += ev[1].elapsed_time(ev[2])
    t_parse /= k
    t_query /= k
    return {"workload": f"twitter-like document ({B} bytes, statuses with nested user objects, "
                        "200,000 user ids), distinct user.id",
            "distinct_values": int(vals.numel()),
            "parse_GB_per_s": round(B / (t_parse * 1e-3) / 1e9, 2),
            "query_GB_per_s": round(B / (t_query * 1e-3) / 1e9, 2),
            "parse_and_query_GB_per_s": round(B / ((t_parse + t_query) * 1e-3) / 1e9, 2),
            "ms_parse": round(t_parse, 4), "ms_query": round(t_query, 4), "steps": k}


def serving_leg(args) -> dict:
    """Serving (config4): the arrival trace replayed natively against the
    continuous-batching server (latency = result seen minus arrival).  The
    timed replay runs three times; the line reports the run with the median
    p99 and lists every run's p50, p99 and maximum (the host is shared: a
    replay now and then meets a stall of the polling thread)."""
    import gen
    import paper_1902_08318_gb300 as sj
    arrival, buf, off = gen.config4(workers=max(1, min(16, os.cpu_count() or 1)))
    n = arrival.size
    srv = sj.Server(max_batch_bytes=16 << 20, max_batch_docs=4096, max_slots=8,
                    mem_budget=8 << 30)
    # warm-up: a slice of the trace (the graphs of every batch size are
    # captured when the server is created)
    w = 20_000
    srv.replay(buf, off[: w + 1], arrival[:w] - arrival[0])
    runs = []
    for _ in range(3):
        b0 = srv.batches
        lat, wall = srv.replay(buf, off, arrival)
        runs.append({"p50": pct(lat, 50) * 1e3, "p99": pct(lat, 99) * 1e3,
                     "max": float(lat.max()) * 1e3, "wall": wall, "batches": srv.batches - b0})
    med = sorted(runs, key=lambda r: r["p99"])[1]
    wall, batches = med["wall"], med["batches"]
    capacity = serving_capacity(srv, buf, off, arrival)
    return {
        "workload": "config4: 200,000 requests, Poisson arrivals at 50,000/s, log-normal sizes "
                    "(median 4 KB, sigma 2, 64 B - 8 MB), 60% records / 25% number-heavy / "
                    "15% string-heavy",
        "requests": int(n), "bytes": int(off[-1]), "offered_req_per_s": round(n / float(arrival[-1]), 1),
        "docs_per_s": round(n / wall, 1), "GB_per_s": round(int(off[-1]) / wall / 1e9, 3),
        "latency_ms_p50": round(med["p50"], 4), "latency_ms_p99": round(med["p99"], 4),
        "latency_ms_max": round(med["max"], 3),
        "runs_ms": [{k: round(r[k], 3) for k in ("p50", "p99", "max")} for r in runs],
        "slots": srv.slots, "device_bytes": srv.device_bytes, "mem_budget": 8 << 30,
        "batches": int(batches), "docs_per_batch": round(n / max(1, batches), 2),
        "timing": "host clock; arrival = scheduled time, done = result seen by the polling loop; "
                  "the run with the median p99 of three timed replays",
        "capacity": capacity,
    }


def serving_capacity(srv, buf, off, arrival, p99_limit_ms: float = 2.0) -> dict:
    """The highest offered rate the server sustains with p99 latency under
    p99_limit_ms: the first 100,000 requests of the config-4 trace replayed
    with their arrival times compressed by rising factors (the same documents
    and Poisson pattern at 1x, 2x, ... the trace's rate).  Each rate is
    replayed three times and judged by the median p99; the sweep stops at the
    first rate over the limit."""
    n = min(arrival.size, 100_000)
    arr0 = arrival[:n] - arrival[0]
    rows, best = [], None
    for mult in (1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 16, 24, 32):
        arr = arr0 / mult
        reps = []
        for _ in range(3):
            lat, wall = srv.replay(buf, off[: n + 1], arr)
            reps.append((pct(lat, 99) * 1e3, pct(lat, 50) * 1e3, wall))
        p99, p50, wall = sorted(reps)[1]
        rate = n / float(arr[-1])
        rows.append({"offered_req_per_s": round(rate), "p50_ms": round(p50, 4),
                     "p99_ms": round(p99, 4), "served_req_per_s": round(n / wall),
                     "GB_per_s": round(int(off[n]) / wall / 1e9, 3)})
        if p99 >= p99_limit_ms:
            break
        best = rows[-1]
    return {"p99_limit_ms": p99_limit_ms, "requests": int(n),
            "highest_rate_req_per_s": best["offered_req_per_s"] if best else None,
            "GB_per_s_at_highest": best["GB_per_s"] if best else None, "sweep": rows,
            "timing": "each rate: the median p99 of three replays"}


def cost_model(args) -> dict:
    """Per-stage time per input byte over a mix of synthetic documents (the
    GPU analogue of the paper's Fig. "stacked"), the effect of minification
    (Table "tab:minification"), and a least-squares refit of the paper's cost
    model (Sec. 4.3): time = a*B + b*S + c*F + d over input bytes B,
    structural indices S and floats F."""
    import torch

    import gen
    import paper_1902_08318_gb300 as sj
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    mb = args.doc_mb or 64
    docs = {}
    for size in (mb << 18, mb << 20):  # a quarter and the whole size: fixed costs separate
        tag = f" {size >> 20} MiB"
        docs["records, pretty" + tag] = gen.records(1, size, root_array=True, pretty=True)
        docs["records, minified" + tag] = gen.records(1, size, root_array=True, pretty=False)
        docs["records, non-ASCII, pretty" + tag] = gen.records(
            2, size, root_array=True, pretty=True, nonascii_p=gen.NONASCII_P)
        docs["records, non-ASCII, minified" + tag] = gen.records(
            2, size, root_array=True, pretty=False, nonascii_p=gen.NONASCII_P)
        docs["config2-shaped (deep 1%)" + tag] = gen.config2(3, size=size)
        docs["number-heavy (geo)" + tag] = gen.geo(4, size)
        docs["string-heavy" + tag] = gen.strings_heavy(5, size)
        docs["tweets" + tag] = gen.tweets(6, size, 100_000)
    p = sj.Parser(max_bytes=max(int(d.size) for d in docs.values()) + 64)
    p.set_profiling(True)
    rows = []
    for name, doc in docs.items():
        d = torch.from_numpy(np.require(doc, requirements=["W"])).to(dev)
        r = p.parse(d)
        assert r.error == 0, (name, r.error_name)
        tape = r.tape().cpu().numpy()
        tags = (tape >> np.uint64(56)).astype(np.uint8)
        is_val = np.concatenate([[False], (tags[:-1] != ord("l")) & (tags[:-1] != ord("d"))])
        floats = int(np.count_nonzero((tags == ord("d")) & is_val))
        ints = int(np.count_nonzero((tags == ord("l")) & is_val))
        st = {k: 0.0 for k in sj.STAGES}
        for _ in range(max(3, min(args.steps, 5))):
            p.parse_async(d)
            for k, v in p.stage_times().items():
                st[k] += v
        n = max(3, min(args.steps, 5))
        st = {k: v / n for k, v in st.items()}
        ms = sum(st.values())
        B = int(doc.size)
        rows.append({"doc": name, "B": B, "S": r.n_indices, "F": floats, "I": ints,
                     "T": r.tape_words, "SB": r.string_bytes, "ms": round(ms, 4),
                     "GB_per_s": round(B / ms / 1e6, 2),
                     "ns_per_byte": {k: round(v * 1e6 / B, 5) for k, v in st.items()}})
    y = np.array([r["ms"] * 1e6 for r in rows])  # ns

    def fit(cols):
        A = np.array([[r[c] for c in cols] + [1.0] for r in rows], dtype=np.float64)
        try:  # non-negative coefficients (a cost per unit cannot be negative)
            from scipy.optimize import nnls
            coef, _ = nnls(A, y)
        except ImportError:
            coef, *_ = np.linalg.lstsq(A, y, rcond=None)
        pred = A @ coef
        r2 = 1.0 - float(((y - pred) ** 2).sum() / ((y - y.mean()) ** 2).sum())
        return coef, r2

    coef, r2 = fit(["B", "S", "F"])
    coef_sb, r2_sb = fit(["B", "S", "F", "SB"])
    # minification: the same kind of records with and without white space;
    # compared per input byte and per tape word (the content parsed)
    mini = {}
    for base in ("records", "records, non-ASCII"):
        a = next(r for r in rows if r["doc"] == f"{base}, pretty {mb} MiB")
        b = next(r for r in rows if r["doc"] == f"{base}, minified {mb} MiB")
        mini[base] = {"pretty_ns_per_byte": round(a["ms"] * 1e6 / a["B"], 5),
                      "minified_ns_per_byte": round(b["ms"] * 1e6 / b["B"], 5),
                      "pretty_ns_per_tape_word": round(a["ms"] * 1e6 / a["T"], 4),
                      "minified_ns_per_tape_word": round(b["ms"] * 1e6 / b["T"], 4),
                      "bytes_per_tape_word": [round(a["B"] / a["T"], 2), round(b["B"] / b["T"], 2)]}
    ablations = ablation_table(args, dev)
    return {"mode": "cost-model", "documents": rows, "ablations": ablations,
            "fit_ns": {"per_byte": round(coef[0], 5), "per_index": round(coef[1], 4),
                       "per_float": round(coef[2], 4), "fixed": round(coef[3], 1), "r2": round(r2, 4)},
            "fit_ns_with_string_bytes": {"per_byte": round(coef_sb[0], 5),
                                         "per_index": round(coef_sb[1], 4),
                                         "per_float": round(coef_sb[2], 4),
                                         "per_string_byte": round(coef_sb[3], 5),
                                         "fixed": round(coef_sb[4], 1), "r2": round(r2_sb, 4)},
            "minification": mini,
            "note": "per-stage ns per input byte from CUDA events; one GB300; synthetic documents "
                    f"of about {mb} MiB"}


def ablation_table(args, dev) -> dict:
    """The GPU analogue of Table "tab:optimization": stage-1 kernel times with
    one optimisation at a time replaced by its plain form (the variant
    libraries of sj.ABLATIONS), on a config-2 shaped document of --doc-mb MiB
    (default 64), ASCII-only records of the same size (where the UTF-8 check
    can skip blocks) and the config-1 document.  Each variant's indices, tape size
    and string bytes are checked equal to the default library's on the device
    (their parity with the oracle is a GPU test); times are medians over the
    profiled parses (CUDA events between the stages)."""
    import torch

    import gen
    import paper_1902_08318_gb300 as sj
    mb = args.doc_mb or 64
    sj.build_variants()
    libs = {"default": sj.load()}
    libs.update({name: sj.load_variant(name) for name in sj.ABLATIONS})
    docs = {f"config2-shaped {mb} MiB": gen.config2(3, size=mb << 20),
            f"records, ASCII only, pretty {mb} MiB": gen.records(1, mb << 20, root_array=True),
            "config1 (2.5 MB)": gen.config1(1000)}
    reps = max(5, min(args.steps, 20))
    out = {}
    for dname, doc in docs.items():
        d = torch.from_numpy(np.require(doc, requirements=["W"])).to(dev)
        ref = None
        rows = {}
        for vname, lib in libs.items():
            p = sj.Parser(max_bytes=int(doc.size) + 64, lib=lib)
            p.set_profiling(True)
            r = p.parse(d)
            assert r.error == 0, (vname, dname, r.error_name)
            got = (r.indices().clone(), r.tape_words, r.string_bytes)
            if ref is None:
                ref = got
            else:
                assert torch.equal(got[0], ref[0]) and got[1:] == ref[1:], (vname, dname)
            t = {k: [] for k in ("s1_blocks", "s1_scan", "s1_flatten")}
            for _ in range(reps):
                p.parse(d)
                st = p.stage_times()
                for k in t:
                    t[k].append(st[k])
            p.close()
            med = {k: float(np.median(v)) for k, v in t.items()}
            rows[vname] = {"s1_blocks_ms": round(med["s1_blocks"], 4),
                           "s1_flatten_ms": round(med["s1_flatten"], 4),
                           "stage1_ms": round(sum(med.values()), 4)}
        base = rows["default"]["stage1_ms"]
        for v in rows.values():
            v["stage1_vs_default"] = round(v["stage1_ms"] / base, 3)
        out[dname] = rows
    out["variants"] = {k: v for k, v in sj.ABLATIONS.items()}
    out["timing"] = f"median of {reps} profiled parses per variant; stage 1 = blocks + scan + flatten"
    return out


def oracle_gbs(sample: bytes, repeats: int = 1) -> tuple[float, float]:
    import oracle
    oracle.parse(sample[:1024])  # build + warm
    t0 = time.perf_counter()
    for _ in range(repeats):
        r = oracle.parse(sample)
    dt = time.perf_counter() - t0
    assert r["error"] == 0, r["error"]
    return len(sample) * repeats / dt / 1e9, dt


def cpu_baseline(args) -> dict:
    sample_bytes = 512 << 20 if args.workload == "config2" else None
    if args.workload == "config2":
        doc = make_doc("config2", 2000, size=sample_bytes + (1 << 20))
        sample = record_prefix(doc, sample_bytes)
        what = f"first whole records ({len(sample)} bytes) of a config-2 document, single-threaded"
    else:
        sample = make_doc(args.workload, 1000 if args.workload == "config1" else 0).tobytes()
        what = f"the whole {args.workload} document ({len(sample)} bytes), single-threaded"
    gbs, dt = oracle_gbs(sample)
    out = {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": what, "seconds": round(dt, 2), "host_cores": os.cpu_count()}
    if not args.no_batch:
        out["batch"] = oracle_batch()
    return out


def _oracle_errors(args):
    """Worker: the oracle over documents [a, b) of a batch held in shared memory."""
    from multiprocessing import shared_memory

    import oracle
    name, size, off, a, b = args
    shm = shared_memory.SharedMemory(name=name)
    try:
        buf = np.ndarray((size,), dtype=np.uint8, buffer=shm.buf)
        lo, hi = int(off[a]), int(off[b])
        errs = oracle.parse_many_errors(buf[lo:hi], off[a: b + 1] - off[a])
        del buf
        return int(np.count_nonzero(errs))
    finally:
        shm.close()


def oracle_batch() -> dict:
    """The oracle over the whole config3 batch, one worker process per host
    core (the batch in shared memory; only the parse is timed)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    import gen
    buf, off = gen.config3()
    n = off.size - 1
    workers = os.cpu_count() or 1
    shm = shared_memory.SharedMemory(create=True, size=int(buf.size))
    try:
        np.ndarray((buf.size,), dtype=np.uint8, buffer=shm.buf)[:] = buf
        cuts = np.linspace(0, n, workers + 1).astype(np.int64)
        jobs = [(shm.name, int(buf.size), off, int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:])]
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_oracle_errors, [(shm.name, int(buf.size), off, 0, 1)] * workers)  # start-up
            t0 = time.perf_counter()
            bad = sum(pool.map(_oracle_errors, jobs))
            dt = time.perf_counter() - t0
    finally:
        shm.close()
        shm.unlink()
    return {"docs_per_s": round(n / dt, 1), "GB_per_s": round(int(off[-1]) / dt / 1e9, 3),
            "cores": workers, "kind": "oracle", "invalid_docs": bad,
            "sample": f"all {n} documents of config3 ({int(off[-1])} bytes), one process per core",
            "seconds": round(dt, 3)}


def run_reference(args, rank: int) -> dict | None:
    if rank != 0:
        return None
    desc, _ = WORKLOADS[args.workload]
    if args.workload == "config2":
        doc = make_doc("config2", 2000, size=(32 << 20) + (1 << 20))
        sample = record_prefix(doc, 32 << 20)
        what = f"first whole records ({len(sample)} bytes) of a config-2 document per step"
    else:
        sample = make_doc(args.workload, 1000 if args.workload == "config1" else 0).tobytes()
        what = f"the whole {args.workload} document per step"
    import oracle
    oracle.parse(sample[:1024])
    for _ in range(args.warmup):
        oracle.parse(sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle.parse(sample)
        assert r["error"] == 0
    dt = time.perf_counter() - t0
    gbs = len(sample) * args.steps / dt / 1e9
    return {
        "impl": "reference",
        "metric": "parse GB/s (input bytes, device-timed)",
        "value": round(gbs, 4), "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "bytes_per_step": len(sample)},
        "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": what},
        "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="config2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched (config3) leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--no-query", action="store_true", help="skip the tape-query leg")
    ap.add_argument("--cost-model", action="store_true",
                    help="per-stage breakdown, minification and cost-model fit (one JSON line)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving (config4) leg")
    ap.add_argument("--doc-mb", type=int, default=0,
                    help="config2 document size in MiB (default 1024; smaller for ncu captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        out = run_reference(args, rank)
        if out:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if args.cost_model:
        if rank == 0:
            print(json.dumps(cost_model(args)), flush=True)
        return
    if dist:
        dist.barrier()
    out = run_ours(args, rank, world, dist)
    if out is not None:
        import torch
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        if not args.no_batch:
            out["batch"] = batch_leg(args, dev)
        if not args.no_query:
            out["query"] = query_leg(args, dev)
        out["small_docs"] = small_doc_leg(args, dev)
        if not args.no_serving:
            out["serving"] = serving_leg(args)
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
