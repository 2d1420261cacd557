"""Benchmark: stable sort of 10^9 uint32 key / uint32 value pairs (uniform
keys, values = original index) on one GB300, through the dtsort C-ABI.

One step = one complete sort of the whole array (sampling, every
distribution level, the on-chip base case, dovetail merges).  Inputs are
synthetic (seeded generator) and resident in HBM when a timed step starts; the
pristine input is restored before every step (untimed, device to device), and
at 8 GB per step the working set is far larger than L2.  Device time is taken
with CUDA events on the sorting stream.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores on a bounded sample of the same workload instead.
"""
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
sys.path.insert(0, ROOT)

METRIC = "sorted keys/s (10^9 keys, u32/u64 KV) and fraction of GB300 HBM roofline"
# algorithmic bytes per record (key read for the level-0 histogram, then two
# distribution passes and the on-chip base case, each reading and writing the
# record): K + 3 * 2 * (K + V)
B_ALG = {"u32kv": 4 + 3 * 2 * 8, "u64kv": 8 + 3 * 2 * 16, "u64": 8 + 3 * 2 * 8,
         "u32": 4 + 3 * 2 * 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000_000)
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--op", default="u32kv", choices=["u32kv", "u32", "u64kv", "u64"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=100_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--launch-mode", type=int, default=0,
                    help="1: one launch per phase (profiling aid)")
    ap.add_argument("--workload", default="single", choices=["single", "segmented"])
    ap.add_argument("--seg-total", default="2e8",
                    help="segmented: total records ('literal' = sizes as drawn)")
    ap.add_argument("--segments", type=int, default=4096)
    ap.add_argument("--graph", action="store_true",
                    help="segmented: capture the call once, replay it per step")
    ap.add_argument("--baseline-calls", action="store_true",
                    help="segmented: also time one dtsort_u32_kv call per array")
    ap.add_argument("--block-tiles", type=int, default=0,
                    help="option block_tiles (0: the library's default)")
    ap.add_argument("--gamma-max", type=int, default=0,
                    help="option gamma_max (0: the library's default)")
    ap.add_argument("--capacity", type=int, default=0,
                    help="option finisher_capacity (0: the library's default)")
    ap.add_argument("--bucketing", default="digit",
                    choices=["digit", "learned", "learned-always"],
                    help="learned: model zones when the device's estimate says they pay; "
                         "learned-always: model zones regardless")
    ap.add_argument("--autotune", action="store_true",
                    help="run the autotuner on the workload first and use its choice")
    ap.add_argument("--heavy", default="on", choices=["on", "off"],
                    help="off: no heavy-key detection (the paper's 'Plain' ablation)")
    ap.add_argument("--parallel", default="replicas", choices=["replicas", "sharded"],
                    help="N > 1: independent replicas, or one array of N*n records "
                         "sharded over the ranks (sample, partition, one all-to-all, "
                         "local sorts)")
    ap.add_argument("--merge", default="dovetail", choices=["dovetail", "generic"],
                    help="generic: merge-path merging of the heavy zones instead of "
                         "dovetail merging (the paper's merge ablation)")
    return ap.parse_args()


def kernel_source_id():
    """Short hash of the CUDA sources and the C header (names + code): comments
    and blank space are left out, so that a documentation edit does not mark
    the committed DRAM traffic of unchanged kernels as stale."""
    import glob
    import hashlib
    import re
    d = os.path.join(ROOT, "paper_2401_00710_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(d, "*.cu")) + glob.glob(os.path.join(d, "*.cuh")) +
                   glob.glob(os.path.join(d, "*.h")))
    files.append(os.path.join(ROOT, "include", "dtsort.h"))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "r") as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)  # block comments
        code = re.sub(r"//[^\n]*", " ", code)                # line comments
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def dram_traffic(op, dist, n):
    """DRAM bytes of one sort from the committed ncu summary, scaled to n;
    None when there is none for this workload or the kernels have changed
    since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            d = json.load(f)
        if d.get("kernel_source") != kernel_source_id():
            return None
        return float(d["%s/%s" % (op, dist)]["bytes_per_record"]) * n
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for nm, val in zip(names, r[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- N > 1: independent replicas (every rank sorts its own array) ----------
def replica_seed(seed, rank):
    """Each rank sorts a different seeded array of the same workload."""
    return seed + rank


def replica_ms(ms, world, device=None):
    """Time of one step of the whole job: the slowest rank's (max over ranks)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_rate(n_per_rank, world, ms):
    """Whole-job throughput: the records all ranks sorted, per second."""
    return world * n_per_rank / (ms / 1e3)


def key_dtype(op):
    return np.uint32 if op.startswith("u32") else np.uint64


def sample_keys(args, count):
    """The first `count` keys of the benchmark's seeded stream."""
    import gen
    kd = key_dtype(args.op)
    table = gen.U32_FAMILIES if kd == np.uint32 else gen.U64_FAMILIES
    kind, dt, p1, p2 = table[args.dist]
    if p1 is None:  # the exponential's rate is fixed by the full n
        p1 = 10.0 / args.n
    return gen.keys(count, kind, kd, args.seed, p1, p2)


def cpu_oracle_time(args, sample):
    """The oracle, as it stands, on `sample` records, all host cores."""
    import gen
    import oracle
    kd = key_dtype(args.op)
    keys = sample_keys(args, sample)
    vals = None
    if args.op.endswith("kv"):
        vals = (gen.edge_src(sample, kd, E=args.n) if args.dist == "edges"
                else gen.iota(sample, kd))
    cores = oracle.default_threads()
    t0 = time.perf_counter()
    oracle.stable_sort(keys, vals, nthreads=cores)
    dt = time.perf_counter() - t0
    return sample / dt, cores, dt


def single_config(args, world, tuned=None):
    """The `config` of a single-array sort line; both arms print the same."""
    rec_bytes = np.dtype(key_dtype(args.op)).itemsize * (2 if args.op.endswith("kv") else 1)
    n = args.n
    return {"workload": "stable sort, %s, n=%d, keys %s seed %d, values = %s%s%s%s"
                        % (args.op, n, args.dist, args.seed,
                           "the edges' sources (graph transpose of a power-law "
                           "edge list over 2^26 vertices)" if args.dist == "edges"
                           else "index",
                           "" if args.bucketing == "digit" else ", bucketing " + args.bucketing,
                           ", heavy-key detection off" if args.heavy == "off" else "",
                           ", generic merge-path merging" if args.merge == "generic" else ""),
            "n": n, "dist": args.dist, "autotuned": tuned,
            "l2": ("inputs %.1f GB per step >> L2 (129 MB)" % (rec_bytes * n / 1e9)
                   if rec_bytes * n > 4 * 129e6 else
                   "inputs %.0f MB per step: not much larger than L2 (129 MB)"
                   % (rec_bytes * n / 1e6)),
            "parallelism": "replicas" if world > 1 else "single"}


def reference_config(args, world, sample):
    """The reference arm's config: the same workload, of which the CPU oracle
    sorts the first `sample` records per step (a bounded sample)."""
    cfg = single_config(args, world)
    if sample < args.n:
        cfg["workload"] += " (the CPU oracle sorts its first %d records per step)" % sample
        cfg["sample_n"] = sample
    return cfg


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import gen  # noqa: F401
    sample = args.cpu_sample
    times = []
    cores = 0
    for i in range(args.warmup + args.steps):
        v, cores, dt = cpu_oracle_time(args, sample)
        if i >= args.warmup:
            times.append(dt)
    t = statistics.mean(times)
    value = sample / t
    line = {"metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.op, "data": "synthetic",
            "config": reference_config(args, world, sample),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "keys/s", "cores": cores,
                             "kind": "oracle",
                             "sample": "first %d records of the same seeded stream" % sample},
            "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def device_error_text(h, st):
    """Status text plus the first failed internal check, if one was recorded."""
    import paper_2401_00710_gb300 as dts

    text = dts.status_string(st)
    if st == dts.DTSORT_ERR_INTERNAL:
        try:
            d = dts.dtsort_get_stats(h).as_dict()
            text += " (check site %d, values %s)" % (d["check_site"], d["check_values"])
        except Exception:  # the context itself may be gone
            pass
    return text


def run_ours(args):
    import torch

    import gen
    import paper_2401_00710_gb300 as dts

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    kd = key_dtype(args.op)
    kbytes = np.dtype(kd).itemsize
    has_v = args.op.endswith("kv")
    n = args.n
    tdt = torch.int32 if kbytes == 4 else torch.int64
    # inputs: generated on the host into pinned memory, one pristine device copy
    hk = torch.empty(n, dtype=tdt, pin_memory=True)
    gen.fill_family(args.dist, hk.data_ptr(), n, kd, seed=replica_seed(args.seed, rank))
    hv = None
    if has_v:
        hv = torch.empty(n, dtype=tdt, pin_memory=True)
        if args.dist == "edges":  # graph transpose: values = the edges' sources
            gen.fill_edge_src(hv.data_ptr(), n, kbytes)
        else:
            gen.fill_iota(hv.data_ptr(), n, kbytes)
    pk = hk.to(dev)
    pv = hv.to(dev) if has_v else None
    k = torch.empty_like(pk)
    v = torch.empty_like(pv) if has_v else None
    op = {"u32kv": dts.DTSORT_OP_U32_KV, "u32": dts.DTSORT_OP_U32,
          "u64kv": dts.DTSORT_OP_U64_KV, "u64": dts.DTSORT_OP_U64}[args.op]
    h = dts.dtsort_create(local)
    if (args.launch_mode or args.bucketing != "digit" or args.block_tiles or args.gamma_max or
            args.capacity or args.heavy == "off" or args.merge != "dovetail"):
        o = dts.dtsort_get_options(h)
        o.heavy_detection = -1 if args.heavy == "off" else 0
        o.launch_mode = args.launch_mode
        o.block_tiles = args.block_tiles
        o.gamma_max = args.gamma_max
        o.finisher_capacity = args.capacity
        o.merge = (dts.DTSORT_MERGE_GENERIC if args.merge == "generic"
                   else dts.DTSORT_MERGE_DOVETAIL)
        o.bucketing = {"digit": dts.DTSORT_BUCKETING_DIGIT,
                       "learned": dts.DTSORT_BUCKETING_LEARNED,
                       "learned-always": dts.DTSORT_BUCKETING_LEARNED_ALWAYS}[args.bucketing]
        dts.dtsort_set_options(h, o)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    tuned = None
    if args.autotune:
        # time the autotuner's candidates on this input, then sort with its
        # cached choice
        o_ = dts.dtsort_get_options(h)
        o_.autotune = 1
        dts.dtsort_set_options(h, o_)
        sb = dts.dtsort_autotune_scratch_bytes(h, op, n, 1)
        scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
        st, best = dts.dtsort_autotune(h, op, pk.data_ptr(), pv.data_ptr() if has_v else None,
                                       None, 0, n, scratch.data_ptr(), sb, sp)
        if st != 0:
            raise RuntimeError(dts.status_string(st))
        tuned = {"gamma_max": best.gamma_max, "finisher_capacity": best.finisher_capacity,
                 "block_tiles": best.block_tiles}
        del scratch
    wsb = dts.dtsort_workspace_bytes(h, op, n)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    fn = {dts.DTSORT_OP_U32_KV: dts.dtsort_u32_kv, dts.DTSORT_OP_U64_KV: dts.dtsort_u64_kv,
          dts.DTSORT_OP_U32: dts.dtsort_u32, dts.DTSORT_OP_U64: dts.dtsort_u64}[op]

    def sort_once(kp, vp):
        if has_v:
            st = fn(h, kp, vp, n, ws.data_ptr(), wsb, sp)
        else:
            st = fn(h, kp, n, ws.data_ptr(), wsb, sp)
        if st != 0:
            raise RuntimeError(dts.status_string(st))

    def restore():
        k.copy_(pk)
        if has_v:
            v.copy_(pv)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()

    for _ in range(args.warmup):
        restore()
        sort_once(k.data_ptr(), v.data_ptr() if has_v else None)
    st = dts.dtsort_last_device_error(h, sp)
    if st != 0:
        raise RuntimeError("device: " + device_error_text(h, st))
    # ---- timed: K sorts, CUDA events around each sort on its stream ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            restore()
            ev[i][0].record(stream)
            sort_once(k.data_ptr(), v.data_ptr() if has_v else None)
            ev[i][1].record(stream)
        barrier()
    st = dts.dtsort_last_device_error(h, sp)
    if st != 0:
        raise RuntimeError("device: " + device_error_text(h, st))
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = replica_ms(sum(ms) / len(ms), world, dev)
    stats = dts.dtsort_get_stats(h).as_dict()
    # ---- end to end: host buffers in, sorted host buffers out ----
    e2e = None
    if not args.no_e2e:
        # through the host-buffer entry point: it copies the pinned host arrays
        # in, sorts, and copies the result back over them; the pristine input
        # is restored on the host between steps (untimed)
        wk = torch.empty_like(hk, pin_memory=True)
        wv = torch.empty_like(hv, pin_memory=True) if has_v else None
        e_ms = []
        for i in range(max(1, min(args.steps, 3))):
            wk.copy_(hk)
            if has_v:
                wv.copy_(hv)
            barrier()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            st = dts.dtsort_sort_host(h, op, wk.data_ptr(), wv.data_ptr() if has_v else None, n,
                                      k.data_ptr(), v.data_ptr() if has_v else None,
                                      ws.data_ptr(), wsb, sp)
            if st != 0:
                raise RuntimeError(dts.status_string(st))
            t1.record(stream)
            barrier()
            e_ms.append(t0.elapsed_time(t1))
        e_ms_step = replica_ms(sum(e_ms) / len(e_ms), world, dev)
        by = n * (kbytes * (2 if has_v else 1))
        e2e = {"value": job_rate(n, world, e_ms_step), "unit": "keys/s",
               "h2d_bytes_per_step": by, "d2h_bytes_per_step": by,
               "ms_per_step": e_ms_step}
    if rank != 0:
        return 0
    peak, peak_kind = peaks()
    b_alg = B_ALG[args.op] * n
    achieved = b_alg / (ms_step / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": job_rate(n, world, ms_step), "unit": "keys/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.op, "data": "synthetic",
        "config": single_config(args, world, tuned),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": dram_traffic(args.op, args.dist, n)
                     if args.bucketing == "digit" else None,
                     "peak_kind": peak_kind, "bytes_per_record": B_ALG[args.op],
                     "kernel": "one sort: the queued per-phase launches (dts::dtsort_phase_one: "
                               "levels, their merges, statistics) + the persistent "
                               "dts::dtsort_kernel; achieved = algorithmic bytes / CUDA-event "
                               "time of the sort"},
        "gpu_launches": args.steps * stats["kernel_launches"],
        "clocks": clk.summary(),
        "e2e": e2e,
        "stats": {"levels": stats["levels"], "phase_ms": stats["phase_ms"],
                  "heavy_keys": stats["heavy_keys"][:4],
                  "records": stats["records"][:6],
                  "finisher_tasks": stats["finisher_tasks"],
                  "finisher_lsd_tasks": stats["finisher_lsd_tasks"],
                  "merge_records": stats["merge_records"],
                  "bucketing": args.bucketing,
                  "learned_zones_used": stats["learned_zones_used"],
                  "learned_estimate": stats["learned_estimate"],
                  "level0_bucket_cv": stats["learned_bucket_cv"],
                  "level0_bucket_max_over_mean": stats["learned_bucket_max_over_mean"],
                  "fixup_records": stats["learned_fixup_records"],
                  "fixup_steps": stats["learned_fixup_steps"]},
        "ms_steps": ms,
    }
    if not args.no_cpu_baseline and world == 1:
        sample = min(args.cpu_sample, n)
        val, cores, dt = cpu_oracle_time(args, sample)
        line["cpu_baseline"] = {"value": val, "unit": "keys/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "first %d records of the same seeded stream "
                                          "(%.1f s)" % (sample, dt)}
    print(json.dumps(line), flush=True)
    dts.dtsort_destroy(h)
    return 0


def segmented_passes(size, cap, gamma=9):
    """Distribution passes + base case the method needs for one array."""
    import math
    if size <= cap:
        return 1
    return 1 + max(1, math.ceil(math.log2(size / (0.85 * cap)) / gamma))


def run_segmented(args):
    """4096 arrays with log-uniform sizes in [100, 10^7], u32 keys (uniform or
    Zipf 1.0 per array) with int32 values, sorted by one persistent launch."""
    import torch

    import gen
    import paper_2401_00710_gb300 as dts

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    total = None if args.seg_total == "literal" else float(args.seg_total)
    off, fam = gen.segmented_layout(nseg=args.segments, lo=100, hi=1e7, seed=args.seed,
                                    total=total)
    n = int(off[-1])
    nseg = len(off) - 1
    hk = torch.empty(n, dtype=torch.int32, pin_memory=True)
    hv = torch.empty(n, dtype=torch.int32, pin_memory=True)
    gen.fill_segmented_u32(hk.data_ptr(), hv.data_ptr(), off, fam,
                           seed=replica_seed(args.seed, rank))
    pk, pv = hk.to(dev), hv.to(dev)
    k, v = torch.empty_like(pk), torch.empty_like(pv)
    o = torch.from_numpy(off).to(dev)
    h = dts.dtsort_create(local)
    op = dts.DTSORT_OP_U32_KV
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    tuned = None
    if args.autotune:
        o_ = dts.dtsort_get_options(h)
        o_.autotune = 1
        dts.dtsort_set_options(h, o_)
        sb = dts.dtsort_autotune_scratch_bytes(h, op, n, nseg)
        scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
        st, best = dts.dtsort_autotune(h, op, pk.data_ptr(), pv.data_ptr(), o.data_ptr(),
                                       nseg, n, scratch.data_ptr(), sb, sp)
        if st != 0:
            raise RuntimeError(dts.status_string(st))
        tuned = {"gamma_max": best.gamma_max, "finisher_capacity": best.finisher_capacity,
                 "block_tiles": best.block_tiles}
        del scratch
    wsb = dts.dtsort_workspace_bytes(h, op, n, nseg)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)

    def call():
        st = dts.dtsort_segmented_u32_kv(h, k.data_ptr(), v.data_ptr(), o.data_ptr(), nseg,
                                         n, ws.data_ptr(), wsb, sp)
        if st != 0:
            raise RuntimeError(dts.status_string(st))

    graph = None
    if args.graph:
        k.copy_(pk)
        v.copy_(pv)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            sp = torch.cuda.current_stream(dev).cuda_stream
            call()
        sp = stream.cuda_stream

    def step():
        if graph is not None:
            graph.replay()
        else:
            call()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            k.copy_(pk)
            v.copy_(pv)
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            k.copy_(pk)
            v.copy_(pv)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return sum(ms) / len(ms), ms

    if world > 1:
        torch.cuda.synchronize(dev)
        tdist.barrier()
    with ClockSampler(local) as clk:
        ms_step, ms_list = timed(step, args.steps, args.warmup)
    ms_step = replica_ms(ms_step, world, dev)
    st = dts.dtsort_last_device_error(h, sp)
    if st != 0:
        raise RuntimeError("device: " + device_error_text(h, st))
    stats = dts.dtsort_get_stats(h).as_dict()
    base = None
    if args.baseline_calls:
        sizes = np.diff(off)

        def separate():
            for s_ in range(nseg):
                a_, b_ = int(off[s_]), int(off[s_ + 1])
                if b_ - a_ < 2:
                    continue
                st_ = dts.dtsort_u32_kv(h, k.data_ptr() + 4 * a_, v.data_ptr() + 4 * a_, b_ - a_,
                                        ws.data_ptr(), wsb, sp)
                if st_ != 0:
                    raise RuntimeError(dts.status_string(st_))
        b_ms, _ = timed(separate, max(1, min(args.steps, 2)), 1)
        base = {"ms_per_step": b_ms, "value": n / (b_ms / 1e3), "unit": "keys/s",
                "what": "one dtsort_u32_kv call per array, same GPU, same stream"}
        del sizes
    cap = 4608  # the base-case capacity for 32-bit keys (9 items x 512 threads)
    if rank != 0:
        dts.dtsort_destroy(h)
        return 0
    b_alg = sum(int(sz) * (4 + segmented_passes(int(sz), cap) * 2 * 8) for sz in np.diff(off))
    peak, peak_kind = peaks()
    achieved = b_alg / (ms_step / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": job_rate(n, world, ms_step), "unit": "keys/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32kv",
        "data": "synthetic",
        "config": {"workload": "batched segmented sort: %d arrays, sizes log-uniform in "
                               "[100, 1e7]%s, u32 keys uniform or Zipf 1.0 per array, int32 "
                               "values" % (nseg, "" if total is None else
                                           " scaled to %.3g records" % total),
                   "n": n, "segments": nseg, "graph": bool(args.graph),
                   "autotuned": tuned},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "bytes": b_alg},
        "gpu_launches": args.steps * stats["kernel_launches"], "clocks": clk.summary(),
        "baseline_separate_calls": base,
        "stats": {"levels": stats["levels"], "phase_ms": stats["phase_ms"],
                  "finisher_tasks": stats["finisher_tasks"]},
        "ms_steps": ms_list,
    }
    print(json.dumps(line), flush=True)
    dts.dtsort_destroy(h)
    return 0


def run_sharded(args):
    """One array of world * n records, rank r holding records [r n, (r+1) n)
    of the seeded stream; one step = the whole sharded sort (sample, gather,
    splitters, partition, one all-to-all, local sort); max over ranks."""
    import torch
    import torch.distributed as tdist

    import gen
    import paper_2401_00710_gb300 as dts
    from paper_2401_00710_gb300 import sharded

    rank, world, local = dist_env()
    tdist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    kd = key_dtype(args.op)
    kbytes = np.dtype(kd).itemsize
    has_v = args.op.endswith("kv")
    n = args.n
    tdt = torch.int32 if kbytes == 4 else torch.int64
    table = gen.U32_FAMILIES if kbytes == 4 else gen.U64_FAMILIES
    kind, _, p1, p2 = table[args.dist]
    if p1 is None:
        p1 = 10.0 / max(n * world, 1)
    hk = torch.empty(n, dtype=tdt, pin_memory=True)
    gen.fill_keys(hk.data_ptr(), n, kind, kbytes, args.seed, p1, p2, first=rank * n)
    pk = hk.to(dev)
    pv = None
    if has_v:
        hv = torch.empty(n, dtype=tdt, pin_memory=True)
        gen.fill_iota(hv.data_ptr(), n, kbytes, first=rank * n)
        pv = hv.to(dev)
    ops = sharded.GpuShardOps(dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        k = pk.clone()
        v = pv.clone() if has_v else None
        torch.cuda.synchronize(dev)
        tdist.barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = sharded.sharded_sort(k, v, ops, seed=args.seed)
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b), res

    for _ in range(args.warmup):
        step()
    with ClockSampler(local) as clk:
        ms = [step()[0] for _ in range(args.steps)]
    ms_step = replica_ms(sum(ms) / len(ms), world, dev)
    if rank != 0:
        tdist.destroy_process_group()
        return 0
    peak, peak_kind = peaks()
    achieved = B_ALG[args.op] * n / (ms_step / 1e3) / 1e9
    cfg = single_config(args, world)
    cfg["workload"] = ("stable sort of one array of %d records sharded over %d GPUs, %s, "
                       "keys %s seed %d, values = global index" % (n * world, world, args.op,
                                                                   args.dist, args.seed))
    cfg["parallelism"] = "sharded: sample, partition, one all-to-all (NCCL), local sort"
    line = {"metric": METRIC, "value": n * world / (ms_step / 1e3), "unit": "keys/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.op, "data": "synthetic", "config": cfg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "bytes_per_record": B_ALG[args.op],
                         "kernel": "one rank's share of the sharded sort (algorithmic bytes "
                                   "of its n records / step time, exchange included)"},
            "gpu_launches": None, "clocks": clk.summary(), "e2e": None, "ms_steps": ms}
    print(json.dumps(line), flush=True)
    tdist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "segmented":
        return run_segmented(args)
    if args.parallel == "sharded" and dist_env()[1] > 1:
        return run_sharded(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
