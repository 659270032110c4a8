"""Benchmark of the word-count hot path on GB300.

Default workload: the large single-pass count -- 1e9 bytes of Zipf(1.0) text
over a 1M-word vocabulary (~170M words), one document, 64-bit counts.  A
step is one whole pass of the path: tokenise + two-level count, compaction
and the radix sort into (count desc, word asc).  Inputs are resident in HBM
when the timed region starts; 1 GB is larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  With --impl reference it times the CPU oracle
(test infrastructure) on a bounded sample of the same workload instead.
Under torchrun each rank counts its own replica of the workload (no
collectives on the data path; timing barrier + max over ranks only).
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "word-count input GB/s (1 GB Zipf corpus)"
UNIT = "GB/s"
WORKLOAD = ("large: 1e9 B synthetic Zipf(s=1.0) text, 1M-word vocabulary (lengths 1-24), mixed case, "
            "digits and punctuation as separators, ~169M words, one document, uint64 global counts")
ORACLE_MBPS_GUESS = 13.0  # single-core oracle throughput, MB/s, used only to size its sample


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks: a job step lasts as long as its slowest
    rank's.  dist is torch.distributed (initialised) or None for one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms_step: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's step."""
    return units_per_rank * world / (ms_step * 1e-3)


def replica_seed(rank: int) -> int:
    """Each replica counts its own corpus (independent problems, no exchange)."""
    import corpus
    return corpus.RECIPES["large"].seed + rank


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash() -> str:
    """Hash of the counting kernel's source code: the files it is built
    from, with // comments and blank lines left out (a comment edit does not
    change the kernel the traffic capture measured)."""
    h = hashlib.sha256()
    for f in ("wc_count.cu", "wc_device.cuh", "wc_internal.h"):
        with open(os.path.join(ROOT, "paper_2206_05269_gb300", "csrc", f), "r", encoding="utf-8") as fh:
            lines = []
            for ln in fh.read().splitlines():
                i = ln.find("//")
                ln = (ln[:i] if i >= 0 else ln).rstrip()
                if ln:
                    lines.append(ln)
        h.update("\n".join(lines).encode())
    return h.hexdigest()[:16]


TRAFFIC_FILE = os.path.join("profiles", "count_kernel_large_1GB_traffic.txt")


def profiled_traffic(kind: str):
    """DRAM bytes per launch of the counting kernel from the committed ncu
    summary (a profiler cannot run inside the timed benchmark), and a note
    saying where the figure comes from or why there is none: the summary
    must have been taken on the current kernel source."""
    p = os.path.join(ROOT, TRAFFIC_FILE)
    if not os.path.exists(p):
        return None, f"no traffic capture ({TRAFFIC_FILE} missing)"
    d = {}
    with open(p) as f:
        for ln in f:
            k, sep, v = ln.partition(":")
            if sep and not ln.startswith((" ", "#", "|")):
                d[k.strip()] = v.strip()
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None, (f"{TRAFFIC_FILE} was captured on kernel source {d.get('kernel_source_hash')}, "
                      f"not the current {kernel_source_hash()}: traffic unmeasured for the current kernel source")
    v = d.get(kind)
    return (float(v) if v else None), f"ncu capture in {TRAFFIC_FILE} (kernel source {kernel_source_hash()})"


def oracle_sample(text: np.ndarray, nbytes: int) -> np.ndarray:
    """A prefix of the corpus of about nbytes, cut after a space."""
    n = min(nbytes, text.size)
    while n < text.size and text[n - 1] != 0x20:
        n += 1
    return text[:n]


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores, per step on a bounded
    sample of the workload."""
    if rank != 0:
        return
    import corpus
    import oracle
    oracle.build()
    c = corpus.generate("large")
    per_step = int(max(1 << 20, min(200e6, 150.0 * ORACLE_MBPS_GUESS * 1e6 / max(1, args.steps + args.warmup))))
    sample = oracle_sample(c.text, per_step)
    for _ in range(args.warmup):
        oracle.count(sample, keep_docs=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.count(sample, keep_docs=False)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    val = sample.size / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_bytes_per_step": int(sample.size)},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"first {sample.size} bytes of the workload per step (single-threaded C++ oracle)"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, rank, world, local, subs=None):
    import torch
    import corpus
    from paper_2206_05269_gb300 import wc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    c = corpus.generate("large", seed=replica_seed(rank), size_a=args.bytes)
    nbytes = c.nbytes
    host = torch.from_numpy(c.text).pin_memory()
    text = host.to(f"cuda:{local}", non_blocking=False)
    ctr = wc.Counter(local)
    stream = torch.cuda.current_stream()

    def step():
        return ctr.count(text, stream)

    # warm-up (also settles the pool and checks the result is valid)
    for _ in range(args.warmup):
        t = step()
        if t.status() != wc.WC_OK:
            raise RuntimeError(f"count failed: {wc.wc_last_error(ctr.ctx)}")
        nwords, ntok, nbytes_words = t.size()
        cbits = wc.wc_table_count_bits(t.handle)
        t.free()

    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    wc.wc_profile_enable(ctr.ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tables, done = [], []
    ev0.record(stream)
    for _ in range(args.steps):
        tables.append(step())
        if len(tables) > 32:  # bound device memory (about 1 GB of tables): the oldest step is long finished
            done.append(tables.pop(0).status())
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_head, ms_count, ms_finish, n_count, launches = wc.wc_profile_read(ctr.ctx)
    wc.wc_profile_enable(ctr.ctx, False)
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1)
    done += [t.status() for t in tables]
    if any(st != wc.WC_OK for st in done):
        raise RuntimeError("a timed step failed")
    del tables
    ms_step = max_over_ranks(elapsed / args.steps, dist, f"cuda:{local}")
    value = job_rate(nbytes, world, ms_step) / 1e9

    # end to end through the C ABI: pinned host text -> device (copied in
    # pieces that are counted as they land: wc_count_host), table -> host
    e2e_steps = max(3, min(args.steps, 10))
    dev2 = torch.empty_like(text)
    d2h = 0
    t_e2e = []
    # pinned host buffers for the result, sized from the device steps' table
    cnt_t = torch.int64 if cbits == 64 else torch.int32
    hw = torch.empty(max(1, nbytes_words + 4096), dtype=torch.uint8).pin_memory()
    ho = torch.empty(nwords + 1, dtype=torch.int64).pin_memory()
    hc = torch.empty(max(1, nwords), dtype=cnt_t).pin_memory()
    for i in range(e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tab = ctr.count_host(host, stream, out=dev2)
        n_rows, n_wb = tab.export_into(hw, ho, hc, stream)
        t_e2e.append(time.perf_counter() - t0)
        d2h = n_wb + (n_rows + 1) * 8 + n_rows * hc.element_size()
        tab.free()
    # the median step (host scheduling hiccups land in single steps); the
    # mean and the extremes are reported beside it
    e2e_s = statistics.median(t_e2e[1:])
    e2e_val = nbytes * world / e2e_s / 1e9
    e2e_spread = {"mean": nbytes * world / statistics.mean(t_e2e[1:]) / 1e9,
                  "slowest_step": nbytes * world / max(t_e2e[1:]) / 1e9,
                  "fastest_step": nbytes * world / min(t_e2e[1:]) / 1e9, "steps": len(t_e2e) - 1,
                  "statistic": "median step"}
    # the host link measured in the same run: one plain pinned host -> device
    # copy of the whole text (the end-to-end figure cannot pass it)
    t_copy = []
    for _ in range(3):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        with torch.cuda.stream(stream):
            dev2.copy_(host, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        t_copy.append(c0.elapsed_time(c1))
    h2d_gbps = nbytes / (min(t_copy) * 1e-3) / 1e9

    peak, peak_kind = measured_peaks()
    avg_count_s = ms_count / max(1, n_count) * 1e-3
    alg_bytes = nbytes + nwords * 24
    achieved = alg_bytes / avg_count_s / 1e9
    traffic, traffic_note = profiled_traffic("dram_bytes_per_launch")

    # the practical ceiling of one pass over this text: a kernel that only reads it
    sink = torch.zeros(4096, dtype=torch.int64, device=f"cuda:{local}")
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        wc.wc_read_ceiling(text.data_ptr(), nbytes, sink.data_ptr(), 4096, stream.cuda_stream)
    ev2.record(stream)
    for _ in range(20):
        wc.wc_read_ceiling(text.data_ptr(), nbytes, sink.data_ptr(), 4096, stream.cuda_stream)
    ev3.record(stream)
    torch.cuda.synchronize()
    read_ceiling = nbytes / (ev2.elapsed_time(ev3) / 20 * 1e-3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        sample = oracle_sample(c.text, int(args.cpu_sample_mb * 1e6))
        t0 = time.perf_counter()
        r = oracle.count(sample, keep_docs=False)
        dt = time.perf_counter() - t0
        r_tokens = int(r.glob().counts.sum())
        del r
        cpu = {"value": sample.size / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {sample.size} bytes of the same corpus, single-threaded C++ oracle, {dt:.1f} s"}
        # the paper's multicore map + reduce on every host core, same sample
        import cpu_parallel
        cp = cpu_parallel.count(sample)
        if cp["tokens"] != r_tokens:
            raise RuntimeError("parallel CPU baseline disagrees with the oracle on the token count")
        cpu_par = {"value": sample.size / cp["seconds"] / 1e9, "unit": UNIT, "cores": cp["threads"],
                   "cpu_model": cpu_parallel.cpu_model(), "kind": "paper-style parallel (per-thread maps + merge)",
                   "sample": f"first {sample.size} bytes of the same corpus, {cp['seconds']:.2f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "bytes": nbytes, "words": ntok, "distinct": nwords,
                       "l2": "input (1e9 B) larger than L2, no flush", "parallelism": f"replicas x{world}"},
            "words_per_s": ntok * world / (ms_step * 1e-3),
            "stages_ms": {"head_selection": ms_head / max(1, n_count), "count_kernel": ms_count / max(1, n_count),
                          "compact_sort": ms_finish / max(1, n_count)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_note,
                         "kernel": "k_count3<HEAD> (main counting kernel)", "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "read_ceiling_GBps": read_ceiling, "frac_of_read_ceiling": achieved / read_ceiling,
                         "nominal_peak_GBps": 7900.0, "frac_of_nominal": achieved / 7900.0},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": d2h,
                    "h2d_copy_GBps": h2d_gbps, "spread": e2e_spread},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        if cpu:
            line["cpu_baseline"] = cpu
            line["cpu_parallel_baseline"] = cpu_par
        line.update(subs or {})
        print(json.dumps(line), flush=True)
    ctr.close()
    if dist:
        dist.destroy_process_group()


def _dev_docs(c, local):
    import torch
    dev = torch.device("cuda", local)
    host = torch.from_numpy(c.text).pin_memory()
    text = host.to(dev)
    offs = torch.from_numpy(c.offsets.view(np.int64)).to(dev)
    cls = torch.from_numpy(c.classes.view(np.int32)).to(dev) if c.nclasses > 1 else None
    return host, text, offs, cls


def docs_oracle_baseline(c, seconds: float = 8.0) -> dict:
    """The oracle (single-threaded C++) on the first documents of the same
    corpus, as many as about `seconds` of CPU work: documents per second with
    per-document tables (and class/global sums where the corpus has them)."""
    import oracle
    oracle.build()
    per_doc = max(1, c.nbytes // max(1, c.ndocs))
    nd = int(max(1, min(c.ndocs, seconds * ORACLE_MBPS_GUESS * 1e6 / per_doc)))
    offs = c.offsets[:nd + 1].copy()
    text = c.text[:int(offs[-1])]
    cls = c.classes[:nd] if c.nclasses > 1 else None
    t0 = time.perf_counter()
    oracle.count(text, offs, cls, c.nclasses if c.nclasses > 1 else 0)
    dt = time.perf_counter() - t0
    return {"value": nd / dt, "unit": "docs/s", "cores": 1, "kind": "oracle",
            "sample": f"first {nd} of {c.ndocs} documents ({text.size} bytes), single-threaded C++ oracle, {dt:.1f} s"}


def run_docs_workload(args, local, print_line: bool = True):
    """Batched per-document counting through a replayed plan: 'tiny' (200
    documents: per-document + global tables), 'classes' (4 x 250 documents:
    per-document, per-class and global tables + top-50 class-ratio words) or
    'batched' (100,000 log-normal documents: per-document tables).  Returns
    the result line (printed unless print_line is false)."""
    import torch
    import corpus
    from paper_2206_05269_gb300 import wc
    torch.cuda.set_device(local)
    c = corpus.generate(args.workload, **({"ndocs": args.docs} if args.docs else {}))
    host, text, offs, cls = _dev_docs(c, local)
    stream = torch.cuda.current_stream()
    # shapes tuned on this workload's own input (a cache entry is used untimed)
    tune = os.path.join(ROOT, "paper_2206_05269_gb300", "_build", f"tune_cache_{args.workload}.json")
    ctr = wc.Counter(local, count_bits=32, autotune=True, tune_cache_path=tune)
    plan = ctr.plan(c.offsets, c.nclasses if c.nclasses > 1 else 0, stream)
    tables = args.workload in ("tiny", "classes")

    def step():
        b = plan.run(text, offs, cls, stream)
        if tables:  # class and global tables (built on the device), ratio ranking
            g = b.table(wc.WC_TABLE_GLOBAL)
            for k in range(c.nclasses if c.nclasses > 1 else 0):
                b.table(wc.WC_TABLE_CLASS, k)
                wc.wc_class_ratio_topk(ctr.ctx, b.handle, k, 50, int(stream.cuda_stream))
            g.size()
        return b

    for _ in range(args.warmup):
        b = step()
        if b.status() != wc.WC_OK:
            raise RuntimeError(wc.wc_last_error(ctr.ctx))
    nent, _ = wc.wc_batch_size(b.handle)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    wc.wc_profile_enable(ctr.ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # inputs smaller than L2 (129 MB): L2 flushed before every timed step by
    # writing a 256 MB buffer, each step timed on its own
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}") if c.nbytes < (256 << 20) else None
    ms_sum, wall = 0.0, 0.0
    if flush is None:
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            b = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms_sum = ev0.elapsed_time(ev1)
    else:
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev0.record(stream)
            b = step()
            ev1.record(stream)
            torch.cuda.synchronize()
            wall += time.perf_counter() - t0
            ms_sum += ev0.elapsed_time(ev1)
    launches = wc.wc_profile_read(ctr.ctx)[4]
    clocks = sampler.stop()
    ms = ms_sum / args.steps
    if tables:
        ms = max(ms, wall * 1e3 / args.steps)  # host waits inside the step count too
    docs_s = c.ndocs / (ms * 1e-3)
    # one wc_count launch per document, on a sample of the same documents
    nsamp = min(c.ndocs, 2000)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    outs = []
    for d in range(nsamp):
        outs.append(ctr.count(text[int(c.offsets[d]):int(c.offsets[d + 1])], stream))
        if len(outs) > 64:
            outs.pop(0).status()
    for t in outs:
        t.status()
    per_launch = nsamp / (time.perf_counter() - t1)
    # end to end: host text -> the plan's device buffer, the step (the plan's
    # batched count, and for tiny/classes the class/global tables and
    # rankings), every per-document table -> pinned host buffers
    nent, nwb = wc.wc_batch_size(b.handle)
    pin = lambda n, dt: torch.empty(max(1, n), dtype=dt).pin_memory()
    hds, hdn = pin(c.ndocs, torch.int64), pin(c.ndocs, torch.int32)
    hw, ho, hc = pin(nwb + 4096, torch.uint8), pin(nent + 1, torch.int64), pin(nent, torch.int32)
    te = []
    d2h = 0
    for i in range(7):
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        text.copy_(host, non_blocking=True)
        bb = step()
        n_rows, n_wb = bb.export_into(hds, hdn, hw, ho, hc, stream)
        te.append(time.perf_counter() - t2)
        d2h = c.ndocs * 12 + n_wb + (n_rows + 1) * 8 + n_rows * 4
    e2e = c.ndocs / statistics.median(te[1:])  # the median step, the mean beside it
    # the same end to end with the vocabulary-id export: every document's
    # (id, count) rows plus the vocabulary (words, offsets, global counts) once
    hi, hcn = pin(nent, torch.int32), pin(nent, torch.int32)
    # the vocabulary's pinned buffers, sized by one untimed run (the text is
    # the same every step)
    nv, _, nvb = step().vocab().size()
    vw, vo, vc = pin(nvb + 16, torch.uint8), pin(nv + 1, torch.int64), pin(nv, torch.int64)
    te_ids, d2h_ids = [], 0
    for i in range(7):
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        text.copy_(host, non_blocking=True)
        bb = step()
        n_rows = bb.export_ids_into(hds, hdn, hi, hcn, stream)
        voc = bb.vocab()
        nv, _, nvb = voc.size()
        voc.export_into(vw, vo, vc, stream)
        te_ids.append(time.perf_counter() - t2)
        d2h_ids = c.ndocs * 12 + n_rows * 8 + nvb + (nv + 1) * 8 + nv * 8
    e2e_ids = c.ndocs / statistics.median(te_ids[1:])
    peak, peak_kind = measured_peaks()
    alg = c.nbytes + nent * 24
    line = {
        "metric": f"{args.workload}: documents/s (per-document tables)", "value": docs_s, "unit": "docs/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": args.workload, "docs": c.ndocs, "bytes": c.nbytes, "words": c.tokens,
                   "entries": nent,
                   "l2": "input smaller than L2: flushed (256 MB write) before each timed step" if flush is not None
                         else "input larger than L2, no flush",
                   "autotuned_shapes": json.load(open(tune)) if os.path.exists(tune) else None},
        "input_GBps": c.nbytes / (ms * 1e-3) / 1e9,
        "per_launch_docs_s": per_launch, "speedup_vs_per_launch": docs_s / per_launch,
        "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg / (ms * 1e-3) / 1e9 / peak, "traffic": None, "kernel": "whole batched step",
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg},
        "e2e": {"value": e2e, "unit": "docs/s", "h2d_bytes_per_step": c.nbytes, "d2h_bytes_per_step": d2h,
                "mean": c.ndocs / statistics.mean(te[1:]), "statistic": "median step"},
        "e2e_vocab_ids": {"value": e2e_ids, "unit": "docs/s", "h2d_bytes_per_step": c.nbytes,
                          "d2h_bytes_per_step": d2h_ids,
                          "mean": c.ndocs / statistics.mean(te_ids[1:]), "statistic": "median step",
                          "note": "per-document (vocabulary id, count) rows + the vocabulary once"},
        "gpu_launches": launches, "clocks": clocks,
    }
    del plan
    ctr.close()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = docs_oracle_baseline(c)
    if print_line:
        print(json.dumps(line), flush=True)
    return line


def run_served_workload(args, local, print_line: bool = True):
    """Served counting: a Poisson stream of requests (2,000/s for
    --serve-seconds, sizes log-uniform 1 KB - 64 MB) through the
    continuous-batching loop, then the first --fifo-seconds of the same
    stream through the plain one-launch-per-request path.  Returns the
    result line (printed unless print_line is false)."""
    import torch
    import corpus
    from paper_2206_05269_gb300 import serve, wc
    torch.cuda.set_device(local)
    pool = corpus.generate("served_pool", size_a=args.pool_bytes).text
    host = torch.from_numpy(pool).pin_memory()
    trip = corpus.poisson_requests(pool, 2000.0, args.serve_seconds, 1 << 10, 64 << 20, 0x5EED0105)
    reqs = [serve.Request(i, a, host[s:e]) for i, (a, s, e) in enumerate(trip)]
    ctr = wc.Counter(local, count_bits=32, budget=40 << 30)
    # warm-up on a few requests
    serve.serve_batched(ctr, [serve.Request(i, 0.0, r.data) for i, r in enumerate(reqs[:16])])
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = wc.wc_profile_read(ctr.ctx)[4]
    ans, st = serve.serve_batched(ctr, reqs, topk=100)
    launches = wc.wc_profile_read(ctr.ctx)[4] - launches0
    clocks = sampler.stop()
    lat = np.array([a.latency for a in ans]) * 1e3
    nbytes = sum(r.data.numel() for r in reqs)
    fifo_reqs = [r for r in reqs if r.arrival < args.fifo_seconds]
    fans, fst = serve.serve_fifo(ctr, fifo_reqs, topk=100)
    flat = np.array([a.latency for a in fans]) * 1e3
    bl = np.array([a.latency for a in ans[:len(fans)]]) * 1e3
    line = {
        "metric": "served: p99 latency ms (Poisson 2,000 req/s, 1 KB - 64 MB)", "value": float(np.percentile(lat, 99)),
        "unit": "ms", "n_gpus": 1, "steps": len(reqs), "warmup": 16, "ms_per_step": st["wall_s"] * 1e3 / len(reqs),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "served", "requests": len(reqs), "seconds": args.serve_seconds,
                   "bytes": nbytes, "rounds": st["rounds"], "large_requests": st["large"],
                   "recounted": st["recounted"], "budget_GB": 40,
                   "first_capacity_error": st["capacity_errors"][0] if st["capacity_errors"] else None},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "req_per_s": len(reqs) / st["wall_s"], "GBps": nbytes / st["wall_s"] / 1e9,
        "fifo": {"requests": len(fans), "p50_ms": float(np.percentile(flat, 50)) if len(fans) else None,
                 "p99_ms": float(np.percentile(flat, 99)) if len(fans) else None,
                 "req_per_s": len(fans) / fst["wall_s"] if len(fans) else None,
                 "batched_same_requests_p99_ms": float(np.percentile(bl, 99)) if len(fans) else None},
        # every latency runs from the request's arrival (its text in pinned
        # host memory) to its top-100 rows read back to the host
        "e2e": {"value": float(np.percentile(lat, 99)), "unit": "ms", "h2d_bytes_per_step": nbytes / len(reqs),
                "d2h_bytes_per_step": sum(a.words.nbytes + a.offs.nbytes + a.counts.nbytes for a in ans) / len(ans)},
        "gpu_launches": launches,
        "clocks": clocks,
        "budget_waits": st.get("budget_waits", 0),
    }
    ctr.close()
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        # the oracle on the first requests of the same stream, about 8 s of CPU work
        t0, done_b, k = time.perf_counter(), 0, 0
        while k < len(trip) and time.perf_counter() - t0 < 8.0:
            a, s0, e0 = trip[k]
            oracle.count(pool[s0:e0], keep_docs=False)
            done_b += e0 - s0
            k += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": k / dt, "unit": "req/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {k} requests of the stream ({done_b} bytes) counted one after "
                                          f"another, single-threaded C++ oracle, {dt:.1f} s"}
    if print_line:
        print(json.dumps(line), flush=True)
    return line


# fp64 thread instructions per term of k_series_part<0> and <1>
# (sm__inst_executed_pipe_fp64 x 32 / n, n = 1e8)
FP64_INSTR_PER_TERM = {0: 16.15, 1: 14.15}


def run_numeric(args, local) -> dict:
    """The paper's numeric MapReduce (Sec. 4.2) at n = 1e8: sum of sqrt(i)
    and the alternating harmonic sum, each term a correctly rounded double,
    compensated sums (wc_series_sum).  FP64-pipe bound: reported against the
    nominal FP64 rate of the part (no measured FP64 peak is available)."""
    import torch
    import oracle
    from paper_2206_05269_gb300 import wc
    torch.cuda.set_device(local)
    ctr = wc.Counter(local)
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device=f"cuda:{local}")
    n = 100_000_000
    res = {}
    for series, name in ((wc.WC_SERIES_SQRT, "sum_sqrt"), (wc.WC_SERIES_ALT_HARMONIC, "alt_harmonic")):
        for _ in range(3):
            wc.wc_series_sum(ctr.ctx, series, n, out.data_ptr(), stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            wc.wc_series_sum(ctr.ctx, series, n, out.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        got = float(out.cpu()[0])
        t0 = time.perf_counter()
        m = 10_000_000  # the oracle on a tenth of the terms (about a second of CPU work)
        oracle.series_sum(series, m)
        cpu_s = time.perf_counter() - t0
        # FP64-pipe bound: fp64 instructions per term from the ncu count of
        # this kernel (sm__inst_executed_pipe_fp64), against the part's
        # nominal FP64 rate, 1.25 TFLOP/s with an FMA counted twice
        per_term = FP64_INSTR_PER_TERM[series]
        ginstr = per_term * n / (ms * 1e-3) / 1e9
        res[name] = {"n": n, "value": got, "oracle": oracle.series_sum(series, n), "ms": ms,
                     "terms_per_s": n / (ms * 1e-3),
                     "roofline": {"bound": "fp64", "achieved": ginstr, "peak": 625.0,
                                  "unit": "G fp64 instructions/s", "frac": ginstr / 625.0,
                                  "peak_kind": "nominal FP64 rate of the part (1.25 TFLOP/s, FMA = 2)",
                                  "instr_per_term": per_term,
                                  "instr_source": "ncu sm__inst_executed_pipe_fp64 (profiles/numeric_series_fp64.md)"},
                     "cpu_baseline": {"value": m / cpu_s, "unit": "terms/s", "cores": 1, "kind": "oracle",
                                      "sample": f"first {m} terms, single-threaded compensated sum, {cpu_s:.2f} s"},
                     "paper_v100_ms": 73.372 if series == wc.WC_SERIES_SQRT else 65.323}
    ctr.close()
    return res


def run_hybrid(args, local) -> dict:
    """The paper's hybrid pipeline (Sec. 3.3, Sec. 4.1) on the class-split
    workload's 1,000 documents: CPU map into per-document dictionaries on
    every host core, grouped into a zero-padded count matrix, copied to the
    device, summed by rows on the GPU (wc_row_sums) -- beside the on-device
    path (text copied in, wc_count_batched, global table out) on the same
    documents.  Context for the host -> device cost the paper reports."""
    import torch
    import corpus
    import cpu_parallel
    from paper_2206_05269_gb300 import wc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c = corpus.generate("classes")
    stream = torch.cuda.current_stream()
    runs = []
    for _ in range(4):
        t0 = time.perf_counter()
        hy = cpu_parallel.HybridMap(c.text, c.offsets)
        m = torch.empty((hy.rows, hy.cols), dtype=torch.int32).pin_memory()
        hy.fill(m)
        t1 = time.perf_counter()
        dm = m.to(dev, non_blocking=True)
        sums = torch.empty(max(1, hy.rows), dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        wc.wc_row_sums(dm.data_ptr(), hy.rows, hy.cols, sums.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        h_sums = sums.cpu()
        t3 = time.perf_counter()
        runs.append({"map_and_group_ms": hy.seconds["map_and_group"] * 1e3, "matrix_ms": hy.seconds["matrix"] * 1e3,
                     "h2d_ms": (t2 - t1) * 1e3, "kernel_ms": e0.elapsed_time(e1), "total_ms": (t3 - t0) * 1e3,
                     "rows": hy.rows, "cols": hy.cols, "matrix_bytes": hy.rows * hy.cols * 4})
        del dm, m, hy
    best = min(runs[1:], key=lambda r: r["total_ms"])
    kb = best["matrix_bytes"] / (best["kernel_ms"] * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    best["row_sum_roofline"] = {"bound": "hbm", "achieved": kb, "peak": peak, "unit": "GB/s", "frac": kb / peak,
                                "peak_kind": peak_kind}
    # the on-device path on the same documents: text in, batched count, global table out
    host = torch.from_numpy(c.text).pin_memory()
    offs = torch.from_numpy(c.offsets.view(np.int64)).to(dev)
    ctr = wc.Counter(local, count_bits=32)
    tms = []
    for _ in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        text = host.to(dev, non_blocking=True)
        b = ctr.count_batched(text, offs, c.offsets)
        g = b.table(wc.WC_TABLE_GLOBAL)
        g.export()
        tms.append((time.perf_counter() - t0) * 1e3)
        b.free()
    ctr.close()
    best["on_device_total_ms"] = min(tms[1:])
    best["workload"] = "classes: 1,000 documents, 29.6 MB (the paper ran 4n speeches, n <= 500)"
    # the paper's own timings for 4n = 1,000 documents (Sec. 4.1, n = 250; a
    # 32-thread CPU and a V100; speech texts, sizes not given): context only
    best["paper_n250"] = {"map_cpu_ms": 49.808, "map_and_reduce_cpu_ms": 82.518,
                          "reduce_gpu_incl_matrix_and_copy_ms": 7.256,
                          "hardware": "32-thread CPU + V100", "docs": 1000}
    best["cpu_threads"] = os.cpu_count()
    return best


def run_mid(args, local) -> dict:
    """Single documents of 1, 4 and 15 MB (prefixes of the 1 GB corpus),
    counted whole by wc_count with the claim-as-you-go shared-memory table
    these sizes use, and with it switched off (every word to the global
    tables).  L2 is flushed before each timed count; the time is the whole
    count (tables, kernel, compaction, sort) on the launching stream."""
    import torch
    import corpus
    from paper_2206_05269_gb300 import wc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ctr = wc.Counter(local)
    out = {}
    for size in (1e6, 4e6, 15e6):
        c = corpus.generate("large", size_a=size)
        text = torch.from_numpy(c.text).to(dev)
        row = {"bytes": int(c.text.size)}
        for name, nl in (("level1", 0), ("all_global", 1)):
            ms = []
            for rep in range(23):
                flush.fill_(rep & 0xFF)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                t = ctr.count(text, stream, (0, 0, 0, nl))
                e1.record(stream)
                torch.cuda.synchronize()
                if t.status() != wc.WC_OK:
                    raise RuntimeError(f"mid-size count failed: {t.status()}")
                t.free()
                if rep >= 3:
                    ms.append(e0.elapsed_time(e1))
            ms.sort()
            med = ms[len(ms) // 2]
            row[name] = {"ms": med, "GBps": c.text.size / (med * 1e-3) / 1e9}
        row["speedup"] = row["all_global"]["ms"] / row["level1"]["ms"]
        out[f"{size / 1e6:.0f}MB"] = row
    ctr.close()
    out["l2"] = "flushed (256 MB written) before each timed count"
    return out


def _sub(line: dict) -> dict:
    """The parts of a workload's own result line that the default line carries."""
    keep = ("metric", "value", "unit", "ms_per_step", "higher_is_better", "config", "input_GBps", "per_launch_docs_s",
            "speedup_vs_per_launch", "roofline", "e2e", "e2e_vocab_ids", "gpu_launches", "clocks", "cpu_baseline",
            "p50_ms", "p99_ms",
            "req_per_s", "GBps", "fifo", "budget_waits")
    return {k: line[k] for k in keep if k in line}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="large",
                    choices=["large", "tiny", "classes", "batched", "served", "numeric", "hybrid", "mid"])
    ap.add_argument("--cpu-sample-mb", type=float, default=400.0)
    ap.add_argument("--bytes", type=float, default=1e9, help="corpus size (smaller only for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--docs", type=int, default=0, help="document count of a docs workload (smaller only for profiling)")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--fifo-seconds", type=float, default=2.0)
    ap.add_argument("--pool-bytes", type=float, default=2e9)
    ap.add_argument("--no-sub", action="store_true",
                    help="large workload only (no batched / served sub-objects in the default line)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if args.workload == "large":
        subs = {}
        if world == 1 and not args.no_sub and args.bytes == 1e9:
            # the batched (100,000 documents) and served (Poisson requests)
            # workloads, measured first and carried in the default line
            import copy
            for name in ("batched", "served"):
                a2 = copy.copy(args)
                a2.workload, a2.steps, a2.warmup, a2.docs = name, 10, 3, 0
                subs[name] = _sub(run_docs_workload(a2, local, False) if name == "batched"
                                  else run_served_workload(a2, local, False))
            subs["numeric"] = run_numeric(args, local)
            subs["hybrid"] = run_hybrid(args, local)
            subs["mid_sizes"] = run_mid(args, local)
        run_gpu(args, rank, world, local, subs)
    elif args.workload == "served":
        run_served_workload(args, local)
    elif args.workload in ("numeric", "hybrid", "mid"):  # one sub-measurement alone (profiling)
        fn = {"numeric": run_numeric, "hybrid": run_hybrid, "mid": run_mid}[args.workload]
        print(json.dumps({"workload": args.workload, "result": fn(args, local)}), flush=True)
    else:
        run_docs_workload(args, local)


if __name__ == "__main__":
    main()
