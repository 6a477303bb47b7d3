"""Benchmark: repairs/s of the batched, device-resident repair loop.

One step = the whole hot path over one batch of synthetic programs already
resident in device memory: the address traces of the programs the general
check kernel reads (a global array, or blocks that differ; none in the
default workload), every program's conflict relation (the check kernels:
Verify of Algorithm 1 under the empty mask), then the loop kernel (check by
the relation, clauses, exact hitting set, to the fixed point for every
program).  Default workload: 4,096 uneven programs (threads log-uniform
32-1024, blocks 1-16, statements 4-24, half repair / half removal mode),
the largest single-GPU batch of the paper-shaped workloads.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank repairs its own batch (programs offset by rank:
weak scaling, no collective on the data path); rank 0 prints one JSON line.
`--impl reference` times the CPU oracle (the slow plain-C definition) on a
bounded sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2011_08373_gb300 import synth  # noqa: E402

WORKLOAD = "uneven4096_mixed"
# further workloads timed on the device in the same run (extra keys)
EXTRA_WORKLOADS = ("batch1024_4x256_s24", "interblock256_64x256_s16")
CSRC = os.path.join(ROOT, "paper_2011_08373_gb300", "csrc")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._thr = None

    def sample_now(self):
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                 timeout=5).stdout.strip()
            if out:
                self.samples.append([x.strip() for x in out.split(",")])
        except Exception:
            pass

    def _run(self):
        while not self._stop.is_set():
            self.sample_now()
            self._stop.wait(0.2)

    def __enter__(self):
        self._thr = threading.Thread(target=self._run, daemon=True)
        self._thr.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._thr.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# CTA shapes (threads, CTAs per SM) the kernels are built for, in the order
# gr_tune_packed indexes them: the relation kernel's and the general check
# kernel's
REL_SHAPES = [(512, 3), (256, 4), (512, 2), (1024, 1), (256, 6), (128, 8)]
GEN_SHAPES = [(512, 2), (256, 3), (256, 4), (1024, 1), (384, 3)]


def shape_dict(shape, picked_by="autotuner"):
    rel, gen = shape & 0xFF, (shape >> 8) & 0xFF
    return {"relation": {"threads": REL_SHAPES[rel][0], "ctas_per_sm": REL_SHAPES[rel][1]},
            "general_check": {"threads": GEN_SHAPES[gen & 15][0], "ctas_per_sm": GEN_SHAPES[gen & 15][1],
                              "balanced_grid": bool(gen & 16)},
            "relation_runs_loop": bool((shape >> 16) & 1),
            "word": hex(shape), "picked_by": picked_by}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# the oracle's hitting set is brute force over 2^slots masks: beyond 24 slots
# one solve takes minutes, so no bounded sample exists
ORACLE_MAX_SLOTS = 24


def _oracle_feasible(workload):
    return synth.generate(workload, 1)[0].n_slots <= ORACLE_MAX_SLOTS


def run_reference(args, rank, world):
    """The CPU oracle, as it stands, on a bounded sample of the workload."""
    import oracle

    if rank != 0:
        return
    if not _oracle_feasible(args.workload):
        print(json.dumps({"impl": "reference", "unavailable": f"{args.workload} has more than "
                          f"{ORACLE_MAX_SLOTS} slots: the oracle's brute-force hitting set over 2^slots "
                          "masks has no bounded sample"}), flush=True)
        return
    cores = os.cpu_count() or 1
    wl = synth.WORKLOADS[args.workload]
    sample_n = args.ref_sample
    progs = synth.generate(args.workload, sample_n)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = oracle.repair_batch(progs, n_threads=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = sample_n * len(times) / total
    checks = sum(r["iters"] for r in res)
    line = {
        "impl": "reference", "metric": "repairs/s", "value": value, "unit": "repairs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "programs_per_step": sample_n,
                   "blocks": wl.blocks, "threads": wl.threads, "stmts": wl.n_stmts},
        "cpu_baseline": {"value": value, "unit": "repairs/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {sample_n} programs of {args.workload}, all-thread-pair "
                                   f"enumeration + brute-force hitting set, {cores} threads"},
        "e2e": {"value": value, "unit": "repairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "checks_per_step": checks,
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_leg(workload, n_sample):
    import oracle

    if not _oracle_feasible(workload):
        return None
    cores = os.cpu_count() or 1
    progs = synth.generate(workload, n_sample)
    oracle.repair_batch(progs[:2], n_threads=cores)  # build + warm
    t0 = time.perf_counter()
    oracle.repair_batch(progs, n_threads=cores)
    dt = time.perf_counter() - t0
    return {"value": n_sample / dt, "unit": "repairs/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n_sample} programs of {workload}, all-thread-pair enumeration + "
                      f"brute-force hitting set, {cores} threads, {dt:.1f} s"}


# Packed program records (DevProg, 1,440 bytes): n_stmts at byte 0, blocks
# 8, threads 12, the statement instances (32 bytes each: op, space, kind,
# flags, a, b, c, perm_off, guard k and r as u16 at 20 and 22) from byte 640;
# the arena header's u64 at byte 16 is the records' offset, its u32 at byte
# 120 the number of programs the relation kernel takes.
DEVPROG_BYTES = 1440
STMT0 = 640
WITNESS_BYTES = 272
RESULT_BYTES = 2944


def _guard_count(T, k, r):
    return T if k == 0 else ((T - 1 - r) // k + 1 if r < T else 0)


def check_bytes(arena, n):
    """Bytes one check of every program moves, two ways:

    expanded: the traces an expanded check reads, 4 bytes per active access
      over every block, plus, since the maps are evaluated in the kernel, a
      2-byte table entry per access of a permutation statement; plus the
      program record and the relation rows written;
    fused: what the relation kernel must move: the program record, the
      permutation entries of block 0 (blocks alike: block 0 decides every
      block), the relation rows.
    """
    off0 = int(arena[16:24].view(np.uint64)[0])
    expanded = fused = 0
    for i in range(n):
        off = off0 + DEVPROG_BYTES * i
        f = arena[off:off + 16].view(np.uint32)
        S, B, T = int(f[0]), int(f[2]), int(f[3])
        st = arena[off + STMT0:off + STMT0 + 32 * S].reshape(S, 32)
        for s in range(S):
            k = int(st[s, 20:22].view(np.uint16)[0])
            r = int(st[s, 22:24].view(np.uint16)[0])
            act = _guard_count(T, k, r)
            perm = int(st[s, 2]) == 2
            expanded += act * B * (4 + (2 if perm else 0))
            fused += act * 2 if perm else 0
        expanded += DEVPROG_BYTES + WITNESS_BYTES
        fused += DEVPROG_BYTES + WITNESS_BYTES
    return expanded, fused


def kernel_source_sha(files=("relation.cu", "loop.cuh", "device.cuh", "engine.cuh")):
    """Hash of the sources a kernel is built from (first 16 hex digits)."""
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# the sources each profiled kernel is built from, in hash order
KERNEL_SOURCES = {"k_relation": ("relation.cu", "loop.cuh", "device.cuh", "engine.cuh"),
                  "k_check": ("kernels.cu", "device.cuh", "engine.cuh")}


def profile_counters(kernel, workload):
    """Per-launch counters from the committed ncu summary of `kernel` on
    `workload`, if its recorded source hash is this build's (else None).  The
    summary carries one line `counters: source=<sha> wavefronts=<n>
    dram_bytes=<n>`."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    m = re.search(r"counters: source=(\w+) wavefronts=(\d+) dram_bytes=(\d+)", text)
    if not m or kernel not in KERNEL_SOURCES or m.group(1) != kernel_source_sha(KERNEL_SOURCES[kernel]):
        return None
    return {"wavefronts": int(m.group(2)), "dram_bytes": int(m.group(3)), "source": m.group(1)}


def shard(workload, n, rank):
    """Rank r repairs programs [r*n, (r+1)*n) of the workload: disjoint
    batches, no data exchanged between ranks."""
    return synth.generate(workload, n, start=rank * n)


def whole_job(n_per_rank, t_step_local, world, device="cuda"):
    """(whole-job repairs/s, max-over-ranks step time): every rank's batch
    counts, the slowest rank sets the time."""
    t = t_step_local
    if world > 1:
        import torch
        import torch.distributed as dist

        x = torch.tensor([t_step_local], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return n_per_rank * world / t, t


def _events(n):
    import torch

    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def time_steps(batch, steps, flush, stream):
    """CUDA-event times (ms) of each part of `steps` device steps: expansion of
    the general programs' traces, the relations, the loop.  The L2 is flushed
    before each step, outside the events."""
    import torch

    evs = []
    for _ in range(steps):
        flush.zero_()
        e = _events(4)
        e[0].record(stream)
        if batch.has_general:
            batch.expand()
        e[1].record(stream)
        batch.relation()
        e[2].record(stream)
        batch.loop()
        e[3].record(stream)
        evs.append(e)
    torch.cuda.synchronize()
    return [[a.elapsed_time(b) for a, b in zip(e[:-1], e[1:])] for e in evs]


def time_runs(batch, steps, flush, stream):
    """CUDA-event times (ms) of `steps` whole repairs of the batch, each one
    gr_repair_packed call (the relation and loop kernels, after the
    expansion and general check when the batch has general programs; one
    launch when the shape word has bit 16).  The L2 is flushed before each,
    outside the events."""
    import torch

    evs = []
    for _ in range(steps):
        flush.zero_()
        a, b = _events(2)
        a.record(stream)
        batch.run()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def fused(batch):
    """Whether run() of the batch is the one-launch relation + loop (bit 16
    of the shape word, given through --shape)."""
    return bool((getattr(batch, "shape", 0) >> 16) & 1)


def launches_per_step(batch):
    """Our kernels one run() launches: the fused relation + loop kernel, or
    the expansion (only with general programs), the split clearing and the
    general check kernel (general programs), the relation kernel (fast ones)
    and the loop kernel."""
    if fused(batch):
        return 1
    return 3 * int(batch.has_general) + int(batch.n_fast > 0) + 1


def device_workload(name, n, warmup, steps, flush, stream):
    """repairs/s and kernel times of one workload's batch, device-timed."""
    from paper_2011_08373_gb300 import binding

    progs = synth.generate(name, n)
    batch = binding.DeviceBatch(progs)
    batch.tune()
    for _ in range(warmup):
        batch.run()
    ms = statistics.mean(time_runs(batch, steps, flush, stream))
    t = time_steps(batch, steps, flush, stream)
    parts = [statistics.mean(x[i] for x in t) for i in range(3)]
    batch.run()
    res = batch.results_raw()
    status = np.bincount(res["status"].astype(np.int64), minlength=4)[:4].tolist()
    return {"repairs_per_s": n / (ms / 1000.0), "programs": n, "ms_per_step": ms, "one_launch": fused(batch),
            "expand_ms": parts[0], "relation_ms": parts[1], "loop_ms": parts[2],
            "checks_per_repair": float(res["iters"].mean()),
            "status_counts": {"repaired": status[0], "unrepairable": status[1], "iter_cap": status[2],
                              "timeout": status[3]}}


def serve_stream(rate, n, budget_gb, slots, local):
    """A Poisson request stream through the repair server: p50/p99 latency
    from submit to the poll that sees the result (host clock)."""
    from paper_2011_08373_gb300 import binding

    n_large = max(1, n // 20)
    small = synth.generate("uneven4096_mixed", n - n_large, start=100000)
    large = synth.generate("large_128x1024_s24", n_large)
    rng = synth.SplitMix64(synth.program_seed(11, 0))
    progs = list(small)
    for p in large:  # 5% large programs at seeded positions
        progs.insert(rng.randint(0, len(progs)), p)
    with binding.Server(mem_budget_bytes=budget_gb << 30, n_slots=slots) as srv:
        tk = [srv.submit(p) for p in progs[:64]]  # warm the server and the kernels
        srv.drain(600000)
        for t in tk:
            srv.poll(t)
        arrivals = synth.poisson_arrivals(rate, n, seed=int(rate))
        tickets, lat = [], {}
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            for p, at in zip(progs, arrivals):
                while time.perf_counter() - t0 < at:
                    pass
                tickets.append(srv.submit(p))
                if len(tickets) % 64 == 0:  # harvesting keeps the done map small
                    for t in tickets[-128:-64]:
                        if t not in lat:
                            r = srv.poll(t)
                            if r is not None:
                                lat[t] = r[1]
            srv.drain(600000)
            t_end = time.perf_counter()
        for t in tickets:
            if t not in lat:
                lat[t] = srv.poll(t)[1]
        ls = np.array([lat[t] for t in tickets]) * 1e6
        return {"rate_per_s": rate, "requests": n, "p50_us": float(np.percentile(ls, 50)),
                "p99_us": float(np.percentile(ls, 99)), "repairs_per_s": n / (t_end - t0),
                "offered_per_s": n / float(arrivals[-1]),
                "config": {"workload": "uneven4096_mixed + 5% large_128x1024_s24", "budget_gb": budget_gb,
                           "slots": slots},
                "launches": srv.stats()["launches"], "clocks": clk.summary()}


def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist

    from paper_2011_08373_gb300 import binding
    from paper_2011_08373_gb300.build import build

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    build()
    wl = synth.WORKLOADS[args.workload]
    n = args.programs or wl.n_programs
    progs = shard(args.workload, n, rank)
    batch = binding.DeviceBatch(progs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # twice the 126 MB L2
    props = torch.cuda.get_device_properties(local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    if args.shape is None:
        shape = batch.tune()  # the autotuner picks the CTA shapes for this batch
    else:  # a word an earlier run's autotuner printed (its config.cta_shape.word)
        shape = batch.set_shape(args.shape)
    for _ in range(args.warmup):
        batch.run()
    barrier()
    with ClockSampler(local) as clk:
        barrier()
        wall0 = time.perf_counter()
        step_ms = time_runs(batch, args.steps, flush, stream)  # the timed steps: whole repairs
        clk.sample_now()
        barrier()
        wall = time.perf_counter() - wall0
    # the parts of a step, timed apart (the stage calls: expansion, relations,
    # loop) for the kernel rooflines and the breakdown
    t = time_steps(batch, args.steps, flush, stream)
    expand_ms, rel_ms, loop_ms = ([x[i] for x in t] for i in range(3))
    batch.run()
    t_step = statistics.mean(step_ms) / 1000.0
    _, t_step = whole_job(n, t_step, world)
    res = batch.results_raw()
    checks = int(res["iters"].sum())
    pairs = int(res["access_pairs"].sum())
    status = np.bincount(res["status"].astype(np.int64), minlength=4)[:4].tolist()
    lat = (res["t_end_ns"].astype(np.int64) - int(res["t_start_ns"].min())) / 1e3
    value = n * world / t_step
    clocks = clk.summary()
    hbm_peak, peak_kind = _peaks()

    # rooflines.  The check kernel (relation) does one check per program, the
    # empty-mask one; its bytes per check are those of an expanded check (4-byte
    # trace reads of every active access over every block), next to the bytes
    # the fused kernel must move.  Its shared-memory fraction takes the
    # wavefronts per launch from the committed ncu summary of this kernel
    # build and workload over this run's kernel time and the SMs' 128 bytes
    # per clock at the sampled SM clock.
    t_rel = statistics.mean(rel_ms) / 1000.0
    t_loop = statistics.mean(loop_ms) / 1000.0
    expanded_b, fused_b = check_bytes(batch.host_arena, n)
    # the check kernel: the relation kernel for programs on the shared array
    # with alike blocks, the general check kernel (after the expansion) for
    # the others
    check_kernel = ("k_relation" if not batch.has_general else
                    "k_check" if batch.n_fast == 0 else "k_relation + k_check")
    prof = profile_counters(check_kernel, args.workload)
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    smem_peak = props.multi_processor_count * 128 * sm_mhz * 1e6 / 1e9  # GB/s
    check = {"kernel": check_kernel, "ms": t_rel * 1000, "checks_per_launch": n, "bound": "hbm",
             "algorithmic_bytes": expanded_b, "fused_bytes": fused_b,
             "achieved": expanded_b / t_rel / 1e9, "peak": hbm_peak, "unit": "GB/s",
             "frac": expanded_b / t_rel / 1e9 / hbm_peak, "peak_kind": peak_kind,
             "fused_frac": fused_b / t_rel / 1e9 / hbm_peak,
             "traffic": prof["dram_bytes"] if prof else None,
             "smem": ({"achieved": prof["wavefronts"] * 128 / t_rel / 1e9, "peak": smem_peak, "unit": "GB/s",
                       "frac": prof["wavefronts"] * 128 / t_rel / 1e9 / smem_peak,
                       "wavefronts_per_launch": prof["wavefronts"], "source": prof["source"],
                       "peak_def": f"{props.multi_processor_count} SMs x 128 B/clk x {sm_mhz:.0f} MHz"}
                      if prof else None)}
    loop_b = n * (DEVPROG_BYTES + WITNESS_BYTES + RESULT_BYTES)
    loop_rf = {"kernel": "k_loop", "ms": t_loop * 1000, "bound": "hbm", "algorithmic_bytes": loop_b,
               "achieved": loop_b / t_loop / 1e9, "peak": hbm_peak, "unit": "GB/s",
               "frac": loop_b / t_loop / 1e9 / hbm_peak, "peak_kind": peak_kind, "traffic": None}
    dominant = check if t_rel >= t_loop else loop_rf
    roofline = {k: dominant[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel",
                                         "algorithmic_bytes", "peak_kind")}

    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        # the C-ABI call with host buffers: validate + pack into pinned staging
        # + H2D + relations + loop + D2H of the results (marshalling of the
        # Python objects into C structs happens once, outside the timed region)
        pb = binding.ProgramBatch(progs)
        host_out = np.zeros(n, dtype=binding.RESULT_DTYPE)
        binding.repair_batch_raw(pb, out=host_out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            binding.repair_batch_raw(pb, out=host_out)
        e2e_t = (time.perf_counter() - t0) / args.e2e_steps
        e2e = {"value": n / e2e_t, "unit": "repairs/s", "h2d_bytes_per_step": int(batch.arena_bytes),
               "d2h_bytes_per_step": int(n * binding.RESULT_DTYPE.itemsize),
               "note": "gr_repair_batch on host program structs: validate + pack + H2D + kernels + D2H",
               "same_results": bool(np.array_equal(host_out["mask"], res["mask"])
                                    and np.array_equal(host_out["iters"], res["iters"]))}
    plain = plain_device = None
    if rank == 0 and args.plain_programs > 0:
        # the plain path: one check launch and one solve launch per loop
        # iteration, the host reading the done flag between them.  Host rate:
        # whole calls (validate + pack + upload + loop); device rate: the
        # CUDA-event time of the launch loop alone, summed over the programs
        sub = progs[:args.plain_programs]
        binding.repair_plain(sub[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain_ms = 0.0
        for p in sub:
            _, ms = binding.repair_plain_timed(p)
            plain_ms += ms
        plain = len(sub) / (time.perf_counter() - t0)
        plain_device = len(sub) / (plain_ms * 1e-3)
    strategies = None
    if rank == 0 and args.strategy_steps > 0:
        # the paper's mhs strategy against the exact (MaxSAT) strategy on the
        # same batch: masks checked per repair (the verifier-call analogue) and
        # the loop kernel's time; both must end at the same masks
        gb = binding.DeviceBatch(progs, strategy=binding.STRATEGY_MHS)
        gb.tune()
        gb.run()
        tg = time_steps(gb, args.strategy_steps, flush, stream)
        gres = gb.results_raw()
        strategies = {
            "maxsat": {"checks_per_repair": checks / n, "loop_ms": statistics.mean(loop_ms)},
            "mhs": {"checks_per_repair": int(gres["iters"].sum()) / n,
                    "loop_ms": statistics.mean(x[2] for x in tg)},
            "same_final_mask": float(np.mean((gres["mask"] == res["mask"]) & (gres["status"] == res["status"]))),
        }
        del gb
    check_leg = None
    if rank == 0 and args.check_steps > 0:
        # gr_check_expanded: one check per program under the empty mask, with
        # its divergence and pair count, on the relation kernel
        batch.check([0] * n)
        torch.cuda.synchronize()
        c_ms = []
        for _ in range(args.check_steps):
            flush.zero_()
            a, b = _events(2)
            a.record(stream)
            batch.check(None, expanded=True)
            b.record(stream)
            torch.cuda.synchronize()
            c_ms.append(a.elapsed_time(b))
        check_leg = {"checks_per_s": n / (statistics.mean(c_ms) / 1000), "check_call_ms": statistics.mean(c_ms),
                     "mask": 0}
    wide = None
    if rank == 0 and args.wide_steps > 0:
        # the wide lane on the same batch: one CTA per (program, block) per
        # check, the loop as a device-side graph; host wall time per call
        batch.run_wide()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.wide_steps):
            batch.run_wide()
            torch.cuda.synchronize()
        t_w = (time.perf_counter() - t0) / args.wide_steps
        wres = batch.results_raw()
        wide = {"repairs_per_s": n / t_w, "ms_per_call": t_w * 1000,
                "same_results": bool(np.array_equal(wres["mask"], res["mask"])
                                     and np.array_equal(wres["iters"], res["iters"])),
                "note": "gr_repair_packed_wide, host wall clock per call incl. synchronisation"}
    extra = None
    if rank == 0 and args.extra_steps > 0:
        extra = {w: device_workload(w, synth.WORKLOADS[w].n_programs, 3, args.extra_steps, flush, stream)
                 for w in EXTRA_WORKLOADS}
    serving = None
    if rank == 0 and args.serve_requests > 0 and args.serve_rate > 0:
        serving = serve_stream(args.serve_rate, args.serve_requests, args.serve_budget_gb, args.serve_slots,
                               local)
    cpu = None
    if rank == 0 and args.cpu_sample > 0:
        cpu = cpu_baseline_leg(args.workload, args.cpu_sample)
    if rank == 0:
        line = {
            "metric": "repairs/s", "value": value, "unit": "repairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1000,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": args.workload, "programs": n, "blocks": wl.blocks, "threads": wl.threads,
                       "stmts": wl.n_stmts, "m_words": wl.m_words, "seed": wl.seed,
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "cta_shape": shape_dict(shape, "autotuner" if args.shape is None else "--shape"),
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e,
            "gpu_launches": launches_per_step(batch) * args.steps,
            "roofline": roofline,
            "check_roofline": check,
            "loop_roofline": loop_rf,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "checks_per_s": checks * world / t_step,
            "access_pair_checks_per_s": pairs * world / t_step,
            "plain_repairs_per_s": plain,
            "plain_device_repairs_per_s": plain_device,
            "one_launch": fused(batch),
            "expand_ms": statistics.mean(expand_ms), "relation_ms": t_rel * 1000, "loop_ms": t_loop * 1000,
            "latency_in_batch_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "status_counts": {"repaired": status[0], "unrepairable": status[1], "iter_cap": status[2],
                              "timeout": status[3]},
            "checks_per_repair": checks / n, "strategies": strategies, "wide_lane": wide,
            "check_kernel": check_leg, "workloads": extra, "serving": serving, "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_serve(args, rank, world, local):
    """Poisson request streams through the repair server (p50/p99 latency)."""
    import torch

    from paper_2011_08373_gb300.build import build

    if rank != 0:
        return
    torch.cuda.set_device(local)
    build()
    lines = []
    for rate in args.serve_rates:
        line = {"metric": "p50/p99 repair latency (serving)"}
        line.update(serve_stream(rate, args.serve_requests, args.serve_budget_gb, args.serve_slots, local))
        lines.append(line)
        print(json.dumps(line), flush=True)
    return lines


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--programs", type=int, default=0)
    ap.add_argument("--shape", type=lambda x: int(x, 0), default=None,
                    help="CTA shape word to use instead of running the autotuner (config.cta_shape.word of "
                         "an earlier run): profilers serialise launches, which changes the autotuner's pick")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--plain-programs", type=int, default=64)
    ap.add_argument("--check-steps", type=int, default=5,
                    help="timed launches of the check kernel alone on the same batch (0: skip)")
    ap.add_argument("--wide-steps", type=int, default=3,
                    help="calls of the wide lane on the same batch (0: skip)")
    ap.add_argument("--strategy-steps", type=int, default=5,
                    help="timed launches of the mhs strategy on the same batch (0: skip)")
    ap.add_argument("--extra-steps", type=int, default=10,
                    help="timed steps of each further workload (batch of 1,024; inter-block), 0: skip")
    ap.add_argument("--cpu-sample", type=int, default=64)
    ap.add_argument("--ref-sample", type=int, default=64)
    ap.add_argument("--serve", action="store_true", help="Poisson request streams through the server")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[200.0, 500.0, 2000.0])
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-rate", type=float, default=2000.0,
                    help="Poisson rate of the serving leg of the default run (0: skip)")
    ap.add_argument("--serve-budget-gb", type=int, default=40)
    ap.add_argument("--serve-slots", type=int, default=4)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.serve:
        run_serve(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
