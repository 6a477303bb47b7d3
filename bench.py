"""Benchmark: repairs/s of the batched, device-resident repair loop.

One step = the whole hot path over one batch of synthetic programs already
resident in device memory: address-trace expansion, then the persistent
repair launch (check -> clauses -> exact hitting set, to the fixed point for
every program).  Default workload: 1,024 programs, 4 blocks x 256 threads,
24 statements, 23 block slots, 1,024-word shared array.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank repairs its own batch (programs offset by rank:
weak scaling, no collective on the data path); rank 0 prints one JSON line.
`--impl reference` times the CPU oracle (the slow plain-C definition) on a
bounded sample of the same workload, on the host cores.
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
sys.path.insert(0, ROOT)

from paper_2011_08373_gb300 import synth  # noqa: E402

WORKLOAD = "batch1024_4x256_s24"
# DRAM bytes (read + write) of one k_repair launch, from the ncu capture summarised in
# profiles/k_repair_batch1024_4x256_s24.md; reset to None whenever k_repair changes.
NCU_TRAFFIC = {"batch1024_4x256_s24": 13_618_432}
# the same for one k_check launch (profiles/k_check_batch1024_4x256_s24.md)
NCU_CHECK_TRAFFIC = {"batch1024_4x256_s24": 13_586_432}


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


def shape_dict(shape):
    rel, gen = shape & 0xFF, (shape >> 8) & 0xFF
    return {"relation": {"threads": REL_SHAPES[rel][0], "ctas_per_sm": REL_SHAPES[rel][1]},
            "general_check": {"threads": GEN_SHAPES[gen & 15][0], "ctas_per_sm": GEN_SHAPES[gen & 15][1],
                              "balanced_grid": bool(gen & 16)},
            "picked_by": "autotuner"}


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


# DevProg fields of a packed arena (bytes): n_stmts 0, blocks 8, threads 12,
# shared_rows 44, global_rows 48, blocks alike 56; records of 1,440 bytes
DEVPROG_BYTES = 1440


def check_bytes(arena, i):
    """Trace bytes one check of packed program i reads."""
    off = int(arena[16:24].view(np.uint64)[0]) + DEVPROG_BYTES * i
    f = arena[off:off + 64].view(np.uint32)
    n_inst, blocks, threads = int(f[0]), int(f[2]), int(f[3])
    shared, glob, alike = int(f[11]), int(f[12]), int(f[14])
    if alike and blocks > 1:
        return (bin(shared).count("1") + bin(glob).count("1") * blocks) * threads * 2
    return n_inst * blocks * threads * 2


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
    l2_flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    shape = batch.tune()  # the autotuner picks the CTA shape for this batch
    for _ in range(args.warmup):
        batch.run()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        wall0 = time.perf_counter()
        for i in range(args.steps):
            l2_flush.zero_()  # inputs fit in L2: flush it between steps (outside the events)
            e0, e1, e2 = ev[i]
            e0.record(stream)
            batch.expand()
            e1.record(stream)
            batch.repair_expanded()
            e2.record(stream)
        clk.sample_now()  # the queued steps are still running on the device
        barrier()
        wall = time.perf_counter() - wall0
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    repair_ms = [b.elapsed_time(c) for a, b, c in ev]
    expand_ms = [a.elapsed_time(b) for a, b, c in ev]
    t_step = sum(step_ms) / len(step_ms) / 1000.0
    _, t_step = whole_job(n, t_step, world)
    res = batch.results_raw()
    checks = int(res["iters"].sum())
    pairs = int(res["access_pairs"].sum())
    status = np.bincount(res["status"].astype(np.int64), minlength=3)[:3].tolist()
    lat = (res["t_end_ns"].astype(np.int64) - int(res["t_start_ns"].min())) / 1e3
    value, _ = whole_job(n, t_step, 1)
    value *= world

    # algorithmic bytes of the repair kernel: each check reads the traces it
    # needs once (u16 addresses of T threads per (statement instance, block):
    # every block, or block 0 of the shared-array statements when the
    # program's blocks are alike); the arena and results once per launch
    trace_bytes = sum(check_bytes(batch.host_arena, i) * int(r["iters"]) for i, r in enumerate(res))
    launch_bytes = trace_bytes + batch.arena_bytes + n * binding.RESULT_DTYPE.itemsize
    t_rep = statistics.mean(repair_ms) / 1000.0
    peak, peak_kind = _peaks()
    achieved = launch_bytes / t_rep / 1e9
    traffic = NCU_TRAFFIC.get(args.workload)
    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        # the C-ABI call with host buffers: validate + pack into pinned staging
        # + H2D + expansion + repair + D2H of the results (marshalling of the
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
               "note": "gr_repair_batch on host program structs: validate + pack + H2D + kernels + D2H"}
    plain = None
    if rank == 0 and args.plain_programs > 0:
        sub = progs[:args.plain_programs]
        binding.repair_plain(sub[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for p in sub:
            binding.repair_plain(p)
        plain = len(sub) / (time.perf_counter() - t0)
    strategies = None
    if rank == 0 and args.strategy_steps > 0:
        # the paper's mhs strategy against the exact (MaxSAT) strategy on the
        # same batch: masks checked per repair (the verifier-call analogue) and
        # the repair kernel's time; both must end at the same masks
        gb = binding.DeviceBatch(progs, strategy=binding.STRATEGY_MHS)
        gb.tune()
        gb.expand()
        gb.repair_expanded()
        torch.cuda.synchronize()
        g_ms = []
        for _ in range(args.strategy_steps):
            l2_flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            gb.expand()
            a.record(stream)
            gb.repair_expanded()
            b.record(stream)
            torch.cuda.synchronize()
            g_ms.append(a.elapsed_time(b))
        gres = gb.results_raw()
        strategies = {
            "maxsat": {"checks_per_repair": checks / n, "repair_kernel_ms": statistics.mean(repair_ms)},
            "mhs": {"checks_per_repair": int(gres["iters"].sum()) / n,
                    "repair_kernel_ms": statistics.mean(g_ms)},
            "same_final_mask": float(np.mean((gres["mask"] == res["mask"]) & (gres["status"] == res["status"]))),
        }
        del gb
    check = None
    if rank == 0 and args.check_steps > 0:
        # the check kernel alone (gr_check_expanded): one check per program
        # under the empty mask, where every statement pair is a candidate
        batch.check([0] * n)
        torch.cuda.synchronize()
        c_ms = []
        for _ in range(args.check_steps):
            l2_flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch.check(None, expanded=True)
            b.record(stream)
            torch.cuda.synchronize()
            c_ms.append(a.elapsed_time(b))
        t_c = statistics.mean(c_ms) / 1000.0
        c_bytes = (sum(check_bytes(batch.host_arena, i) for i in range(n)) + batch.arena_bytes
                   + n * binding.WITNESS_DTYPE.itemsize)
        check = {"checks_per_s": n / t_c, "check_kernel_ms": t_c * 1000, "mask": 0,
                 "roofline": {"bound": "hbm", "achieved": c_bytes / t_c / 1e9, "peak": peak, "unit": "GB/s",
                              "frac": c_bytes / t_c / 1e9 / peak, "kernel": "k_check",
                              "algorithmic_bytes": c_bytes, "traffic": NCU_CHECK_TRAFFIC.get(args.workload)}}
    wide = None
    if rank == 0 and args.wide_steps > 0:
        # the wide lane on the same batch: one CTA per (program, block) per
        # check, the loop as a device-side graph; host wall time per call
        # (header read, expansion, graph build and launch, completion)
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
                       "cta_shape": shape_dict(shape),
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e,
            "gpu_launches": 2 * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": "k_repair",
                         "algorithmic_bytes": launch_bytes, "peak_kind": peak_kind},
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "checks_per_s": checks * world / t_step,
            "access_pair_checks_per_s": pairs * world / t_step,
            "plain_repairs_per_s": plain,
            "expand_ms": statistics.mean(expand_ms), "repair_kernel_ms": statistics.mean(repair_ms),
            "latency_in_batch_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "status_counts": {"repaired": status[0], "unrepairable": status[1], "iter_cap": status[2]},
            "checks_per_repair": checks / n, "strategies": strategies, "wide_lane": wide,
            "check_kernel": check, "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_serve(args, rank, world, local):
    """Poisson request streams through the repair server (p50/p99 latency)."""
    import torch

    from paper_2011_08373_gb300 import binding
    from paper_2011_08373_gb300.build import build

    if rank != 0:
        return
    torch.cuda.set_device(local)
    build()
    n = args.serve_requests
    n_large = max(1, n // 20)
    small = synth.generate("uneven4096_mixed", n - n_large, start=100000)
    large = synth.generate("large_128x1024_s24", n_large)
    rng = synth.SplitMix64(synth.program_seed(11, 0))
    progs = list(small)
    for p in large:  # 5% large programs at seeded positions
        progs.insert(rng.randint(0, len(progs)), p)
    lines = []
    with binding.Server(mem_budget_bytes=args.serve_budget_gb << 30, n_slots=args.serve_slots) as srv:
        # warm the server and the kernels
        tk = [srv.submit(p) for p in progs[:64]]
        srv.drain(600000)
        for t in tk:
            srv.poll(t)
        for rate in args.serve_rates:
            arrivals = synth.poisson_arrivals(rate, n, seed=int(rate))
            tickets = []
            lat = {}
            with ClockSampler(local) as clk:
                t0 = time.perf_counter()
                for p, at in zip(progs, arrivals):
                    while time.perf_counter() - t0 < at:
                        pass
                    tickets.append(srv.submit(p))
                    # opportunistic harvesting keeps the done map small
                    if len(tickets) % 64 == 0:
                        for t in tickets[-128:-64]:
                            if t not in lat:
                                r = srv.poll(t)
                                if r is not None:
                                    lat[t] = r[1]
                srv.drain(600000)
                t_end = time.perf_counter()
            for t in tickets:
                if t not in lat:
                    r = srv.poll(t)
                    lat[t] = r[1]
            ls = np.array([lat[t] for t in tickets]) * 1e6
            line = {"metric": "p50/p99 repair latency (serving)", "rate_per_s": rate, "requests": n,
                    "p50_us": float(np.percentile(ls, 50)), "p99_us": float(np.percentile(ls, 99)),
                    "repairs_per_s": n / (t_end - t0), "offered_per_s": n / float(arrivals[-1]),
                    "config": {"workload": "uneven4096_mixed + 5% large_128x1024_s24",
                               "budget_gb": args.serve_budget_gb, "slots": args.serve_slots},
                    "launches": srv.stats()["launches"], "clocks": clk.summary()}
            lines.append(line)
            print(json.dumps(line), flush=True)
    return lines


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--programs", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--plain-programs", type=int, default=64)
    ap.add_argument("--check-steps", type=int, default=5,
                    help="timed launches of the check kernel alone on the same batch (0: skip)")
    ap.add_argument("--wide-steps", type=int, default=5,
                    help="calls of the wide lane on the same batch (0: skip)")
    ap.add_argument("--strategy-steps", type=int, default=5,
                    help="timed launches of the mhs strategy on the same batch (0: skip)")
    ap.add_argument("--cpu-sample", type=int, default=32)
    ap.add_argument("--ref-sample", type=int, default=16)
    ap.add_argument("--serve", action="store_true", help="Poisson request streams through the server")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[200.0, 500.0, 2000.0])
    ap.add_argument("--serve-requests", type=int, default=1000)
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
