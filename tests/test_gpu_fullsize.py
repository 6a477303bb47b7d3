"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (the packed, device-resident batch, persistent launch).

Every program of every batch is compared with the oracle's own loop on every
field.  Where the oracle's thread-pair enumeration is too slow for a whole
batch (64 x 256 global arrays, launches of up to 16 x 1,024 or 128 x 1,024
threads) its loop verifies with the same definition grouped by word
(orc_check_words, pinned against the enumeration on CPU).  Independently of
that, the one-pair enumeration gives the unconstrained witness set W(0) pair
by pair for sampled programs, its solver the expected final mask from W(0)
(clauses are exact, so the loop ends at the lowest-key mask over all masks
whose own check is clean, whatever the trajectory), and a launch-independent
copy of the program (same threads and slot guards, no accesses) gives the
divergent slots."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
from paper_2011_08373_gb300 import synth
from paper_2011_08373_gb300.synth import MODE_REPAIR, OP_W

pytestmark = pytest.mark.gpu

KEYS = ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses", "forbidden",
        "access_pairs")
N_THREADS = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def gb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08373_gb300.build import build
    from paper_2011_08373_gb300 import binding

    build()
    binding.lib()
    return binding


def _run(gb, progs):
    import torch

    db = gb.DeviceBatch(progs)
    db.run()
    torch.cuda.synchronize()
    return db, db.results()


def _properties(p, r):
    """Facts every result must satisfy, at any size."""
    n = p.n_slots
    assert r["iters"] <= n + 3
    assert r["weight"] == sum(int(p.slot_weight[k]) for k in range(n) if (r["mask"] >> k) & 1)
    assert r["clauses"] == sorted(set(r["clauses"]))
    # repair mode starts at MHS(empty) = E, removal mode probes E
    assert (r["iters"] == 0 and r["status"] == 1) or r["traj"][0] == p.existing_mask
    if r["status"] == 0:
        assert r["mask"] == r["traj"][-1]
        assert all(r["mask"] & c for c in r["clauses"])
        assert not (r["mask"] & r["forbidden"])


def _w0_by_pairs(p, mask=0):
    S = p.n_stmts
    cand = [(i, j) for i in range(S) for j in range(i, S)
            if p.space[i] == p.space[j] and (p.op[i] == OP_W or p.op[j] == OP_W)]
    with cf.ThreadPoolExecutor(N_THREADS) as ex:
        res = list(ex.map(lambda ij: oracle.check_pair(p, mask, *ij), cand))
    intra, inter = [0] * S, [0] * S
    pairs = 0
    for (i, j), (a, b, n) in zip(cand, res):
        intra[i] |= int(a) << j
        inter[i] |= int(b) << j
        pairs += n
    return {"intra": intra, "inter": inter, "diverge": 0, "access_pairs": pairs}


def _divergent_slots(p):
    """Divergence depends only on the slot guards and the thread count: check
    a copy with the same threads and slots whose statements touch nothing
    that could race, under all slots on."""
    q = synth.make_program([{"op": "R"} for _ in range(p.n_stmts)], blocks=1, threads=p.threads,
                           m_shared=1, slot_level=p.slot_level.tolist(),
                           slot_guard=list(zip(p.slot_guard_k.tolist(), p.slot_guard_r.tolist())),
                           slot_weight=p.slot_weight.tolist())
    return oracle.check(q, (1 << p.n_slots) - 1)["diverge"]


def _expected_final(p, w0):
    n = p.n_slots
    forced = p.existing_mask if p.mode == MODE_REPAIR else 0
    cls = oracle.clauses(p, w0)
    sol = oracle.solve(n, [int(x) for x in p.slot_weight], cls, (), forced, _divergent_slots(p))
    return sol, cls


def test_batch1024_full_size(gb):
    progs = synth.generate("batch1024_4x256_s24")
    assert len(progs) == 1024
    _, got = _run(gb, progs)
    for p, r in zip(progs, got):
        _properties(p, r)
    # every program, every field (about 30 s of oracle time on 16 cores)
    want = oracle.repair_batch(progs, n_threads=N_THREADS)
    for i, w in enumerate(want):
        for k in KEYS:
            assert got[i][k] == w[k], (i, k)


def test_uneven4096_full_size(gb):
    progs = synth.generate("uneven4096_mixed")
    assert len(progs) == 4096
    _, got = _run(gb, progs)
    for p, r in zip(progs, got):
        _properties(p, r)
    # every program, every field: the oracle's loop verifying by thread-pair
    # enumeration on the programs of at most 1,024 threads in all, by the
    # word-grouped check on all (about a minute of oracle time on 16 cores)
    small = [i for i, p in enumerate(progs) if p.blocks * p.threads <= 1024]
    assert len(small) > 1000
    big = max(range(len(progs)), key=lambda i: progs[i].blocks * progs[i].threads * progs[i].n_stmts)
    want = oracle.repair_batch([progs[i] for i in small], n_threads=N_THREADS)
    for i, w in zip(small, want):
        for k in KEYS:
            assert got[i][k] == w[k], (i, k)
    want = oracle.repair_batch(progs, n_threads=N_THREADS, words=True)
    for i, w in enumerate(want):
        for k in KEYS:
            assert got[i][k] == w[k], (i, k)
    # the host-pointer call (chunks packed on the host, its own tuned shapes)
    # agrees with the device-resident launch on every program and field
    host = gb.repair_batch(progs)
    for i in range(len(progs)):
        for k in KEYS:
            assert host[i][k] == got[i][k], (i, k)
    # the largest program of the batch: W(0) by sampled pairs, final mask by path independence
    p = progs[big]
    sol, _ = _expected_final(p, _w0_by_pairs(p))
    r = got[big]
    if sol is None:
        assert r["status"] == 1
    else:
        assert r["status"] == 0 and (r["mask"], r["weight"]) == sol


@pytest.mark.parametrize("idx", [3, 77])
def test_interblock_full_size_sampled(gb, idx):
    progs = synth.generate("interblock256_64x256_s16")
    assert len(progs) == 256 and progs[idx].blocks == 64 and progs[idx].m_global == 65536
    db, got = _run(gb, progs)
    db.check([0] * len(progs))
    import torch

    torch.cuda.synchronize()
    w_gpu = db.witnesses(progs)[idx]
    p = progs[idx]
    w0 = _w0_by_pairs(p)
    assert w_gpu["intra"] == w0["intra"] and w_gpu["inter"] == w0["inter"]
    assert w_gpu["access_pairs"] == w0["access_pairs"]
    sol, cls = _expected_final(p, w0)
    r = got[idx]
    _properties(p, r)
    if sol is None:
        assert r["status"] == 1
    else:
        assert r["status"] == 0 and (r["mask"], r["weight"]) == sol
    # repair mode with no existing barriers: the first check (mask 0) sees every race
    assert r["clauses"] == cls


def test_interblock_full_size_every_field(gb):
    """Every program of the inter-block batch (64 blocks x 256 threads over a
    65,536-word global array) at full size, compared with the oracle's own
    loop on every field: trajectory, iterations, clauses, access pairs (the
    loop verifying with the word-grouped check; eight programs also with the
    thread-pair enumeration)."""
    progs = synth.generate("interblock256_64x256_s16")
    _, got = _run(gb, progs)
    want = oracle.repair_batch(progs, n_threads=N_THREADS, words=True)
    for i, w in enumerate(want):
        for k in KEYS:
            assert got[i][k] == w[k], (i, k)
    idx = list(range(5, 256, 32))
    want = oracle.repair_batch([progs[i] for i in idx], n_threads=N_THREADS)
    for i, w in zip(idx, want):
        for k in KEYS:
            assert got[i][k] == w[k], (i, k)


def test_large_program_full_size(gb):
    progs = synth.generate("large_128x1024_s24", 2)
    _, got = _run(gb, progs)
    for p, r in zip(progs, got):
        _properties(p, r)
        sol, _ = _expected_final(p, _w0_by_pairs(p))
        if sol is None:
            assert r["status"] == 1
        else:
            assert r["status"] == 0 and (r["mask"], r["weight"]) == sol
    # every field, the oracle's loop verifying with the word-grouped check
    want = oracle.repair_batch(progs, n_threads=N_THREADS, words=True)
    for i, w in enumerate(want):
        for k in KEYS:
            assert got[i][k] == w[k], (i, k)


def test_loops512_full_size(gb):
    progs = synth.generate("loops512_4x256_s12")
    assert len(progs) == 512 and all(p.loops for p in progs)
    _, got = _run(gb, progs)
    for p, r in zip(progs, got):
        _properties(p, r)
    sample = list(range(0, 512, 16))
    want = oracle.repair_batch([progs[i] for i in sample], n_threads=N_THREADS)
    for i, w in zip(sample, want):
        for k in KEYS:
            assert got[i][k] == w[k], (i, k)
    want = oracle.repair_batch(progs, n_threads=N_THREADS, words=True)
    for i, w in enumerate(want):
        for k in KEYS:
            assert got[i][k] == w[k], (i, k)


def test_sites128_full_size(gb):
    """The batch with 30 barrier variables per program (a block and a grid
    candidate at 15 sites; 16 blocks x 256 threads over a global array) at
    full size, every program.  The oracle's brute-force solve cannot reach 30
    variables, so: the device's check under the empty mask equals the
    oracle's (word-grouped) on every field; the repair ends at the lowest-key
    mask over the clauses of those witnesses (path independence), found by
    integer programming; its clauses are among those; and the check of its
    final mask is equal on both sides."""
    pytest.importorskip("scipy.optimize")
    import torch
    from test_oracle_pins import milp_lowest_key

    progs = synth.generate("sites128_16x256_s16")
    assert len(progs) == 128 and all(p.n_slots == 30 for p in progs)
    db, got = _run(gb, progs)
    db.check([0] * len(progs))
    torch.cuda.synchronize()
    w_dev = db.witnesses(progs)
    db.check([r["mask"] for r in got])
    torch.cuda.synchronize()
    w_fin = db.witnesses(progs)
    for i, (p, r) in enumerate(zip(progs, got)):
        _properties(p, r)
        w0 = oracle.check(p, 0, words=True)
        assert w_dev[i] == w0, i
        cls = oracle.clauses(p, w0)
        div = oracle.check(p, (1 << p.n_slots) - 1, words=True)["diverge"]
        forced = p.existing_mask if p.mode == MODE_REPAIR else 0
        want = milp_lowest_key(p.n_slots, [int(x) for x in p.slot_weight], cls, p.neg_clauses, forced, div)
        if want is None:
            assert r["status"] == 1, i
        else:
            assert r["status"] == 0 and (r["mask"], r["weight"]) == want, i
            assert set(r["clauses"]) <= set(cls), i
            assert w_fin[i] == oracle.check(p, r["mask"], words=True), i


def test_wide_lane_full_size(gb):
    """The wide lane at full size: the inter-block batch and large programs
    give the same results as the persistent launch (itself pinned above)."""
    import torch

    for progs in (synth.generate("interblock256_64x256_s16"), synth.generate("large_128x1024_s24", 3)):
        db = gb.DeviceBatch(progs)
        db.run()
        torch.cuda.synchronize()
        narrow = db.results()
        db.run_wide()
        torch.cuda.synchronize()
        wide = db.results()
        for p, w, n in zip(progs, wide, narrow):
            _properties(p, w)
            for k in KEYS:
                assert w[k] == n[k], k
    p = synth.generate("large_128x1024_s24", 1)[0]
    sol, _ = _expected_final(p, _w0_by_pairs(p))
    w = wide[0]
    if sol is None:
        assert w["status"] == 1
    else:
        assert w["status"] == 0 and (w["mask"], w["weight"]) == sol
