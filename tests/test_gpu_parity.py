"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything here is integer and exact, so every comparison is bit-exact:
witness bitmaps, divergence masks, access-pair counts, clause lists, masks,
weights, trajectories and statuses."""
import numpy as np
import pytest

import oracle
from conftest import load_golden, program_from_spec
from _tiny import random_program
from paper_2011_08373_gb300 import synth
from paper_2011_08373_gb300.synth import MAP_AFFINE, MAP_STRIDED, SPACE_SHARED

pytestmark = pytest.mark.gpu

GOLD = load_golden("listings.json")
RESULT_KEYS = ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses",
               "forbidden", "access_pairs")


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


def _same_result(got, want, ctx=""):
    for k in RESULT_KEYS:
        assert got[k] == want[k], (ctx, k, got[k], want[k])


@pytest.mark.parametrize("case", GOLD["cases"], ids=[c["name"] for c in GOLD["cases"]])
def test_listings(gb, case):
    p = program_from_spec(case["program"])
    for chk in case["checks"]:
        got = gb.check(p, chk["mask"])
        assert got["intra"] == chk["intra"] and got["inter"] == chk["inter"]
        assert got["diverge"] == chk["diverge"]
        if "access_pairs" in chk:
            assert got["access_pairs"] == chk["access_pairs"]
    for exp in case["repairs"]:
        for fn in (gb.repair, gb.repair_plain):
            got = fn(p, mode=exp["mode"])
            for key in ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses",
                        "forbidden"):
                assert got[key] == exp[key], (fn.__name__, key)


def test_solver_paper_example(gb):
    for case in GOLD["solver_cases"]:
        got = gb.solve(case["n_vars"], case["weights"], case["pos"], case["neg"], case["forced"],
                       case["forbidden"])
        assert got == (case["expect"]["mask"], case["expect"]["weight"])


def test_solver_random_vs_oracle(gb):
    for seed in range(120):
        rng = synth.SplitMix64(synth.program_seed(99, seed))
        n = rng.randint(1, 24 if seed % 10 == 0 else 14)
        full = (1 << n) - 1
        w = [rng.randint(1, 1 << rng.randint(0, 12)) for _ in range(n)]
        pos = [(rng.randint(1, full) & rng.randint(1, full)) or 1 for _ in range(rng.randint(0, 40))]
        neg = [rng.randint(1, full) | rng.randint(1, full) for _ in range(rng.randint(0, 4))]
        forced = rng.randint(0, full) & rng.randint(0, full) & rng.randint(0, full)
        forbidden = rng.randint(0, full) & rng.randint(0, full) & rng.randint(0, full) & ~forced
        got = gb.solve(n, w, pos, neg, forced, forbidden)
        want = oracle.solve(n, w, pos, neg, forced, forbidden)
        assert got == want, (seed, n)


def test_interval_solve_key_widths(gb):
    """The loop's interval stabbing program packs each (weight, mask) key in
    32 bits, (weight << r) | compact mask, when the weights of the r compact
    slots sum below 2^(32 - r), and keeps 64-bit keys otherwise.  Straight-line
    programs on the shared array with small weights (packed keys) and with
    weights near the 2^24 maximum (64-bit keys) give the oracle's results."""
    progs = synth.generate("batch1024_4x256_s24", 40, start=5000, blocks=2, threads=32, n_stmts=14,
                           m_words=128)
    for k, p in enumerate(progs):
        if k % 2:
            rng = synth.SplitMix64(synth.program_seed(61, k))
            p.slot_weight = np.array([(1 << 24) - rng.randint(0, 1000) for _ in range(p.n_slots)], np.uint32)
    got = gb.repair_batch(progs)
    wide = 0
    for p, g in zip(progs, got):
        want = oracle.repair(p)
        _same_result(g, want)
        wide += int(p.slot_weight[0]) > 1000 and g["status"] == 0 and bin(g["mask"]).count("1") > 1
    assert wide >= 3  # repaired programs with several large-weight slots on


def test_tiny_checks_all_masks(gb):
    progs, masks, refs = [], [], []
    for seed in range(150):
        p = random_program(10000 + seed, s_max=5, b_max=3, t_max=9, m_max=16)
        for m in range(1 << p.n_slots):
            progs.append(p)
            masks.append(m)
    got = gb.check_batch(progs, masks)
    for p, m, g in zip(progs, masks, got):
        assert g == oracle.check(p, m), m


def test_tiny_repairs(gb):
    progs = [random_program(20000 + seed, s_max=6, b_max=3, t_max=12, m_max=24) for seed in range(200)]
    for grid_enabled in (True, False):
        got = gb.repair_batch(progs, grid_enabled=grid_enabled)
        for p, g in zip(progs, got):
            _same_result(g, oracle.repair(p, grid_enabled=grid_enabled), p.mode)


def test_iteration_cap(gb):
    progs = [random_program(30000 + seed, s_min=4, s_max=8, b_max=2, t_max=16, m_max=24)
             for seed in range(60)]
    for cap in (1, 2):
        got = gb.repair_batch(progs, max_iters=cap)
        for p, g in zip(progs, got):
            _same_result(g, oracle.repair(p, max_iters=cap))


def test_medium_programs_all_paths(gb):
    """Several chunks, ragged thread counts, guards and both array kinds."""
    progs = [random_program(40000 + seed, s_min=6, s_max=14, b_min=1, b_max=4, t_min=20, t_max=200,
                            m_max=3000, a_max=9, c_max=700) for seed in range(24)]
    got = gb.repair_batch(progs)
    for p, g in zip(progs, got):
        want = oracle.repair(p)
        _same_result(g, want)
    for p in progs[:6]:
        _same_result(gb.repair(p), oracle.repair(p))
        _same_result(gb.repair_plain(p), oracle.repair(p))


def test_single_workload(gb):
    p = synth.generate("single_1x64_s8", 1)[0]
    want = oracle.repair(p)
    for fn in (gb.repair, gb.repair_plain):
        _same_result(fn(p), want, fn.__name__)


def test_batch_workload_sample_full_size(gb):
    progs = synth.generate("batch1024_4x256_s24", 12)
    want = oracle.repair_batch(progs, n_threads=12)
    got = gb.repair_batch(progs)
    for g, w in zip(got, want):
        _same_result(g, w)


def test_interblock_workload_reduced(gb):
    progs = synth.generate("interblock256_64x256_s16", 8, blocks=6, threads=32, m_words=4096)
    want = oracle.repair_batch(progs, n_threads=8)
    got = gb.repair_batch(progs)
    for g, w in zip(got, want):
        _same_result(g, w)


def test_uneven_workload_sample(gb):
    progs = [p for p in synth.generate("uneven4096_mixed", 200) if p.blocks * p.threads <= 1200][:40]
    want = oracle.repair_batch(progs, n_threads=16)
    got = gb.repair_batch(progs)
    for g, w in zip(got, want):
        _same_result(g, w)


def test_device_resident_matches_host_path(gb):
    import torch

    progs = synth.generate("uneven4096_mixed", 64)
    host = gb.repair_batch(progs)
    db = gb.DeviceBatch(progs)
    db.run()
    torch.cuda.synchronize()
    dev = db.results()
    for a, b in zip(host, dev):
        _same_result(a, b)
    db.run()  # a second launch on the same buffers gives the same results
    torch.cuda.synchronize()
    for a, b in zip(host, db.results()):
        _same_result(a, b)


def test_mhs_strategy_matches_oracle(gb):
    """The paper's default mhs strategy (greedy proposals, MaxSAT fallback,
    one exact query at the end): every field, trajectories included."""
    progs = [random_program(50000 + seed, s_max=8, b_max=3, t_max=12, m_max=24) for seed in range(150)]
    progs += synth.generate("batch1024_4x256_s24", 6, blocks=2, threads=64, n_stmts=14, m_words=256)
    for grid_enabled in (True, False):
        got = gb.repair_batch(progs, grid_enabled=grid_enabled, strategy=gb.STRATEGY_MHS)
        for p, g in zip(progs, got):
            _same_result(g, oracle.repair(p, grid_enabled=grid_enabled, strategy=1))
    for p in progs[:4]:
        _same_result(gb.repair_plain(p, strategy=gb.STRATEGY_MHS), oracle.repair(p, strategy=1))


def test_mhs_strategy_listings(gb):
    for case in GOLD["cases"]:
        p = program_from_spec(case["program"])
        for exp in case["repairs"]:
            got = gb.repair(p, mode=exp["mode"], strategy=gb.STRATEGY_MHS)
            want = oracle.repair(p, mode=exp["mode"], strategy=1)
            _same_result(got, want, case["name"])
            assert (got["status"], got["mask"]) == (exp["status"], exp["mask"])


# --------------------------------------------------------------------------
# Counted loops: witnesses over executed instances, clauses over slots
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLD["loop_cases"], ids=[c["name"] for c in GOLD["loop_cases"]])
def test_loop_cases(gb, case):
    p = program_from_spec(case["program"])
    for chk in case["checks"]:
        got = gb.check(p, chk["mask"])
        for key in ("intra", "inter", "diverge", "access_pairs"):
            if key in chk:
                assert got[key] == chk[key], (key, chk["mask"])
    for exp in case["repairs"]:
        for fn in (gb.repair, gb.repair_plain):
            got = fn(p, mode=exp["mode"])
            for key in ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses",
                        "forbidden"):
                assert got[key] == exp[key], (fn.__name__, key)


def test_loop_checks_all_masks(gb):
    from _tiny import random_loop_program

    progs, masks = [], []
    for seed in range(120):
        p = random_loop_program(60000 + seed, s_min=2, s_max=5, b_max=3, t_max=9, m_max=16)
        for m in range(1 << p.n_slots):
            progs.append(p)
            masks.append(m)
    got = gb.check_batch(progs, masks)
    for p, m, g in zip(progs, masks, got):
        assert g == oracle.check(p, m), (p.loops, m)


def test_loop_repairs_both_strategies(gb):
    from _tiny import random_loop_program

    progs = [random_loop_program(61000 + seed, s_min=2, s_max=7, b_max=3, t_max=12, m_max=24)
             for seed in range(160)]
    for strategy in (0, 1):
        for grid_enabled in (True, False):
            got = gb.repair_batch(progs, grid_enabled=grid_enabled, strategy=strategy)
            for p, g in zip(progs, got):
                _same_result(g, oracle.repair(p, grid_enabled=grid_enabled, strategy=strategy), p.loops)
    for p in progs[:6]:
        _same_result(gb.repair_plain(p), oracle.repair(p))


def test_loop_medium_programs(gb):
    """Several address chunks, ragged thread counts, loop-counter terms that
    move a statement's addresses between iterations."""
    from _tiny import random_loop_program

    progs = [random_loop_program(62000 + seed, s_min=4, s_max=10, b_min=1, b_max=3, t_min=20, t_max=160,
                                 m_max=2500, a_max=9, c_max=700, d_max=70, trips_max=4)
             for seed in range(20)]
    got = gb.repair_batch(progs)
    for p, g in zip(progs, got):
        _same_result(g, oracle.repair(p), p.loops)


# --------------------------------------------------------------------------
# Wide lane: one CTA per (program, block), the loop as a device-side graph
# --------------------------------------------------------------------------

def _wide(gb, progs, **kw):
    import torch

    db = gb.DeviceBatch(progs, **kw)
    db.run_wide()
    torch.cuda.synchronize()
    wide = db.results()
    db.run()
    torch.cuda.synchronize()
    return wide, db.results()


def test_wide_lane_matches_oracle(gb):
    from _tiny import random_loop_program

    progs = [random_program(70000 + seed, s_max=7, b_max=4, t_max=12, m_max=24) for seed in range(80)]
    progs += [random_loop_program(71000 + seed, s_min=3, s_max=6, b_max=3, t_max=10, m_max=20)
              for seed in range(40)]
    progs += [random_program(72000 + seed, s_min=6, s_max=12, b_min=1, b_max=5, t_min=20, t_max=160,
                             m_max=2500, a_max=9, c_max=700) for seed in range(12)]
    for strategy in (0, 1):
        for grid_enabled in (True, False):
            wide, narrow = _wide(gb, progs, grid_enabled=grid_enabled, strategy=strategy)
            for p, w, n in zip(progs, wide, narrow):
                _same_result(w, oracle.repair(p, grid_enabled=grid_enabled, strategy=strategy))
                assert w["t_end_ns"] >= w["t_start_ns"]
                _same_result(w, n)


def test_wide_lane_iteration_cap(gb):
    progs = [random_program(30000 + seed, s_min=4, s_max=8, b_max=2, t_max=16, m_max=24)
             for seed in range(40)]
    for cap in (1, 2):
        wide, _ = _wide(gb, progs, max_iters=cap)
        for p, w in zip(progs, wide):
            _same_result(w, oracle.repair(p, max_iters=cap))


def test_wide_lane_workload_samples(gb):
    progs = synth.generate("interblock256_64x256_s16", 6, blocks=6, threads=32, m_words=4096)
    progs += synth.generate("batch1024_4x256_s24", 8)
    progs += [p for p in synth.generate("uneven4096_mixed", 120) if p.blocks * p.threads <= 1200][:20]
    want = oracle.repair_batch(progs, n_threads=16)
    wide, narrow = _wide(gb, progs)
    for w, n, o in zip(wide, narrow, want):
        _same_result(w, o)
        _same_result(n, o)


# --------------------------------------------------------------------------
# Negative clauses given with the program
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLD["neg_cases"], ids=[c["name"] for c in GOLD["neg_cases"]])
def test_neg_cases(gb, case):
    p = program_from_spec(case["program"])
    for exp in case["repairs"]:
        for fn in (gb.repair, gb.repair_plain):
            got = fn(p, mode=exp["mode"], strategy=exp["strategy"])
            for key in ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses", "forbidden"):
                assert got[key] == exp[key], (fn.__name__, key)


def test_negative_clauses_random(gb):
    from _tiny import random_loop_program
    from test_oracle_pins import _random_negs

    progs = []
    for seed in range(120):
        p = random_program(80000 + seed, s_min=3, s_max=8, b_max=3, t_max=12, m_max=24) if seed % 3 else \
            random_loop_program(80000 + seed, s_min=3, s_max=6, b_max=3, t_max=10, m_max=20)
        p.neg_clauses = _random_negs(seed, p.n_slots)
        progs.append(p)
    for strategy in (0, 1):
        got = gb.repair_batch(progs, strategy=strategy)
        for p, g in zip(progs, got):
            _same_result(g, oracle.repair(p, strategy=strategy), p.neg_clauses)
        wide, narrow = _wide(gb, progs, strategy=strategy)
        for w, n in zip(wide, got):
            _same_result(w, n)


# --------------------------------------------------------------------------
# Two barrier variables per site (slots with explicit places), up to 32 slots
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLD["site_cases"], ids=[c["name"] for c in GOLD["site_cases"]])
def test_site_cases(gb, case):
    p = program_from_spec(case["program"])
    for chk in case["checks"]:
        got = gb.check(p, chk["mask"])
        for key in ("intra", "inter", "diverge", "access_pairs"):
            if key in chk:
                assert got[key] == chk[key], (key, chk["mask"])
    for exp in case["repairs"]:
        for fn in (gb.repair, gb.repair_plain):
            got = fn(p, mode=exp["mode"], grid_enabled=exp["grid_enabled"])
            for key in ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses", "forbidden"):
                assert got[key] == exp[key], (fn.__name__, key)


def test_greedy_counts_distinct_clauses(gb):
    """The greedy strategy's hit counts are over the clause set: two witness
    pairs with the same clause (a site's block and grid candidates make such
    pairs) count once.  Seed 3048 of this family is a program whose greedy
    trajectory changes if they count twice."""
    from _tiny import with_sites

    progs = [with_sites(random_program(s, s_max=7), s) for s in range(3000, 3100)]
    want = oracle.repair_batch(progs, strategy=1)
    for p, g, w in zip(progs, gb.repair_batch(progs, strategy=gb.STRATEGY_MHS), want):
        _same_result(g, w, p.slot_pos)
    _same_result(gb.repair_plain(progs[48], strategy=gb.STRATEGY_MHS), want[48], progs[48].slot_pos)
    wide, _ = _wide(gb, progs, strategy=1)
    for w, o in zip(wide, want):
        _same_result(w, o, None)


def test_site_programs_match_oracle(gb):
    from _tiny import random_loop_program, with_sites

    progs = [with_sites(random_program(90000 + s, s_min=2, s_max=7, b_max=3, t_max=10, m_max=20), s)
             for s in range(100)]
    progs += [with_sites(random_loop_program(91000 + s, s_min=3, s_max=5, b_max=3, t_max=8, m_max=16), s)
              for s in range(40)]
    for strategy in (0, 1):
        for grid_enabled in (True, False):
            got = gb.repair_batch(progs, grid_enabled=grid_enabled, strategy=strategy)
            for p, g in zip(progs, got):
                _same_result(g, oracle.repair(p, grid_enabled=grid_enabled, strategy=strategy), p.slot_pos)
    tiny = [p for p in progs if p.n_slots <= 8][:40]
    ps, ms = [], []
    for p in tiny:
        for m in range(1 << p.n_slots):
            ps.append(p)
            ms.append(m)
    for p, m, g in zip(ps, ms, gb.check_batch(ps, ms)):
        assert g == oracle.check(p, m)
    wide, narrow = _wide(gb, progs[:60])
    for w, n in zip(wide, narrow):
        _same_result(w, n)


def test_solver_up_to_32_variables(gb):
    pytest.importorskip("scipy.optimize")
    from test_oracle_pins import milp_lowest_key

    for seed in range(24):
        rng = synth.SplitMix64(synth.program_seed(321, seed))
        n = rng.randint(25, 32)
        full = (1 << n) - 1
        w = [rng.randint(1, 1 << rng.randint(0, 8)) for _ in range(n)]
        pos = [rng.randint(1, full) & rng.randint(1, full) & rng.randint(1, full) or 1
               for _ in range(rng.randint(1, 30))]
        neg = [rng.randint(1, full) | rng.randint(1, full) for _ in range(rng.randint(0, 3))]
        forced = rng.randint(0, full) & rng.randint(0, full) & rng.randint(0, full) & rng.randint(0, full)
        forbidden = rng.randint(0, full) & rng.randint(0, full) & rng.randint(0, full) & ~forced
        got = gb.solve(n, w, pos, neg, forced, forbidden)
        assert got == milp_lowest_key(n, w, pos, neg, forced, forbidden), (seed, n)


def test_sites_workload_reduced(gb):
    """30 barrier variables per program (a block and a grid candidate at 15
    sites): the check against the oracle, the final repair against the
    lowest-key mask over the oracle's unconstrained witnesses (path
    independence), solved by integer programming."""
    pytest.importorskip("scipy.optimize")
    from test_oracle_pins import milp_lowest_key

    progs = synth.generate("sites128_16x256_s16", 12, blocks=3, threads=16, m_words=1024)
    assert all(p.n_slots == 30 for p in progs)
    got = gb.repair_batch(progs)
    for p, g in zip(progs, got):
        w0 = oracle.check(p, 0)
        assert gb.check(p, 0) == w0
        cls = oracle.clauses(p, w0)
        div = oracle.check(p, (1 << p.n_slots) - 1)["diverge"]
        want = milp_lowest_key(p.n_slots, [int(x) for x in p.slot_weight], cls, (), 0, div)
        if want is None:
            assert g["status"] == 1
        else:
            assert g["status"] == 0 and (g["mask"], g["weight"]) == want
            assert set(g["clauses"]) <= set(cls)
            assert oracle.check(p, g["mask"]) == gb.check(p, g["mask"])


def test_blocks_that_differ(gb):
    """Block offsets on shared and global arrays (blocks see different access
    patterns, or the same one up to a shift): every block's same-block
    witnesses must be found, whichever blocks the engine checks."""
    progs = [random_program(95000 + s, s_min=2, s_max=7, b_min=2, b_max=5, t_max=10, m_max=24, c_max=6,
                            shared_c=True) for s in range(160)]
    got = gb.repair_batch(progs)
    for p, g in zip(progs, got):
        _same_result(g, oracle.repair(p))
    ps, ms = [], []
    for p in progs[:40]:
        for m in (0, (1 << p.n_slots) - 1, 1 if p.n_slots else 0):
            ps.append(p)
            ms.append(m)
    for p, m, g in zip(ps, ms, gb.check_batch(ps, ms)):
        assert g == oracle.check(p, m)
    wide, narrow = _wide(gb, progs[:60])
    for w, n in zip(wide, narrow):
        _same_result(w, n)
    for p in progs[:8]:
        _same_result(gb.repair_plain(p), oracle.repair(p))


def test_batch_rejects_bad_permutation_tables(gb):
    """Batch calls reject a permutation table with a repeated entry: the
    host-pointer repair checks repeats on the device and the range on the
    host, the check batch and the plain path on the host; the lowest bad
    program is reported and the outputs stay untouched."""
    good = synth.generate("batch1024_4x256_s24", 3)
    bad = synth.generate("batch1024_4x256_s24", 3, start=10)
    for p in bad:
        assert (p.kind == 2).any()
    import copy
    progs = [good[0], copy.deepcopy(bad[0]), good[1], copy.deepcopy(bad[1])]
    for p in (progs[1], progs[3]):
        s = int(np.nonzero(p.kind == 2)[0][0])
        i0, i1 = _window_entries(p, s)
        p.perm = p.perm.copy()
        p.perm[i1] = p.perm[i0]  # a repeated entry among those the statement reads
    for fn in (lambda: gb.repair_batch(progs), lambda: gb.check_batch(progs, [0] * 4)):
        with pytest.raises(gb.GrError) as e:
            fn()
        assert e.value.code == gb.EINVAL and "program 1 stmt" in str(e.value) and "permutation" in str(e.value)
    with pytest.raises(gb.GrError) as e:
        gb.repair_plain(progs[1])
    assert e.value.code == gb.EINVAL
    # the same batch without the bad tables goes through
    got = gb.repair_batch([progs[0], progs[2]])
    for p, g in zip([progs[0], progs[2]], got):
        _same_result(g, oracle.repair(p))
    # a large batch goes in chunks: a bad table in the last chunk is still
    # reported (after earlier chunks ran), and the next call is unaffected
    # (2,100 programs: four chunks, the last from program 1,800)
    big = synth.generate("batch1024_4x256_s24", 2100, blocks=2, threads=32, n_stmts=8, m_words=128)
    k = next(i for i in range(2090, 2100) if (big[i].kind == 2).any())
    s = int(np.nonzero(big[k].kind == 2)[0][0])
    big[k] = copy.deepcopy(big[k])
    big[k].perm = big[k].perm.copy()
    i0, i1 = _window_entries(big[k], s)
    big[k].perm[i0] = big[k].perm[i1]
    out = np.zeros(2100, dtype=gb.RESULT_DTYPE)
    with pytest.raises(gb.GrError) as e:
        gb.repair_batch_raw(big, out=out)
    assert e.value.code == gb.EINVAL and f"program {k} stmt" in str(e.value)
    assert not out.view(np.uint8).any()  # results untouched
    good_big = big[:k] + big[k + 1:]
    got = gb.repair_batch(good_big)
    for i in (0, 650, 1300, 1950, len(good_big) - 1):
        _same_result(got[i], oracle.repair(good_big[i]))



def _window_entries(p, s):
    """Positions in p.perm of the first two table entries statement s reads:
    threads 0 and 1 read entries b and b + 1 (mod M) of its table."""
    M = p.m_shared if p.space[s] == 0 else p.m_global
    off, b = int(p.perm_off[s]), int(p.b[s]) % M
    return off + b, off + (b + 1) % M


def _spoil(p, how):
    """A copy of p whose first permutation statement reads a repeated entry
    ("repeat") or an entry past the array ("range")."""
    import copy

    q = copy.deepcopy(p)
    s = int(np.nonzero(q.kind == 2)[0][0])
    i0, i1 = _window_entries(q, s)
    q.perm = q.perm.copy()
    if how == "repeat":
        q.perm[i1] = q.perm[i0]
    else:
        q.perm[i0] = (q.m_shared if q.space[s] == 0 else q.m_global) + 5
    return q, s


def test_batch_reports_lowest_bad_table(gb):
    """A repeat (found on the device) below an out-of-range entry (found by
    the packer) is still the one reported, in the same chunk and across
    chunks; an out-of-range entry alone is reported too."""
    small = synth.generate("batch1024_4x256_s24", 8, blocks=2, threads=32, n_stmts=8, m_words=128)
    perm_idx = [i for i, p in enumerate(small) if (p.kind == 2).any()]
    assert len(perm_idx) >= 3
    a, b = perm_idx[0], perm_idx[2]
    progs = list(small)
    progs[a], sa = _spoil(small[a], "repeat")
    progs[b], _ = _spoil(small[b], "range")
    with pytest.raises(gb.GrError) as e:
        gb.repair_batch(progs)
    assert e.value.code == gb.EINVAL and f"program {a} stmt {sa}:" in str(e.value)
    progs = list(small)
    progs[b], sb = _spoil(small[b], "range")
    with pytest.raises(gb.GrError) as e:
        gb.repair_batch(progs)
    assert f"program {b} stmt {sb}:" in str(e.value)
    # 2,100 programs go in four chunks (from 0, 600, 1,200, 1,800): a repeat
    # in the first, a bad range in the second
    big = synth.generate("batch1024_4x256_s24", 2100, blocks=2, threads=32, n_stmts=8, m_words=128)
    i = next(j for j in range(10, 100) if (big[j].kind == 2).any())
    k = next(j for j in range(700, 800) if (big[j].kind == 2).any())
    big[i], si = _spoil(big[i], "repeat")
    big[k], _ = _spoil(big[k], "range")
    out = np.zeros(2100, dtype=gb.RESULT_DTYPE)
    with pytest.raises(gb.GrError) as e:
        gb.repair_batch_raw(big, out=out)
    assert f"program {i} stmt {si}:" in str(e.value)
    assert not out.view(np.uint8).any()
