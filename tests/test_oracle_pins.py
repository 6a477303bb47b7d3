"""Pins of the CPU oracle against facts that do not come from the oracle:
values the paper fixes (its listings and the Section 2.4 clause set),
independent algorithms (a flag-reset race detector written from Section 2.2's
description of barriers, a number-theoretic closed form for affine maps,
interval stabbing by dynamic programming, scipy's MILP solver) and invariants
of the model.  All CPU-only."""
import itertools
import math

import numpy as np
import pytest

import oracle
from conftest import load_golden, program_from_spec
from _tiny import random_program
from paper_2011_08373_gb300 import synth
from paper_2011_08373_gb300.synth import (LEVEL_GRID, MAP_AFFINE, MAP_PERM, MAP_STRIDED,
                                          MODE_REMOVE, MODE_REPAIR, SPACE_GLOBAL, SPACE_SHARED)

GOLD = load_golden("listings.json")


# --------------------------------------------------------------------------
# Paper listings (hand-derived fixtures)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLD["cases"], ids=[c["name"] for c in GOLD["cases"]])
def test_listing_checks(case):
    p = program_from_spec(case["program"])
    for chk in case["checks"]:
        got = oracle.check(p, chk["mask"])
        assert got["intra"] == chk["intra"], case["cite"]
        assert got["inter"] == chk["inter"], case["cite"]
        assert got["diverge"] == chk["diverge"], case["cite"]
        if "access_pairs" in chk:
            assert got["access_pairs"] == chk["access_pairs"]


@pytest.mark.parametrize("case", GOLD["cases"], ids=[c["name"] for c in GOLD["cases"]])
def test_listing_repairs(case):
    p = program_from_spec(case["program"])
    for exp in case["repairs"]:
        got = oracle.repair(p, mode=exp["mode"])
        for key in ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses",
                    "forbidden"):
            assert got[key] == exp[key], (key, case["cite"])


@pytest.mark.parametrize("case", GOLD["solver_cases"], ids=[c["name"] for c in GOLD["solver_cases"]])
def test_solver_paper_example(case):
    got = oracle.solve(case["n_vars"], case["weights"], case["pos"], case["neg"],
                       case["forced"], case["forbidden"])
    assert got == (case["expect"]["mask"], case["expect"]["weight"]), case["cite"]
    for bad in case["rejected_masks"]:
        # the greedy mhs answer hits every positive clause but breaks a negative one
        assert all(bad & c for c in case["pos"])
        assert any(bad & n == n for n in case["neg"])


# --------------------------------------------------------------------------
# Independent race detector: per pair of threads, read/write flags that an
# enabled barrier resets (Section 2.2: block barriers reset the flags of two
# threads of one block, grid barriers reset them for any two threads)
# --------------------------------------------------------------------------

def _addr(p, s, blk, tid):
    M = p.m_shared if p.space[s] == SPACE_SHARED else p.m_global
    if p.kind[s] == MAP_PERM:
        return int(p.perm[int(p.perm_off[s]) + (tid + int(p.c[s]) * blk + int(p.b[s])) % M])
    return (int(p.a[s]) * tid + int(p.c[s]) * blk + int(p.b[s])) % M


def _runs(k, r, tid):
    return k == 0 or tid % k == r


def flag_reset_detector(p, mask):
    S, B, T = p.n_stmts, p.blocks, p.threads
    intra, inter = [0] * S, [0] * S
    threads = [(b, t) for b in range(B) for t in range(T)]
    for x, y in itertools.combinations(range(len(threads)), 2):
        pair = (threads[x], threads[y])
        same = pair[0][0] == pair[1][0]
        logs = ([], [])
        for s in range(S):
            if s > 0 and (mask >> (s - 1)) & 1 and (same or p.slot_level[s - 1] == LEVEL_GRID):
                logs = ([], [])
            fresh = []
            for who, (b, t) in enumerate(pair):
                if _runs(int(p.guard_k[s]), int(p.guard_r[s]), t):
                    inst = ("shared", b) if p.space[s] == SPACE_SHARED else ("global",)
                    e = (inst, _addr(p, s, b, t), p.op[s] == 1, s)
                    logs[who].append(e)
                    fresh.append((who, e))
            for who, e in fresh:
                for f in logs[1 - who]:
                    if f[0] == e[0] and f[1] == e[1] and (e[2] or f[2]):
                        i, j = min(e[3], f[3]), max(e[3], f[3])
                        if same:
                            intra[i] |= 1 << j
                        else:
                            inter[i] |= 1 << j
    diverge = 0
    for k in range(S - 1):
        if not (mask >> k) & 1:
            continue
        gk, gr = int(p.slot_guard_k[k]), int(p.slot_guard_r[k])
        for t1, t2 in itertools.combinations(range(T), 2):
            if _runs(gk, gr, t1) != _runs(gk, gr, t2):
                diverge |= 1 << k
    return intra, inter, diverge


@pytest.mark.parametrize("seed", range(48))
def test_check_matches_flag_reset_detector(seed):
    p = random_program(seed, s_max=4, b_max=3, t_max=6, m_max=12)
    n = p.n_slots
    masks = sorted({0, (1 << n) - 1} | {(seed * 2654435761 + k * 40503) % (1 << n) for k in range(3)}) \
        if n > 0 else [0]
    for m in masks:
        got = oracle.check(p, m)
        intra, inter, div = flag_reset_detector(p, m)
        assert got["intra"] == intra
        assert got["inter"] == inter
        assert got["diverge"] == div


# --------------------------------------------------------------------------
# Affine closed form: f_i(g1) == f_j(g2) is the linear congruence
# a_j*t2 == rhs (mod M); its solutions form one residue class mod M/gcd(a_j, M)
# --------------------------------------------------------------------------

def _congruence_solutions(a, rhs, M, T):
    a %= M
    if a == 0:
        return range(T) if rhs % M == 0 else range(0)
    g = math.gcd(a, M)
    if rhs % g:
        return range(0)
    step = M // g
    t0 = (rhs // g) * pow(a // g, -1, step) % step if step > 1 else 0
    return range(t0, T, step)


def affine_closed_form(p):
    S, B, T = p.n_stmts, p.blocks, p.threads
    intra, inter = [0] * S, [0] * S
    act = [[_runs(int(p.guard_k[s]), int(p.guard_r[s]), t) for t in range(T)] for s in range(S)]
    for i in range(S):
        for j in range(i, S):
            if p.space[i] != p.space[j] or not (p.op[i] == 1 or p.op[j] == 1):
                continue
            shared = p.space[i] == SPACE_SHARED
            M = p.m_shared if shared else p.m_global
            for b1 in range(B):
                for b2 in range(B):
                    if shared and b1 != b2:
                        continue
                    for t1 in range(T):
                        if not act[i][t1]:
                            continue
                        lhs = int(p.a[i]) * t1 + int(p.c[i]) * b1 + int(p.b[i])
                        rhs = (lhs - int(p.c[j]) * b2 - int(p.b[j])) % M
                        for t2 in _congruence_solutions(int(p.a[j]), rhs, M, T):
                            if act[j][t2] and (b1, t1) != (b2, t2):
                                if b1 == b2:
                                    intra[i] |= 1 << j
                                else:
                                    inter[i] |= 1 << j
                                break
    return intra, inter


def pair_count_closed_form(p, mask):
    """Thread pairs a naive checker examines under ``mask`` (closed form)."""
    S, B, T = p.n_stmts, p.blocks, p.threads
    act = [[_runs(int(p.guard_k[s]), int(p.guard_r[s]), t) for t in range(T)] for s in range(S)]
    total = 0
    for i in range(S):
        for j in range(i, S):
            if p.space[i] != p.space[j] or not (p.op[i] == 1 or p.op[j] == 1):
                continue
            ks = range(i, j)
            open_same = not any((mask >> k) & 1 for k in ks)
            open_cross = p.space[i] == SPACE_GLOBAL and not any(
                (mask >> k) & 1 and p.slot_level[k] == LEVEL_GRID for k in ks)
            ni, nj = sum(act[i]), sum(act[j])
            nij = sum(1 for t in range(T) if act[i][t] and act[j][t])
            if i < j:
                total += open_same * B * (ni * nj - nij) + open_cross * B * (B - 1) * ni * nj
            else:
                total += open_same * B * ni * (ni - 1) // 2 + open_cross * (B * (B - 1) // 2) * ni * ni
    return total


@pytest.mark.parametrize("seed", range(40))
def test_check_matches_affine_closed_form(seed):
    p = random_program(1000 + seed, s_max=6, b_max=3, t_max=48, m_max=160,
                       kinds=(MAP_AFFINE, MAP_STRIDED), a_max=6, c_max=64,
                       guard_ks=(0, 0, 2, 3, 4, 8))
    got = oracle.check(p, 0)
    intra, inter = affine_closed_form(p)
    assert got["intra"] == intra
    assert got["inter"] == inter


@pytest.mark.parametrize("seed", range(40))
def test_access_pairs_closed_form(seed):
    p = random_program(2000 + seed, s_max=6, b_max=3, t_max=24, m_max=64)
    n = p.n_slots
    for m in {0, (1 << n) - 1, (seed * 7919) % (1 << n) if n else 0}:
        assert oracle.check(p, m)["access_pairs"] == pair_count_closed_form(p, m)


# --------------------------------------------------------------------------
# Hitting-set solver vs interval stabbing DP and vs MILP
# --------------------------------------------------------------------------

def interval_stabbing(n, w, intervals, forced, forbidden):
    """Least (weight, mask) set of allowed slots meeting every interval
    [l, r] and containing ``forced``: dynamic programming over the last chosen
    slot (textbook weighted interval stabbing, kept lexicographic)."""
    if any(l > r for l, r in intervals):
        return None

    def gap_ok(q, p_):
        if any(l > q and r < p_ for l, r in intervals):
            return False
        return not any((forced >> k) & 1 for k in range(q + 1, p_))

    best = {}
    for p_ in range(n):
        if (forbidden >> p_) & 1:
            continue
        cands = []
        if gap_ok(-1, p_):
            cands.append((w[p_], 1 << p_))
        for q, (bw, bm) in best.items():
            if gap_ok(q, p_):
                cands.append((bw + w[p_], bm | (1 << p_)))
        if cands:
            best[p_] = min(cands)
    finals = [(0, 0)] if gap_ok(-1, n) else []
    finals += [v for q, v in best.items() if gap_ok(q, n)]
    return min(finals) if finals else None


def _as_interval(mask):
    if mask == 0:
        return (1, 0)
    lo = (mask & -mask).bit_length() - 1
    hi = mask.bit_length() - 1
    assert mask == ((1 << (hi + 1)) - (1 << lo)), "race clauses of block slots are intervals"
    return (lo, hi)


@pytest.mark.parametrize("seed", range(60))
def test_solve_matches_interval_dp(seed):
    p = random_program(3000 + seed, s_min=3, s_max=12, b_max=2, t_max=8, m_max=10,
                       spaces=(SPACE_SHARED,), weight_max=6)
    p.slot_level[:] = 0
    n = p.n_slots
    w0 = oracle.check(p, 0)
    cls = oracle.clauses(p, w0)
    rng = synth.SplitMix64(seed)
    forced = rng.randint(0, (1 << n) - 1) & rng.randint(0, (1 << n) - 1) & rng.randint(0, (1 << n) - 1)
    forbidden = rng.randint(0, (1 << n) - 1) & rng.randint(0, (1 << n) - 1) & ~forced
    w = [int(x) for x in p.slot_weight]
    got = oracle.solve(n, w, cls, (), forced, forbidden)
    ref = interval_stabbing(n, w, [_as_interval(c) for c in cls], forced, forbidden)
    assert got == (None if ref is None else (ref[1], ref[0]))


def _milp_min(n, w, pos, neg, forced, forbidden, extra_zero=(), weight_eq=None):
    from scipy.optimize import LinearConstraint, milp, Bounds
    rows, lo, hi = [], [], []
    for c in pos:
        rows.append([1 if (c >> k) & 1 else 0 for k in range(n)]); lo.append(1); hi.append(np.inf)
    for c in neg:
        rows.append([1 if (c >> k) & 1 else 0 for k in range(n)]); lo.append(-np.inf)
        hi.append(bin(c).count("1") - 1)
    if weight_eq is not None:
        rows.append(list(w)); lo.append(weight_eq); hi.append(weight_eq)
    lb = [1 if (forced >> k) & 1 else 0 for k in range(n)]
    ub = [0 if ((forbidden >> k) & 1 or k in extra_zero) else 1 for k in range(n)]
    if any(l > u for l, u in zip(lb, ub)):
        return None
    cons = [LinearConstraint(np.array(rows, float), lo, hi)] if rows else []
    obj = np.array(w, float) if weight_eq is None else np.zeros(n)
    res = milp(obj, constraints=cons, integrality=np.ones(n), bounds=Bounds(lb, ub))
    if res.status != 0:
        return None
    return np.rint(res.x).astype(int)


def milp_lowest_key(n, w, pos, neg=(), forced=0, forbidden=0):
    """The least (weight, mask) hitting set by integer programming: the minimum
    weight, then the lowest mask among the sets of that weight (clear bits from
    the top while a set of that weight stays feasible).  None if infeasible."""
    x = _milp_min(n, w, pos, neg, forced, forbidden)
    if x is None:
        return None
    wstar = int(np.dot(w, x))
    zero, mask = [], 0
    for k in reversed(range(n)):
        if _milp_min(n, w, pos, neg, forced, forbidden, extra_zero=zero + [k], weight_eq=wstar) is not None:
            zero.append(k)
        else:
            mask |= 1 << k
    return mask, wstar


@pytest.mark.parametrize("seed", range(40))
def test_solve_matches_milp(seed):
    pytest.importorskip("scipy.optimize")
    rng = synth.SplitMix64(synth.program_seed(77, seed))
    n = rng.randint(1, 9)
    full = (1 << n) - 1
    w = [rng.randint(1, 9) for _ in range(n)]
    pos = [rng.randint(1, full) & rng.randint(1, full) or 1 for _ in range(rng.randint(0, 8))]
    neg = [rng.randint(1, full) | rng.randint(1, full) for _ in range(rng.randint(0, 3))]
    forced = rng.randint(0, full) & rng.randint(0, full) & rng.randint(0, full)
    forbidden = rng.randint(0, full) & rng.randint(0, full) & rng.randint(0, full)
    got = oracle.solve(n, w, pos, neg, forced, forbidden)
    x = _milp_min(n, w, pos, neg, forced, forbidden)
    if x is None:
        assert got is None
        return
    wstar = int(np.dot(w, x))
    assert got is not None and got[1] == wstar
    # lowest mask among the minimum-weight sets: clear bits from the top while feasible
    zero = []
    mask = 0
    for k in reversed(range(n)):
        if _milp_min(n, w, pos, neg, forced, forbidden, extra_zero=zero + [k], weight_eq=wstar) is not None:
            zero.append(k)
        else:
            mask |= 1 << k
    assert got[0] == mask


# --------------------------------------------------------------------------
# Invariants of the check
# --------------------------------------------------------------------------

def _rows_subset(a, b):
    return all((x & ~y) == 0 for x, y in zip(a, b))


@pytest.mark.parametrize("seed", range(40))
def test_check_antitone_in_mask(seed):
    """Enabling barriers never adds a race (Section 2.4: inserting barriers may
    only cause divergence, removing them only races)."""
    p = random_program(4000 + seed, s_max=5, b_max=3, t_max=8, m_max=12)
    n = p.n_slots
    rng = synth.SplitMix64(seed)
    for _ in range(4):
        m = rng.randint(0, (1 << n) - 1) if n else 0
        m2 = m | (rng.randint(0, (1 << n) - 1) if n else 0)
        a, b = oracle.check(p, m), oracle.check(p, m2)
        assert _rows_subset(b["intra"], a["intra"])
        assert _rows_subset(b["inter"], a["inter"])


@pytest.mark.parametrize("seed", range(40))
def test_clause_is_exact_filter(seed):
    """A witness of the unconstrained check stays under mask m exactly when m
    misses its clause: pins the clause builder against the check."""
    p = random_program(5000 + seed, s_max=5, b_max=3, t_max=8, m_max=12)
    n, S = p.n_slots, p.n_stmts
    w0 = oracle.check(p, 0)
    masks = range(1 << n)
    checks = {m: oracle.check(p, m) for m in masks}
    for i in range(S):
        for j in range(S):
            for scope in ("intra", "inter"):
                if not (w0[scope][i] >> j) & 1:
                    continue
                single = {"intra": [0] * S, "inter": [0] * S, "diverge": 0}
                single[scope][i] = 1 << j
                (cl,) = oracle.clauses(p, single)
                for m in masks:
                    assert bool((checks[m][scope][i] >> j) & 1) == ((m & cl) == 0)


def test_shared_programs_have_no_cross_block_witness():
    for seed in range(30):
        p = random_program(6000 + seed, spaces=(SPACE_SHARED,), b_max=4)
        for m in range(1 << p.n_slots):
            assert not any(oracle.check(p, m)["inter"])


def test_all_barriers_race_free_on_generated_programs():
    """With every slot on (grid level for global arrays) only a statement that
    collides with itself can still race."""
    for wl, over in (("batch1024_4x256_s24", dict(blocks=2, threads=32, n_stmts=8, m_words=128)),
                     ("interblock256_64x256_s16", dict(blocks=3, threads=16, n_stmts=6,
                                                       m_words=256))):
        for p in synth.generate(wl, 6, **over):
            p.slot_level[:] = LEVEL_GRID
            got = oracle.check(p, (1 << p.n_slots) - 1)
            for i in range(p.n_stmts):
                assert (got["intra"][i] | got["inter"][i]) & ~(1 << i) == 0


# --------------------------------------------------------------------------
# Repair loop: path independence and iteration bound
# --------------------------------------------------------------------------

def _lowest_safe_mask(p, mode, grid_enabled):
    n = p.n_slots
    forced = p.existing_mask if mode == MODE_REPAIR else 0
    grid = p.grid_mask()
    best = None
    for x in range(1 << n):
        if (x & forced) != forced or (not grid_enabled and x & grid):
            continue
        c = oracle.check(p, x)
        if any(c["intra"]) or any(c["inter"]) or c["diverge"]:
            continue
        key = (sum(int(p.slot_weight[k]) for k in range(n) if (x >> k) & 1), x)
        best = key if best is None or key < best else best
    return best


@pytest.mark.parametrize("seed", range(60))
def test_repair_path_independence(seed):
    """Clauses are exact, so the loop ends at the lowest (weight, mask) among
    all masks whose own check is clean, whatever the trajectory."""
    p = random_program(7000 + seed, s_max=5, b_max=2, t_max=6, m_max=10)
    for mode in (MODE_REPAIR, MODE_REMOVE):
        for grid_enabled in (True, False):
            got = oracle.repair(p, mode=mode, grid_enabled=grid_enabled)
            ref = _lowest_safe_mask(p, mode, grid_enabled)
            assert got["iters"] <= p.n_slots + 3
            if ref is None:
                assert got["status"] == 1 and got["mask"] == 0
            else:
                assert got["status"] == 0
                assert (got["weight"], got["mask"]) == ref
                assert got["added"] == got["mask"] & ~p.existing_mask
                assert got["removed"] == p.existing_mask & ~got["mask"]


@pytest.mark.parametrize("seed", range(30))
def test_check_pair_matches_check(seed):
    """The one-pair form used to sample full-size launches agrees with the
    whole check on every pair."""
    p = random_program(8000 + seed, s_max=5, b_max=3, t_max=8, m_max=12)
    for m in {0, (1 << p.n_slots) - 1, (seed * 31) % (1 << p.n_slots) if p.n_slots else 0}:
        full = oracle.check(p, m)
        total = 0
        for i in range(p.n_stmts):
            for j in range(i, p.n_stmts):
                a, b, n = oracle.check_pair(p, m, i, j)
                assert a == bool((full["intra"][i] >> j) & 1)
                assert b == bool((full["inter"][i] >> j) & 1)
                total += n
        assert total == full["access_pairs"]


@pytest.mark.parametrize("seed", range(40))
def test_check_words_matches_check(seed):
    """The word-grouped check (used at full size) gives every field of the
    thread-pair enumeration: witnesses of both scopes, divergent slots and
    the pairs examined, on random programs with guards, permutation maps,
    both arrays, block-offset shared maps, counted loops and candidate
    sites, under several masks."""
    from _tiny import random_loop_program, with_sites

    progs = [random_program(9100 + seed, s_max=6, b_max=3, t_max=9, m_max=12),
             random_program(9200 + seed, s_max=5, b_max=4, t_max=12, m_max=20, shared_c=True),
             random_loop_program(9300 + seed),
             with_sites(random_program(9400 + seed, s_max=5, b_max=3, t_max=8, m_max=12), seed),
             random_program(9500 + seed, s_min=4, s_max=8, b_min=2, b_max=6, t_min=16, t_max=48, m_max=200,
                            a_max=3, c_max=60)]
    for p in progs:
        n = p.n_slots
        for m in {0, (1 << n) - 1, (seed * 2654435761) % (1 << n) if n else 0, (seed * 40503) % (1 << n) if n else 0}:
            assert oracle.check(p, m, words=True) == oracle.check(p, m), (seed, m)


@pytest.mark.parametrize("seed", range(20))
def test_repair_words_matches_repair(seed):
    """Algorithm 1 verified by the word-grouped check follows the same
    trajectory to the same result, both strategies, one program at a time and
    in a batch."""
    from _tiny import random_loop_program

    progs = [random_program(9600 + seed, s_max=7, b_max=3, t_max=10, m_max=16),
             random_loop_program(9700 + seed),
             random_program(9800 + seed, s_min=5, s_max=9, b_min=1, b_max=4, t_min=8, t_max=40, m_max=160,
                            a_max=3, c_max=40, p_write=0.35)]
    for strategy in (0, 1):
        for p in progs:
            assert oracle.repair(p, strategy=strategy, words=True) == oracle.repair(p, strategy=strategy)
    assert oracle.repair_batch(progs, n_threads=2, words=True) == oracle.repair_batch(progs)


# --------------------------------------------------------------------------
# The mhs strategy (Section 2.4): greedy minimal hitting sets
# --------------------------------------------------------------------------

def test_greedy_paper_example():
    """Section 2.4: on the positive clauses of the example the mhs is {b1, b2},
    which breaks the negative clause; the strategy then falls back."""
    case = GOLD["solver_cases"][0]
    g = oracle.greedy(case["n_vars"], case["weights"], case["pos"])
    assert g == case["greedy_mhs"]
    assert any(g & n == n for n in case["neg"])


@pytest.mark.parametrize("seed", range(60))
def test_greedy_minimal_and_within_johnson_bound(seed):
    """A greedy hitting set is minimal (no element can be dropped) and within
    H(d) of the optimum, d the most clauses one variable hits (Johnson 1974,
    Chvatal 1979 for weights)."""
    rng = synth.SplitMix64(synth.program_seed(555, seed))
    n = rng.randint(1, 12)
    full = (1 << n) - 1
    w = [rng.randint(1, 6) for _ in range(n)]
    pos = [(rng.randint(1, full) & rng.randint(1, full)) or 1 for _ in range(rng.randint(1, 14))]
    forced = rng.randint(0, full) & rng.randint(0, full) & rng.randint(0, full)
    forbidden = rng.randint(0, full) & rng.randint(0, full) & rng.randint(0, full) & ~forced
    g = oracle.greedy(n, w, pos, forced, forbidden)
    opt = oracle.solve(n, w, pos, (), forced, forbidden)
    if opt is None:
        assert g is None
        return
    assert g is not None
    assert (g & forced) == forced and not (g & forbidden)
    assert all(g & c for c in pos)
    for k in range(n):
        if (g >> k) & 1 and not (forced >> k) & 1:
            assert not all((g & ~(1 << k)) & c for c in pos), "not minimal"
    live = [c for c in pos if not (c & forced)]
    d = max([sum(1 for c in live if (c >> k) & 1) for k in range(n)] + [1])
    harmonic = sum(1.0 / i for i in range(1, d + 1))
    wf = sum(w[k] for k in range(n) if (forced >> k) & 1)
    wg = sum(w[k] for k in range(n) if (g >> k) & 1)
    assert wg - wf <= harmonic * (opt[1] - wf) + 1e-9


@pytest.mark.parametrize("seed", range(40))
def test_mhs_strategy_reaches_the_same_repair(seed):
    """Clauses are exact, so the mhs strategy ends at the same lowest-key clean
    mask as the MaxSAT strategy; only the trajectory differs."""
    p = random_program(9500 + seed, s_max=6, b_max=2, t_max=8, m_max=12)
    for grid_enabled in (True, False):
        a = oracle.repair(p, grid_enabled=grid_enabled, strategy=0)
        b = oracle.repair(p, grid_enabled=grid_enabled, strategy=1)
        assert (a["status"], a["mask"], a["weight"]) == (b["status"], b["mask"], b["weight"])
        assert b["iters"] <= 2 * p.n_slots + 4


@pytest.mark.parametrize("case", GOLD["greedy_cases"], ids=[c["name"] for c in GOLD["greedy_cases"]])
def test_greedy_worked_cases(case):
    got = oracle.greedy(case["n_vars"], case["weights"], case["pos"], case["forced"], case["forbidden"])
    assert got == case["expect"], case["cite"]


# --------------------------------------------------------------------------
# Counted loops: hand-derived cases, a control-flow interpreter with flag
# resets (written from Section 2.2's barrier semantics, independent of the
# oracle's unrolled ranges), and the invariants on loop programs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLD["loop_cases"], ids=[c["name"] for c in GOLD["loop_cases"]])
def test_loop_cases(case):
    p = program_from_spec(case["program"])
    assert [list(x) for x in oracle.unroll(p)] == case["unrolled"]
    for chk in case["checks"]:
        got = oracle.check(p, chk["mask"])
        for key in ("intra", "inter", "diverge", "access_pairs"):
            if key in chk:
                assert got[key] == chk[key], (key, chk["mask"], case["cite"])
    for exp in case["repairs"]:
        got = oracle.repair(p, mode=exp["mode"])
        for key in ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses",
                    "forbidden"):
            assert got[key] == exp[key], (key, case["cite"])


def _interpret(p):
    """Run the program's control flow once: a program counter over the
    statements that jumps back to a loop's first statement while iterations
    remain.  The barrier of slot k is passed each time control arrives at
    statement k+1.  Returns events ('bar', k) and ('st', s, counter)."""
    S = p.n_stmts
    loops = list(p.loops)
    count = [0] * len(loops)
    events, pc = [], 0
    while pc < S:
        if pc > 0:
            events.append(("bar", pc - 1))
        inner = [q for q, (lo, hi, _) in enumerate(loops) if lo <= pc <= hi]
        q_in = max(inner, key=lambda q: loops[q][0]) if inner else None
        events.append(("st", pc, count[q_in] if q_in is not None else 0))
        nxt = pc + 1
        for q in sorted((q for q, l in enumerate(loops) if l[1] == pc), key=lambda q: -loops[q][0]):
            if count[q] + 1 < loops[q][2]:
                count[q] += 1
                nxt = loops[q][0]
                break
            count[q] = 0
        pc = nxt
    return events


def _addr_it(p, s, blk, tid, it):
    M = p.m_shared if p.space[s] == SPACE_SHARED else p.m_global
    d = int(p.iter_coef[s]) * it
    if p.kind[s] == MAP_PERM:
        return int(p.perm[int(p.perm_off[s]) + (tid + int(p.c[s]) * blk + int(p.b[s]) + d) % M])
    return (int(p.a[s]) * tid + int(p.c[s]) * blk + int(p.b[s]) + d) % M


def loop_flag_reset_detector(p, mask):
    events = _interpret(p)
    X = sum(1 for e in events if e[0] == "st")
    B, T = p.blocks, p.threads
    intra, inter = [0] * X, [0] * X
    threads = [(b, t) for b in range(B) for t in range(T)]
    for x, y in itertools.combinations(range(len(threads)), 2):
        pair = (threads[x], threads[y])
        same = pair[0][0] == pair[1][0]
        logs = ([], [])
        n = -1
        for e in events:
            if e[0] == "bar":
                k = e[1]
                if (mask >> k) & 1 and (same or p.slot_level[k] == LEVEL_GRID):
                    logs = ([], [])
                continue
            _, s, it = e
            n += 1
            fresh = []
            for who, (b, t) in enumerate(pair):
                if _runs(int(p.guard_k[s]), int(p.guard_r[s]), t):
                    inst = ("shared", b) if p.space[s] == SPACE_SHARED else ("global",)
                    ev = (inst, _addr_it(p, s, b, t, it), p.op[s] == 1, n)
                    logs[who].append(ev)
                    fresh.append((who, ev))
            for who, ev in fresh:
                for f in logs[1 - who]:
                    if f[0] == ev[0] and f[1] == ev[1] and (ev[2] or f[2]):
                        i, j = min(ev[3], f[3]), max(ev[3], f[3])
                        if same:
                            intra[i] |= 1 << j
                        else:
                            inter[i] |= 1 << j
    return intra, inter


@pytest.mark.parametrize("seed", range(60))
def test_loop_check_matches_interpreter(seed):
    from _tiny import random_loop_program

    p = random_loop_program(seed, s_min=3, s_max=5, b_max=2, t_max=5, m_max=10)
    n = p.n_slots
    masks = sorted({0, (1 << n) - 1} | {(seed * 2654435761 + k * 40503) % (1 << n) for k in range(3)}) \
        if n > 0 else [0]
    for m in masks:
        got = oracle.check(p, m)
        intra, inter = loop_flag_reset_detector(p, m)
        assert got["intra"] == intra, (p.loops, m)
        assert got["inter"] == inter, (p.loops, m)


def test_loop_interpreter_order_is_the_unrolled_order():
    from _tiny import random_loop_program

    for seed in range(80):
        p = random_loop_program(seed, s_max=6)
        ev = [(e[1], e[2]) for e in _interpret(p) if e[0] == "st"]
        assert ev == oracle.unroll(p), p.loops


def test_one_trip_loops_change_nothing():
    """A loop that runs once is the straight-line program."""
    from _tiny import random_loops

    for seed in range(40):
        p = random_program(11000 + seed, s_max=6, b_max=2, t_max=6, m_max=10)
        rng = synth.SplitMix64(seed)
        q = random_program(11000 + seed, s_max=6, b_max=2, t_max=6, m_max=10)
        q.loops = tuple((lo, hi, 1) for lo, hi, _ in random_loops(rng, q.n_stmts))
        q.iter_coef = np.arange(q.n_stmts, dtype=np.uint32)
        for m in (0, (1 << p.n_slots) - 1):
            assert oracle.check(p, m) == oracle.check(q, m)
        assert oracle.repair(p) == oracle.repair(q)


@pytest.mark.parametrize("seed", range(80))
def test_loop_repair_path_independence(seed):
    from _tiny import random_loop_program

    p = random_loop_program(12000 + seed, s_min=3, s_max=5 + seed % 2, b_max=2, t_max=5, m_max=10)
    for mode in (MODE_REPAIR, MODE_REMOVE):
        got = oracle.repair(p, mode=mode)
        ref = _lowest_safe_mask(p, mode, True)
        assert got["iters"] <= p.n_slots + 3
        if ref is None:
            assert got["status"] == 1 and got["mask"] == 0
        else:
            assert got["status"] == 0 and (got["weight"], got["mask"]) == ref


@pytest.mark.parametrize("seed", range(30))
def test_loop_clause_is_exact_filter(seed):
    from _tiny import random_loop_program

    p = random_loop_program(13000 + seed, s_min=3, s_max=5, b_max=2, t_max=5, m_max=10)
    n = p.n_slots
    w0 = oracle.check(p, 0)
    X = len(w0["intra"])
    checks = {m: oracle.check(p, m) for m in range(1 << n)}
    for i in range(X):
        for j in range(X):
            for scope in ("intra", "inter"):
                if not (w0[scope][i] >> j) & 1:
                    continue
                single = {"intra": [0] * X, "inter": [0] * X, "diverge": 0}
                single[scope][i] = 1 << j
                (cl,) = oracle.clauses(p, single)
                for m in checks:
                    assert bool((checks[m][scope][i] >> j) & 1) == ((m & cl) == 0)


# --------------------------------------------------------------------------
# Negative clauses given with the program (Section 2.4: phi holds positive and
# negative monotone clauses; the mhs strategy falls back to MaxSAT)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLD["neg_cases"], ids=[c["name"] for c in GOLD["neg_cases"]])
def test_neg_cases(case):
    p = program_from_spec(case["program"])
    n = p.n_slots
    w = [int(x) for x in p.slot_weight]
    g = oracle.greedy(n, w, case["repairs"][0]["clauses"])
    assert g == case["greedy_mhs"]
    if case["program"]["neg_clauses"]:
        # the greedy hitting set breaks a negative clause: the strategy must fall back
        assert any(g & c == c for c in case["program"]["neg_clauses"])
    for exp in case["repairs"]:
        got = oracle.repair(p, mode=exp["mode"], strategy=exp["strategy"])
        for key in ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses", "forbidden"):
            assert got[key] == exp[key], (key, case["cite"])


def _random_negs(seed, n):
    rng = synth.SplitMix64(synth.program_seed(4242, seed))
    negs = []
    for _ in range(rng.randint(0, 3)):
        m = 0
        for _ in range(rng.randint(1, 2)):
            m |= 1 << rng.randint(0, n - 1)
        negs.append(m)
    return tuple(negs)


@pytest.mark.parametrize("seed", range(60))
def test_repair_path_independence_with_negative_clauses(seed):
    """With negative clauses the loop ends at the lowest-key clean mask that
    contains none of them, for both strategies."""
    from _tiny import random_loop_program

    p = random_program(14000 + seed, s_min=3, s_max=6, b_max=2, t_max=6, m_max=10) if seed % 2 else \
        random_loop_program(14000 + seed, s_min=3, s_max=5, b_max=2, t_max=5, m_max=10)
    p.neg_clauses = _random_negs(seed, p.n_slots)
    for mode in (MODE_REPAIR, MODE_REMOVE):
        forced = p.existing_mask if mode == MODE_REPAIR else 0
        best = None
        for x in range(1 << p.n_slots):
            if (x & forced) != forced or any(x & c == c for c in p.neg_clauses):
                continue
            c = oracle.check(p, x)
            if any(c["intra"]) or any(c["inter"]) or c["diverge"]:
                continue
            key = (sum(int(p.slot_weight[k]) for k in range(p.n_slots) if (x >> k) & 1), x)
            best = key if best is None or key < best else best
        for strategy in (0, 1):
            got = oracle.repair(p, mode=mode, strategy=strategy)
            if best is None:
                assert got["status"] == 1 and got["mask"] == 0
            else:
                assert got["status"] == 0 and (got["weight"], got["mask"]) == best, (strategy, p.neg_clauses)


# --------------------------------------------------------------------------
# Two barrier variables per site (slots with explicit places)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLD["site_cases"], ids=[c["name"] for c in GOLD["site_cases"]])
def test_site_cases(case):
    p = program_from_spec(case["program"])
    for chk in case["checks"]:
        got = oracle.check(p, chk["mask"])
        for key in ("intra", "inter", "diverge", "access_pairs"):
            if key in chk:
                assert got[key] == chk[key], (key, chk["mask"], case["cite"])
    for exp in case["repairs"]:
        got = oracle.repair(p, mode=exp["mode"], grid_enabled=exp["grid_enabled"])
        for key in ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses", "forbidden"):
            assert got[key] == exp[key], (key, case["cite"])


def _interpret_sites(p):
    """_interpret with several slots per place: every slot placed after
    statement q is passed when control arrives at statement q+1."""
    pos = list(range(p.n_stmts - 1)) if p.slot_pos is None else [int(x) for x in p.slot_pos]
    out = []
    for e in _interpret(p):
        if e[0] == "bar":
            out += [("bar", k) for k in range(len(pos)) if pos[k] == e[1]]
        else:
            out.append(e)
    return out


@pytest.mark.parametrize("seed", range(50))
def test_site_check_matches_interpreter(seed):
    from _tiny import random_loop_program, with_sites

    p = with_sites(random_loop_program(15000 + seed, s_min=2, s_max=5, b_max=3, t_max=5, m_max=10), seed)
    n = p.n_slots
    masks = sorted({0, (1 << n) - 1} | {(seed * 2654435761 + k * 40503) % (1 << n) for k in range(4)})
    events = _interpret_sites(p)
    for m in masks:
        got = oracle.check(p, m)
        intra, inter = _flag_reset_on_events(p, events, m)
        assert got["intra"] == intra, (m, p.slot_pos)
        assert got["inter"] == inter, (m, p.slot_pos)


def _flag_reset_on_events(p, events, mask):
    X = sum(1 for e in events if e[0] == "st")
    B, T = p.blocks, p.threads
    intra, inter = [0] * X, [0] * X
    threads = [(b, t) for b in range(B) for t in range(T)]
    for x, y in itertools.combinations(range(len(threads)), 2):
        pair = (threads[x], threads[y])
        same = pair[0][0] == pair[1][0]
        logs = ([], [])
        n = -1
        for e in events:
            if e[0] == "bar":
                k = e[1]
                if (mask >> k) & 1 and (same or p.slot_level[k] == LEVEL_GRID):
                    logs = ([], [])
                continue
            _, s, it = e
            n += 1
            fresh = []
            for who, (b, t) in enumerate(pair):
                if _runs(int(p.guard_k[s]), int(p.guard_r[s]), t):
                    inst = ("shared", b) if p.space[s] == SPACE_SHARED else ("global",)
                    ev = (inst, _addr_it(p, s, b, t, it), p.op[s] == 1, n)
                    logs[who].append(ev)
                    fresh.append((who, ev))
            for who, ev in fresh:
                for f in logs[1 - who]:
                    if f[0] == ev[0] and f[1] == ev[1] and (ev[2] or f[2]):
                        i, j = min(ev[3], f[3]), max(ev[3], f[3])
                        if same:
                            intra[i] |= 1 << j
                        else:
                            inter[i] |= 1 << j
    return intra, inter


@pytest.mark.parametrize("seed", range(50))
def test_site_repair_path_independence(seed):
    """Two variables per site: the loop still ends at the lowest-key clean
    mask; a site never needs both of its variables (grid orders all a block
    barrier orders, and costs less than both)."""
    from _tiny import random_loop_program, with_sites

    p = with_sites(random_program(16000 + seed, s_min=3, s_max=6, b_max=3, t_max=6, m_max=10) if seed % 2 else
                   random_loop_program(16000 + seed, s_min=3, s_max=5, b_max=2, t_max=5, m_max=10), seed)
    for mode in (MODE_REPAIR, MODE_REMOVE):
        for grid_enabled in (True, False):
            for strategy in (0, 1):
                got = oracle.repair(p, mode=mode, grid_enabled=grid_enabled, strategy=strategy)
                ref = _lowest_safe_mask(p, mode, grid_enabled)
                if ref is None:
                    assert got["status"] == 1 and got["mask"] == 0
                else:
                    assert got["status"] == 0 and (got["weight"], got["mask"]) == ref
                    if mode == MODE_REPAIR:
                        continue  # forced existing barriers may hold both variables of a site
                    pos = [int(x) for x in p.slot_pos]
                    for a in range(p.n_slots):
                        for b in range(a + 1, p.n_slots):
                            if pos[a] == pos[b]:
                                assert not ((got["mask"] >> a) & 1 and (got["mask"] >> b) & 1)
