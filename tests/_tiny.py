"""Seeded tiny and medium random programs for tests (draws only, no method
arithmetic)."""
import numpy as np

from paper_2011_08373_gb300.synth import (
    LEVEL_BLOCK, LEVEL_GRID, MAP_AFFINE, MAP_PERM, MAP_STRIDED, MODE_REMOVE, MODE_REPAIR,
    SPACE_GLOBAL, SPACE_SHARED, SplitMix64, make_program, program_seed)


def random_program(seed, *, s_max=5, b_max=3, t_max=8, m_max=16, spaces=(0, 1),
                   kinds=(MAP_AFFINE, MAP_STRIDED, MAP_PERM), a_max=5, c_max=8,
                   guard_ks=(0, 0, 1, 2, 3, 4), p_write=0.5, weight_max=5, s_min=1,
                   t_min=1, b_min=1, shared_c=False):
    rng = SplitMix64(program_seed(0xC0FFEE, seed))
    S = rng.randint(s_min, s_max)
    B = rng.randint(b_min, b_max)
    T = rng.randint(t_min, t_max)
    m_sh = rng.randint(1, m_max)
    m_gl = rng.randint(1, m_max)
    stmts, perms = [], []
    for _ in range(S):
        space = rng.choice(spaces)
        kind = rng.choice(kinds)
        M = m_sh if space == SPACE_SHARED else m_gl
        gk = rng.choice(guard_ks)
        gr = rng.randint(0, gk - 1) if gk > 0 else 0
        st = {"op": 1 if rng.bernoulli(p_write) else 0, "space": space, "kind": kind,
              "a": rng.randint(0, a_max), "b": rng.randint(0, 3 * m_max),
              "c": rng.randint(0, c_max) if (space == SPACE_GLOBAL or shared_c) else 0, "guard": (gk, gr)}
        if kind == MAP_PERM:
            st["perm"] = len(perms)
            perms.append(rng.permutation(M))
        stmts.append(st)
    n = S - 1
    levels = [LEVEL_GRID if rng.bernoulli(0.5) else LEVEL_BLOCK for _ in range(n)]
    sguard = []
    for _ in range(n):
        gk = rng.choice(guard_ks)
        sguard.append((gk, rng.randint(0, gk - 1) if gk > 0 else 0))
    weights = [rng.randint(1, weight_max) for _ in range(n)]
    existing = rng.randint(0, (1 << n) - 1) if n > 0 else 0
    mode = MODE_REMOVE if rng.bernoulli(0.5) else MODE_REPAIR
    return make_program(stmts, blocks=B, threads=T, m_shared=m_sh, m_global=m_gl,
                        slot_level=levels, slot_guard=sguard, slot_weight=weights,
                        perms=perms, existing_mask=existing, mode=mode)


def random_loops(rng, S, max_exec=25, trips_max=3):
    """Up to two counted loops over statements 1..S-1 (nested or disjoint, a
    nested loop starting strictly inside its parent), with at most
    ``max_exec`` executed statement instances."""
    if S < 2:
        return []
    for _ in range(20):
        loops = []
        lo = rng.randint(1, S - 1)
        hi = rng.randint(lo, S - 1)
        t1 = rng.randint(1, trips_max)
        loops.append((lo, hi, t1))
        count = S + (t1 - 1) * (hi - lo + 1)
        if rng.bernoulli(0.5):
            if hi > lo and rng.bernoulli(0.5):  # nested
                lo2 = rng.randint(lo + 1, hi)
                hi2 = rng.randint(lo2, hi)
                t2 = rng.randint(1, trips_max)
                loops.append((lo2, hi2, t2))
                count += t1 * (t2 - 1) * (hi2 - lo2 + 1)
            elif hi + 1 <= S - 1:  # disjoint, after the first
                lo2 = rng.randint(hi + 1, S - 1)
                hi2 = rng.randint(lo2, S - 1)
                t2 = rng.randint(1, trips_max)
                loops.append((lo2, hi2, t2))
                count += (t2 - 1) * (hi2 - lo2 + 1)
        if count <= max_exec:
            return loops
    return []


def random_loop_program(seed, *, s_max=5, b_max=3, t_max=6, m_max=12, d_max=3, trips_max=3,
                        max_exec=25, **kw):
    """random_program plus counted loops and per-statement loop-counter
    coefficients."""
    p = random_program(seed, s_max=s_max, b_max=b_max, t_max=t_max, m_max=m_max, **kw)
    rng = SplitMix64(program_seed(0x100F5, seed))
    p.loops = tuple(random_loops(rng, p.n_stmts, max_exec, trips_max))
    p.iter_coef = np.array([rng.randint(0, d_max) for _ in range(p.n_stmts)], np.uint32)
    return p


def with_sites(p, seed, p_both=0.5):
    """Re-lay the slots of p as candidate sites: each place between two
    statements gets one slot of its drawn level or, with probability p_both,
    two slots (a block and a grid candidate, the grid one heavier)."""
    rng = SplitMix64(program_seed(0x517E5, seed))
    pos, lv, gk, gr, w = [], [], [], [], []
    for g in range(p.n_stmts - 1):
        kinds = [LEVEL_BLOCK, LEVEL_GRID] if rng.bernoulli(p_both) else [int(p.slot_level[g])]
        for level in kinds:
            pos.append(g)
            lv.append(level)
            gk.append(int(p.slot_guard_k[g]))
            gr.append(int(p.slot_guard_r[g]))
            w.append(rng.randint(1, 4) + (rng.randint(1, 6) if level == LEVEL_GRID else 0))
    n = len(pos)
    p.slot_pos = np.array(pos, np.uint32)
    p.slot_level = np.array(lv, np.uint8)
    p.slot_guard_k = np.array(gk, np.uint16)
    p.slot_guard_r = np.array(gr, np.uint16)
    p.slot_weight = np.array(w, np.uint32)
    p.existing_mask = rng.randint(0, (1 << n) - 1) if n else 0
    return p
