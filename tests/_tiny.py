"""Seeded tiny and medium random programs for tests (draws only, no method
arithmetic)."""
import numpy as np

from paper_2011_08373_gb300.synth import (
    LEVEL_BLOCK, LEVEL_GRID, MAP_AFFINE, MAP_PERM, MAP_STRIDED, MODE_REMOVE, MODE_REPAIR,
    SPACE_GLOBAL, SPACE_SHARED, SplitMix64, make_program, program_seed)


def random_program(seed, *, s_max=5, b_max=3, t_max=8, m_max=16, spaces=(0, 1),
                   kinds=(MAP_AFFINE, MAP_STRIDED, MAP_PERM), a_max=5, c_max=8,
                   guard_ks=(0, 0, 1, 2, 3, 4), p_write=0.5, weight_max=5, s_min=1,
                   t_min=1, b_min=1):
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
              "c": rng.randint(0, c_max) if space == SPACE_GLOBAL else 0, "guard": (gk, gr)}
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
