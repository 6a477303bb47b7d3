"""Seeded synthetic instrumented access programs.

This module only draws inputs: it holds none of the repair method's arithmetic
(no address-map evaluation, no race test, no clause or hitting-set logic), so
both the CUDA path and the CPU oracle can consume what it produces.

A program is the concrete restatement of the paper's instrumented kernel
(Section 2.2): S straight-line statements, each one shared- or global-memory
read or write at an address given by a per-thread map, optionally under a
thread-dependent guard ``tid % k == r``; a candidate barrier slot sits between
consecutive statements (Section 2.2, "instrumented barrier"), each slot either
block-level or grid-level, with a weight (Section 2.4, ``(gw*gb) + lw^ld``).

Random numbers come from splitmix64 (Steele, Lea, Flood, OOPSLA 2014).  The
program ``p`` of a workload with seed ``s`` draws from the stream started at
``mix(s ^ (p * 0x9E3779B97F4A7C15))``.  Permutation tables are the argsort of
one 64-bit key per position drawn from the same stream (ties are impossible to
matter: the argsort is stable and keys are 64-bit).

The shapes follow the paper's corpus statistics (Section 5, Appendix A.2:
median 11 Boogie commands, 91% of kernels with at most 20 instrumented
barriers); the exact distributions are free choices and are listed per
workload in ``WORKLOADS``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

# Encodings shared by every consumer (plain integers, no arithmetic).
OP_R, OP_W = 0, 1
SPACE_SHARED, SPACE_GLOBAL = 0, 1
MAP_AFFINE, MAP_STRIDED, MAP_PERM = 0, 1, 2
LEVEL_BLOCK, LEVEL_GRID = 0, 1
MODE_REPAIR, MODE_REMOVE = 0, 1


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _mix_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    """splitmix64 stream: state += golden; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + GOLDEN) & MASK64
        return _mix(self.state)

    def bulk(self, n: int) -> np.ndarray:
        """n consecutive outputs as uint64 (advances the stream by n)."""
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            st = np.uint64(self.state) + idx * np.uint64(GOLDEN)
            out = _mix_np(st)
        self.state = (self.state + n * GOLDEN) & MASK64
        return out

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + self.next() % (hi - lo + 1)

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def bernoulli(self, p: float) -> bool:
        return self.uniform() < p

    def choice(self, items):
        return items[self.next() % len(items)]

    def permutation(self, m: int) -> np.ndarray:
        keys = self.bulk(m)
        return np.argsort(keys, kind="stable").astype(np.uint32)


def program_seed(workload_seed: int, p: int) -> int:
    return _mix((workload_seed ^ ((p * GOLDEN) & MASK64)) & MASK64)


@dataclass
class Program:
    """One instrumented access program plus its launch and repair mode.

    Arrays are per statement (length S) or per slot (length S-1); slot k sits
    between statements k and k+1.  ``guard_k == 0`` means unguarded.
    """

    op: np.ndarray          # uint8  [S]  OP_R / OP_W
    space: np.ndarray       # uint8  [S]  SPACE_SHARED / SPACE_GLOBAL
    kind: np.ndarray        # uint8  [S]  MAP_*
    a: np.ndarray           # uint32 [S]  tid multiplier (AFFINE, STRIDED)
    b: np.ndarray           # uint32 [S]  offset
    c: np.ndarray           # uint32 [S]  block multiplier
    perm_off: np.ndarray    # uint32 [S]  offset of the statement's table in perm
    guard_k: np.ndarray     # uint16 [S]
    guard_r: np.ndarray     # uint16 [S]
    slot_level: np.ndarray  # uint8  [n_slots] (S-1 unless slot_pos is given)
    slot_guard_k: np.ndarray  # uint16 [n_slots]
    slot_guard_r: np.ndarray  # uint16 [n_slots]
    slot_weight: np.ndarray   # uint32 [n_slots]
    m_shared: int
    m_global: int
    perm: np.ndarray        # uint32 concatenated permutation tables
    existing_mask: int
    blocks: int
    threads: int
    mode: int = MODE_REPAIR
    # counted loops (lo, hi, trips): statements lo..hi run `trips` times; the
    # slot before statement lo is the loop head (it runs before every
    # iteration).  Ranges are nested or disjoint, lo >= 1, nested loops start
    # strictly inside their parent.
    loops: tuple = ()
    # per-statement coefficient d of the innermost enclosing loop's counter
    # (0..trips-1) in the address map; None = all zero
    iter_coef: Optional[np.ndarray] = None
    # negative clauses given with the program: no repair may enable every
    # slot of one of these masks (constraints from outside the model, e.g. a
    # pair of barriers the programmer rules out)
    neg_clauses: tuple = ()
    # per slot, the statement it follows (several slots may share a place,
    # e.g. a block and a grid candidate at every site); None: slot k follows
    # statement k
    slot_pos: Optional[np.ndarray] = None

    @property
    def n_stmts(self) -> int:
        return int(self.op.shape[0])

    @property
    def n_slots(self) -> int:
        return int(self.slot_level.shape[0])

    def grid_mask(self) -> int:
        m = 0
        for k, lv in enumerate(self.slot_level.tolist()):
            if lv == LEVEL_GRID:
                m |= 1 << k
        return m


def make_program(stmts: List[dict], *, blocks: int, threads: int, m_shared: int = 0,
                 m_global: int = 0, slot_level=None, slot_guard=None, slot_weight=None,
                 perms: Optional[List[np.ndarray]] = None, existing_mask: int = 0,
                 mode: int = MODE_REPAIR, loops=(), neg_clauses=(), slot_pos=None) -> Program:
    """Build a Program from a list of statement dicts.

    Each dict: op ('R'/'W' or 0/1), space ('shared'/'global' or 0/1), kind
    ('affine'/'strided'/'perm' or 0/1/2), a, b, c, perm (index into ``perms``),
    guard (k, r), d (coefficient of the innermost loop counter).  Missing
    fields default to an unguarded shared affine read.  ``loops``: (lo, hi,
    trips) triples.
    """
    S = len(stmts)
    enc_op = {"R": OP_R, "W": OP_W, OP_R: OP_R, OP_W: OP_W}
    enc_sp = {"shared": SPACE_SHARED, "global": SPACE_GLOBAL, 0: 0, 1: 1}
    enc_kd = {"affine": MAP_AFFINE, "strided": MAP_STRIDED, "perm": MAP_PERM, 0: 0, 1: 1, 2: 2}
    perms = perms or []
    offs = []
    o = 0
    for pt in perms:
        offs.append(o)
        o += len(pt)
    perm = np.concatenate(perms).astype(np.uint32) if perms else np.zeros(0, np.uint32)
    cols = {n: [] for n in ("op", "space", "kind", "a", "b", "c", "perm_off", "gk", "gr", "d")}
    for st in stmts:
        cols["op"].append(enc_op[st.get("op", "R")])
        cols["space"].append(enc_sp[st.get("space", "shared")])
        cols["kind"].append(enc_kd[st.get("kind", "affine")])
        cols["a"].append(int(st.get("a", 1)))
        cols["b"].append(int(st.get("b", 0)))
        cols["c"].append(int(st.get("c", 0)))
        cols["perm_off"].append(offs[st["perm"]] if "perm" in st else 0)
        gk, gr = st.get("guard", (0, 0))
        cols["gk"].append(gk)
        cols["gr"].append(gr)
        cols["d"].append(int(st.get("d", 0)))
    n = S - 1 if slot_pos is None else len(slot_pos)
    if slot_level is None:
        slot_level = [LEVEL_BLOCK] * n
    if slot_guard is None:
        slot_guard = [(0, 0)] * n
    if slot_weight is None:
        slot_weight = [12 * int(lv) + 1 for lv in slot_level]
    return Program(
        op=np.array(cols["op"], np.uint8), space=np.array(cols["space"], np.uint8),
        kind=np.array(cols["kind"], np.uint8), a=np.array(cols["a"], np.uint32),
        b=np.array(cols["b"], np.uint32), c=np.array(cols["c"], np.uint32),
        perm_off=np.array(cols["perm_off"], np.uint32),
        guard_k=np.array(cols["gk"], np.uint16), guard_r=np.array(cols["gr"], np.uint16),
        slot_level=np.array(slot_level, np.uint8).reshape(n),
        slot_guard_k=np.array([g[0] for g in slot_guard], np.uint16).reshape(n),
        slot_guard_r=np.array([g[1] for g in slot_guard], np.uint16).reshape(n),
        slot_weight=np.array(slot_weight, np.uint32).reshape(n),
        m_shared=int(m_shared), m_global=int(m_global), perm=perm,
        existing_mask=int(existing_mask), blocks=int(blocks), threads=int(threads), mode=int(mode),
        loops=tuple((int(lo), int(hi), int(tr)) for lo, hi, tr in loops),
        iter_coef=np.array(cols["d"], np.uint32), neg_clauses=tuple(int(x) for x in neg_clauses),
        slot_pos=None if slot_pos is None else np.array(slot_pos, np.uint32).reshape(n))


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    """Distribution of one synthetic workload (all sizes overridable)."""

    name: str
    seed: int
    n_programs: int
    blocks: object            # int, or ("uniform", lo, hi)
    threads: object           # int, or ("loguniform", lo, hi)
    n_stmts: object           # int, or ("uniform", lo, hi)
    space: int
    m_words: object           # int, or ("times_threads", k)
    maps: Dict[str, float]    # kind -> probability
    p_write: float
    guard_fraction: object    # float, or ("uniform", lo, hi) per program
    guard_ks: tuple = (2, 4, 8, 32)
    p_grid_slot: float = 0.0
    grid_weight: int = 4
    mode: object = MODE_REPAIR  # int, or ("mixed", p_remove)
    affine_as: tuple = (1, 2)
    affine_b_max: int = 4
    strided_max: int = 32
    block_offset: bool = False  # global block-offset maps a*(tid + T*blk) + b
    p_halo: float = 0.0         # block-offset maps: fraction with a halo offset b in [1, 4]
    p_collide: float = 0.01     # programs given one deliberately colliding write
    # counted loops: probability that a program has one, trip counts of the
    # outer / nested loop, probability of a nested loop, the loop-counter
    # coefficients d of statements inside loops (0, 1, 2 or "T" = threads)
    p_loop: float = 0.0
    loop_len: tuple = (2, 5)
    outer_trips: tuple = (2, 4)
    p_nested: float = 0.5
    inner_len: tuple = (1, 3)
    inner_trips: tuple = (2, 3)
    iter_coefs: Dict[object, float] = field(default_factory=lambda: {0: 0.4, 1: 0.2, 2: 0.1, "T": 0.3})
    loop_weight_base: int = 10  # lw of the weight (gw*gb) + lw^ld
    both_sites: bool = False    # a block and a grid candidate at every site (two slots per place)
    extra: dict = field(default_factory=dict)


WORKLOADS: Dict[str, Workload] = {
    # one program, 1 block x 64 threads, 8 statements, 7 block slots,
    # 128-word shared array, (a*tid+b) mod 128, a in {1,2}, b in [0,4], 50% writes
    "single_1x64_s8": Workload(
        name="single_1x64_s8", seed=0, n_programs=1, blocks=1, threads=64, n_stmts=8,
        space=SPACE_SHARED, m_words=128, maps={"affine": 1.0}, p_write=0.5,
        guard_fraction=0.0, p_collide=0.0),
    # 1,024 programs, 4 blocks x 256 threads, 24 statements, 23 block slots,
    # 1,024-word shared array; 40% affine / 30% strided / 30% permutation maps,
    # 60% reads, 25% of statements under tid % k == r guards (if-blocks)
    "batch1024_4x256_s24": Workload(
        name="batch1024_4x256_s24", seed=1, n_programs=1024, blocks=4, threads=256,
        n_stmts=24, space=SPACE_SHARED, m_words=1024,
        maps={"affine": 0.4, "strided": 0.3, "perm": 0.3}, p_write=0.4,
        guard_fraction=0.25),
    # 256 programs, 64 blocks x 256 threads, 16 statements over a 65,536-word
    # global array, block-offset affine maps a*(tid + T*blk) + b (one stride
    # a in {1,2} per program; b = 0, or a halo offset in [1,4] for 15% of the
    # statements), 15 slots each block or grid (grid w.p. 0.75; grid weight 4,
    # block weight 1)
    "interblock256_64x256_s16": Workload(
        name="interblock256_64x256_s16", seed=2, n_programs=256, blocks=64, threads=256,
        n_stmts=16, space=SPACE_GLOBAL, m_words=65536, maps={"affine": 1.0}, p_write=0.5,
        guard_fraction=0.0, p_grid_slot=0.75, grid_weight=4, block_offset=True, p_halo=0.15),
    # 4,096 uneven programs: threads log-uniform 32-1024, blocks uniform 1-16,
    # statements uniform 4-24, shared array of 4*threads words, guards on 0-30%
    # of statements, half repair (E=0) / half removal (E = all slots)
    "uneven4096_mixed": Workload(
        name="uneven4096_mixed", seed=3, n_programs=4096, blocks=("uniform", 1, 16),
        threads=("loguniform", 32, 1024), n_stmts=("uniform", 4, 24), space=SPACE_SHARED,
        m_words=("times_threads", 4), maps={"affine": 0.4, "strided": 0.3, "perm": 0.3},
        p_write=0.4, guard_fraction=("uniform", 0.0, 0.3), mode=("mixed", 0.5)),
    # 512 programs with counted loops: 4 blocks x 256 threads, 12 statements
    # (11 block slots) over a 1,024-word shared array, maps and reads as in
    # the 1,024-program batch, guards on 15% of statements; every program has
    # a loop of 2-5 statements run 2-4 times, half of them a nested loop of
    # 1-3 statements run 2-3 times (at most 25 statement instances run);
    # addresses inside loops move by d*t, d in {0, 1, 2, threads}; slot
    # weights lw^ld with lw = 10 (1, 10, 100 by loop depth)
    "loops512_4x256_s12": Workload(
        name="loops512_4x256_s12", seed=5, n_programs=512, blocks=4, threads=256,
        n_stmts=12, space=SPACE_SHARED, m_words=1024,
        maps={"affine": 0.4, "strided": 0.3, "perm": 0.3}, p_write=0.4,
        guard_fraction=0.15, p_loop=1.0),
    # 128 programs, 16 blocks x 256 threads, 16 statements over a 16,384-word
    # global array with block-offset maps as in the inter-block workload, and
    # at each of the 15 sites both a block candidate (weight 1) and a grid
    # candidate (weight 13 = gw + lw^0 with the paper's gw = 12): 30 barrier
    # variables per program
    "sites128_16x256_s16": Workload(
        name="sites128_16x256_s16", seed=6, n_programs=128, blocks=16, threads=256,
        n_stmts=16, space=SPACE_GLOBAL, m_words=16384, maps={"affine": 1.0}, p_write=0.5,
        guard_fraction=0.0, grid_weight=13, block_offset=True, p_halo=0.15, both_sites=True),
    # the large programs mixed into the serving stream: 128 blocks x 1,024
    # threads, 24 statements, 4,096-word shared array
    "large_128x1024_s24": Workload(
        name="large_128x1024_s24", seed=4, n_programs=1, blocks=128, threads=1024,
        n_stmts=24, space=SPACE_SHARED, m_words=4096,
        maps={"affine": 0.4, "strided": 0.3, "perm": 0.3}, p_write=0.4,
        guard_fraction=("uniform", 0.0, 0.3), mode=("mixed", 0.5)),
}


def _draw_size(rng: SplitMix64, spec) -> int:
    if isinstance(spec, int):
        return spec
    kind = spec[0]
    if kind == "uniform":
        return rng.randint(spec[1], spec[2])
    if kind == "loguniform":
        u = rng.uniform()
        v = math.exp(math.log(spec[1]) + u * (math.log(spec[2]) - math.log(spec[1])))
        return int(min(spec[2], max(spec[1], round(v))))
    raise ValueError(spec)


def _injective_on_threads(mult: int, m: int, threads: int) -> bool:
    """(mult*tid + const) mod m takes distinct values for tid in [0, threads)
    iff threads <= m / gcd(mult, m)  (elementary number theory)."""
    if m == 0:
        return False
    return threads <= m // math.gcd(mult % m if mult % m else m, m)


def _draw_map(rng: SplitMix64, wl: Workload, m: int, T: int, kinds, probs, stride: int = 1):
    u = rng.uniform()
    acc = 0.0
    kind = kinds[-1]
    for kd, pr in zip(kinds, probs):
        acc += pr
        if u < acc:
            kind = kd
            break
    if kind == "affine":
        if wl.block_offset:
            a = stride
            b = rng.randint(1, wl.affine_b_max) if rng.bernoulli(wl.p_halo) else 0
            return MAP_AFFINE, a, b, a * T, a
        a = rng.choice(wl.affine_as)
        b = rng.randint(0, wl.affine_b_max)
        return MAP_AFFINE, a, b, 0, a
    if kind == "strided":
        s = rng.randint(1, wl.strided_max)
        b = rng.randint(0, s - 1)
        return MAP_STRIDED, s, b, 0, s
    return MAP_PERM, 0, 0, 0, None


def generate_program(wl: Workload, p: int, **override) -> Program:
    """Draw program ``p`` of workload ``wl`` (sizes may be overridden)."""
    rng = SplitMix64(program_seed(wl.seed, p))
    B = override.get("blocks") or _draw_size(rng, wl.blocks)
    T = override.get("threads") or _draw_size(rng, wl.threads)
    S = override.get("n_stmts") or _draw_size(rng, wl.n_stmts)
    if isinstance(wl.m_words, tuple):
        M = wl.m_words[1] * T
    else:
        M = wl.m_words
    M = override.get("m_words") or M
    gf = wl.guard_fraction
    if isinstance(gf, tuple):
        gf = gf[1] + rng.uniform() * (gf[2] - gf[1])
    mode = wl.mode
    if isinstance(mode, tuple):
        mode = MODE_REMOVE if rng.bernoulli(mode[1]) else MODE_REPAIR
    mode = override.get("mode", mode)
    kinds = list(wl.maps.keys())
    probs = [wl.maps[k] for k in kinds]

    # Guards form if-blocks: runs of 1-4 consecutive statements sharing one
    # guard (tid % k == r); the run-start probability gives the requested
    # guarded fraction on average (mean run length 2.5).
    guards = [(0, 0)] * S
    if gf > 0:
        p_start = gf / (2.5 - 1.5 * gf)
        s = 0
        while s < S:
            if rng.bernoulli(p_start):
                run = rng.randint(1, 4)
                k = rng.choice(wl.guard_ks)
                r = rng.randint(0, k - 1)
                for t in range(s, min(S, s + run)):
                    guards[t] = (k, r)
                s += run
            else:
                s += 1

    stride = rng.choice(wl.affine_as) if wl.block_offset else 1
    collide_at = -1
    if wl.p_collide > 0 and rng.bernoulli(wl.p_collide):
        collide_at = rng.randint(0, S - 1)

    stmts = []
    perms = []
    for s in range(S):
        is_w = rng.bernoulli(wl.p_write) or s == collide_at
        while True:
            kind, a, b, c, mult = _draw_map(rng, wl, M, T, kinds, probs, stride)
            if kind == MAP_PERM:
                break  # a permutation restricted to T <= M threads is injective
            if not is_w or s == collide_at:
                break
            if wl.block_offset:
                # a write must be injective over the whole grid: c == a*T makes
                # the map a*(tid + T*blk) + b, injective iff B*T <= M / gcd(a, M)
                if c == a * T and _injective_on_threads(a, M, B * T):
                    break
            elif _injective_on_threads(mult, M, T):
                break
        st = {"op": OP_W if is_w else OP_R, "space": wl.space, "kind": kind,
              "a": a, "b": b, "c": c, "guard": guards[s]}
        if s == collide_at:
            # a deliberately colliding write: every active thread hits one word
            st.update(kind=MAP_AFFINE, a=0, b=rng.randint(0, M - 1), c=0)
        elif kind == MAP_PERM:
            st["perm"] = len(perms)
            perms.append(rng.permutation(M))
            if wl.block_offset:
                st["c"] = T
        stmts.append(st)

    n = S - 1
    levels = [LEVEL_GRID if (wl.p_grid_slot > 0 and rng.bernoulli(wl.p_grid_slot)) else LEVEL_BLOCK
              for _ in range(n)]
    # Slot guard: a slot strictly inside an if-block (both neighbours carry the
    # same guard) is under that guard; otherwise it sits at a join point.
    sguard = []
    for k in range(n):
        g0, g1 = guards[k], guards[k + 1]
        sguard.append(g0 if (g0[0] != 0 and g0 == g1) else (0, 0))
    loops = _draw_loops(wl, p, S) if wl.p_loop > 0 else []
    depth = [sum(1 for lo, hi, _ in loops if lo <= s <= hi) for s in range(S)]
    if loops:
        rng_d = SplitMix64(program_seed(wl.seed ^ 0x100F5, p))
        dk = list(wl.iter_coefs.keys())
        dp = [wl.iter_coefs[k] for k in dk]
        for s in range(S):
            if depth[s] and s != collide_at:
                d = dk[_choose(rng_d, dp)]
                stmts[s]["d"] = T if d == "T" else int(d)
    # weight (gw*gb) + lw^ld; the barrier of slot k runs at statement k+1, so
    # its loop depth is that statement's
    weights = [(wl.grid_weight - 1 if lv == LEVEL_GRID else 0) + wl.loop_weight_base ** depth[k + 1]
               for k, lv in enumerate(levels)]
    slot_pos = None
    if wl.both_sites:  # every place gets a block and a grid slot
        slot_pos = [k for k in range(n) for _ in (0, 1)]
        levels = [lv for _ in range(n) for lv in (LEVEL_BLOCK, LEVEL_GRID)]
        sguard = [g for g in sguard for _ in (0, 1)]
        weights = [(wl.grid_weight - 1 if lv == LEVEL_GRID else 0) + wl.loop_weight_base ** depth[slot_pos[k] + 1]
                   for k, lv in enumerate(levels)]
        n = len(slot_pos)
    existing = ((1 << n) - 1) if mode == MODE_REMOVE else 0
    return make_program(
        stmts, blocks=B, threads=T,
        m_shared=M if wl.space == SPACE_SHARED else 0,
        m_global=M if wl.space == SPACE_GLOBAL else 0,
        slot_level=levels, slot_guard=sguard, slot_weight=weights, perms=perms,
        existing_mask=existing, mode=mode, loops=loops, slot_pos=slot_pos)


def _choose(rng: SplitMix64, probs) -> int:
    u = rng.uniform()
    acc = 0.0
    for i, q in enumerate(probs):
        acc += q
        if u < acc:
            return i
    return len(probs) - 1


def _draw_loops(wl: Workload, p: int, S: int, max_exec: int = 25) -> list:
    """A counted loop over statements lo..hi (lo >= 1, so its head slot
    exists) and, with probability p_nested, a loop nested strictly inside it;
    trip counts are lowered until at most max_exec instances run."""
    rng = SplitMix64(program_seed(wl.seed ^ 0x1009, p))
    if S < 3 or not rng.bernoulli(wl.p_loop):
        return []
    length = min(rng.randint(*wl.loop_len), S - 1)
    lo = rng.randint(1, S - length)
    hi = lo + length - 1
    t1 = rng.randint(*wl.outer_trips)
    inner = None
    if hi > lo and rng.bernoulli(wl.p_nested):
        l2 = min(rng.randint(*wl.inner_len), hi - lo)
        lo2 = rng.randint(lo + 1, hi - l2 + 1)
        inner = [lo2, lo2 + l2 - 1, rng.randint(*wl.inner_trips)]

    def count():
        c = S + (t1 - 1) * length
        if inner:
            c += t1 * (inner[2] - 1) * (inner[1] - inner[0] + 1)
        return c

    while count() > max_exec:
        if inner and inner[2] > 1:
            inner[2] -= 1
        else:
            t1 -= 1
    loops = [(lo, hi, t1)]
    if inner:
        loops.append(tuple(inner))
    return loops


def generate(workload: str, n_programs: Optional[int] = None, start: int = 0,
             **override) -> List[Program]:
    """Programs ``start .. start+n-1`` of a named workload."""
    wl = WORKLOADS[workload]
    n = wl.n_programs if n_programs is None else n_programs
    return [generate_program(wl, p, **override) for p in range(start, start + n)]


def poisson_arrivals(rate_per_s: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream: exponential gaps drawn by
    inversion from the splitmix64 stream ``seed``."""
    rng = SplitMix64(program_seed(seed, 0x5EED))
    u = (rng.bulk(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)
