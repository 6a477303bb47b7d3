"""C ABI contract tests that need no GPU: the library loads, exports every
entry point declared in include/gpurepair.h, and rejects invalid input with
GR_EINVAL before any device work; packing is deterministic."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2011_08373_gb300 import binding as gb
from paper_2011_08373_gb300 import synth
from paper_2011_08373_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return gb.lib()


def declared_entry_points():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(gr_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_entry_points()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(gb.EXPORTS) <= set(names)


def test_version(lib):
    assert "sm_103a" in gb.version()


def test_struct_sizes_match_header(lib):
    assert C.sizeof(gb.gr_stmt) == 24
    assert C.sizeof(gb.gr_witnesses) == 272
    assert C.sizeof(gb.gr_repair_result) == 2944
    assert C.sizeof(gb.gr_program) == 120
    assert C.sizeof(gb.gr_loop) == 12
    assert C.sizeof(gb.gr_options) == 16 and gb.gr_options.deadline_us.offset == 8


@pytest.mark.parametrize("over", [{"deadline_us": (1 << 40) + 1}, {"max_iters": 65}, {"strategy": 2}])
def test_options_rejected_before_device_work(lib, over):
    """Out-of-range options: GR_EINVAL before any CUDA call (this host has no GPU)."""
    good = synth.generate("single_1x64_s8", 1)[0]
    kw = {"max_iters": 64, "strategy": 0, "deadline_us": 0}
    kw.update(over)
    with pytest.raises(gb.GrError) as e:
        gb.repair_batch([good], **kw)
    assert e.value.code == gb.EINVAL


def _prog(**over):
    p = synth.generate("single_1x64_s8", 1)[0]
    for k, v in over.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("mutate,msg", [
    (lambda p: setattr(p, "threads", 2000), "threads"),
    (lambda p: setattr(p, "threads", 0), "threads"),
    (lambda p: setattr(p, "blocks", 0), "blocks"),
    (lambda p: setattr(p, "blocks", 70000), "blocks"),
    (lambda p: setattr(p, "m_shared", 0), "0 words"),
    (lambda p: setattr(p, "m_shared", 70000), "array size"),
    (lambda p: p.guard_k.__setitem__(0, 4) or p.guard_r.__setitem__(0, 4), "guard"),
    (lambda p: p.guard_r.__setitem__(0, 1), "guard"),
    (lambda p: p.slot_weight.__setitem__(0, 0), "weight"),
    (lambda p: p.slot_level.__setitem__(0, 2), "level"),
    (lambda p: setattr(p, "existing_mask", 1 << 7), "existing_mask"),
    (lambda p: p.op.__setitem__(0, 3), "op"),
])
def test_validation_rejects(lib, mutate, msg):
    p = _prog()
    mutate(p)
    with pytest.raises(gb.GrError) as e:
        gb.validate(p)
    assert e.value.code == gb.EINVAL
    assert msg in str(e.value)


def test_validation_rejects_bad_permutation(lib):
    p = synth.make_program([{"op": "W", "kind": "perm", "perm": 0}, {"op": "R"}], blocks=1,
                           threads=4, m_shared=4, perms=[np.array([0, 1, 1, 3], np.uint32)])
    with pytest.raises(gb.GrError):
        gb.validate(p)
    p = synth.make_program([{"op": "W", "kind": "perm", "perm": 0}, {"op": "R"}], blocks=1,
                           threads=4, m_shared=4, perms=[np.array([0, 1, 2], np.uint32)])
    with pytest.raises(gb.GrError):
        gb.validate(p)


def test_permutation_check_covers_the_entries_read(lib):
    """A permutation statement's table must hold distinct indices below M
    where the statement reads it: from b on, one entry per thread, when its
    address does not depend on the block; the whole table when it does.
    Entries nobody reads are not checked."""
    table = np.array([5, 5, 0, 1, 7, 7, 7, 7], np.uint32)  # distinct only at 2..3 (and 0 at 2)

    def prog(b, c=0, blocks=1, threads=2):
        return synth.make_program([{"op": "W", "kind": "perm", "perm": 0, "b": b, "c": c}, {"op": "R"}],
                                  blocks=blocks, threads=threads, m_shared=8, perms=[table])

    gb.validate(prog(b=2))  # reads entries 2, 3: distinct, below 8
    for bad in (prog(b=0), prog(b=4), prog(b=3, threads=3)):  # a repeat, or 7 then 7, among those read
        with pytest.raises(gb.GrError) as e:
            gb.validate(bad)
        assert e.value.code == gb.EINVAL and "permutation" in str(e.value)
    # the block term moves the window across the table: all of it must be a permutation
    with pytest.raises(gb.GrError):
        gb.validate(prog(b=2, c=2, blocks=2))
    gb.validate(prog(b=2, c=8, blocks=2))  # c = 0 mod M: every block reads entries 2, 3
    # wrapping past the end: entries 7, 0 of a table whose others repeat
    wrap = np.array([3, 9, 9, 9, 9, 9, 9, 4], np.uint32)
    gb.validate(synth.make_program([{"op": "W", "kind": "perm", "perm": 0, "b": 7}, {"op": "R"}],
                                   blocks=1, threads=2, m_shared=8, perms=[wrap]))


def test_invalid_batch_rejected_before_device_work(lib):
    good = synth.generate("single_1x64_s8", 1)[0]
    bad = _prog(threads=5000)
    with pytest.raises(gb.GrError) as e:
        gb.repair_batch([good, bad])
    assert e.value.code == gb.EINVAL and "program 1" in str(e.value)


def test_solve_rejects_bad_arguments(lib):
    with pytest.raises(gb.GrError):
        gb.solve(0, [], [1])
    with pytest.raises(gb.GrError):
        gb.solve(3, [1, 0, 1], [1])
    with pytest.raises(gb.GrError):
        gb.solve(3, [1, 1, 1], [8])
    with pytest.raises(gb.GrError):
        gb.solve(3, [1, 1, 1], [1], neg=[0])


def test_pack_is_deterministic_and_sized(lib):
    progs = synth.generate("uneven4096_mixed", 24)
    a1, s1 = gb.pack(progs)
    a2, s2 = gb.pack(progs)
    assert s1 == s2 and a1.nbytes == a2.nbytes
    assert np.array_equal(a1, a2)
    assert a1.nbytes % 256 == 0 and s1 % 256 == 0
    # the arena header records the program count and the packer's magic
    hdr = a1[:16].view(np.uint32)
    assert hdr[0] == 0x47525031 and hdr[1] == 24


def test_generator_is_deterministic():
    a = synth.generate("batch1024_4x256_s24", 3)
    b = synth.generate("batch1024_4x256_s24", 3)
    for x, y in zip(a, b):
        for f in ("op", "space", "kind", "a", "b", "c", "guard_k", "guard_r", "slot_guard_k", "perm"):
            assert np.array_equal(getattr(x, f), getattr(y, f))
    p = synth.generate("batch1024_4x256_s24", 1, start=5)[0]
    assert p.n_stmts == 24 and p.blocks == 4 and p.threads == 256 and p.m_shared == 1024


def test_workload_shapes():
    for name, (B, T, S, M) in {"single_1x64_s8": (1, 64, 8, 128),
                               "interblock256_64x256_s16": (64, 256, 16, 65536)}.items():
        p = synth.generate(name, 1)[0]
        assert (p.blocks, p.threads, p.n_stmts) == (B, T, S)
        assert max(p.m_shared, p.m_global) == M
    p = synth.generate("interblock256_64x256_s16", 1)[0]
    assert set(p.slot_weight.tolist()) <= {1, 4}
    for p in synth.generate("uneven4096_mixed", 40):
        assert 1 <= p.blocks <= 16 and 32 <= p.threads <= 1024 and 4 <= p.n_stmts <= 24
        assert p.m_shared == 4 * p.threads


def _loop_prog(loops, S=6):
    p = synth.make_program([{"op": "W" if s % 2 else "R", "a": 1, "b": s} for s in range(S)],
                           blocks=1, threads=8, m_shared=64, loops=loops)
    return p


@pytest.mark.parametrize("loops,msg", [
    ([(0, 2, 2)], "lo <= hi"),           # no head slot before statement 0
    ([(3, 2, 2)], "lo <= hi"),
    ([(2, 6, 2)], "hi < n_stmts"),
    ([(2, 3, 0)], "trips"),
    ([(1, 3, 2), (2, 4, 2)], "neither disjoint nor nested"),
    ([(1, 3, 2), (1, 2, 2)], "neither disjoint nor nested"),  # nested loops need their own heads
    ([(1, 5, 6)], "statement instances"),
    ([(1, 1, 2), (2, 2, 2), (3, 3, 2), (4, 4, 2), (5, 5, 2)], "loops"),
])
def test_validation_rejects_bad_loops(lib, loops, msg):
    with pytest.raises(gb.GrError) as e:
        gb.validate(_loop_prog(loops))
    assert e.value.code == gb.EINVAL
    assert msg in str(e.value)


def test_validation_accepts_loops(lib):
    for loops in ([(1, 5, 4)], [(1, 4, 2), (2, 3, 3)], [(1, 2, 3), (3, 5, 2)], [(5, 5, 20)]):
        gb.validate(_loop_prog(loops))


# DevProg layout (bytes): n_stmts 0, n_slots 4, general 60, gapslots
# 368..495, n_neg 496, neg 512..639, stmts 640 + 32*k (op 0, space 1, kind 2,
# bm 8, gk 20, gr 22)
DEVPROG_BYTES, STMT0, GAPS0, NEG0 = 1440, 640, 368, 496


def _devprog(arena, i):
    progs_off = int(arena[16:24].view(np.uint64)[0])
    base = progs_off + DEVPROG_BYTES * i
    return arena[base:base + DEVPROG_BYTES]


def test_packer_lays_out_executed_instances(lib):
    """Host-side packing of loop programs: one packed statement per executed
    instance, in the oracle's execution order, with the loop-counter term in
    its offset, and the slot whose barrier runs between consecutive instances."""
    import oracle
    from _tiny import random_loop_program

    progs = [random_loop_program(seed, s_min=3, s_max=8, m_max=40) for seed in range(40)]
    arena, _ = gb.pack(progs)
    for i, p in enumerate(progs):
        d = _devprog(arena, i)
        order = oracle.unroll(p)
        assert int(d[0:4].view(np.uint32)[0]) == len(order)
        assert int(d[4:8].view(np.uint32)[0]) == p.n_slots
        assert int(d[60:64].view(np.uint32)[0]) == (1 if p.loops else 0)
        for z, (s, ctr) in enumerate(order):
            st = d[STMT0 + 32 * z:STMT0 + 32 * z + 32]
            M = p.m_shared if p.space[s] == 0 else p.m_global
            assert st[0] == p.op[s] and st[1] == p.space[s] and st[2] == p.kind[s]
            want_b = (int(p.b[s]) % M + (int(p.iter_coef[s]) % M) * ctr) % M
            if p.kind[s] == 2:
                # a permutation instance reads its window, the table rotated to
                # start at its offset (which becomes 0)
                assert int(st[8:12].view(np.uint32)[0]) == 0
                off, need = int(st[16:20].view(np.uint32)[0]), int(st[28:32].view(np.uint32)[0])
                perm_off = int(arena[:128].view(np.uint64)[5])
                win = arena[perm_off + 2 * off:perm_off + 2 * (off + need)].view(np.uint16)
                idx = (want_b + np.arange(need)) % M
                assert np.array_equal(win, p.perm[int(p.perm_off[s]) + idx].astype(np.uint16))
            else:
                assert int(st[8:12].view(np.uint32)[0]) == want_b
            assert int(st[20:22].view(np.uint16)[0]) == p.guard_k[s]
            if z + 1 < len(order):
                k = order[z + 1][0] - 1
                assert int(d[GAPS0 + 4 * z:GAPS0 + 4 * z + 4].view(np.uint32)[0]) == 1 << k


def test_expansion_items_cover_every_segment_once(lib):
    """The packer's trace-expansion work items: runs of at most 64 (statement,
    block) segments of one program (kind 0), or block 0 of a program's
    shared-array statements when its blocks are alike (kind 1), together
    covering each segment a check reads exactly once; the general programs'
    items first (the repair path expands only those), each part larger
    programs first; the program order puts the relation kernel's programs
    (shared array only, blocks alike or one block) first."""
    import oracle
    from _tiny import random_loop_program, random_program

    progs = synth.generate("uneven4096_mixed", 30) + [random_loop_program(s, s_min=3, m_max=40) for s in range(10)]
    progs += [random_program(50 + s, s_min=2, s_max=6, b_min=2, b_max=5, c_max=3, shared_c=True) for s in range(20)]
    arena, _ = gb.pack(progs)
    h = arena[:128].view(np.uint64)
    segbase_off, items_off, n_items = int(h[4]), int(h[12]), int(h[13]) & 0xFFFFFFFF
    n = len(progs)
    segbase = arena[segbase_off:segbase_off + 8 * (n + 1)].view(np.uint64)
    items = arena[items_off:items_off + 16 * n_items].view(np.uint32).reshape(-1, 4)
    covered = [np.zeros(int(segbase[p + 1] - segbase[p]), np.int64) for p in range(n)]
    order = []
    for p, lo, hi, kind in items.tolist():
        B = progs[p].blocks
        if kind == 1:
            for x, (s, _) in enumerate(oracle.unroll(progs[p])):
                if lo <= x < hi and progs[p].space[s] == 0:
                    covered[p][x * B] += 1
        else:
            assert 0 < hi - lo <= 64
            covered[p][lo:hi] += 1
        if not order or order[-1] != p:
            order.append(p)
    alike_seen = 0
    for p in range(n):
        alike = int(_devprog(arena, p)[56:60].view(np.uint32)[0]) and progs[p].blocks > 1
        alike_seen += bool(alike)
        B = progs[p].blocks
        for x, (s, _) in enumerate(oracle.unroll(progs[p])):
            for b in range(B):
                need = not alike or progs[p].space[s] == 1 or b == 0
                assert covered[p][x * B + b] == (1 if need else 0), (p, x, b)
    assert alike_seen > 10
    assert sorted(order) == list(range(n))
    n_fast, n_items_gen = (int(x) for x in arena[120:128].view(np.uint32))
    fast = [int(_devprog(arena, p)[NEG0 + 4:NEG0 + 8].view(np.uint32)[0]) for p in range(n)]
    for p in range(n):
        alike = int(_devprog(arena, p)[56:60].view(np.uint32)[0])
        want = all(sp == 0 for sp in progs[p].space) and (alike or progs[p].blocks == 1)
        assert fast[p] == int(want), p
    assert n_fast == sum(fast) and 0 < n_fast < n
    gen_items = {int(x) for x in items[:n_items_gen, 0]}
    assert gen_items == {p for p in range(n) if not fast[p]}
    assert {int(x) for x in items[n_items_gen:, 0]} == {p for p in range(n) if fast[p]}
    def cost(p):
        # the packer's work estimate: block 0's accesses when the blocks are
        # alike, every block's otherwise, plus every block's global accesses
        B, tp = progs[p].blocks, (progs[p].threads + 7) // 8 * 8
        inst = [s for s, _ in oracle.unroll(progs[p])]
        alike = int(_devprog(arena, p)[56:60].view(np.uint32)[0])
        G = sum(int(progs[p].space[s]) == 1 for s in inst)
        return len(inst) * tp * (1 if alike else B) + (G * B * tp if B > 1 else 0)

    prog_order = arena[int(h[3]):int(h[3]) + 4 * n].view(np.uint32).tolist()
    k = n - n_fast
    costs = [cost(p) for p in prog_order]
    assert [fast[p] for p in prog_order] == [1] * n_fast + [0] * k
    assert costs[:n_fast] == sorted(costs[:n_fast], reverse=True)
    assert costs[n_fast:] == sorted(costs[n_fast:], reverse=True)
    # the expansion items: the general programs first, each part in program order
    assert order[:k] == prog_order[n_fast:] and order[k:] == prog_order[:n_fast]
    # the check items: the general programs in program order, one item each,
    # or one per range of blocks (at most 16, covering every block once) when
    # the blocks differ; the first range is the primary item
    ch = arena[128:192].view(np.uint32)
    citems_off, n_citems, n_split = int(arena[128:136].view(np.uint64)[0]), int(ch[2]), int(ch[3])
    citems = arena[citems_off:citems_off + 16 * n_citems].view(np.uint32).reshape(-1, 4).tolist()
    seen, at = [], 0
    for p in prog_order[n_fast:]:
        alike = int(_devprog(arena, p)[56:60].view(np.uint32)[0])
        B = progs[p].blocks
        K = 1 if alike else min(B, 16)
        mine = citems[at:at + K]
        at += K
        assert [c[0] for c in mine] == [p] * K
        assert mine[0][1] == 0 and mine[-1][2] == B
        assert all(a[2] == b[1] and a[1] < a[2] for a, b in zip(mine, mine[1:]))
        assert [c[3] for c in mine] == [1 | (2 if K > 1 else 0)] + [2] * (K - 1)
        seen.append(K > 1)
    assert at == n_citems and sum(seen) == n_split > 0


@pytest.mark.parametrize("negs,msg", [([0], "empty"), ([1 << 7], "beyond slot"), ([1] * 33, "negative clauses")])
def test_validation_rejects_bad_negative_clauses(lib, negs, msg):
    with pytest.raises(gb.GrError) as e:
        gb.validate(_prog(neg_clauses=tuple(negs)))
    assert e.value.code == gb.EINVAL and msg in str(e.value)


def test_packer_copies_negative_clauses(lib):
    progs = [_prog(neg_clauses=(3, 96)), _prog(), _prog(neg_clauses=(64,))]
    arena, _ = gb.pack(progs)
    for i, p in enumerate(progs):
        d = _devprog(arena, i)
        n = int(d[NEG0:NEG0 + 4].view(np.uint32)[0])
        assert n == len(p.neg_clauses)
        assert d[NEG0 + 16:NEG0 + 16 + 4 * n].view(np.uint32).tolist() == list(p.neg_clauses)


def test_packer_places_slots(lib):
    """Explicit slot places: the slots whose barriers run in each gap between
    executed instances."""
    import oracle
    from _tiny import random_loop_program, random_program, with_sites

    progs = [with_sites(random_program(s, s_min=3, s_max=8), s) for s in range(20)]
    progs += [with_sites(random_loop_program(100 + s, s_min=3, s_max=6), s) for s in range(20)]
    arena, _ = gb.pack(progs)
    for i, p in enumerate(progs):
        d = _devprog(arena, i)
        order = oracle.unroll(p)
        assert int(d[4:8].view(np.uint32)[0]) == p.n_slots
        assert int(d[60:64].view(np.uint32)[0]) == 1
        for z in range(len(order) - 1):
            place = order[z + 1][0] - 1
            want = sum(1 << k for k in range(p.n_slots) if int(p.slot_pos[k]) == place)
            assert int(d[GAPS0 + 4 * z:GAPS0 + 4 * z + 4].view(np.uint32)[0]) == want


def test_program_without_slots_takes_empty_places(lib):
    """A one-statement program laid out as sites has no slot and an empty
    place list: the binding gives no places and the program validates and
    packs."""
    from _tiny import random_program, with_sites

    p = with_sites(random_program(0, s_min=1, s_max=1), 0)
    assert p.n_stmts == 1 and len(p.slot_pos) == 0
    gb.validate(p)
    gb.pack([p, _prog()])


@pytest.mark.parametrize("pos,msg", [([0, 7], "place"), ([0] * 33, "more than 32 slots")])
def test_validation_rejects_bad_places(lib, pos, msg):
    p = _prog()
    n = len(pos)
    p.slot_pos = np.array(pos, np.uint32)
    p.slot_level = np.zeros(n, np.uint8)
    p.slot_guard_k = np.zeros(n, np.uint16)
    p.slot_guard_r = np.zeros(n, np.uint16)
    p.slot_weight = np.ones(n, np.uint32)
    p.existing_mask = 0
    with pytest.raises(gb.GrError) as e:
        gb.validate(p)
    assert e.value.code == gb.EINVAL and msg in str(e.value)


def test_block_invariance_flag_is_sound(lib):
    """The packer marks a program block-invariant only when, for every pair of
    statements of one array and every pair of threads, two addresses agree in
    block b exactly when they agree in block 0 (so block 0's same-block
    witnesses are every block's)."""
    from _tiny import random_program

    flagged = 0
    progs = [random_program(s, s_min=2, s_max=5, b_min=2, b_max=4, t_max=6, m_max=12, c_max=3) for s in range(300)]
    arena, _ = gb.pack(progs)
    for i, p in enumerate(progs):
        inv = int(_devprog(arena, i)[56:60].view(np.uint32)[0])
        if not inv:
            continue
        flagged += 1
        def addr(s, t, b):
            M = p.m_shared if p.space[s] == 0 else p.m_global
            if p.kind[s] == 2:
                return int(p.perm[int(p.perm_off[s]) + (t + int(p.c[s]) * b + int(p.b[s])) % M])
            return (int(p.a[s]) * t + int(p.c[s]) * b + int(p.b[s])) % M
        for s1 in range(p.n_stmts):
            for s2 in range(p.n_stmts):
                if p.space[s1] != p.space[s2]:
                    continue
                for b in range(1, p.blocks):
                    for t1 in range(p.threads):
                        for t2 in range(p.threads):
                            assert (addr(s1, t1, b) == addr(s2, t2, b)) == (addr(s1, t1, 0) == addr(s2, t2, 0))
    assert flagged >= 50
