"""Edge cases of the CUDA path against the oracle (or, where the oracle's
enumeration is too slow, against results fixed by reasoning): degenerate
programs, the largest sizes the ABI allows."""
import numpy as np
import pytest

import oracle
from _tiny import random_program
from paper_2011_08373_gb300 import synth

pytestmark = pytest.mark.gpu

KEYS = ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses", "forbidden",
        "access_pairs")


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


def _same(g, w):
    for k in KEYS:
        assert g[k] == w[k], (k, g[k], w[k])


def test_degenerate_programs(gb):
    """One statement (no slot), one thread, one block, one-word arrays."""
    progs = [
        synth.make_program([{"op": "W"}], blocks=1, threads=1, m_shared=1),
        synth.make_program([{"op": "W", "a": 0}], blocks=1, threads=5, m_shared=1),  # self race, no slot
        synth.make_program([{"op": "R"}, {"op": "W"}], blocks=1, threads=1, m_shared=1),
        synth.make_program([{"op": "W", "space": "global", "a": 0}, {"op": "R", "space": "global"}],
                           blocks=3, threads=1, m_global=1),
        synth.make_program([{"op": "R", "a": 0}, {"op": "R", "a": 0}], blocks=2, threads=7, m_shared=1),
    ]
    progs += [random_program(97000 + s, s_max=2, b_max=2, t_max=2, m_max=2) for s in range(60)]
    for fn in (gb.repair_batch, lambda ps: [gb.repair(p) for p in ps], lambda ps: [gb.repair_plain(p) for p in ps]):
        for p, g in zip(progs, fn(progs)):
            _same(g, oracle.repair(p))
    assert gb.repair(progs[1])["status"] == 1


def test_largest_statement_count(gb):
    """25 statements and 24 slots, 1,024 threads, 4,096-word shared array."""
    progs = synth.generate("batch1024_4x256_s24", 3, n_stmts=25, blocks=1, threads=1024, m_words=4096)
    assert all(p.n_stmts == 25 and p.n_slots == 24 for p in progs)
    got = gb.repair_batch(progs)
    want = oracle.repair_batch(progs, n_threads=8)
    for g, w in zip(got, want):
        _same(g, w)


def test_largest_address_space(gb):
    """65,536-word arrays: addresses up to 65,535 in the u16 traces."""
    p = synth.make_program([{"op": "W", "space": "global", "a": 1, "b": 65535 - 63},
                            {"op": "R", "space": "global", "a": 1, "b": 65535 - 62},
                            {"op": "W", "a": 2, "b": 65534}, {"op": "R", "a": 2, "b": 0}],
                           blocks=2, threads=64, m_global=65536, m_shared=65536)
    for g, w in zip(gb.repair_batch([p]), [oracle.repair(p)]):
        _same(g, w)
    assert gb.check(p, 0) == oracle.check(p, 0)


def test_most_blocks(gb):
    """65,533 blocks of one thread (the owner tables hold block indices up to
    65,532): block b writes word b and reads word b+1, which block b+1 writes,
    so the one race is cross-block and only a grid barrier between the two
    statements fixes it."""
    B = 65533
    p = synth.make_program([{"op": "R", "space": "global", "a": 0, "c": 1, "b": 1},
                            {"op": "W", "space": "global", "a": 0, "c": 1, "b": 0}],
                           blocks=B, threads=1, m_global=65536, slot_level=[1], slot_weight=[13])
    w = gb.check(p, 0)
    assert w["intra"] == [0, 0] and w["inter"] == [2, 0] and w["diverge"] == 0
    # ordered pairs (read block b1, write block b2 != b1) plus unordered write pairs
    assert w["access_pairs"] == B * (B - 1) + B * (B - 1) // 2
    r = gb.repair(p)
    assert (r["status"], r["mask"], r["weight"], r["traj"], r["clauses"]) == (0, 1, 13, [0, 1], [1])
    assert gb.repair(p, grid_enabled=False)["status"] == 1


def test_thirty_two_slots(gb):
    """32 barrier variables (a block and a grid candidate at 16 sites): the
    final repair is the lowest-key mask over the oracle's unconstrained
    witnesses, found by integer programming (path independence)."""
    pytest.importorskip("scipy.optimize")
    from test_oracle_pins import milp_lowest_key

    progs = synth.generate("sites128_16x256_s16", 6, n_stmts=17, blocks=2, threads=16, m_words=512)
    assert all(p.n_slots == 32 for p in progs)
    for p, g in zip(progs, gb.repair_batch(progs)):
        w0 = oracle.check(p, 0)
        assert gb.check(p, 0) == w0
        cls = oracle.clauses(p, w0)
        div = oracle.check(p, 0xFFFFFFFF)["diverge"]
        want = milp_lowest_key(32, [int(x) for x in p.slot_weight], cls, (), 0, div)
        if want is None:
            assert g["status"] == 1
        else:
            assert g["status"] == 0 and (g["mask"], g["weight"]) == want


def test_many_blocks_that_differ(gb):
    """More than 64 blocks whose access patterns differ (the check walks every
    block and reads their chunk masks one block at a time), on the persistent
    launch, the plain path and the wide lane."""
    import torch

    progs = []
    for s in range(6):
        p = random_program(98000 + s, s_min=3, s_max=5, b_min=1, b_max=1, t_min=3, t_max=4, m_max=3000,
                           c_max=9, a_max=3, spaces=(1,))
        p.blocks = 70 + s
        p.c[0] = p.c[0] + 1  # blocks differ
        progs.append(p)
    want = oracle.repair_batch(progs, n_threads=4)
    assert sum(w["status"] == 0 for w in want) >= 3
    for p, g, w in zip(progs, gb.repair_batch(progs), want):
        _same(g, w)
        assert gb.check(p, 0) == oracle.check(p, 0)
    _same(gb.repair_plain(progs[0]), want[0])
    timed, loop_ms = gb.repair_plain_timed(progs[1])
    _same(timed, want[1])
    assert loop_ms > 0.0
    db = gb.DeviceBatch(progs)
    db.run_wide()
    torch.cuda.synchronize()
    for g, w in zip(db.results(), want):
        _same(g, w)


def test_clause_of_all_slots(gb):
    """A clause holding all 32 slots (every bit set) among more than 128
    clauses: 25 statements that all write one shared word, so every pair of
    statements races and pair (0, 24) is separated by every slot; the empty
    clause of each statement's self race makes the program unrepairable after
    the first check."""
    pos = [g for g in range(24) for _ in range(2 if g < 8 else 1)]
    level = [1 if (g < 8 and k == 1) else 0 for g in range(24) for k in range(2 if g < 8 else 1)]
    p = synth.make_program([{"op": "W", "a": 0, "b": 0}] * 25, blocks=1, threads=4, m_shared=1,
                           slot_pos=pos, slot_level=level, slot_weight=[1] * 32)
    assert p.n_slots == 32
    w0 = oracle.check(p, 0)
    cls = oracle.clauses(p, w0)
    assert len(cls) == 301 and cls[0] == 0 and cls[-1] == 0xFFFFFFFF
    for strategy in (0, 1):
        for g in (gb.repair_batch([p], strategy=strategy)[0], gb.repair_plain(p, strategy=strategy)):
            assert (g["status"], g["iters"], g["traj"]) == (1, 1, [0])
            assert g["clauses"] == cls


def test_launch_checks_n_and_scratch_against_the_arena(gb):
    """A device-resident repair given a program count or a scratch size that
    does not match its packed arena does no work: every kernel compares them
    with the arena header first, leaves the results untouched and sets the
    argument bit (4) of the device error word (scratch word 1).  A matching
    call afterwards repairs the batch as usual."""
    import ctypes as C

    import torch

    progs = synth.generate("batch1024_4x256_s24", 6, blocks=2, threads=32, n_stmts=8, m_words=128)
    progs += [synth.generate("interblock256_64x256_s16", 1, blocks=3, threads=32, n_stmts=5, m_words=512)[0]]
    db = gb.DeviceBatch(progs)
    n = len(progs)
    lib = gb.lib()
    scratch_words = db.scratch.view(torch.uint8)
    base = db._scratch_ptr - db.scratch.data_ptr()

    def call(n_arg, scratch_bytes):
        db.out.view(torch.uint8).fill_(0xA5)
        scratch_words[base:base + 256].zero_()
        gb._check(lib.gr_repair_packed(C.c_void_p(db._arena_ptr), n_arg, None, C.c_void_p(db._scratch_ptr),
                                       C.c_uint64(scratch_bytes), C.c_void_p(db._out_ptr), None))
        torch.cuda.synchronize()
        err = int(scratch_words[base + 4:base + 8].cpu().numpy().view(np.uint32)[0])
        untouched = bool((db.out.view(torch.uint8) == 0xA5).all())
        return err, untouched

    for n_arg, sb in ((n - 1, db.scratch_bytes), (n, db.scratch_bytes - 256)):
        err, untouched = call(n_arg, sb)
        assert err & 4 and untouched, (n_arg, sb, err)
    err, untouched = call(n, db.scratch_bytes)
    assert err == 0 and not untouched
    want = oracle.repair_batch(progs, n_threads=4)
    for g, w in zip(db.results(), want):
        _same(g, w)


def test_one_launch_equals_the_two_kernels(gb):
    """gr_relation_loop_packed (the relation kernel running the loop too, each
    program's loop waiting on its relation's flag) writes the results the
    oracle gives on a small batch, and the two-kernel repair's results on the
    1,024-program batch of 4 x 256 threads and 24 statements and on the
    4,096-program uneven batch; the device error word stays 0.  A batch with
    a program that needs expanded traces is refused with nothing launched."""
    import ctypes as C

    import torch

    def err_word(db):
        base = db._scratch_ptr - db.scratch.data_ptr()
        return int(db.scratch.view(torch.uint8)[base + 4:base + 8].cpu().numpy().view(np.uint32)[0])

    small = synth.generate("batch1024_4x256_s24", 40, blocks=2, threads=32, n_stmts=8, m_words=128)
    db = gb.DeviceBatch(small)
    assert db.simple and not db.has_general
    db.relation_loop()
    torch.cuda.synchronize()
    assert err_word(db) == 0
    for g, w in zip(db.results(), oracle.repair_batch(small, n_threads=4)):
        _same(g, w)

    for name in ("batch1024_4x256_s24", "uneven4096_mixed"):
        full = synth.generate(name)
        db = gb.DeviceBatch(full)
        db.tune()
        db.relation()
        db.loop()
        torch.cuda.synchronize()
        two = db.results_raw().copy()
        db.out.view(torch.uint8).fill_(0xA5)
        db.relation_loop()
        torch.cuda.synchronize()
        assert err_word(db) == 0
        one = db.results_raw()
        for k in one.dtype.names:
            if k not in ("_pad", "t_start_ns", "t_end_ns"):
                assert np.array_equal(one[k], two[k]), (name, k)

    general = small[:3] + synth.generate("interblock256_64x256_s16", 1, blocks=3, threads=32, n_stmts=5,
                                         m_words=512)
    db = gb.DeviceBatch(general)
    assert db.has_general
    db.out.view(torch.uint8).fill_(0xA5)
    with pytest.raises(gb.GrError):
        db.relation_loop()
    torch.cuda.synchronize()
    assert bool((db.out.view(torch.uint8) == 0xA5).all())


def test_a_recorded_shape_word_replaces_the_autotuner(gb):
    """gr_set_shape_packed: the word gr_tune_packed returned (never with the
    one-launch bit), set on a fresh arena of the same batch, gives the tuned
    batch's results; so does that word with the one-launch bit added, on a
    batch that allows it.  Words that name no
    built shape, and the one-launch bit on a batch with a general program,
    are refused."""
    import torch

    progs = synth.generate("batch1024_4x256_s24", 24, blocks=2, threads=32, n_stmts=8, m_words=128)
    want = oracle.repair_batch(progs, n_threads=4)
    a = gb.DeviceBatch(progs)
    word = a.tune()
    assert not word >> 16  # the autotuner keeps two launches
    for w in (word, word | (1 << 16)):
        b = gb.DeviceBatch(progs)
        assert b.set_shape(w) == w
        b.run()
        torch.cuda.synchronize()
        for g, x in zip(b.results(), want):
            _same(g, x)
    b = gb.DeviceBatch(progs)
    for bad in (6, 5 << 8, 0x20 << 8, 1 << 17):
        with pytest.raises(gb.GrError):
            b.set_shape(bad)
    general = progs[:2] + synth.generate("interblock256_64x256_s16", 1, blocks=3, threads=32, n_stmts=5,
                                         m_words=512)
    with pytest.raises(gb.GrError):
        gb.DeviceBatch(general).set_shape(1 << 16)
