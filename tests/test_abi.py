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
