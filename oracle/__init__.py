"""CPU oracle for the barrier-repair loop (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import this package.  The product path never does.  It
shares no code with the CUDA engine: it compiles ``oracle.c`` (plain C) with
gcc on first use and calls it through ctypes.

Functions take duck-typed programs (any object with the attributes of
``paper_2011_08373_gb300.synth.Program``) and return plain Python values.

Parity status: every C function is pinned by ``tests/test_oracle_pins.py``
(paper listings, the Section 2.4 mhs counterexample, an independent flag-reset
race detector, a closed form for affine maps, interval-stabbing DP, scipy
MILP, invariants, the path-independence lemma).  The synthetic workload
distributions themselves are free choices and carry no pin.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_TRAJ = 64
MAX_CLAUSES = 656
MAX_STMTS = 25


def _check_loops(loops, S):
    """Loops must be counted ranges lo..hi (1 <= lo <= hi < S, trips >= 1),
    pairwise nested or disjoint, a nested loop starting strictly after its
    parent (so that every loop has its own head slot)."""
    for lo, hi, trips in loops:
        if not (1 <= lo <= hi < S) or trips < 1:
            raise ValueError(f"bad loop {(lo, hi, trips)} for {S} statements")
    for x, (lo1, hi1, _) in enumerate(loops):
        for lo2, hi2, _ in loops[x + 1:]:
            disjoint = hi1 < lo2 or hi2 < lo1
            nested = (lo1 < lo2 and hi2 <= hi1) or (lo2 < lo1 and hi1 <= hi2)
            if not (disjoint or nested):
                raise ValueError("loops must be nested (starting strictly inside) or disjoint")


def unroll_count(prog_struct) -> int:
    st = (C.c_uint32 * MAX_STMTS)()
    it = (C.c_uint32 * MAX_STMTS)()
    return int(_load().orc_unroll(C.byref(prog_struct), st, it))


def unroll(p):
    """The executed statement instances of p in order: (statement, counter of
    its innermost loop) pairs."""
    m = _Marshalled(p)
    st = (C.c_uint32 * MAX_STMTS)()
    it = (C.c_uint32 * MAX_STMTS)()
    n = int(_load().orc_unroll(C.byref(m.s), st, it))
    return [(st[x], it[x]) for x in range(n)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, plain -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Prog(C.Structure):
    _fields_ = [
        ("n_stmts", C.c_uint32),
        ("op", C.c_void_p), ("space", C.c_void_p), ("kind", C.c_void_p),
        ("a", C.c_void_p), ("b", C.c_void_p), ("c", C.c_void_p), ("perm_off", C.c_void_p),
        ("guard_k", C.c_void_p), ("guard_r", C.c_void_p),
        ("slot_level", C.c_void_p),
        ("slot_guard_k", C.c_void_p), ("slot_guard_r", C.c_void_p),
        ("slot_weight", C.c_void_p),
        ("m_shared", C.c_uint32), ("m_global", C.c_uint32),
        ("perm", C.c_void_p), ("perm_len", C.c_uint32),
        ("existing_mask", C.c_uint32),
        ("blocks", C.c_uint32), ("threads", C.c_uint32),
        ("n_loops", C.c_uint32),
        ("loop_lo", C.c_void_p), ("loop_hi", C.c_void_p), ("loop_trips", C.c_void_p),
        ("iter_coef", C.c_void_p),
        ("n_neg", C.c_uint32), ("neg", C.c_void_p),
        ("n_slots", C.c_uint32), ("slot_pos", C.c_void_p),
    ]


class _Witness(C.Structure):
    _fields_ = [("intra", C.c_uint32 * 32), ("inter", C.c_uint32 * 32),
                ("diverge", C.c_uint32), ("access_pairs", C.c_uint64)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("mask", C.c_uint32), ("weight", C.c_uint32),
                ("added", C.c_uint32), ("removed", C.c_uint32), ("iters", C.c_uint32),
                ("traj", C.c_uint32 * MAX_TRAJ), ("n_clauses", C.c_uint32),
                ("clauses", C.c_uint32 * MAX_CLAUSES), ("forbidden", C.c_uint32),
                ("access_pairs", C.c_uint64)]


def _configure(path):
    lib = C.CDLL(path)
    lib.orc_check.argtypes = [C.POINTER(_Prog), C.c_uint32, C.POINTER(_Witness)]
    lib.orc_check.restype = None
    lib.orc_check_words.argtypes = lib.orc_check.argtypes
    lib.orc_check_words.restype = None
    lib.orc_clauses.argtypes = [C.POINTER(_Prog), C.POINTER(_Witness),
                                C.POINTER(C.c_uint32), C.c_uint32]
    lib.orc_clauses.restype = C.c_uint32
    lib.orc_solve.argtypes = [C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                              C.c_uint32, C.POINTER(C.c_uint32), C.c_uint32, C.c_uint32,
                              C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)]
    lib.orc_solve.restype = C.c_int
    lib.orc_repair.argtypes = [C.POINTER(_Prog), C.c_int, C.c_int, C.c_uint32, C.c_int,
                               C.POINTER(_Result)]
    lib.orc_greedy.argtypes = [C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.c_uint32,
                               C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32)]
    lib.orc_greedy.restype = C.c_int
    lib.orc_repair.restype = None
    lib.orc_repair_batch.argtypes = [C.POINTER(_Prog), C.POINTER(C.c_int32), C.c_uint32,
                                     C.c_int, C.c_uint32, C.c_int, C.POINTER(_Result), C.c_uint32]
    lib.orc_repair_batch.restype = None
    lib.orc_repair_words.argtypes = lib.orc_repair.argtypes
    lib.orc_repair_words.restype = None
    lib.orc_repair_batch_words.argtypes = lib.orc_repair_batch.argtypes
    lib.orc_repair_batch_words.restype = None
    lib.orc_check_pair.argtypes = [C.POINTER(_Prog), C.c_uint32, C.c_uint32, C.c_uint32,
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_uint64)]
    lib.orc_check_pair.restype = None
    lib.orc_unroll.argtypes = [C.POINTER(_Prog), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    lib.orc_unroll.restype = C.c_uint32
    assert lib.orc_sizeof_result() == C.sizeof(_Result)
    assert lib.orc_sizeof_prog() == C.sizeof(_Prog)
    assert lib.orc_sizeof_witness() == C.sizeof(_Witness)
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(build())
    return _lib


class using_library:
    """Temporarily route every call through another build of oracle.c (the
    mutation tests use it to show that the pins reject planted mistakes)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _load()
        _lib = _configure(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _u32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint32))


def _u8(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8))


class _Marshalled:
    """Keeps the numpy buffers of one program alive while C reads them."""

    def __init__(self, p):
        n = len(p.slot_level)
        self.keep = [
            _u8(p.op), _u8(p.space), _u8(p.kind), _u32(p.a), _u32(p.b), _u32(p.c),
            _u32(p.perm_off), _u32(p.guard_k), _u32(p.guard_r), _u8(p.slot_level),
            _u32(p.slot_guard_k), _u32(p.slot_guard_r), _u32(p.slot_weight),
            _u32(p.perm) if len(p.perm) else np.zeros(1, np.uint32),
        ]
        pos = getattr(p, "slot_pos", None)
        if pos is None:
            assert n == p.op.shape[0] - 1
        loops = list(getattr(p, "loops", ()) or ())
        _check_loops(loops, p.op.shape[0])
        coef = getattr(p, "iter_coef", None)
        self.keep += [_u32([l[0] for l in loops] or [0]), _u32([l[1] for l in loops] or [0]),
                      _u32([l[2] for l in loops] or [0]),
                      _u32(coef) if coef is not None else np.zeros(p.op.shape[0], np.uint32)]
        negs = [int(x) for x in (getattr(p, "neg_clauses", ()) or ())]
        self.keep.append(_u32(negs or [0]))
        self.keep.append(_u32(pos) if pos is not None else np.zeros(1, np.uint32))
        k = self.keep
        ptr = lambda arr: arr.ctypes.data
        self.s = _Prog(p.op.shape[0], ptr(k[0]), ptr(k[1]), ptr(k[2]), ptr(k[3]), ptr(k[4]),
                       ptr(k[5]), ptr(k[6]), ptr(k[7]), ptr(k[8]), ptr(k[9]), ptr(k[10]),
                       ptr(k[11]), ptr(k[12]), int(p.m_shared), int(p.m_global), ptr(k[13]),
                       len(p.perm), int(p.existing_mask), int(p.blocks), int(p.threads),
                       len(loops), ptr(k[14]), ptr(k[15]), ptr(k[16]), ptr(k[17]),
                       len(negs), ptr(k[18]), n, ptr(k[19]) if pos is not None else 0)
        self.n_exec = unroll_count(self.s) if loops else p.op.shape[0]
        if self.n_exec > MAX_STMTS:
            raise ValueError(f"{self.n_exec} executed statement instances (at most {MAX_STMTS})")


def check(p, mask: int, words: bool = False) -> dict:
    """Witnesses of program ``p`` under barrier mask ``mask``; rows index the
    executed statement instances (the statements themselves without loops).
    words=True: the same definition grouped by word (orc_check_words), for
    launches whose thread-pair enumeration is too slow."""
    lib = _load()
    m = _Marshalled(p)
    w = _Witness()
    (lib.orc_check_words if words else lib.orc_check)(C.byref(m.s), mask, C.byref(w))
    S = m.n_exec
    return {"intra": [w.intra[i] for i in range(S)], "inter": [w.inter[i] for i in range(S)],
            "diverge": w.diverge, "access_pairs": w.access_pairs}


def check_pair(p, mask: int, i: int, j: int) -> tuple:
    """(same-block witness, cross-block witness, thread pairs examined) for
    executed instances i <= j under ``mask``: the check's definition on one
    pair."""
    lib = _load()
    m = _Marshalled(p)
    a, b, n = C.c_int32(), C.c_int32(), C.c_uint64()
    lib.orc_check_pair(C.byref(m.s), mask, i, j, C.byref(a), C.byref(b), C.byref(n))
    return bool(a.value), bool(b.value), n.value


def clauses(p, witness: dict) -> list:
    """Sorted unique clause masks generated by one check's witnesses."""
    lib = _load()
    m = _Marshalled(p)
    w = _Witness()
    for i, v in enumerate(witness["intra"]):
        w.intra[i] = v
    for i, v in enumerate(witness["inter"]):
        w.inter[i] = v
    w.diverge = witness["diverge"]
    buf = (C.c_uint32 * (2 * 32 * 32))()
    n = lib.orc_clauses(C.byref(m.s), C.byref(w), buf, 0)
    return [buf[i] for i in range(n)]


def solve(n_vars: int, weights, pos, neg=(), forced: int = 0, forbidden: int = 0):
    """Lowest (weight, mask) hitting set, or None if unsatisfiable."""
    lib = _load()
    w = (C.c_uint32 * max(1, n_vars))(*[int(x) for x in weights])
    pa = (C.c_uint32 * max(1, len(pos)))(*[int(x) for x in pos])
    na = (C.c_uint32 * max(1, len(neg)))(*[int(x) for x in neg])
    mask = C.c_uint32()
    wt = C.c_uint64()
    rc = lib.orc_solve(n_vars, w, pa, len(pos), na, len(neg), forced, forbidden,
                       C.byref(mask), C.byref(wt))
    if rc:
        return None
    return mask.value, wt.value


def _result_dict(r: _Result) -> dict:
    return {"status": r.status, "mask": r.mask, "weight": r.weight, "added": r.added,
            "removed": r.removed, "iters": r.iters,
            "traj": [r.traj[i] for i in range(min(r.iters, MAX_TRAJ))],
            "clauses": [r.clauses[i] for i in range(r.n_clauses)], "forbidden": r.forbidden,
            "access_pairs": r.access_pairs}


def greedy(n_vars: int, weights, pos, forced: int = 0, forbidden: int = 0):
    """The mhs strategy's greedy minimal hitting set, or None if infeasible."""
    lib = _load()
    w = (C.c_uint32 * max(1, n_vars))(*[int(x) for x in weights])
    pa = (C.c_uint32 * max(1, len(pos)))(*[int(x) for x in pos])
    mask = C.c_uint32()
    if lib.orc_greedy(n_vars, w, pa, len(pos), forced, forbidden, C.byref(mask)):
        return None
    return mask.value


def repair(p, mode=None, grid_enabled: bool = True, max_iters: int = 64, strategy: int = 0,
           words: bool = False) -> dict:
    """Algorithm 1 on one program (mode defaults to ``p.mode``); strategy 0 =
    MaxSAT proposals, 1 = the mhs strategy; words=True verifies with the
    word-grouped check."""
    lib = _load()
    m = _Marshalled(p)
    r = _Result()
    (lib.orc_repair_words if words else lib.orc_repair)(C.byref(m.s), int(p.mode if mode is None else mode),
                                                        int(grid_enabled), max_iters, strategy, C.byref(r))
    return _result_dict(r)


def repair_batch(progs, grid_enabled: bool = True, max_iters: int = 64,
                 n_threads: int = 1, strategy: int = 0, words: bool = False) -> list:
    """Algorithm 1 on many programs, spread over ``n_threads`` CPU threads
    (words=True: Verify by the word-grouped check)."""
    lib = _load()
    ms = [_Marshalled(p) for p in progs]
    arr = (_Prog * len(progs))(*[m.s for m in ms])
    modes = (C.c_int32 * len(progs))(*[int(p.mode) for p in progs])
    out = (_Result * len(progs))()
    fn = lib.orc_repair_batch_words if words else lib.orc_repair_batch
    fn(arr, modes, len(progs), int(grid_enabled), max_iters, strategy, out, n_threads)
    return [_result_dict(out[i]) for i in range(len(progs))]
