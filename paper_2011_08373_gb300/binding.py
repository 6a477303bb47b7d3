"""ctypes binding of libgpurepair.so (include/gpurepair.h).

Argument marshalling only: every step of the repair path runs in the
library's CUDA kernels.  The library must have been built (``build()`` in
``paper_2011_08373_gb300.build``); loading raises if it is missing.  Names
follow the C entry points without the ``gr_`` prefix.  Device memory and
streams for the device-resident calls come from PyTorch.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpurepair.so")

MAX_STMTS, MAX_SLOTS, MAX_ITERS, MAX_CLAUSES = 25, 32, 64, 656
OK, UNSAT, EINVAL, ENOMEM, ECUDA, EBUSY, ECAPACITY = 0, 1, -1, -2, -4, -5, -6
REPAIRED, UNREPAIRABLE, ITER_CAP, TIMEOUT = 0, 1, 2, 3


class GrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gpurepair error {code}: {msg}")
        self.code = code


class gr_stmt(C.Structure):
    _fields_ = [("op", C.c_uint8), ("space", C.c_uint8), ("kind", C.c_uint8), ("_pad", C.c_uint8),
                ("a", C.c_uint32), ("b", C.c_uint32), ("c", C.c_uint32), ("perm_off", C.c_uint32),
                ("guard_k", C.c_uint16), ("guard_r", C.c_uint16)]


class gr_loop(C.Structure):
    _fields_ = [("lo", C.c_uint32), ("hi", C.c_uint32), ("trips", C.c_uint32)]


class gr_program(C.Structure):
    _fields_ = [("n_stmts", C.c_uint32), ("stmts", C.POINTER(gr_stmt)),
                ("slot_level", C.POINTER(C.c_uint8)), ("slot_guard", C.POINTER(C.c_uint16)),
                ("slot_weight", C.POINTER(C.c_uint32)), ("m_shared", C.c_uint32),
                ("m_global", C.c_uint32), ("perm", C.POINTER(C.c_uint32)), ("perm_len", C.c_uint32),
                ("existing_mask", C.c_uint32), ("n_loops", C.c_uint32),
                ("loops", C.POINTER(gr_loop)), ("iter_coef", C.POINTER(C.c_uint32)),
                ("n_slots", C.c_uint32), ("slot_pos", C.POINTER(C.c_uint8)),
                ("n_neg", C.c_uint32), ("neg", C.POINTER(C.c_uint32))]


class gr_launch(C.Structure):
    _fields_ = [("blocks", C.c_uint32), ("threads", C.c_uint32)]


class gr_witnesses(C.Structure):
    _fields_ = [("race_intra", C.c_uint32 * 32), ("race_inter", C.c_uint32 * 32),
                ("diverge", C.c_uint32), ("n_stmts", C.c_uint32), ("access_pairs", C.c_uint64)]


class gr_options(C.Structure):
    _fields_ = [("grid_enabled", C.c_uint8), ("strategy", C.c_uint8), ("_pad", C.c_uint8 * 2),
                ("max_iters", C.c_uint32), ("deadline_us", C.c_uint64)]


class gr_repair_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("mask", C.c_uint32), ("weight", C.c_uint32),
                ("added", C.c_uint32), ("removed", C.c_uint32), ("iters", C.c_uint32),
                ("traj", C.c_uint32 * MAX_ITERS), ("n_clauses", C.c_uint32),
                ("clauses", C.c_uint32 * MAX_CLAUSES), ("forbidden", C.c_uint32), ("_pad", C.c_uint32),
                ("access_pairs", C.c_uint64), ("t_start_ns", C.c_uint64), ("t_end_ns", C.c_uint64)]


RESULT_DTYPE = np.dtype(gr_repair_result)
WITNESS_DTYPE = np.dtype(gr_witnesses)

_lock = threading.Lock()
_lib = None

EXPORTS = ["gr_version", "gr_last_error", "gr_validate", "gr_check", "gr_repair", "gr_repair_plain",
           "gr_solve", "gr_repair_batch", "gr_check_batch", "gr_pack_size", "gr_pack",
           "gr_repair_packed", "gr_check_packed", "gr_expand_packed", "gr_repair_expanded",
           "gr_repair_packed_noalloc", "gr_server_create", "gr_server_submit", "gr_server_poll",
           "gr_server_drain", "gr_server_stats", "gr_server_destroy", "gr_tune_packed",
           "gr_repair_packed_wide", "gr_check_expanded", "gr_relation_packed", "gr_loop_packed",
           "gr_repair_plain_timed", "gr_relation_loop_packed", "gr_set_shape_packed"]


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2011_08373_gb300.build` (nvcc, sm_103a)")
            L = C.CDLL(LIB_PATH)
            P = C.POINTER
            L.gr_version.restype = C.c_char_p
            L.gr_last_error.restype = C.c_char_p
            L.gr_validate.argtypes = [P(gr_program), gr_launch]
            L.gr_check.argtypes = [P(gr_program), gr_launch, C.c_uint32, P(gr_witnesses)]
            L.gr_repair.argtypes = [P(gr_program), gr_launch, C.c_int32, P(gr_options),
                                    P(gr_repair_result)]
            L.gr_repair_plain.argtypes = L.gr_repair.argtypes
            L.gr_repair_plain_timed.argtypes = L.gr_repair.argtypes + [P(C.c_float)]
            L.gr_solve.argtypes = [C.c_uint32, P(C.c_uint32), P(C.c_uint32), C.c_uint32, P(C.c_uint32),
                                   C.c_uint32, C.c_uint32, C.c_uint32, P(C.c_uint32), P(C.c_uint32)]
            L.gr_repair_batch.argtypes = [P(gr_program), P(gr_launch), P(C.c_int32), C.c_uint32,
                                          P(gr_options), C.c_void_p, C.c_void_p]
            L.gr_check_batch.argtypes = [P(gr_program), P(gr_launch), P(C.c_uint32), C.c_uint32,
                                         C.c_void_p, C.c_void_p]
            L.gr_pack_size.argtypes = [P(gr_program), P(gr_launch), C.c_uint32, P(C.c_uint64),
                                       P(C.c_uint64)]
            L.gr_pack.argtypes = [P(gr_program), P(gr_launch), P(C.c_int32), C.c_uint32, C.c_void_p,
                                  C.c_uint64]
            L.gr_repair_packed.argtypes = [C.c_void_p, C.c_uint32, P(gr_options), C.c_void_p,
                                           C.c_uint64, C.c_void_p, C.c_void_p]
            L.gr_expand_packed.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p]
            L.gr_repair_packed_wide.argtypes = L.gr_repair_packed.argtypes
            L.gr_repair_expanded.argtypes = L.gr_repair_packed.argtypes
            L.gr_repair_packed_noalloc.argtypes = [C.c_void_p, C.c_uint32, P(gr_options), C.c_void_p,
                                                   C.c_void_p]
            L.gr_server_create.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, P(gr_options),
                                           P(C.c_void_p)]
            L.gr_server_submit.argtypes = [C.c_void_p, P(gr_program), gr_launch, C.c_int32,
                                           P(C.c_uint64)]
            L.gr_server_poll.argtypes = [C.c_void_p, C.c_uint64, P(gr_repair_result), P(C.c_uint64)]
            L.gr_server_drain.argtypes = [C.c_void_p, C.c_uint32]
            L.gr_server_stats.argtypes = [C.c_void_p, P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
            L.gr_server_destroy.argtypes = [C.c_void_p]
            L.gr_tune_packed.argtypes = [C.c_void_p, C.c_uint32, P(gr_options), C.c_void_p, C.c_uint64,
                                         C.c_void_p, C.c_void_p, P(C.c_uint32)]
            L.gr_check_packed.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_uint64,
                                          C.c_void_p, C.c_void_p]
            L.gr_check_expanded.argtypes = L.gr_check_packed.argtypes
            L.gr_relation_packed.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint64, C.c_void_p]
            L.gr_loop_packed.argtypes = L.gr_repair_packed.argtypes
            L.gr_relation_loop_packed.argtypes = L.gr_repair_packed.argtypes
            L.gr_set_shape_packed.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p]
            for name in EXPORTS[2:]:
                getattr(L, name).restype = C.c_int32
            _lib = L
    return _lib


def version() -> str:
    return lib().gr_version().decode()


def last_error() -> str:
    return lib().gr_last_error().decode()


def _check(code: int, allowed=(OK,)) -> int:
    if code not in allowed:
        raise GrError(code, last_error())
    return code


# ---------------------------------------------------------------------------
# Program marshalling
# ---------------------------------------------------------------------------

class CProgram:
    """A Program marshalled into C structs (keeps its buffers alive)."""

    def __init__(self, p):
        S = int(p.op.shape[0])
        n = int(len(p.slot_level))
        st = (gr_stmt * S)()
        for s in range(S):
            st[s].op, st[s].space, st[s].kind = int(p.op[s]), int(p.space[s]), int(p.kind[s])
            st[s].a, st[s].b, st[s].c = int(p.a[s]), int(p.b[s]), int(p.c[s])
            st[s].perm_off = int(p.perm_off[s])
            st[s].guard_k, st[s].guard_r = int(p.guard_k[s]), int(p.guard_r[s])
        self.stmts = st
        self.level = np.ascontiguousarray(p.slot_level, dtype=np.uint8)
        sg = np.zeros(2 * max(n, 1), np.uint16)
        sg[0:2 * n:2] = p.slot_guard_k
        sg[1:2 * n:2] = p.slot_guard_r
        self.guard = sg
        self.weight = np.ascontiguousarray(p.slot_weight, dtype=np.uint32)
        self.perm = np.ascontiguousarray(p.perm, dtype=np.uint32) if len(p.perm) else None
        self.s = gr_program()
        self.s.n_stmts = S
        self.s.stmts = C.cast(st, C.POINTER(gr_stmt))
        self.s.slot_level = self.level.ctypes.data_as(C.POINTER(C.c_uint8)) if n else None
        self.s.slot_guard = self.guard.ctypes.data_as(C.POINTER(C.c_uint16))
        self.s.slot_weight = self.weight.ctypes.data_as(C.POINTER(C.c_uint32)) if n else None
        self.s.m_shared, self.s.m_global = int(p.m_shared), int(p.m_global)
        if self.perm is not None:
            self.s.perm = self.perm.ctypes.data_as(C.POINTER(C.c_uint32))
            self.s.perm_len = len(self.perm)
        self.s.existing_mask = int(p.existing_mask)
        loops = list(getattr(p, "loops", ()) or ())
        if loops:
            self.loops = (gr_loop * len(loops))(*[gr_loop(int(a), int(b), int(c)) for a, b, c in loops])
            self.s.n_loops = len(loops)
            self.s.loops = C.cast(self.loops, C.POINTER(gr_loop))
        coef = getattr(p, "iter_coef", None)
        if coef is not None:
            self.coef = np.ascontiguousarray(coef, dtype=np.uint32)
            self.s.iter_coef = self.coef.ctypes.data_as(C.POINTER(C.c_uint32))
        pos = getattr(p, "slot_pos", None)
        if pos is not None and len(pos):  # no slots: no places to give
            self.pos = np.ascontiguousarray(np.asarray(pos, dtype=np.uint8))
            self.s.n_slots = n
            self.s.slot_pos = self.pos.ctypes.data_as(C.POINTER(C.c_uint8))
        negs = list(getattr(p, "neg_clauses", ()) or ())
        if negs:
            self.neg = np.ascontiguousarray(np.array(negs, np.uint32))
            self.s.n_neg = len(negs)
            self.s.neg = self.neg.ctypes.data_as(C.POINTER(C.c_uint32))
        self.launch = gr_launch(int(p.blocks), int(p.threads))
        self.mode = int(p.mode)


STRATEGY_MAXSAT, STRATEGY_MHS = 0, 1


def _options(grid_enabled: bool = True, max_iters: int = 64, strategy: int = 0,
             deadline_us: int = 0) -> gr_options:
    o = gr_options()
    o.grid_enabled = 1 if grid_enabled else 0
    o.strategy = strategy
    o.max_iters = max_iters
    o.deadline_us = deadline_us
    return o


class ProgramBatch:
    """Many programs marshalled into a few contiguous numpy buffers (one
    gr_stmt array, one slot array of each kind, one permutation array) and a
    gr_program array pointing into them.  Keeps every buffer alive."""

    STMT_DTYPE = np.dtype(gr_stmt)
    PROG_DTYPE = np.dtype([("n_stmts", np.uint32), ("stmts", np.uint64), ("slot_level", np.uint64),
                           ("slot_guard", np.uint64), ("slot_weight", np.uint64),
                           ("m_shared", np.uint32), ("m_global", np.uint32), ("perm", np.uint64),
                           ("perm_len", np.uint32), ("existing_mask", np.uint32),
                           ("n_loops", np.uint32), ("loops", np.uint64), ("iter_coef", np.uint64),
                           ("n_slots", np.uint32), ("slot_pos", np.uint64),
                           ("n_neg", np.uint32), ("neg", np.uint64)],
                          align=True)

    def __init__(self, progs: Sequence):
        assert self.PROG_DTYPE.itemsize == C.sizeof(gr_program)
        n = len(progs)
        S = np.array([p.op.shape[0] for p in progs], np.int64)
        nsl = np.array([len(p.slot_level) for p in progs], np.int64)
        s_off = np.concatenate([[0], np.cumsum(S)])
        k_off = np.concatenate([[0], np.cumsum(nsl)])
        st = np.zeros(int(s_off[-1]), self.STMT_DTYPE)
        for name, attr in (("op", "op"), ("space", "space"), ("kind", "kind"), ("a", "a"), ("b", "b"),
                           ("c", "c"), ("perm_off", "perm_off"), ("guard_k", "guard_k"),
                           ("guard_r", "guard_r")):
            st[name] = np.concatenate([getattr(p, attr) for p in progs])
        self.stmts = st
        self.level = np.ascontiguousarray(np.concatenate([p.slot_level for p in progs]).astype(np.uint8))
        guard = np.zeros(2 * int(k_off[-1]) + 2, np.uint16)
        guard[0:2 * int(k_off[-1]):2] = np.concatenate([p.slot_guard_k for p in progs])
        guard[1:2 * int(k_off[-1]):2] = np.concatenate([p.slot_guard_r for p in progs])
        self.guard = guard
        self.weight = np.ascontiguousarray(np.concatenate([p.slot_weight for p in progs]).astype(np.uint32))
        plen = np.array([len(p.perm) for p in progs], np.int64)
        p_off = np.concatenate([[0], np.cumsum(plen)])
        self.perm = (np.ascontiguousarray(np.concatenate([p.perm for p in progs]).astype(np.uint32))
                     if p_off[-1] else np.zeros(1, np.uint32))
        pa = np.zeros(n, self.PROG_DTYPE)
        pa["n_stmts"] = S
        pa["stmts"] = st.ctypes.data + s_off[:-1] * self.STMT_DTYPE.itemsize
        has_slots = nsl > 0
        pa["slot_level"] = np.where(has_slots, self.level.ctypes.data + k_off[:-1], 0)
        pa["slot_guard"] = self.guard.ctypes.data + 4 * k_off[:-1]
        pa["slot_weight"] = np.where(has_slots, self.weight.ctypes.data + 4 * k_off[:-1], 0)
        pa["m_shared"] = [p.m_shared for p in progs]
        pa["m_global"] = [p.m_global for p in progs]
        pa["perm"] = np.where(plen > 0, self.perm.ctypes.data + 4 * p_off[:-1], 0)
        pa["perm_len"] = plen
        pa["existing_mask"] = [p.existing_mask for p in progs]
        # counted loops (lo, hi, trips) and loop-counter coefficients
        nloop = np.array([len(getattr(p, "loops", ()) or ()) for p in progs], np.int64)
        if nloop.any():
            l_off = np.concatenate([[0], np.cumsum(nloop)])
            self.loop_arr = np.ascontiguousarray(
                np.array([l for p in progs for l in (getattr(p, "loops", ()) or ())], np.uint32).reshape(-1, 3))
            pa["n_loops"] = nloop
            pa["loops"] = np.where(nloop > 0, self.loop_arr.ctypes.data + 12 * l_off[:-1], 0)
        has_coef = np.array([getattr(p, "iter_coef", None) is not None for p in progs])
        if has_coef.any():
            self.coef = np.ascontiguousarray(np.concatenate(
                [p.iter_coef if c else np.zeros(len(p.op), np.uint32) for p, c in zip(progs, has_coef)]
            ).astype(np.uint32))
            pa["iter_coef"] = np.where(has_coef, self.coef.ctypes.data + 4 * s_off[:-1], 0)
        has_pos = np.array([getattr(p, "slot_pos", None) is not None and len(p.slot_pos) > 0 for p in progs])
        if has_pos.any():
            self.pos_arr = np.ascontiguousarray(np.concatenate(
                [np.asarray(p.slot_pos, np.uint8) if h else np.zeros(0, np.uint8) for p, h in zip(progs, has_pos)]
                + [np.zeros(1, np.uint8)]))
            pos_len = np.array([len(p.slot_level) if h else 0 for p, h in zip(progs, has_pos)], np.int64)
            p_off2 = np.concatenate([[0], np.cumsum(pos_len)])
            pa["n_slots"] = np.where(has_pos, nsl, 0)
            pa["slot_pos"] = np.where(has_pos, self.pos_arr.ctypes.data + p_off2[:-1], 0)
        nneg = np.array([len(getattr(p, "neg_clauses", ()) or ()) for p in progs], np.int64)
        if nneg.any():
            n_off = np.concatenate([[0], np.cumsum(nneg)])
            self.neg_arr = np.ascontiguousarray(
                np.array([c for p in progs for c in (getattr(p, "neg_clauses", ()) or ())], np.uint32))
            pa["n_neg"] = nneg
            pa["neg"] = np.where(nneg > 0, self.neg_arr.ctypes.data + 4 * n_off[:-1], 0)
        self.progs = pa
        la = np.zeros((n, 2), np.uint32)
        la[:, 0] = [p.blocks for p in progs]
        la[:, 1] = [p.threads for p in progs]
        self.launches = la
        self.modes = np.ascontiguousarray(np.array([p.mode for p in progs], np.int32))
        self.n = n

    @property
    def prog_ptr(self):
        return C.cast(self.progs.ctypes.data, C.POINTER(gr_program))

    @property
    def launch_ptr(self):
        return C.cast(self.launches.ctypes.data, C.POINTER(gr_launch))

    @property
    def mode_ptr(self):
        return C.cast(self.modes.ctypes.data, C.POINTER(C.c_int32))


def _program_array(progs: Sequence) -> tuple:
    b = ProgramBatch(progs)
    return b, b.prog_ptr, b.launch_ptr


def witness_dict(w, S: int) -> dict:
    return {"intra": [int(w["race_intra"][i]) for i in range(S)],
            "inter": [int(w["race_inter"][i]) for i in range(S)],
            "diverge": int(w["diverge"]), "access_pairs": int(w["access_pairs"])}


def result_dict(r) -> dict:
    it = int(r["iters"])
    nc = int(r["n_clauses"])
    return {"status": int(r["status"]), "mask": int(r["mask"]), "weight": int(r["weight"]),
            "added": int(r["added"]), "removed": int(r["removed"]), "iters": it,
            "traj": [int(x) for x in r["traj"][:min(it, MAX_ITERS)]],
            "clauses": [int(x) for x in r["clauses"][:nc]], "forbidden": int(r["forbidden"]),
            "access_pairs": int(r["access_pairs"]), "t_start_ns": int(r["t_start_ns"]),
            "t_end_ns": int(r["t_end_ns"])}


# ---------------------------------------------------------------------------
# Host-pointer entry points
# ---------------------------------------------------------------------------

def validate(p) -> None:
    c = CProgram(p)
    _check(lib().gr_validate(C.byref(c.s), c.launch))


def check(p, mask: int) -> dict:
    c = CProgram(p)
    w = gr_witnesses()
    _check(lib().gr_check(C.byref(c.s), c.launch, mask, C.byref(w)))
    arr = np.frombuffer(bytes(w), dtype=WITNESS_DTYPE)[0]
    return witness_dict(arr, int(arr["n_stmts"]))


def repair(p, mode: Optional[int] = None, grid_enabled: bool = True, max_iters: int = 64,
           strategy: int = 0, deadline_us: int = 0) -> dict:
    c = CProgram(p)
    r = gr_repair_result()
    o = _options(grid_enabled, max_iters, strategy, deadline_us)
    _check(lib().gr_repair(C.byref(c.s), c.launch, c.mode if mode is None else mode, C.byref(o),
                           C.byref(r)))
    return result_dict(np.frombuffer(bytes(r), dtype=RESULT_DTYPE)[0])


def repair_plain(p, mode: Optional[int] = None, grid_enabled: bool = True,
                 max_iters: int = 64, strategy: int = 0, deadline_us: int = 0) -> dict:
    c = CProgram(p)
    r = gr_repair_result()
    o = _options(grid_enabled, max_iters, strategy, deadline_us)
    _check(lib().gr_repair_plain(C.byref(c.s), c.launch, c.mode if mode is None else mode,
                                 C.byref(o), C.byref(r)))
    return result_dict(np.frombuffer(bytes(r), dtype=RESULT_DTYPE)[0])


def repair_plain_timed(p, mode: Optional[int] = None, grid_enabled: bool = True,
                       max_iters: int = 64, strategy: int = 0, deadline_us: int = 0):
    """repair_plain, and the CUDA-event time (ms) of its launch loop alone."""
    c = CProgram(p)
    r = gr_repair_result()
    o = _options(grid_enabled, max_iters, strategy, deadline_us)
    ms = C.c_float(0.0)
    _check(lib().gr_repair_plain_timed(C.byref(c.s), c.launch, c.mode if mode is None else mode,
                                       C.byref(o), C.byref(r), C.byref(ms)))
    return result_dict(np.frombuffer(bytes(r), dtype=RESULT_DTYPE)[0]), float(ms.value)


def solve(n_vars: int, weights, pos, neg=(), forced: int = 0, forbidden: int = 0):
    """Lowest (mask, weight) hitting set, or None when unsatisfiable."""
    w = (C.c_uint32 * max(1, n_vars))(*[int(x) for x in weights])
    pa = (C.c_uint32 * max(1, len(pos)))(*[int(x) for x in pos])
    na = (C.c_uint32 * max(1, len(neg)))(*[int(x) for x in neg])
    m, wt = C.c_uint32(), C.c_uint32()
    rc = _check(lib().gr_solve(n_vars, w, pa, len(pos), na, len(neg), forced, forbidden,
                               C.byref(m), C.byref(wt)), allowed=(OK, UNSAT))
    return None if rc == UNSAT else (m.value, wt.value)


def repair_batch_raw(progs, grid_enabled: bool = True, max_iters: int = 64, stream: int = 0,
                     out: Optional[np.ndarray] = None, strategy: int = 0, deadline_us: int = 0) -> np.ndarray:
    """gr_repair_batch.  ``progs`` is a list of programs or a ProgramBatch."""
    b = progs if isinstance(progs, ProgramBatch) else ProgramBatch(progs)
    if out is None:
        out = np.zeros(b.n, dtype=RESULT_DTYPE)
    o = _options(grid_enabled, max_iters, strategy, deadline_us)
    _check(lib().gr_repair_batch(b.prog_ptr, b.launch_ptr, b.mode_ptr, b.n, C.byref(o), out.ctypes.data,
                                 C.c_void_p(stream)))
    return out


def repair_batch(progs: Sequence, grid_enabled: bool = True, max_iters: int = 64,
                 stream: int = 0, strategy: int = 0, deadline_us: int = 0) -> List[dict]:
    return [result_dict(r) for r in repair_batch_raw(progs, grid_enabled, max_iters, stream,
                                                      strategy=strategy, deadline_us=deadline_us)]


def check_batch(progs: Sequence, masks: Sequence[int], stream: int = 0) -> List[dict]:
    b, arr, la = _program_array(progs)
    m = (C.c_uint32 * b.n)(*[int(x) for x in masks])
    out = np.zeros(b.n, dtype=WITNESS_DTYPE)
    _check(lib().gr_check_batch(arr, la, m, b.n, out.ctypes.data, C.c_void_p(stream)))
    return [witness_dict(out[i], int(out[i]["n_stmts"])) for i in range(len(progs))]


# ---------------------------------------------------------------------------
# Device-resident entry points (torch supplies device memory and streams)
# ---------------------------------------------------------------------------

def pack(progs: Sequence) -> tuple:
    """(host arena as a 256-byte-aligned uint8 array, scratch bytes needed)."""
    b, arr, la = _program_array(progs)
    ab, sb = C.c_uint64(), C.c_uint64()
    _check(lib().gr_pack_size(arr, la, b.n, C.byref(ab), C.byref(sb)))
    raw = np.zeros(ab.value + 256, np.uint8)
    off = (-raw.ctypes.data) % 256
    host = raw[off:off + ab.value]
    _check(lib().gr_pack(arr, la, b.mode_ptr, b.n, host.ctypes.data, ab.value))
    return host, sb.value


class DeviceBatch:
    """A packed batch resident in device memory with its scratch and results.

    ``run()`` enqueues the whole repair (trace expansion + persistent repair
    launch) on the current torch stream; nothing is allocated per call.
    """

    def __init__(self, progs: Sequence, device: str = "cuda", grid_enabled: bool = True,
                 max_iters: int = 64, strategy: int = 0, deadline_us: int = 0):
        import torch

        self.n = len(progs)
        host, scratch_bytes = pack(progs)
        self.arena_bytes = host.nbytes
        self.scratch_bytes = scratch_bytes
        self.arena = torch.empty(self.arena_bytes + 256, dtype=torch.uint8, device=device)
        self.scratch = torch.empty(scratch_bytes + 256, dtype=torch.uint8, device=device)
        self.out = torch.empty(self.n * RESULT_DTYPE.itemsize + 256, dtype=torch.uint8, device=device)
        self.wit = None
        self._arena_ptr = _aligned(self.arena.data_ptr())
        self._scratch_ptr = _aligned(self.scratch.data_ptr())
        self._out_ptr = _aligned(self.out.data_ptr())
        a_off = self._arena_ptr - self.arena.data_ptr()
        self.arena[a_off:a_off + self.arena_bytes].copy_(torch.from_numpy(host))
        self.opts = _options(grid_enabled, max_iters, strategy, deadline_us)
        self.host_arena = host
        # programs the relation kernel takes (header u32 at byte 120); the
        # others need their traces expanded
        self.n_fast = int(host[120:124].view(np.uint32)[0])
        self.has_general = self.n_fast < self.n
        # the packer's kArenaSimple flag: straight-line programs on the shared
        # array only; with no general program, a tuned run() is one launch
        self.simple = bool(int(host[108:112].view(np.uint32)[0]) & 1)

    def run(self, stream: Optional[int] = None) -> None:
        import torch

        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(lib().gr_repair_packed(C.c_void_p(self._arena_ptr), self.n, C.byref(self.opts),
                                      C.c_void_p(self._scratch_ptr), self.scratch_bytes,
                                      C.c_void_p(self._out_ptr), C.c_void_p(st)))

    def run_wide(self, stream: Optional[int] = None) -> None:
        """The same repair on the wide lane (gr_repair_packed_wide): one CTA per
        (program, block) per check, the loop as a device-side graph."""
        import torch

        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(lib().gr_repair_packed_wide(C.c_void_p(self._arena_ptr), self.n, C.byref(self.opts),
                                           C.c_void_p(self._scratch_ptr), self.scratch_bytes,
                                           C.c_void_p(self._out_ptr), C.c_void_p(st)))

    def tune(self, stream: Optional[int] = None) -> int:
        """Pick the fastest CTA shapes for this batch (gr_tune_packed): bits 0-7
        index the relation kernel's shape, bits 8-15 the general check kernel's."""
        import torch

        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        shape = C.c_uint32()
        _check(lib().gr_tune_packed(C.c_void_p(self._arena_ptr), self.n, C.byref(self.opts),
                                    C.c_void_p(self._scratch_ptr), self.scratch_bytes,
                                    C.c_void_p(self._out_ptr), C.c_void_p(st), C.byref(shape)))
        self.shape = shape.value
        return shape.value

    def set_shape(self, shape: int, stream: Optional[int] = None) -> int:
        """Use a shape word tune() returned before (gr_set_shape_packed),
        without timing anything."""
        import torch

        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(lib().gr_set_shape_packed(C.c_void_p(self._arena_ptr), self.n, shape, C.c_void_p(st)))
        self.shape = shape
        return shape

    def expand(self, stream: Optional[int] = None) -> None:
        """Only the trace expansion (first half of run())."""
        import torch

        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(lib().gr_expand_packed(C.c_void_p(self._arena_ptr), C.c_void_p(self._scratch_ptr),
                                      self.scratch_bytes, C.c_void_p(st)))

    def repair_expanded(self, stream: Optional[int] = None) -> None:
        """Only the persistent repair launch (second half of run())."""
        import torch

        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(lib().gr_repair_expanded(C.c_void_p(self._arena_ptr), self.n, C.byref(self.opts),
                                        C.c_void_p(self._scratch_ptr), self.scratch_bytes,
                                        C.c_void_p(self._out_ptr), C.c_void_p(st)))

    def relation(self, stream: Optional[int] = None) -> None:
        """Each program's conflict relation into the scratch (gr_relation_packed)."""
        import torch

        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(lib().gr_relation_packed(C.c_void_p(self._arena_ptr), self.n, C.c_void_p(self._scratch_ptr),
                                        self.scratch_bytes, C.c_void_p(st)))

    def loop(self, stream: Optional[int] = None) -> None:
        """Algorithm 1 on the relations relation() wrote (gr_loop_packed)."""
        import torch

        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(lib().gr_loop_packed(C.c_void_p(self._arena_ptr), self.n, C.byref(self.opts),
                                    C.c_void_p(self._scratch_ptr), self.scratch_bytes,
                                    C.c_void_p(self._out_ptr), C.c_void_p(st)))

    def relation_loop(self, stream: Optional[int] = None) -> None:
        """The whole repair as one launch (gr_relation_loop_packed); only for
        straight-line programs on the shared array with no general one."""
        import torch

        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(lib().gr_relation_loop_packed(C.c_void_p(self._arena_ptr), self.n, C.byref(self.opts),
                                             C.c_void_p(self._scratch_ptr), self.scratch_bytes,
                                             C.c_void_p(self._out_ptr), C.c_void_p(st)))

    def check(self, masks, stream: Optional[int] = None, expanded: bool = False):
        """One check per program under masks[p] (gr_check_packed; with
        expanded=True only the check kernel, gr_check_expanded, on traces a
        previous call of this batch wrote)."""
        import torch

        if self.wit is None:
            self.wit = torch.empty(self.n * WITNESS_DTYPE.itemsize + 256, dtype=torch.uint8,
                                   device=self.arena.device)
            self.masks = torch.empty(self.n, dtype=torch.int32, device=self.arena.device)
        if masks is not None:  # None: the masks of the previous call
            self.masks.copy_(torch.as_tensor(np.asarray(masks, np.uint32).view(np.int32)))
        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        fn = lib().gr_check_expanded if expanded else lib().gr_check_packed
        _check(fn(C.c_void_p(self._arena_ptr), self.n, C.c_void_p(self.masks.data_ptr()),
                  C.c_void_p(self._scratch_ptr), self.scratch_bytes, C.c_void_p(_aligned(self.wit.data_ptr())),
                  C.c_void_p(st)))

    def results_raw(self) -> np.ndarray:
        off = self._out_ptr - self.out.data_ptr()
        b = self.out[off:off + self.n * RESULT_DTYPE.itemsize].cpu().numpy()
        return b.view(RESULT_DTYPE)

    def results(self) -> List[dict]:
        return [result_dict(r) for r in self.results_raw()]

    def witnesses(self, progs) -> List[dict]:
        off = _aligned(self.wit.data_ptr()) - self.wit.data_ptr()
        b = self.wit[off:off + self.n * WITNESS_DTYPE.itemsize].cpu().numpy().view(WITNESS_DTYPE)
        return [witness_dict(b[i], int(b[i]["n_stmts"])) for i in range(self.n)]


def _aligned(ptr: int) -> int:
    return (ptr + 255) // 256 * 256


# ---------------------------------------------------------------------------
# Repair server (continuous batching)
# ---------------------------------------------------------------------------

class Server:
    """gr_server_*: submit single programs at any time; poll for results."""

    def __init__(self, mem_budget_bytes: int, n_slots: int = 4, max_inflight: int = 1 << 20,
                 grid_enabled: bool = True, max_iters: int = 64, strategy: int = 0, deadline_us: int = 0):
        self._h = C.c_void_p()
        o = _options(grid_enabled, max_iters, strategy, deadline_us)
        _check(lib().gr_server_create(mem_budget_bytes, n_slots, max_inflight, C.byref(o),
                                      C.byref(self._h)))
        self._keep = {}

    def submit(self, p, mode: Optional[int] = None) -> int:
        c = CProgram(p)
        t = C.c_uint64()
        _check(lib().gr_server_submit(self._h, C.byref(c.s), c.launch,
                                      c.mode if mode is None else mode, C.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """(result dict, latency seconds) when done, else None."""
        r = gr_repair_result()
        lat = C.c_uint64()
        rc = _check(lib().gr_server_poll(self._h, ticket, C.byref(r), C.byref(lat)), allowed=(OK, EBUSY))
        if rc == EBUSY:
            return None
        return result_dict(np.frombuffer(bytes(r), dtype=RESULT_DTYPE)[0]), lat.value * 1e-9

    def drain(self, timeout_ms: int = 60000) -> bool:
        return _check(lib().gr_server_drain(self._h, timeout_ms), allowed=(OK, EBUSY)) == OK

    def stats(self) -> dict:
        a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(lib().gr_server_stats(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return {"pending": a.value, "inflight": b.value, "launches": c.value}

    def close(self) -> None:
        if self._h:
            _check(lib().gr_server_destroy(self._h))
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False
