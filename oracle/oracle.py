"""Python binding of the CPU oracle (oracle.cpp) and its build step.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` import this module.  It shares no code
with the GPU library: it compiles and loads its own C++ source, and takes a
program in the plain-data form of ``paper_2501_13051_gb300.workloads``
(relation arities, rules, input facts).

The oracle computes the least fixpoint of the rules (Section 2) by
semi-naive rounds that apply every rule once per round (Section 3) or, for
cross-checks, by naive rounds; see the header of oracle.cpp.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (plain g++, no GPU code)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp],
                           check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        lib.orc_new.restype = ctypes.c_void_p
        lib.orc_free.argtypes = [ctypes.c_void_p]
        lib.orc_add_relation.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
        lib.orc_load.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64]
        lib.orc_add_rule.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32]
        lib.orc_run.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64]
        lib.orc_run.restype = ctypes.c_int64
        lib.orc_size.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.orc_size.restype = ctypes.c_uint64
        lib.orc_export.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        lib.orc_rounds.argtypes = [ctypes.c_void_p]
        lib.orc_rounds.restype = ctypes.c_uint64
        lib.orc_delta_sizes.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64]
        _lib = lib
    return _lib


@dataclass
class OracleResult:
    relations: dict        # name -> (n, arity) uint32, sorted lexicographically, unique
    iterations: int        # rounds that produced a non-empty delta
    rounds: int            # rounds executed (the last one found nothing new)
    deltas: dict           # name -> list of per-round delta sizes

    def derived(self, program) -> int:
        return sum(len(self.relations[r]) for r in program.idb())


def encode_rule(rule, rel_id: dict, arity: dict) -> list:
    """Flatten a workloads.Rule into the integer form orc_add_rule reads."""
    var_id = {}

    def term(t):
        if isinstance(t, str):
            return [0, var_id.setdefault(t, len(var_id))]
        return [1, int(t)]

    def atom(a):
        name, terms = a
        if len(terms) != arity[name]:
            raise ValueError(f"arity mismatch in atom {a}")
        out = [rel_id[name], len(terms)]
        for t in terms:
            out += term(t)
        return out

    body = []
    for a in rule.body:
        body += atom(a)
    head = atom(rule.head)
    flat = head + [len(rule.body)] + body + [len(rule.neq)]
    for a, b in rule.neq:
        flat += [var_id[a], var_id[b]]
    return flat


def run_program(program, naive: bool = False, max_iters: int = 1 << 40) -> OracleResult:
    """Evaluate ``program`` to its least fixpoint on the CPU."""
    lib = _load()
    h = lib.orc_new()
    try:
        names = list(program.arity)
        rel_id = {}
        for nm in names:
            rid = lib.orc_add_relation(h, program.arity[nm])
            if rid < 0:
                raise ValueError(f"bad arity for {nm}")
            rel_id[nm] = rid
        for nm, rows in program.edb.items():
            rows = np.ascontiguousarray(rows, dtype=np.uint32).reshape(-1, program.arity[nm])
            if lib.orc_load(h, rel_id[nm], rows.ctypes.data, rows.shape[0]) != 0:
                raise ValueError(f"load failed for {nm}")
        for rule in program.rules:
            flat = np.asarray(encode_rule(rule, rel_id, program.arity), dtype=np.int64)
            if lib.orc_add_rule(h, flat.ctypes.data, len(flat)) != 0:
                raise ValueError(f"bad rule {rule}")
        it = lib.orc_run(h, 1 if naive else 0, max_iters)
        if it < 0:
            raise RuntimeError(f"oracle run failed ({it})")
        rels, deltas = {}, {}
        for nm in names:
            n = lib.orc_size(h, rel_id[nm])
            out = np.zeros((n, program.arity[nm]), dtype=np.uint32)
            if n:
                lib.orc_export(h, rel_id[nm], out.ctypes.data)
            rels[nm] = out
            buf = np.zeros(1 << 16, dtype=np.uint64)
            k = lib.orc_delta_sizes(h, rel_id[nm], buf.ctypes.data, len(buf))
            deltas[nm] = [int(x) for x in buf[:k]]
        return OracleResult(rels, int(it), int(lib.orc_rounds(h)), deltas)
    finally:
        lib.orc_free(h)
