"""Python binding of libcdl (include/cdl.h): argument marshalling only.

Every step of the fixpoint runs in the library's sm_103a kernels.  PyTorch
supplies device memory (through the engine's allocator callbacks, or as the
tensors handed to the single-step calls) and the CUDA stream.  There is no
CPU fallback: if libcdl.so is missing or no GPU is visible, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcdl.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "cdl.h")

MAX_ARITY = 8
STATUS = {0: "CDL_OK", -1: "CDL_E_INVALID", -2: "CDL_E_NOMEM", -3: "CDL_E_CAPACITY",
          -4: "CDL_E_VALUE", -5: "CDL_E_MAXITER", -6: "CDL_E_TIMEOUT", -7: "CDL_E_CUDA",
          -8: "CDL_E_STATE"}


class CdlError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {msg}" if msg else self.name)


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("mem_limit", ctypes.c_uint64),
                ("max_iters", ctypes.c_uint64), ("spin_limit", ctypes.c_uint64),
                ("timing", ctypes.c_uint32), ("estimator", ctypes.c_int32),
                ("hash_load", ctypes.c_double), ("radix_bits", ctypes.c_uint32),
                ("log_path", ctypes.c_char_p), ("est_margin", ctypes.c_double),
                ("n_instances", ctypes.c_uint32), ("retire", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("tune_cache", ctypes.c_char_p),
                ("est_min_rows", ctypes.c_uint64), ("graph", ctypes.c_int32),
                ("dense_bits", ctypes.c_int32), ("dedup", ctypes.c_int32),
                ("plan_launch_bytes", ctypes.c_double), ("est_max_rows", ctypes.c_uint64),
                ("host_full", ctypes.c_int32), ("star", ctypes.c_int32)]

MLP_IN = 16
MLP_PARAMS = 5313


class Term(ctypes.Structure):
    _fields_ = [("is_const", ctypes.c_uint32), ("v", ctypes.c_uint32)]


class Atom(ctypes.Structure):
    _fields_ = [("rel", ctypes.c_uint32), ("arity", ctypes.c_uint32),
                ("terms", ctypes.POINTER(Term))]


class RuleS(ctypes.Structure):
    _fields_ = [("head", Atom), ("nbody", ctypes.c_uint32), ("body", ctypes.POINTER(Atom)),
                ("nneq", ctypes.c_uint32), ("neq", ctypes.POINTER(ctypes.c_uint32))]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_uint64), ("rounds", ctypes.c_uint64),
                ("derived_tuples", ctypes.c_uint64), ("seconds", ctypes.c_double),
                ("algo_bytes", ctypes.c_double), ("joins", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("est_predictions", ctypes.c_uint64),
                ("est_overflows", ctypes.c_uint64),
                ("delta_per_round", ctypes.POINTER(ctypes.c_uint64)),
                ("delta_cap", ctypes.c_uint64),
                ("iters_per_instance", ctypes.POINTER(ctypes.c_uint64)),
                ("graph_rounds", ctypes.c_uint64), ("graph_builds", ctypes.c_uint64),
                ("index_merges", ctypes.c_uint64), ("graph_retirements", ctypes.c_uint64),
                ("star_joins", ctypes.c_uint64)]


class ColRef(ctypes.Structure):
    _fields_ = [("side", ctypes.c_uint32), ("v", ctypes.c_uint32)]


_lib = None


def header_functions() -> list:
    """Names of the functions include/cdl.h declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(cdl_\w+)\s*\(", src, flags=re.M)))


def lib():
    """Loads libcdl.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() or "
                           "python -m paper_2501_13051_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    P, U64, U32, VP = ctypes.POINTER, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
    PP = P(ctypes.c_void_p)
    sig = {
        "cdl_options_default": (None, [P(Options)]),
        "cdl_create": (ctypes.c_int, [P(Options), P(VP)]),
        "cdl_destroy": (ctypes.c_int, [VP]),
        "cdl_relation_create": (ctypes.c_int, [VP, ctypes.c_char_p, U32, P(U32)]),
        "cdl_relation_load": (ctypes.c_int, [VP, U32, PP, U64, ctypes.c_int]),
        "cdl_relations_load": (ctypes.c_int, [VP, U32, P(U32), P(PP), P(U64), ctypes.c_int]),
        "cdl_rule_add": (ctypes.c_int, [VP, P(RuleS)]),
        "cdl_run": (ctypes.c_int, [VP, P(Stats)]),
        "cdl_relation_size": (ctypes.c_int, [VP, U32, P(U64)]),
        "cdl_relation_export": (ctypes.c_int, [VP, U32, PP, U64, P(U64), ctypes.c_int]),
        "cdl_relation_export_rows": (ctypes.c_int, [VP, U32, U64, U64, PP, ctypes.c_int]),
        "cdl_checkpoint_save": (ctypes.c_int, [VP, ctypes.c_char_p]),
        "cdl_checkpoint_load": (ctypes.c_int, [VP, ctypes.c_char_p]),
        "cdl_instance_rows": (ctypes.c_int, [VP, U32, U32, P(U64), P(U64)]),
        "cdl_kernel_profile": (ctypes.c_int, [VP, U32, ctypes.c_char_p, ctypes.c_size_t, P(U64),
                                              P(ctypes.c_double), P(ctypes.c_double)]),
        "cdl_last_error": (ctypes.c_char_p, [VP]),
        "cdl_hash_table_bytes": (U64, [U64, ctypes.c_double]),
        "cdl_hash_build": (ctypes.c_int, [VP, U64, VP, U64, VP]),
        "cdl_join_count": (ctypes.c_int, [VP, U64, VP, U64, VP, VP]),
        "cdl_exclusive_scan": (ctypes.c_int, [VP, U64, VP, P(U64), VP, P(ctypes.c_size_t), VP]),
        "cdl_exclusive_scan_noalloc": (ctypes.c_int, [VP, U64, VP, P(U64), VP]),
        "cdl_join": (ctypes.c_int, [PP, U32, U64, U32, PP, U32, U64, U32, P(ColRef), U32,
                                    P(ColRef), U32, PP, U64, P(U64), VP, P(ctypes.c_size_t), VP]),
        "cdl_sort_unique": (ctypes.c_int, [PP, U32, U64, PP, P(U64), VP, P(ctypes.c_size_t), VP]),
        "cdl_diff_merge": (ctypes.c_int, [PP, U64, PP, U64, U32, PP, P(U64), PP, VP,
                                          P(ctypes.c_size_t), VP]),
        "cdl_estimator_log": (ctypes.c_int, [VP, VP, VP, U64, P(U64)]),
        "cdl_estimator_train": (ctypes.c_int, [VP, VP, VP, U64, U32, ctypes.c_float,
                                               ctypes.c_float, U64, P(ctypes.c_float)]),
        "cdl_estimator_params": (ctypes.c_int, [VP, VP, ctypes.c_int]),
        "cdl_mlp_forward": (ctypes.c_int, [VP, VP, U64, VP, VP, P(ctypes.c_size_t), VP]),
        "cdl_mlp_gradient": (ctypes.c_int, [VP, VP, VP, U64, ctypes.c_float, VP, VP, VP,
                                            P(ctypes.c_size_t), VP]),
        "cdl_mlp_infer_bf16": (ctypes.c_int, [VP, VP, U64, VP, VP, P(ctypes.c_size_t), VP]),
        "cdl_mlp_adam": (ctypes.c_int, [VP, VP, VP, VP, U64, ctypes.c_float, VP]),
        "cdl_join_features": (ctypes.c_int, [VP, VP, U64, VP, VP, U64, P(ctypes.c_float), VP,
                                             VP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return _lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libcdl needs a CUDA GPU; none is visible")
    return torch


def _ptrs(tensors) -> ctypes.Array:
    arr = (ctypes.c_void_p * max(1, len(tensors)))()
    for i, t in enumerate(tensors):
        arr[i] = t.data_ptr() if hasattr(t, "data_ptr") else t
    return arr


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class _TorchArena:
    """Allocator callbacks that hand the engine torch-owned device memory."""

    def __init__(self, device):
        self.torch = _torch()
        self.device = device
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, _ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:  # out of memory -> NULL, the engine reports CDL_E_NOMEM
            return None
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, _nbytes, _ctx):
        self.live.pop(ptr, None)


@dataclass
class RunStats:
    iterations: int
    rounds: int
    derived_tuples: int
    seconds: float
    algo_bytes: float
    joins: int
    kernel_launches: int
    delta_per_round: list = field(default_factory=list)
    est_predictions: int = 0
    est_overflows: int = 0
    iters_per_instance: list = field(default_factory=list)
    graph_rounds: int = 0
    graph_builds: int = 0
    index_merges: int = 0
    graph_retirements: int = 0
    star_joins: int = 0


# kernel classes in cdl_kernel_profile order
KERNEL_CLASSES = ("hash_build", "count_heads", "join_count", "scan", "join_write",
                  "radix_upsweep", "radix_scatter", "diff_count", "diff_merge", "select",
                  "misc", "estimator", "join_direct", "retire", "dense", "dedup")


def _timing_mask(timing):
    """options.timing from False / True / an iterable of kernel class names."""
    if timing is True:
        return 1
    if not timing:
        return 0
    m = 0
    for name in timing:
        m |= 1 << (1 + KERNEL_CLASSES.index(name))
    return m


class Engine:
    """One engine on the current CUDA device and stream (cdl_create).

    timing: False, True (every kernel class) or an iterable of class names
    from KERNEL_CLASSES (events wrap only those launches)."""

    def __init__(self, *, device=None, stream=None, mem_limit=0, max_iters=0, spin_limit=0,
                 timing=False, hash_load=0.5, radix_bits=0, torch_alloc=True, estimator=0,
                 est_margin=1.0, est_params=None, n_instances=0, retire=True, autotune=0,
                 tune_cache=None, graph=False, est_min_rows=0, dense_bits=0, dedup=0,
                 plan_launch_bytes=0.0, est_max_rows=0, host_full=0, star=0):
        torch = _torch()
        L = lib()
        self._L = L
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        opts = Options()
        L.cdl_options_default(ctypes.byref(opts))
        self._arena = _TorchArena(self.device) if torch_alloc else None
        if self._arena is not None:
            opts.alloc = self._arena.alloc_cb
            opts.free = self._arena.free_cb
        opts.stream = ctypes.c_void_p(self.stream.cuda_stream)
        opts.mem_limit = mem_limit
        opts.max_iters = max_iters
        opts.spin_limit = spin_limit
        opts.timing = _timing_mask(timing)
        opts.hash_load = hash_load
        opts.radix_bits = radix_bits
        opts.estimator = estimator
        opts.est_margin = est_margin
        opts.n_instances = n_instances
        opts.retire = 0 if retire else -1
        opts.autotune = autotune
        opts.graph = int(graph)  # True / False, or a starting capacity in rows
        opts.est_min_rows = est_min_rows
        opts.dense_bits = dense_bits  # 0 default (28), -1 never
        opts.dedup = dedup  # 0 merge of sorted rows, 1 Algorithm 2 (hybrid index), 2 hash-only
        opts.plan_launch_bytes = plan_launch_bytes
        opts.est_max_rows = est_max_rows
        opts.host_full = host_full  # 1: Full of step-(d)-only relations in pinned host memory
        opts.star = star  # 0: chains ending in two probe-keyed atoms join them at once; -1 never
        opts.tune_cache = os.fsencode(tune_cache) if tune_cache else None
        self.n_instances = n_instances
        self._opts = opts
        h = ctypes.c_void_p()
        self._check(L.cdl_create(ctypes.byref(opts), ctypes.byref(h)), engine=False)
        self._h = h
        self.rels = {}
        self.arity = {}
        if est_params is not None:
            self.estimator_params(est_params)

    def _check(self, st, engine=True):
        if st != 0:
            msg = ""
            if engine and getattr(self, "_h", None):
                msg = (self._L.cdl_last_error(self._h) or b"").decode()
            raise CdlError(st, msg)

    def close(self):
        if getattr(self, "_h", None):
            self._L.cdl_destroy(self._h)
            self._h = None
        if self._arena is not None:
            self._arena.live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ program
    def relation(self, name: str, arity: int) -> int:
        out = ctypes.c_uint32()
        self._check(self._L.cdl_relation_create(self._h, name.encode(), arity, ctypes.byref(out)))
        self.rels[name] = out.value
        self.arity[name] = arity
        return out.value

    def _columns(self, name, rows):
        """(column pointers, n, on_device, objects to keep alive) of one load."""
        ar = self.arity[name]
        if isinstance(rows, (list, tuple)):
            cols = list(rows)
            n = cols[0].numel() if cols else 0
            return _ptrs(cols), n, 1 if (cols and cols[0].is_cuda) else 0, cols
        a = np.ascontiguousarray(np.asarray(rows, dtype=np.uint32).reshape(-1, ar))
        keep = [np.ascontiguousarray(a[:, k]) for k in range(ar)]
        return _ptrs([c.ctypes.data for c in keep]), a.shape[0], 0, keep

    def load(self, name: str, rows) -> None:
        """rows: (n, arity) host array of uint32, or a list of `arity` int32 /
        uint32 column tensors (CUDA tensors are read on the device, CPU
        tensors -- e.g. pinned -- are copied from host memory)."""
        arr, n, on_dev, keep = self._columns(name, rows)
        self._check(self._L.cdl_relation_load(self._h, self.rels[name], arr, n, on_dev))
        del keep

    def load_many(self, relations: dict) -> None:
        """{name: rows} (as for load, all on the device or all in host
        memory) in one call: one check of all values, all added or none."""
        names = list(relations)
        if not names:
            return
        parts = [self._columns(nm, relations[nm]) for nm in names]
        on_dev = {p[2] for p in parts if p[1]}
        if len(on_dev) > 1:
            raise ValueError("load_many: mix of device and host columns")
        rel = (ctypes.c_uint32 * len(names))(*[self.rels[nm] for nm in names])
        cols = (ctypes.POINTER(ctypes.c_void_p) * len(names))(
            *[ctypes.cast(p[0], ctypes.POINTER(ctypes.c_void_p)) for p in parts])
        ns = (ctypes.c_uint64 * len(names))(*[p[1] for p in parts])
        self._check(self._L.cdl_relations_load(self._h, len(names), rel, cols, ns,
                                               on_dev.pop() if on_dev else 0))
        del parts

    def rule(self, head, body, neq=()) -> None:
        var_id = {}

        def atom(a):
            name, terms = a
            ts = (Term * len(terms))()
            for i, t in enumerate(terms):
                if isinstance(t, str):
                    ts[i] = Term(0, var_id.setdefault(t, len(var_id)))
                else:
                    ts[i] = Term(1, int(t))
            return Atom(self.rels[name], len(terms), ts), ts

        body_atoms = (Atom * len(body))()
        keep = []
        for i, a in enumerate(body):
            at, ts = atom(a)
            body_atoms[i] = at
            keep.append(ts)
        h, hts = atom(head)
        nq = (ctypes.c_uint32 * max(1, 2 * len(neq)))()
        for i, (a, b) in enumerate(neq):
            nq[2 * i], nq[2 * i + 1] = var_id[a], var_id[b]
        r = RuleS(h, len(body), body_atoms, len(neq), nq)
        self._check(self._L.cdl_rule_add(self._h, ctypes.byref(r)))

    def load_program(self, program) -> None:
        for name, ar in program.arity.items():
            self.relation(name, ar)
        self.load_many(dict(program.edb))
        for r in program.rules:
            self.rule(r.head, r.body, r.neq)

    # ---------------------------------------------------------------- run
    def run(self) -> RunStats:
        cap = 1 << 16
        buf = (ctypes.c_uint64 * cap)()
        st = Stats()
        st.delta_per_round = ctypes.cast(buf, ctypes.POINTER(ctypes.c_uint64))
        st.delta_cap = cap
        inst = (ctypes.c_uint64 * max(1, self.n_instances))()
        if self.n_instances:
            st.iters_per_instance = ctypes.cast(inst, ctypes.POINTER(ctypes.c_uint64))
        self._check(self._L.cdl_run(self._h, ctypes.byref(st)))
        return RunStats(st.iterations, st.rounds, st.derived_tuples, st.seconds, st.algo_bytes,
                        st.joins, st.kernel_launches, [int(buf[i]) for i in range(min(st.rounds, cap))],
                        st.est_predictions, st.est_overflows,
                        [int(inst[i]) for i in range(self.n_instances)],
                        st.graph_rounds, st.graph_builds, st.index_merges,
                        st.graph_retirements, st.star_joins)

    # ---------------------------------------------------------- estimator
    def estimator_log(self):
        """(X, y) of the joins logged so far (options estimator=2)."""
        n = ctypes.c_uint64()
        self._check(self._L.cdl_estimator_log(self._h, None, None, 0, ctypes.byref(n)))
        X = np.zeros((n.value, MLP_IN), dtype=np.float32)
        y = np.zeros(n.value, dtype=np.float32)
        self._check(self._L.cdl_estimator_log(self._h, X.ctypes.data, y.ctypes.data, n.value,
                                              ctypes.byref(n)))
        return X, y

    def estimator_train(self, X=None, y=None, epochs=2000, lr=3e-3, tau=0.9, seed=1):
        """Trains the network on the GPU (on X, y, or the engine's own log);
        returns the final training loss."""
        loss = ctypes.c_float()
        if X is None:
            st = self._L.cdl_estimator_train(self._h, None, None, 0, epochs, lr, tau, seed,
                                             ctypes.byref(loss))
        else:
            X = np.ascontiguousarray(X, dtype=np.float32)
            y = np.ascontiguousarray(y, dtype=np.float32)
            st = self._L.cdl_estimator_train(self._h, X.ctypes.data, y.ctypes.data, len(y), epochs,
                                             lr, tau, seed, ctypes.byref(loss))
        self._check(st)
        return float(loss.value)

    def estimator_params(self, params=None):
        """Reads the trained FP32 parameters, or installs `params`."""
        if params is None:
            out = np.zeros(MLP_PARAMS, dtype=np.float32)
            self._check(self._L.cdl_estimator_params(self._h, out.ctypes.data, 0))
            return out
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self._L.cdl_estimator_params(self._h, p.ctypes.data, 1))
        return p

    def size(self, name: str) -> int:
        n = ctypes.c_uint64()
        self._check(self._L.cdl_relation_size(self._h, self.rels[name], ctypes.byref(n)))
        return n.value

    def checkpoint_save(self, path: str) -> None:
        """Writes every relation's full and delta versions and the rounds done."""
        self._check(self._L.cdl_checkpoint_save(self._h, os.fsencode(path)))

    def checkpoint_load(self, path: str) -> None:
        """Restores a checkpoint before run(): the run continues from it."""
        self._check(self._L.cdl_checkpoint_load(self._h, os.fsencode(path)))

    def instance_rows(self, name: str, instance: int):
        """Batched runs: (first, count) of the instance's rows in the sorted relation."""
        f, c = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self._L.cdl_instance_rows(self._h, self.rels[name], instance, ctypes.byref(f),
                                              ctypes.byref(c)))
        return f.value, c.value

    def export_instance(self, name: str, instance: int):
        """Batched runs: the instance's tuples, instance column included, as an
        (n, arity) numpy array."""
        ar = self.arity[name]
        first, n = self.instance_rows(name, instance)
        res = np.zeros((ar, max(n, 1)), dtype=np.uint32)
        ptrs = _ptrs([res[k].ctypes.data for k in range(ar)])
        self._check(self._L.cdl_relation_export_rows(self._h, self.rels[name], first, n, ptrs, 0))
        return np.ascontiguousarray(res[:, :n].T)

    def export(self, name: str, device: bool = False, out=None):
        """Sorted unique tuples: (n, arity) numpy array, or with device=True a
        list of CUDA int32 column tensors (uint32 bit patterns).  ``out`` may
        supply host column buffers (e.g. pinned tensors) of sufficient size."""
        torch = _torch()
        ar, n = self.arity[name], self.size(name)
        got = ctypes.c_uint64()
        if device:
            cols = [torch.empty(max(n, 1), dtype=torch.int32, device=self.device) for _ in range(ar)]
            self._check(self._L.cdl_relation_export(self._h, self.rels[name], _ptrs(cols), n,
                                                    ctypes.byref(got), 1))
            return [c[:n] for c in cols]
        if out is not None:
            self._check(self._L.cdl_relation_export(self._h, self.rels[name], _ptrs(out), n,
                                                    ctypes.byref(got), 0))
            return out
        res = np.zeros((ar, max(n, 1)), dtype=np.uint32)
        ptrs = _ptrs([res[k].ctypes.data for k in range(ar)])
        self._check(self._L.cdl_relation_export(self._h, self.rels[name], ptrs, n,
                                                ctypes.byref(got), 0))
        return np.ascontiguousarray(res[:, :n].T)

    def kernel_profile(self) -> list:
        out = []
        for i in range(64):
            name = ctypes.create_string_buffer(64)
            la, ms, by = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
            st = self._L.cdl_kernel_profile(self._h, i, name, 64, ctypes.byref(la), ctypes.byref(ms),
                                            ctypes.byref(by))
            if st != 0:
                break
            out.append({"kernel": name.value.decode(), "launches": la.value, "ms": ms.value,
                        "bytes": by.value})
        return out


def run_program(program, **opts):
    """Loads and runs a workloads.Program; returns ({name: rows}, RunStats)."""
    with Engine(**opts) as e:
        e.load_program(program)
        st = e.run()
        return {nm: e.export(nm) for nm in program.arity}, st


# ---------------------------------------------------------------------------
# single steps on torch tensors (device memory owned by the caller)
# ---------------------------------------------------------------------------

def _u32(t):
    torch = _torch()
    if t.dtype not in (torch.int32, torch.uint32) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("columns must be contiguous CUDA int32/uint32 tensors")
    return t


def _workspace(fn, *args):
    torch = _torch()
    need = ctypes.c_size_t(0)
    st = fn(*args, None, ctypes.byref(need))
    if st != 0:
        raise CdlError(st)
    ws = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device="cuda")
    return ws, need


def hash_table_bytes(n_keys: int, load: float = 0.5) -> int:
    return int(lib().cdl_hash_table_bytes(n_keys, load))


def hash_build(keys, load: float = 0.5, stream=None):
    """Step (a) on a sorted key column; returns the table as a uint8 tensor."""
    torch = _torch()
    keys = _u32(keys)
    nb = hash_table_bytes(keys.numel(), load)
    table = torch.empty(nb, dtype=torch.uint8, device=keys.device)
    st = lib().cdl_hash_build(keys.data_ptr(), keys.numel(), table.data_ptr(), nb,
                              _stream_handle(stream))
    if st != 0:
        raise CdlError(st)
    return table


def join_count(probe, table, stream=None):
    torch = _torch()
    probe = _u32(probe)
    counts = torch.empty(max(1, probe.numel()), dtype=torch.int32, device=probe.device)
    st = lib().cdl_join_count(probe.data_ptr(), probe.numel(), table.data_ptr(), table.numel(),
                              counts.data_ptr(), _stream_handle(stream))
    if st != 0:
        raise CdlError(st)
    return counts[:probe.numel()]


def exclusive_scan(counts, stream=None):
    torch = _torch()
    counts = _u32(counts)
    n = counts.numel()
    out = torch.empty(max(1, n), dtype=torch.int64, device=counts.device)
    L, s = lib(), _stream_handle(stream)
    total = ctypes.c_uint64()
    need = ctypes.c_size_t(0)
    st = L.cdl_exclusive_scan(counts.data_ptr(), n, out.data_ptr(), ctypes.byref(total), None,
                              ctypes.byref(need), s)
    if st != 0:
        raise CdlError(st)
    ws = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device=counts.device)
    st = L.cdl_exclusive_scan(counts.data_ptr(), n, out.data_ptr(), ctypes.byref(total),
                              ws.data_ptr(), ctypes.byref(need), s)
    if st != 0:
        raise CdlError(st)
    return out[:n], int(total.value)


def join(probe_cols, probe_key, build_cols, build_key, spec, neq=(), out_cap=None, stream=None):
    """Step (b): the full three-pass join; spec / neq hold (side, v) pairs
    (side 0 probe column, 1 build column, 2 constant)."""
    torch = _torch()
    probe_cols = [_u32(c) for c in probe_cols]
    build_cols = [_u32(c) for c in build_cols]
    L, s = lib(), _stream_handle(stream)
    npr, nbu = probe_cols[0].numel(), build_cols[0].numel()
    sp = (ColRef * len(spec))(*[ColRef(a, b) for a, b in spec])
    flat = [x for pair in neq for x in pair]
    nq = (ColRef * max(1, len(flat)))(*[ColRef(a, b) for a, b in flat])
    n_out = ctypes.c_uint64()
    need = ctypes.c_size_t(0)
    args_head = (_ptrs(probe_cols), len(probe_cols), npr, probe_key, _ptrs(build_cols),
                 len(build_cols), nbu, build_key, sp, len(spec), nq, len(neq))
    st = L.cdl_join(*args_head, _ptrs([]), 0, ctypes.byref(n_out), None, ctypes.byref(need), s)
    if st != 0:
        raise CdlError(st)
    ws = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device="cuda")
    # size query: out_cap 0 reports the unfiltered size
    outs0 = [torch.empty(1, dtype=torch.int32, device="cuda") for _ in spec]
    st = L.cdl_join(*args_head, _ptrs(outs0), 0, ctypes.byref(n_out), ws.data_ptr(),
                    ctypes.byref(need), s)
    if st not in (0, -3):
        raise CdlError(st)
    total = int(n_out.value)
    cap = total if out_cap is None else out_cap
    outs = [torch.empty(max(1, cap), dtype=torch.int32, device="cuda") for _ in spec]
    st = L.cdl_join(*args_head, _ptrs(outs), cap, ctypes.byref(n_out), ws.data_ptr(),
                    ctypes.byref(need), s)
    if st != 0:
        raise CdlError(st)
    return [o[:n_out.value] for o in outs]


def sort_unique(cols, stream=None):
    """Step (c): sorted unique tuples of the given columns."""
    torch = _torch()
    cols = [_u32(c) for c in cols]
    L, s = lib(), _stream_handle(stream)
    n = cols[0].numel()
    outs = [torch.empty(max(1, n), dtype=torch.int32, device="cuda") for _ in cols]
    n_out = ctypes.c_uint64()
    need = ctypes.c_size_t(0)
    st = L.cdl_sort_unique(_ptrs(cols), len(cols), n, _ptrs(outs), ctypes.byref(n_out), None,
                           ctypes.byref(need), s)
    if st != 0:
        raise CdlError(st)
    ws = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device="cuda")
    st = L.cdl_sort_unique(_ptrs(cols), len(cols), n, _ptrs(outs), ctypes.byref(n_out),
                           ws.data_ptr(), ctypes.byref(need), s)
    if st != 0:
        raise CdlError(st)
    return [o[:n_out.value] for o in outs]


def diff_merge(full_cols, fresh_cols, stream=None):
    """Step (d): (delta, merged) for sorted unique full and sorted fresh."""
    torch = _torch()
    full_cols = [_u32(c) for c in full_cols]
    fresh_cols = [_u32(c) for c in fresh_cols]
    L, s = lib(), _stream_handle(stream)
    nf, nu, k = full_cols[0].numel(), fresh_cols[0].numel(), len(full_cols)
    delta = [torch.empty(max(1, nu), dtype=torch.int32, device="cuda") for _ in range(k)]
    merged = [torch.empty(max(1, nf + nu), dtype=torch.int32, device="cuda") for _ in range(k)]
    nd = ctypes.c_uint64()
    need = ctypes.c_size_t(0)
    args = (_ptrs(full_cols), nf, _ptrs(fresh_cols), nu, k, _ptrs(delta), ctypes.byref(nd),
            _ptrs(merged))
    st = L.cdl_diff_merge(*args, None, ctypes.byref(need), s)
    if st != 0:
        raise CdlError(st)
    ws = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device="cuda")
    st = L.cdl_diff_merge(*args, ws.data_ptr(), ctypes.byref(need), s)
    if st != 0:
        raise CdlError(st)
    d = int(nd.value)
    return [x[:d] for x in delta], [x[:nf + d] for x in merged]


def _f32(t):
    torch = _torch()
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA float32 tensor")
    return t


def mlp_forward(params, X, stream=None):
    """FP32 forward of the join-size network: params (5313,), X (n, 16)."""
    torch = _torch()
    params, X = _f32(params), _f32(X)
    n = X.shape[0]
    out = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    ws, need = _workspace(lambda w, nb: lib().cdl_mlp_forward(params.data_ptr(), X.data_ptr(), n,
                                                               out.data_ptr(), w, nb,
                                                               _stream_handle(stream)))
    st = lib().cdl_mlp_forward(params.data_ptr(), X.data_ptr(), n, out.data_ptr(), ws.data_ptr(),
                               ctypes.byref(need), _stream_handle(stream))
    if st != 0:
        raise CdlError(st)
    return out[:n]


def mlp_gradient(params, X, y, tau=0.9, stream=None):
    """FP32 forward + backward: (predictions, d mean pinball loss / d params)."""
    torch = _torch()
    params, X, y = _f32(params), _f32(X), _f32(y)
    n = X.shape[0]
    out = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    args = (params.data_ptr(), X.data_ptr(), y.data_ptr(), n, tau, out.data_ptr(), grad.data_ptr())
    ws, need = _workspace(lambda w, nb: lib().cdl_mlp_gradient(*args, w, nb, _stream_handle(stream)))
    st = lib().cdl_mlp_gradient(*args, ws.data_ptr(), ctypes.byref(need), _stream_handle(stream))
    if st != 0:
        raise CdlError(st)
    return out[:n], grad


def mlp_infer_bf16(params, X, stream=None):
    """The engine's prediction path: BF16 weights / activations, FP32 sums."""
    torch = _torch()
    params, X = _f32(params), _f32(X)
    n = X.shape[0]
    out = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    args = (params.data_ptr(), X.data_ptr(), n, out.data_ptr())
    ws, need = _workspace(lambda w, nb: lib().cdl_mlp_infer_bf16(*args, w, nb, _stream_handle(stream)))
    st = lib().cdl_mlp_infer_bf16(*args, ws.data_ptr(), ctypes.byref(need), _stream_handle(stream))
    if st != 0:
        raise CdlError(st)
    return out[:n]


def mlp_adam(params, grad, m, v, step, lr, stream=None):
    """One Adam step in place on CUDA float32 tensors of CDL_MLP_PARAMS values."""
    for t in (params, grad, m, v):
        _f32(t)
    st = lib().cdl_mlp_adam(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), step,
                            lr, _stream_handle(stream))
    if st != 0:
        raise CdlError(st)


def join_features(probe, build, host, stream=None):
    """The estimator's 16 features of a join: probe / build are lists of one
    or two CUDA key columns (int32 tensors, uint32 bit patterns); host the 6
    host values.  Returns a CUDA float32 tensor of 16."""
    torch = _torch()
    for t in list(probe) + list(build):
        _u32(t)
    out = torch.empty(MLP_IN, dtype=torch.float32, device=probe[0].device)
    h = (ctypes.c_float * 6)(*[float(x) for x in host])
    p1 = probe[1].data_ptr() if len(probe) > 1 else None
    b1 = build[1].data_ptr() if len(build) > 1 else None
    st = lib().cdl_join_features(probe[0].data_ptr(), p1, probe[0].numel(), build[0].data_ptr(),
                                 b1, build[0].numel(), h, out.data_ptr(), _stream_handle(stream))
    if st != 0:
        raise CdlError(st)
    return out
