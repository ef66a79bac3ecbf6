"""Python binding of libhisa.so (include/hisa.h, include/hisa_prims.h).

Argument marshalling only: every step of evaluation runs in the CUDA library.
PyTorch supplies device memory (its caching allocator, through the library's
allocator hooks) and the CUDA stream.  Importing works without a GPU; any call
that needs the library raises if libhisa.so is missing or cannot run -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhisa.so")

HISA_OK = 0
FLAG_GRAPH = 1
FLAG_PHASE_TIMES = 2
FLAG_LOG_FULL = 4
FLAG_NO_DENSE = 8
FLAG_HASH_INDEX = 16
FLAG_NO_CHAIN = 32
FLAG_NO_PULL = 64
FLAG_LEVELS = 128
FLAG_NO_BITJOIN = 256

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Config(ctypes.Structure):
    _fields_ = [
        ("alloc", _ALLOC_FN),
        ("free", _FREE_FN),
        ("user", ctypes.c_void_p),
        ("cuda_stream", ctypes.c_void_p),
        ("hbm_budget_bytes", ctypes.c_uint64),
        ("load_factor", ctypes.c_float),
        ("ebm_k", ctypes.c_float),
        ("max_iters", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("device", ctypes.c_int32),
        ("pull_ratio", ctypes.c_float),
        ("radix_items", ctypes.c_uint32),
        ("dense_unit", ctypes.c_uint32),
    ]


class Atom(ctypes.Structure):
    _fields_ = [("rel", ctypes.c_uint32), ("var", ctypes.c_uint32 * 2)]


class Rule(ctypes.Structure):
    _fields_ = [
        ("head", Atom),
        ("n_body", ctypes.c_uint32),
        ("body", Atom * 3),
        ("n_neq", ctypes.c_uint32),
        ("neq", (ctypes.c_uint32 * 2) * 2),
    ]


class RunStats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_uint32),
        ("iterations_run", ctypes.c_uint32),
        ("regrows", ctypes.c_uint32),
        ("graph_launches", ctypes.c_uint32),
        ("ms_total", ctypes.c_double),
        ("ms_edb", ctypes.c_double),
        ("ms_join", ctypes.c_double),
        ("ms_sort", ctypes.c_double),
        ("ms_merge", ctypes.c_double),
        ("tuples_joined", ctypes.c_uint64),
        ("peak_bytes", ctypes.c_uint64),
        ("kernel_launches", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServeStats(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_uint32), ("retired", ctypes.c_uint32), ("active", ctypes.c_uint32),
                ("pending", ctypes.c_uint32), ("iterations", ctypes.c_uint32),
                ("ms_admit", ctypes.c_double), ("ms_iterate", ctypes.c_double), ("ms_rows", ctypes.c_double),
                ("ms_retire", ctypes.c_double), ("ms_compact", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


# entry point -> (restype, argtypes); the complete list of include/*.h declarations
_P = ctypes.c_void_p
_U32P = ctypes.POINTER(ctypes.c_uint32)
_U64P = ctypes.POINTER(ctypes.c_uint64)
SIGNATURES = {
    "hisa_config_default": (ctypes.c_int32, [ctypes.POINTER(Config)]),
    "hisa_create": (ctypes.c_int32, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]),
    "hisa_destroy": (ctypes.c_int32, [_P]),
    "hisa_declare_relation": (ctypes.c_int32, [_P, ctypes.c_char_p, ctypes.c_uint32, ctypes.c_int, _U32P]),
    "hisa_load_tuples": (ctypes.c_int32, [_P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint64,
                                          ctypes.c_int]),
    "hisa_add_rule": (ctypes.c_int32, [_P, ctypes.POINTER(Rule)]),
    "hisa_run": (ctypes.c_int32, [_P, ctypes.POINTER(RunStats)]),
    "hisa_reset_edb": (ctypes.c_int32, [_P]),
    "hisa_relation_size": (ctypes.c_int32, [_P, ctypes.c_uint32, _U64P]),
    "hisa_read_relation": (ctypes.c_int32, [_P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint64,
                                            _U64P, ctypes.c_int]),
    "hisa_delta_counts": (ctypes.c_int32, [_P, ctypes.c_uint32, _U64P, ctypes.c_uint32, _U32P]),
    "hisa_load_instance": (ctypes.c_int32, [_P, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.c_uint64, ctypes.c_int]),
    "hisa_instance_size": (ctypes.c_int32, [_P, ctypes.c_uint32, ctypes.c_uint32, _U64P]),
    "hisa_read_instance": (ctypes.c_int32, [_P, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.c_uint64, _U64P, ctypes.c_int]),
    "hisa_instance_delta_counts": (ctypes.c_int32, [_P, ctypes.c_uint32, ctypes.c_uint32, _U64P, ctypes.c_uint32,
                                                    _U32P]),
    "hisa_serve_open": (ctypes.c_int32, [_P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]),
    "hisa_serve_submit": (ctypes.c_int32, [_P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint64,
                                           _U64P]),
    "hisa_serve_step": (ctypes.c_int32, [_P, ctypes.c_uint32, ctypes.POINTER(ServeStats)]),
    "hisa_serve_poll": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
    "hisa_serve_retired": (ctypes.c_int32, [_P, _P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "hisa_serve_result": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.c_uint64, _U64P, _U64P, ctypes.c_uint32, _U32P, ctypes.c_int]),
    "hisa_serve_release": (ctypes.c_int32, [_P, ctypes.c_uint64]),
    "hisa_kernel_stats": (ctypes.c_int32, [_P, ctypes.POINTER(KernelStat), ctypes.c_uint32, _U32P]),
    "hisa_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "hisa_last_error": (ctypes.c_char_p, [_P]),
    "hisa_sort_codes": (ctypes.c_int32, [_P, _P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _P]),
    "hisa_sort_unique_codes": (ctypes.c_int32, [_P, _P, ctypes.c_uint64, _U64P, ctypes.c_int, ctypes.c_int, _P]),
    "hisa_difference_merge": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, ctypes.c_uint64, _P, ctypes.c_uint64, _P,
                                               ctypes.c_uint64, _U64P, ctypes.c_int, _P]),
    "hisa_difference_merge_noalloc": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, ctypes.c_uint64, _P,
                                                       ctypes.c_uint64, _P, ctypes.c_uint64, _U64P, ctypes.c_int,
                                                       _P]),
    "hisa_check_bounded_wait": (ctypes.c_int32, [ctypes.c_int, ctypes.c_uint32, _P]),
    "hisa_column_max": (ctypes.c_int32, [_P, _P, ctypes.c_uint64, _U32P, _P]),
    "hisa_encode_codes": (ctypes.c_int32, [_P, _P, ctypes.c_uint64, ctypes.c_int, _P, ctypes.c_int, _P]),
    "hisa_decode_codes": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "hisa_partition_codes": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_uint32, _P, _U64P, _P]),
    "hisa_join_codes": (ctypes.c_int32, [_P, ctypes.c_uint64, _P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_uint64, _U64P,
                                         ctypes.c_int, _P]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libhisa.so (built by ``paper_2311_02206_gb300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_2311_02206_gb300.build.build() first "
                               "(the CUDA library is required; there is no CPU path)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class HisaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hisa status {status}: {msg}")
        self.status = status


def _check(rc: int, ctx=None):
    if rc < 0:
        lib = load_library()
        detail = lib.hisa_status_string(rc).decode()
        if ctx is not None:
            extra = lib.hisa_last_error(ctx).decode()
            if extra:
                detail += f" ({extra})"
        raise HisaError(rc, detail)
    return rc


def _torch():
    import torch
    return torch


class Context:
    """One engine instance on one CUDA device and stream (include/hisa.h)."""

    def __init__(self, device: int = 0, stream=None, flags: int = FLAG_GRAPH | FLAG_LOG_FULL, max_iters: int = 0,
                 load_factor: float = 0.0, ebm_k: float = 0.0, hbm_budget_bytes: int = 0,
                 torch_allocator: bool = True, allocator=None, pull_ratio: float = 0.0, radix_items: int = 0,
                 dense_unit: int = 0):
        """``allocator``: optional pair (alloc, free) of Python callables,
        alloc(nbytes, stream) -> device pointer or None, free(ptr, nbytes,
        stream), used in place of torch's caching allocator."""
        lib = load_library()
        torch = _torch()
        self._lib = lib
        self.device = device
        cfg = Config()
        _check(lib.hisa_config_default(ctypes.byref(cfg)))
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self._stream = stream
        cfg.cuda_stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        cfg.device = device
        cfg.flags = flags
        cfg.max_iters = max_iters
        cfg.load_factor = load_factor
        cfg.ebm_k = ebm_k
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.pull_ratio = pull_ratio
        cfg.radix_items = radix_items
        cfg.dense_unit = dense_unit
        if allocator is not None:
            user_alloc, user_free = allocator

            def _alloc(nbytes, strm, user):
                try:
                    return user_alloc(int(nbytes), int(strm or 0))
                except Exception:
                    return None

            def _free(ptr, nbytes, strm, user):
                user_free(int(ptr), int(nbytes), int(strm or 0))

            self._alloc_cb = _ALLOC_FN(_alloc)
            self._free_cb = _FREE_FN(_free)
            cfg.alloc = self._alloc_cb
            cfg.free = self._free_cb
        elif torch_allocator:
            def _alloc(nbytes, strm, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(strm or 0))
                except Exception:   # out of memory: the library reports HISA_ERR_OOM
                    return None

            def _free(ptr, nbytes, strm, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._alloc_cb = _ALLOC_FN(_alloc)
            self._free_cb = _FREE_FN(_free)
            cfg.alloc = self._alloc_cb
            cfg.free = self._free_cb
        self._cfg = cfg
        h = ctypes.c_void_p()
        _check(lib.hisa_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.rel_ids: dict[str, int] = {}

    # -- lifecycle --
    def close(self):
        if getattr(self, "_h", None):
            self._lib.hisa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- program --
    def declare_relation(self, name: str, arity: int = 2, idb: bool = False) -> int:
        rid = ctypes.c_uint32()
        _check(self._lib.hisa_declare_relation(self._h, name.encode(), arity, int(idb), ctypes.byref(rid)), self._h)
        self.rel_ids[name] = rid.value
        return rid.value

    def load_tuples(self, rel, c0, c1):
        """Appends tuples; c0/c1 are numpy uint32 arrays (host) or torch uint32/int32
        CUDA tensors (device)."""
        rid = self.rel_ids[rel] if isinstance(rel, str) else rel
        torch = _torch()
        if isinstance(c0, torch.Tensor):
            c0 = c0.contiguous()
            c1 = c1.contiguous()
            assert c0.is_cuda and c0.element_size() == 4 and c0.numel() == c1.numel()
            ptrs = (ctypes.c_void_p * 2)(c0.data_ptr(), c1.data_ptr())
            _check(self._lib.hisa_load_tuples(self._h, rid, ptrs, c0.numel(), 1), self._h)
        else:
            c0 = np.ascontiguousarray(c0, dtype=np.uint32)
            c1 = np.ascontiguousarray(c1, dtype=np.uint32)
            assert len(c0) == len(c1)
            ptrs = (ctypes.c_void_p * 2)(c0.ctypes.data, c1.ctypes.data)
            _check(self._lib.hisa_load_tuples(self._h, rid, ptrs, len(c0), 0), self._h)

    def add_rule(self, head, body, neq=()):
        """head/body atoms as (relation, (var, var)); variables are any hashable
        names (mapped to ids 0..15 in order of first use); neq: pairs of vars."""
        names: dict = {}

        def vid(v):
            if v not in names:
                names[v] = len(names)
            return names[v]

        r = Rule()
        for i, (rel, (a, b)) in enumerate(body):
            r.body[i].rel = self.rel_ids[rel]
            r.body[i].var[0] = vid(a)
            r.body[i].var[1] = vid(b)
        r.n_body = len(body)
        r.head.rel = self.rel_ids[head[0]]
        r.head.var[0] = vid(head[1][0])
        r.head.var[1] = vid(head[1][1])
        r.n_neq = len(neq)
        for i, (a, b) in enumerate(neq):
            r.neq[i][0] = vid(a)
            r.neq[i][1] = vid(b)
        _check(self._lib.hisa_add_rule(self._h, ctypes.byref(r)), self._h)

    def program(self, relations: dict, rules: Iterable):
        """Declares ``relations`` (name -> "edb"/"idb") and adds ``rules``
        ((head, body, neq) tuples)."""
        for name, kind in relations.items():
            self.declare_relation(name, 2, kind == "idb")
        for head, body, neq in rules:
            self.add_rule(head, body, neq)

    def run(self) -> RunStats:
        st = RunStats()
        _check(self._lib.hisa_run(self._h, ctypes.byref(st)), self._h)
        return st

    def reset_edb(self):
        _check(self._lib.hisa_reset_edb(self._h), self._h)

    # -- results --
    def relation_size(self, rel) -> int:
        rid = self.rel_ids[rel] if isinstance(rel, str) else rel
        n = ctypes.c_uint64()
        _check(self._lib.hisa_relation_size(self._h, rid, ctypes.byref(n)), self._h)
        return n.value

    def read_relation(self, rel, device: bool = False, out=None):
        """Returns (c0, c1) in lexicographic order: numpy uint32 arrays, or torch
        int32 CUDA tensors (the uint32 bit patterns) when ``device``.  ``out``
        may give two preallocated host arrays (e.g. pinned) to fill."""
        rid = self.rel_ids[rel] if isinstance(rel, str) else rel
        n = self.relation_size(rid)
        got = ctypes.c_uint64()
        if out is not None:
            c0, c1 = out
            assert len(c0) >= n and len(c1) >= n and c0.dtype.itemsize == 4
            ptrs = (ctypes.c_void_p * 2)(c0.ctypes.data, c1.ctypes.data)
            _check(self._lib.hisa_read_relation(self._h, rid, ptrs, min(len(c0), len(c1)), ctypes.byref(got), 0),
                   self._h)
            return c0[:n], c1[:n]
        if device:
            torch = _torch()
            c0 = torch.empty(max(n, 1), dtype=torch.int32, device=f"cuda:{self.device}")
            c1 = torch.empty(max(n, 1), dtype=torch.int32, device=f"cuda:{self.device}")
            ptrs = (ctypes.c_void_p * 2)(c0.data_ptr(), c1.data_ptr())
            _check(self._lib.hisa_read_relation(self._h, rid, ptrs, n, ctypes.byref(got), 1), self._h)
            return c0[:n], c1[:n]
        c0 = np.empty(max(n, 1), np.uint32)
        c1 = np.empty(max(n, 1), np.uint32)
        ptrs = (ctypes.c_void_p * 2)(c0.ctypes.data, c1.ctypes.data)
        _check(self._lib.hisa_read_relation(self._h, rid, ptrs, n, ctypes.byref(got), 0), self._h)
        return c0[:n], c1[:n]

    # -- batched instances --
    def load_instance(self, rel, instance: int, c0, c1):
        rid = self.rel_ids[rel] if isinstance(rel, str) else rel
        c0 = np.ascontiguousarray(c0, dtype=np.uint32)
        c1 = np.ascontiguousarray(c1, dtype=np.uint32)
        ptrs = (ctypes.c_void_p * 2)(c0.ctypes.data, c1.ctypes.data)
        _check(self._lib.hisa_load_instance(self._h, rid, instance, ptrs, len(c0), 0), self._h)

    def instance_size(self, rel, instance: int) -> int:
        rid = self.rel_ids[rel] if isinstance(rel, str) else rel
        n = ctypes.c_uint64()
        _check(self._lib.hisa_instance_size(self._h, rid, instance, ctypes.byref(n)), self._h)
        return n.value

    def read_instance(self, rel, instance: int):
        rid = self.rel_ids[rel] if isinstance(rel, str) else rel
        n = self.instance_size(rid, instance)
        c0 = np.empty(max(n, 1), np.uint32)
        c1 = np.empty(max(n, 1), np.uint32)
        got = ctypes.c_uint64()
        ptrs = (ctypes.c_void_p * 2)(c0.ctypes.data, c1.ctypes.data)
        _check(self._lib.hisa_read_instance(self._h, rid, instance, ptrs, n, ctypes.byref(got), 0), self._h)
        return c0[:n], c1[:n]

    def instance_delta_counts(self, rel, instance: int) -> list:
        rid = self.rel_ids[rel] if isinstance(rel, str) else rel
        k = ctypes.c_uint32()
        self._lib.hisa_instance_delta_counts(self._h, rid, instance, None, 0, ctypes.byref(k))
        out = (ctypes.c_uint64 * max(k.value, 1))()
        _check(self._lib.hisa_instance_delta_counts(self._h, rid, instance, out, k.value, ctypes.byref(k)), self._h)
        return [int(out[i]) for i in range(k.value)]

    # -- serving --
    def serve_open(self, max_instances: int, max_value: int, budget_bytes: int = 0):
        _check(self._lib.hisa_serve_open(self._h, max_instances, max_value, budget_bytes), self._h)

    def serve_submit(self, rel, c0, c1) -> int:
        rid = self.rel_ids[rel] if isinstance(rel, str) else rel
        c0 = np.ascontiguousarray(c0, dtype=np.uint32)
        c1 = np.ascontiguousarray(c1, dtype=np.uint32)
        ptrs = (ctypes.c_void_p * 2)(c0.ctypes.data, c1.ctypes.data)
        t = ctypes.c_uint64()
        _check(self._lib.hisa_serve_submit(self._h, rid, ptrs, len(c0), ctypes.byref(t)), self._h)
        return t.value

    def serve_step(self, max_iterations: int = 1) -> dict:
        st = ServeStats()
        _check(self._lib.hisa_serve_step(self._h, max_iterations, ctypes.byref(st)), self._h)
        return st.as_dict()

    def serve_retired(self) -> list:
        """Tickets retired by the latest serve_step, in slot order."""
        n = ctypes.c_uint32()
        _check(self._lib.hisa_serve_retired(self._h, None, 0, ctypes.byref(n)), self._h)
        buf = (ctypes.c_uint64 * max(n.value, 1))()
        _check(self._lib.hisa_serve_retired(self._h, ctypes.cast(buf, ctypes.c_void_p), n.value, ctypes.byref(n)),
               self._h)
        return [int(buf[i]) for i in range(n.value)]

    def serve_poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(self._lib.hisa_serve_poll(self._h, ticket, ctypes.byref(d)), self._h)
        return bool(d.value)

    def serve_result(self, ticket: int, rel, device: bool = False):
        """(c0, c1, delta_counts) of a completed request for IDB relation ``rel``:
        numpy uint32 arrays, or int32 CUDA tensors when ``device``."""
        rid = self.rel_ids[rel] if isinstance(rel, str) else rel
        n = ctypes.c_uint64()
        k = ctypes.c_uint32()
        self._lib.hisa_serve_result(self._h, ticket, rid, None, 0, ctypes.byref(n), None, 0, ctypes.byref(k), 0)
        dl = (ctypes.c_uint64 * max(k.value, 1))()
        if device:
            torch = _torch()
            c0 = torch.empty(max(n.value, 1), dtype=torch.int32, device=f"cuda:{self.device}")
            c1 = torch.empty(max(n.value, 1), dtype=torch.int32, device=f"cuda:{self.device}")
            ptrs = (ctypes.c_void_p * 2)(c0.data_ptr(), c1.data_ptr())
        else:
            c0 = np.empty(max(n.value, 1), np.uint32)
            c1 = np.empty(max(n.value, 1), np.uint32)
            ptrs = (ctypes.c_void_p * 2)(c0.ctypes.data, c1.ctypes.data)
        _check(self._lib.hisa_serve_result(self._h, ticket, rid, ptrs, n.value, ctypes.byref(n), dl, k.value,
                                           ctypes.byref(k), 1 if device else 0), self._h)
        return c0[:n.value], c1[:n.value], [int(dl[i]) for i in range(k.value)]

    def serve_release(self, ticket: int):
        _check(self._lib.hisa_serve_release(self._h, ticket), self._h)

    def kernel_stats(self) -> list:
        """Per-kernel launches, device ms and algorithmic bytes of the last run
        made with FLAG_PHASE_TIMES."""
        n = ctypes.c_uint32()
        _check(self._lib.hisa_kernel_stats(self._h, None, 0, ctypes.byref(n)), self._h)
        arr = (KernelStat * max(n.value, 1))()
        _check(self._lib.hisa_kernel_stats(self._h, arr, n.value, ctypes.byref(n)), self._h)
        return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "ms": arr[i].ms,
                 "bytes": arr[i].bytes} for i in range(n.value)]

    def delta_counts(self, rel) -> list:
        rid = self.rel_ids[rel] if isinstance(rel, str) else rel
        k = ctypes.c_uint32()
        self._lib.hisa_delta_counts(self._h, rid, None, 0, ctypes.byref(k))
        out = (ctypes.c_uint64 * max(k.value, 1))()
        _check(self._lib.hisa_delta_counts(self._h, rid, out, k.value, ctypes.byref(k)), self._h)
        return [int(out[i]) for i in range(k.value)]


# ---- primitives (include/hisa_prims.h) on torch CUDA tensors -----------------------------

def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _kb(t):
    return t.element_size()


def sort_codes(codes, key_bits: int = 0, stream=None):
    """Ascending sort of a 1-D int32/int64 CUDA tensor of codes (unsigned order)."""
    torch = _torch()
    out = torch.empty_like(codes)
    _check(load_library().hisa_sort_codes(codes.data_ptr(), out.data_ptr(), codes.numel(), _kb(codes), key_bits,
                                          _stream_ptr(stream)))
    return out


def sort_unique_codes(codes, key_bits: int = 0, stream=None):
    torch = _torch()
    out = torch.empty_like(codes)
    n = ctypes.c_uint64()
    _check(load_library().hisa_sort_unique_codes(codes.data_ptr(), out.data_ptr(), codes.numel(), ctypes.byref(n),
                                                 _kb(codes), key_bits, _stream_ptr(stream)))
    return out[:n.value]


def difference_merge(full, fresh, with_full: bool = True, stream=None):
    """(delta, full') for sorted distinct ``full`` and sorted ``fresh`` codes."""
    torch = _torch()
    d = torch.empty(max(fresh.numel(), 1), dtype=fresh.dtype, device=fresh.device)
    f = torch.empty(max(full.numel() + fresh.numel(), 1), dtype=fresh.dtype, device=fresh.device) if with_full else None
    n = ctypes.c_uint64()
    _check(load_library().hisa_difference_merge(
        full.data_ptr() if full.numel() else None, full.numel(), fresh.data_ptr() if fresh.numel() else None,
        fresh.numel(), d.data_ptr(), d.numel(), f.data_ptr() if f is not None else None,
        f.numel() if f is not None else 0, ctypes.byref(n), _kb(fresh), _stream_ptr(stream)))
    nd = n.value
    return d[:nd], (f[:full.numel() + nd] if f is not None else None)


NOALLOC_MAX_CODES = 1 << 26
HISA_ERR_TOO_LARGE = -10


def difference_merge_noalloc(full, fresh, delta_out, full_out=None, stream=None):
    """hisa_difference_merge_noalloc on caller-provided outputs (the library
    allocates nothing); returns (delta, full') views of the outputs."""
    n = ctypes.c_uint64()
    _check(load_library().hisa_difference_merge_noalloc(
        full.data_ptr() if full.numel() else None, full.numel(), fresh.data_ptr() if fresh.numel() else None,
        fresh.numel(), delta_out.data_ptr(), delta_out.numel(),
        full_out.data_ptr() if full_out is not None else None, full_out.numel() if full_out is not None else 0,
        ctypes.byref(n), _kb(fresh), _stream_ptr(stream)))
    nd = n.value
    return delta_out[:nd], (full_out[:full.numel() + nd] if full_out is not None else None)


def join_codes(outer, inner, b: int, outer_col: int, proj0: int, proj1: int, neq: int = 0, stream=None):
    """Results of Algorithm 3 as codes (outer order, run order inside an outer)."""
    torch = _torch()
    lib = load_library()
    n = ctypes.c_uint64()
    cap = max(outer.numel(), 1)
    for _ in range(2):
        out = torch.empty(cap, dtype=outer.dtype, device=outer.device)
        rc = lib.hisa_join_codes(outer.data_ptr() if outer.numel() else None, outer.numel(),
                                 inner.data_ptr() if inner.numel() else None, inner.numel(), b, outer_col, proj0,
                                 proj1, neq, out.data_ptr(), cap, ctypes.byref(n), _kb(outer), _stream_ptr(stream))
        if rc == -9:   # HISA_ERR_CAPACITY: n holds the size
            cap = max(n.value, 1)
            continue
        _check(rc)
        return out[:n.value]
    raise HisaError(-9, "join output did not fit")


def check_bounded_wait(which: int, spin_limit: int = 64, stream=None) -> int:
    """hisa_check_bounded_wait: the status of one bounded device-side wait run
    on a word that nothing publishes (HISA_ERR_DEVICE_TIMEOUT, -5, expected)."""
    return int(load_library().hisa_check_bounded_wait(which, spin_limit, _stream_ptr(stream)))


def encode_codes(c0, c1, b: int, wide: bool = False, stream=None):
    """Two int32 CUDA tensors (uint32 bit patterns) -> codes (c0 << b) | c1
    (int32, or int64 when ``wide``)."""
    torch = _torch()
    out = torch.empty(max(c0.numel(), 1), dtype=torch.int64 if wide else torch.int32, device=c0.device)
    _check(load_library().hisa_encode_codes(c0.data_ptr() if c0.numel() else None,
                                            c1.data_ptr() if c1.numel() else None, c0.numel(), b,
                                            out.data_ptr(), 8 if wide else 4, _stream_ptr(stream)))
    return out[:c0.numel()]


def decode_codes(codes, b: int, stream=None):
    """Codes -> (c0, c1) int32 CUDA tensors."""
    torch = _torch()
    n = codes.numel()
    c0 = torch.empty(max(n, 1), dtype=torch.int32, device=codes.device)
    c1 = torch.empty(max(n, 1), dtype=torch.int32, device=codes.device)
    _check(load_library().hisa_decode_codes(codes.data_ptr() if n else None, n, b, c0.data_ptr(), c1.data_ptr(),
                                            _kb(codes), _stream_ptr(stream)))
    return c0[:n], c1[:n]


def partition_codes(codes, b: int, key_col: int, nparts: int, stream=None):
    """hisa_partition_codes: (codes grouped by owner, list of part sizes)."""
    torch = _torch()
    n = codes.numel()
    out = torch.empty(max(n, 1), dtype=codes.dtype, device=codes.device)
    counts = (ctypes.c_uint64 * nparts)()
    _check(load_library().hisa_partition_codes(codes.data_ptr() if n else None, n, _kb(codes), b, key_col, nparts,
                                               out.data_ptr(), counts, _stream_ptr(stream)))
    return out[:n], [int(counts[i]) for i in range(nparts)]


def column_max(c0, c1, stream=None) -> int:
    """Largest uint32 value of two int32 CUDA tensors (uint32 bit patterns)."""
    out = ctypes.c_uint32()
    n = c0.numel()
    _check(load_library().hisa_column_max(c0.data_ptr() if n else None, c1.data_ptr() if n else None, n,
                                          ctypes.byref(out), _stream_ptr(stream)))
    return int(out.value)
