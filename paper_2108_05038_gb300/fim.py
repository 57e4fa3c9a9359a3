"""Python binding of the C ABI in include/fim.h (argument marshalling only).

Every step of the mining path runs in libfimgpu.so; this module converts
numpy/torch buffers to pointers, calls the entry point of the same name and
turns the returned CSR arrays into numpy arrays.  There is no CPU fallback:
if the library cannot be built or loaded, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

FIM_OK, FIM_ERR_INVALID, FIM_ERR_OOM, FIM_ERR_OUTPUT_OVERFLOW, FIM_ERR_CUDA, FIM_ERR_TIMEOUT = range(6)
FIM_ORDER_ESTIMATE, FIM_ORDER_UNIFORM = 0, 1
FIM_DFS_NODES, FIM_DFS_FRAMES, FIM_DFS_AUTO, FIM_DFS_SPARSE, FIM_DFS_WARP, FIM_DFS_PROJECTED = 0, 1, 2, 3, 4, 5
FIM_OUTPUT_ALL, FIM_OUTPUT_CLOSED, FIM_OUTPUT_MAXIMAL = 0, 1, 2
FIM_PAIR_AUTO, FIM_PAIR_CORES, FIM_PAIR_TENSOR, FIM_PAIR_TENSOR_E4M3, FIM_PAIR_TENSOR_FUSED = 0, 1, 2, 3, 4
SAMPLE_ITEMSET_LIMIT = 1 << 20  # FIM_SAMPLE_ITEMSET_LIMIT

# every symbol declared in include/fim.h
EXPORTED = [
    "fim_mine_opts_init", "fim_build_vertical_db", "fim_build_vertical_db_device", "fim_db_info", "fim_db_rows",
    "fim_estimate_class_costs", "fim_estimate_class_costs_ex", "fim_estimate_sample_size", "fim_estimate_result", "fim_mine", "fim_result_view", "fim_result_free",
    "fim_db_free", "fim_status_str", "fim_last_error", "fim_mine_pairs_noalloc", "fim_autotune", "fim_plan_create",
    "fim_plan_launch", "fim_plan_result", "fim_plan_stream", "fim_plan_free", "fim_server_create",
    "fim_server_submit", "fim_server_wait", "fim_server_stats", "fim_server_free", "fim_kernel_launches",
    "fim_extension_supports", "fim_result_flags", "fim_pool_memory", "fim_server_wait_ex",
]


class FimError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


STATUS_NAMES = {0: "FIM_OK", 1: "FIM_ERR_INVALID", 2: "FIM_ERR_OOM", 3: "FIM_ERR_OUTPUT_OVERFLOW", 4: "FIM_ERR_CUDA",
                5: "FIM_ERR_TIMEOUT"}


class MineStats(ctypes.Structure):
    _fields_ = [
        ("n_frequent", ctypes.c_uint64), ("n_items_out", ctypes.c_uint64), ("n_frequent_items", ctypes.c_uint32),
        ("max_len", ctypes.c_uint32), ("n_intersections", ctypes.c_uint64), ("n_pair_intersections", ctypes.c_uint64),
        ("n_classes", ctypes.c_uint64), ("n_queue_entries", ctypes.c_uint64), ("n_donations", ctypes.c_uint64),
        ("bytes_algorithmic", ctypes.c_uint64), ("bytes_pair_kernel", ctypes.c_uint64),
        ("bytes_dfs_kernel", ctypes.c_uint64), ("words_per_row", ctypes.c_uint32), ("grid_ctas", ctypes.c_uint32),
        ("threads_per_cta", ctypes.c_uint32), ("vec_per_lane", ctypes.c_uint32), ("ms_pair_kernel", ctypes.c_float),
        ("ms_dfs_kernel", ctypes.c_float), ("ms_device_total", ctypes.c_float),
        ("dfs_cta_busy_max_ms", ctypes.c_float), ("dfs_cta_busy_mean_ms", ctypes.c_float), ("pair_kernel", ctypes.c_uint32),
        ("n_proj_classes", ctypes.c_uint32), ("n_proj_splits", ctypes.c_uint64), ("n_fallback_entries", ctypes.c_uint64),
        ("bytes_projected", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MineOpts(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("class_order", ctypes.c_uint32), ("dfs_mode", ctypes.c_uint32),
        ("threads_per_cta", ctypes.c_uint32), ("vec_per_lane", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
        ("donate", ctypes.c_uint32), ("result_on_device", ctypes.c_uint32), ("collect_times", ctypes.c_uint32),
        ("dfs_depth_first", ctypes.c_uint32), ("pair_kernel", ctypes.c_uint32), ("fault_pair_wait", ctypes.c_uint32),
        ("out_capacity_sets", ctypes.c_uint64),
        ("out_capacity_items", ctypes.c_uint64), ("spin_limit", ctypes.c_uint64), ("max_itemsets", ctypes.c_uint64),
        ("proj_bitmap_words", ctypes.c_uint64), ("proj_stack_words", ctypes.c_uint64),
        ("proj_max_row_words", ctypes.c_uint32), ("output", ctypes.c_uint32), ("diffsets", ctypes.c_uint32),
        ("proj_split_words", ctypes.c_uint32),
        ("out_needed_sets", ctypes.c_uint64),
        ("out_needed_items", ctypes.c_uint64), ("stats", ctypes.POINTER(MineStats)),
        ("class_work_out", ctypes.c_void_p),
    ]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load libfimgpu.so (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_stale and (not os.path.exists(_build.LIB) or _build.stale()):
            _build.build()
        if not os.path.exists(_build.LIB):
            raise FimError(FIM_ERR_CUDA, "load", f"{_build.LIB} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(_build.LIB)
        P, u32, u64, dbl = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        i32 = ctypes.c_int
        lib.fim_mine_opts_init.restype = None
        lib.fim_mine_opts_init.argtypes = [ctypes.POINTER(MineOpts)]
        for name in ("fim_build_vertical_db", "fim_build_vertical_db_device"):
            f = getattr(lib, name)
            f.restype = i32
            f.argtypes = [P, P, u32, u32, u32, u32, P, PP]
        lib.fim_db_info.restype = i32
        lib.fim_db_info.argtypes = [P] + [ctypes.POINTER(u32)] * 5 + [ctypes.POINTER(u64)]
        lib.fim_db_rows.restype = i32
        lib.fim_db_rows.argtypes = [P, P, P]
        lib.fim_estimate_class_costs.restype = i32
        lib.fim_estimate_class_costs.argtypes = [P, dbl, dbl, u64, P, P]
        lib.fim_estimate_class_costs_ex.restype = i32
        lib.fim_estimate_class_costs_ex.argtypes = [P, dbl, dbl, u64, u32, u64, P, P]
        lib.fim_estimate_sample_size.restype = i32
        lib.fim_estimate_sample_size.argtypes = [P, ctypes.POINTER(u64), ctypes.POINTER(u32), ctypes.POINTER(u32)]
        lib.fim_estimate_result.restype = i32
        lib.fim_estimate_result.argtypes = [P, P, P]
        lib.fim_mine.restype = i32
        lib.fim_mine.argtypes = [P, u32, ctypes.POINTER(MineOpts), PP]
        lib.fim_autotune.restype = i32
        lib.fim_autotune.argtypes = [P, u32, ctypes.POINTER(MineOpts), ctypes.POINTER(ctypes.c_float)]
        lib.fim_plan_create.restype = i32
        lib.fim_plan_create.argtypes = [P, u32, ctypes.POINTER(MineOpts), PP]
        lib.fim_plan_launch.restype = i32
        lib.fim_plan_launch.argtypes = [P]
        lib.fim_plan_result.restype = i32
        lib.fim_plan_result.argtypes = [P, ctypes.POINTER(MineOpts), PP]
        lib.fim_plan_stream.restype = i32
        lib.fim_plan_stream.argtypes = [P, PP]
        lib.fim_plan_free.restype = None
        lib.fim_plan_free.argtypes = [P]
        lib.fim_server_create.restype = i32
        lib.fim_server_create.argtypes = [u64, u32, u32, u64, PP]
        lib.fim_server_submit.restype = i32
        lib.fim_server_submit.argtypes = [P, P, P, u32, u32, u32, dbl, ctypes.POINTER(u64)]
        lib.fim_server_wait.restype = i32
        lib.fim_server_wait.argtypes = [P, u64, PP, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
        lib.fim_server_wait_ex.restype = i32
        lib.fim_server_wait_ex.argtypes = [P, u64, PP, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                           ctypes.POINTER(dbl)]
        lib.fim_server_stats.restype = i32
        lib.fim_server_stats.argtypes = [P, ctypes.POINTER(u64), ctypes.POINTER(u32), ctypes.POINTER(u32),
                                         ctypes.POINTER(u64)]
        lib.fim_server_free.restype = None
        lib.fim_server_free.argtypes = [P]
        lib.fim_mine_pairs_noalloc.restype = i32
        lib.fim_mine_pairs_noalloc.argtypes = [P, u32, P, P, u64, ctypes.POINTER(u64)]
        lib.fim_result_flags.restype = i32
        lib.fim_result_flags.argtypes = [P, P]
        lib.fim_extension_supports.restype = i32
        lib.fim_extension_supports.argtypes = [P, P, u32, P, u32, P]
        lib.fim_result_view.restype = i32
        lib.fim_result_view.argtypes = [P, ctypes.POINTER(u64), PP, PP, PP, ctypes.POINTER(i32)]
        lib.fim_result_free.restype = None
        lib.fim_result_free.argtypes = [P]
        lib.fim_db_free.restype = None
        lib.fim_db_free.argtypes = [P]
        lib.fim_status_str.restype = ctypes.c_char_p
        lib.fim_status_str.argtypes = [i32]
        lib.fim_last_error.restype = ctypes.c_char_p
        lib.fim_last_error.argtypes = []
        lib.fim_kernel_launches.restype = u64
        lib.fim_kernel_launches.argtypes = []
        lib.fim_pool_memory.restype = i32
        lib.fim_pool_memory.argtypes = [i32, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        _lib = lib
        return lib


def _check(lib, status: int, where: str):
    if status != FIM_OK:
        raise FimError(status, where, lib.fim_last_error().decode(errors="replace"))


def _ptr(x):
    """Address of a numpy array, a torch tensor, or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class _HostResult:
    """Owns the C result of a host result: its arrays are views of the result's pinned memory, which is
    released (fim_result_free) only when the last of them, and the Result, are gone."""

    def __init__(self, lib, handle):
        self.lib, self.h = lib, handle

    def view(self, ctype, addr, n):
        buf = (ctype * n).from_address(addr)
        buf._owner = self  # the buffer, and so every array made from it, keeps the result alive
        return np.frombuffer(buf, dtype=np.dtype(ctype))

    def __del__(self):
        try:
            self.lib.fim_result_free(self.h)
        except Exception:
            pass


class Result:
    """Frequent itemsets in CSR form; numpy arrays for host results (views of the result's own pinned
    host memory, valid for as long as they are referenced)."""

    def __init__(self, lib, handle, stats: MineStats | None):
        self._lib, self._h = lib, handle
        self._owner = None
        self._flags = None
        n = ctypes.c_uint64()
        po, pi, ps = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        dev = ctypes.c_int()
        _check(lib, lib.fim_result_view(handle, ctypes.byref(n), ctypes.byref(po), ctypes.byref(pi), ctypes.byref(ps),
                                        ctypes.byref(dev)), "fim_result_view")
        self.n_sets = n.value
        self.on_device = bool(dev.value)
        self.stats = stats.as_dict() if stats is not None else None
        self.device_ptrs = (po.value, pi.value, ps.value) if self.on_device else None
        if not self.on_device:
            own = _HostResult(lib, handle)
            off = own.view(ctypes.c_uint64, po.value, self.n_sets + 1)
            n_items = int(off[-1]) if self.n_sets else 0
            items = own.view(ctypes.c_uint32, pi.value, n_items) if n_items else np.zeros(0, dtype=np.uint32)
            supp = own.view(ctypes.c_uint32, ps.value, self.n_sets) if self.n_sets else np.zeros(0, dtype=np.uint32)
            self.set_offsets, self.set_items, self.supports = off, items, supp
            self._owner = own  # fim_result_flags reads the handle until free() (or collection)

    def flags(self) -> np.ndarray:
        """fim_result_flags: u8 per itemset (record order), bit 0 closed, bit 1 maximal (computed once)."""
        if self._flags is None:
            if not self._h:
                raise FimError(FIM_ERR_INVALID, "fim_result_flags", "result already freed")
            f = np.zeros(max(self.n_sets, 1), dtype=np.uint8)
            _check(self._lib, self._lib.fim_result_flags(self._h, f.ctypes.data), "fim_result_flags")
            self._flags = f[: self.n_sets]
        return self._flags

    def free(self):
        """Device result: freed now.  Host result: the Result lets go of it; its memory is released once no
        array of it is referenced any more."""
        if self._h:
            if self._owner is None:
                self._lib.fim_result_free(self._h)
            self._owner = None
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def as_dict(self):
        """{itemset tuple: support} (host results)."""
        so, si, sp = self.set_offsets, self.set_items, self.supports
        return {tuple(int(v) for v in si[so[k]:so[k + 1]]): int(sp[k]) for k in range(self.n_sets)}


class Database:
    """A built vertical database (fim_db)."""

    def __init__(self, lib, handle):
        self._lib, self._h = lib, handle
        self._inputs = None

    @property
    def handle(self):
        return self._h

    def info(self):
        vals = [ctypes.c_uint32() for _ in range(5)]
        nbytes = ctypes.c_uint64()
        _check(self._lib, self._lib.fim_db_info(self._h, *[ctypes.byref(v) for v in vals], ctypes.byref(nbytes)),
               "fim_db_info")
        D, N, rows, words, wb = (v.value for v in vals)
        return dict(D=D, N=N, n_rows=rows, words_per_row=words, word_bits=wb, device_bytes=nbytes.value)

    def rows(self):
        n = self.info()["n_rows"]
        ri = np.zeros(max(n, 1), dtype=np.uint32)
        sp = np.zeros(max(n, 1), dtype=np.uint32)
        _check(self._lib, self._lib.fim_db_rows(self._h, ri.ctypes.data, sp.ctypes.data), "fim_db_rows")
        return ri[:n], sp[:n]

    def estimate_class_costs(self, sample_rate: float, rel_minsup: float, seed: int, cost: str = "itemsets",
                             max_sample_itemsets: int = SAMPLE_ITEMSET_LIMIT, outputs: bool = True):
        """fim_estimate_class_costs_ex: cost "itemsets" (the thesis's measure) or "intersections"; the sample
        minsup doubles while the sample has more than ``max_sample_itemsets`` frequent itemsets (0: never).
        outputs=False passes NULL outputs (the estimate may then stay on the device until the next mine) and
        returns None."""
        kind = {"itemsets": 0, "intersections": 1}[cost]
        if not outputs:
            _check(self._lib, self._lib.fim_estimate_class_costs_ex(self._h, sample_rate, rel_minsup, seed, kind,
                                                                    max_sample_itemsets, None, None),
                   "fim_estimate_class_costs_ex")
            return None
        n = self.info()["n_rows"]
        c = np.zeros(max(n, 1), dtype=np.float64)
        order = np.zeros(max(n, 1), dtype=np.uint32)
        _check(self._lib, self._lib.fim_estimate_class_costs_ex(self._h, sample_rate, rel_minsup, seed, kind,
                                                                max_sample_itemsets, c.ctypes.data,
                                                                order.ctypes.data),
               "fim_estimate_class_costs_ex")
        return c[:n], order[:n]

    def estimate_result(self):
        """fim_estimate_result: the last estimate's (costs, order), waiting for a deferred one."""
        n = self.info()["n_rows"]
        c = np.zeros(max(n, 1), dtype=np.float64)
        order = np.zeros(max(n, 1), dtype=np.uint32)
        _check(self._lib, self._lib.fim_estimate_result(self._h, c.ctypes.data, order.ctypes.data),
               "fim_estimate_result")
        return c[:n], order[:n]

    def estimate_sample_size(self):
        nfs, rows, ms = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(self._lib, self._lib.fim_estimate_sample_size(self._h, ctypes.byref(nfs), ctypes.byref(rows),
                                                             ctypes.byref(ms)), "fim_estimate_sample_size")
        return nfs.value, rows.value, ms.value

    def _opts(self, class_order="estimate", threads_per_cta=0, vec_per_lane=0, ctas_per_sm=0, donate=False,
              result_on_device=False, collect_times=False, out_capacity_sets=0, out_capacity_items=0, spin_limit=0,
              stats=True, shape=None, dfs_mode=None, max_itemsets=0, pair_kernel=FIM_PAIR_AUTO):
        opts = MineOpts()
        self._lib.fim_mine_opts_init(ctypes.byref(opts))
        opts.pair_kernel = pair_kernel
        if dfs_mode is not None:
            opts.dfs_mode = dfs_mode
        opts.class_order = {"estimate": FIM_ORDER_ESTIMATE, "uniform": FIM_ORDER_UNIFORM}[class_order]
        opts.threads_per_cta = threads_per_cta
        opts.vec_per_lane = vec_per_lane
        opts.ctas_per_sm = ctas_per_sm
        opts.donate = 1 if donate else 0
        if shape:
            opts.threads_per_cta, opts.vec_per_lane = shape["threads_per_cta"], shape["vec_per_lane"]
            opts.ctas_per_sm, opts.donate = shape["ctas_per_sm"], shape["donate"]
            opts.dfs_mode = shape.get("dfs_mode", 0)
        opts.result_on_device = 1 if result_on_device else 0
        opts.collect_times = 1 if collect_times else 0
        opts.out_capacity_sets = out_capacity_sets
        opts.out_capacity_items = out_capacity_items
        opts.spin_limit = spin_limit
        opts.max_itemsets = max_itemsets
        st = MineStats() if stats else None
        if st is not None:
            opts.stats = ctypes.pointer(st)
        return opts, st

    def autotune(self, minsup: int, class_order: str = "estimate"):
        """fim_autotune: fastest DFS launch shape for this database and minsup (dict, plus its time)."""
        opts, _ = self._opts(class_order=class_order, stats=False)
        ms = ctypes.c_float()
        _check(self._lib, self._lib.fim_autotune(self._h, minsup, ctypes.byref(opts), ctypes.byref(ms)), "fim_autotune")
        return {"threads_per_cta": opts.threads_per_cta, "vec_per_lane": opts.vec_per_lane,
                "ctas_per_sm": opts.ctas_per_sm, "donate": opts.donate, "dfs_mode": opts.dfs_mode}, ms.value

    def plan(self, minsup: int, **kw):
        """fim_plan_create: the mine captured in a CUDA graph (see Plan)."""
        opts, _ = self._opts(**kw)
        h = ctypes.c_void_p()
        _check(self._lib, self._lib.fim_plan_create(self._h, minsup, ctypes.byref(opts), ctypes.byref(h)),
               "fim_plan_create")
        return Plan(self._lib, h.value, self)

    def mine(self, minsup: int, class_order: str = "estimate", threads_per_cta: int = 0, vec_per_lane: int = 0,
             ctas_per_sm: int = 0, donate: bool = False, result_on_device: bool = False, collect_times: bool = False,
             out_capacity_sets: int = 0, out_capacity_items: int = 0, spin_limit: int = 0, stats: bool = True,
             shape=None, dfs_mode: int | None = None, max_itemsets: int = 0, class_work: bool = False,
             dfs_depth_first: int = 0, pair_kernel: int = FIM_PAIR_AUTO, fault_pair_wait: bool = False,
             proj_bitmap_words: int = 0, proj_stack_words: int = 0, proj_max_row_words: int = 0,
             proj_split_words: int = 0, output: str = "all", diffsets: int = 0):
        """fim_mine; with ``class_work`` the result carries ``class_work`` (u64[n_rows]): the intersections
        of every one-row class, level 2 and below."""
        opts, st = self._opts(class_order, threads_per_cta, vec_per_lane, ctas_per_sm, donate, result_on_device,
                              collect_times, out_capacity_sets, out_capacity_items, spin_limit, stats, shape, dfs_mode,
                              max_itemsets, pair_kernel)
        opts.dfs_depth_first = dfs_depth_first
        opts.fault_pair_wait = 1 if fault_pair_wait else 0
        opts.proj_bitmap_words = proj_bitmap_words
        opts.proj_stack_words = proj_stack_words
        opts.proj_max_row_words = proj_max_row_words
        opts.proj_split_words = proj_split_words
        opts.output = {"all": FIM_OUTPUT_ALL, "closed": FIM_OUTPUT_CLOSED, "maximal": FIM_OUTPUT_MAXIMAL}[output]
        opts.diffsets = diffsets
        cw = None
        if class_work:
            cw = np.zeros(max(1, self.info()["n_rows"]), dtype=np.uint64)
            opts.class_work_out = cw.ctypes.data
        h = ctypes.c_void_p()
        status = self._lib.fim_mine(self._h, minsup, ctypes.byref(opts), ctypes.byref(h))
        if status == FIM_ERR_OUTPUT_OVERFLOW:
            err = FimError(status, "fim_mine", self._lib.fim_last_error().decode(errors="replace"))
            err.needed = (opts.out_needed_sets, opts.out_needed_items)
            raise err
        _check(self._lib, status, "fim_mine")
        res = Result(self._lib, h.value, st)
        if cw is not None:
            res.class_work = cw[: self.info()["n_rows"]]
        return res

    def mine_pairs_noalloc(self, minsup: int, d_pairs, d_supports, capacity: int) -> int:
        """fim_mine_pairs_noalloc into caller-owned device buffers; returns the number of frequent pairs."""
        n = ctypes.c_uint64()
        status = self._lib.fim_mine_pairs_noalloc(self._h, minsup, _ptr(d_pairs), _ptr(d_supports), capacity,
                                                  ctypes.byref(n))
        if status == FIM_ERR_OUTPUT_OVERFLOW:
            err = FimError(status, "fim_mine_pairs_noalloc", self._lib.fim_last_error().decode(errors="replace"))
            err.needed = n.value
            raise err
        _check(self._lib, status, "fim_mine_pairs_noalloc")
        return n.value

    def extension_supports(self, prefix, candidates) -> np.ndarray:
        """fim_extension_supports: supp(P u {c}) for every candidate item c of ``candidates``
        (original ids), P = ``prefix``; returns u32[len(candidates)]."""
        pre = np.ascontiguousarray(prefix, dtype=np.uint32)
        cand = np.ascontiguousarray(candidates, dtype=np.uint32)
        out = np.zeros(len(cand), dtype=np.uint32)
        _check(self._lib, self._lib.fim_extension_supports(self._h, pre.ctypes.data, len(pre), cand.ctypes.data,
                                                            len(cand), out.ctypes.data), "fim_extension_supports")
        return out

    def free(self):
        if self._h:
            self._lib.fim_db_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Plan:
    """A captured mine (fim_plan): launch() enqueues a graph replay, result() waits and returns it."""

    def __init__(self, lib, handle, db):
        self._lib, self._h, self._db = lib, handle, db

    @property
    def stream(self) -> int:
        s = ctypes.c_void_p()
        _check(self._lib, self._lib.fim_plan_stream(self._h, ctypes.byref(s)), "fim_plan_stream")
        return s.value or 0

    def launch(self):
        _check(self._lib, self._lib.fim_plan_launch(self._h), "fim_plan_launch")

    def result(self, result_on_device: bool = False):
        opts, st = self._db._opts(result_on_device=result_on_device)
        h = ctypes.c_void_p()
        _check(self._lib, self._lib.fim_plan_result(self._h, ctypes.byref(opts), ctypes.byref(h)), "fim_plan_result")
        return Result(self._lib, h.value, st)

    def free(self):
        if self._h:
            self._lib.fim_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_vertical_db(tx_offsets, tx_items, N: int, word_bits: int = 64, prefilter_minsup: int = 0, stream=None):
    """fim_build_vertical_db: host CSR (numpy uint32) -> Database."""
    lib = load()
    off = np.ascontiguousarray(tx_offsets, dtype=np.uint32)
    it = np.ascontiguousarray(tx_items, dtype=np.uint32)
    if it.size == 0:
        it = np.zeros(1, dtype=np.uint32)
    h = ctypes.c_void_p()
    _check(lib, lib.fim_build_vertical_db(off.ctypes.data, it.ctypes.data, off.size - 1, N, word_bits,
                                          prefilter_minsup, _stream_handle(stream), ctypes.byref(h)),
           "fim_build_vertical_db")
    return Database(lib, h.value)


def build_vertical_db_device(d_tx_offsets, d_tx_items, D: int, N: int, word_bits: int = 64,
                             prefilter_minsup: int = 0, stream=None):
    """fim_build_vertical_db_device: CSR already in device memory (torch tensors or raw pointers)."""
    lib = load()
    h = ctypes.c_void_p()
    _check(lib, lib.fim_build_vertical_db_device(_ptr(d_tx_offsets), _ptr(d_tx_items), D, N, word_bits,
                                                 prefilter_minsup, _stream_handle(stream), ctypes.byref(h)),
           "fim_build_vertical_db_device")
    db = Database(lib, h.value)
    db._inputs = (d_tx_offsets, d_tx_items)  # read on the stream after the call returns: keep them alive
    return db


def kernel_launches() -> int:
    """fim_kernel_launches: kernels this library has put on a stream so far (graph replays included)."""
    return int(load().fim_kernel_launches())


def pool_memory(device: int = 0):
    """fim_pool_memory: (bytes in use, bytes reserved) of the library's device memory pool."""
    lib = load()
    used, reserved = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib, lib.fim_pool_memory(device, ctypes.byref(used), ctypes.byref(reserved)), "fim_pool_memory")
    return used.value, reserved.value


def status_str(status: int) -> str:
    return load().fim_status_str(status).decode()


class Server:
    """fim_server: continuous-batching request loop (submit / wait)."""

    def __init__(self, hbm_budget_bytes: int = 0, slots: int = 4, ctas_per_sm: int = 1, max_itemsets: int = 0):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib, self._lib.fim_server_create(hbm_budget_bytes, slots, ctas_per_sm, max_itemsets,
                                                      ctypes.byref(h)), "fim_server_create")
        self._h = h.value

    def submit(self, tx_offsets, tx_items, N: int, minsup: int, sample_rate: float = 0.0) -> int:
        off = np.ascontiguousarray(tx_offsets, dtype=np.uint32)
        it = np.ascontiguousarray(tx_items, dtype=np.uint32)
        if it.size == 0:
            it = np.zeros(1, dtype=np.uint32)
        jid = ctypes.c_uint64()
        _check(self._lib, self._lib.fim_server_submit(self._h, off.ctypes.data, it.ctypes.data, off.size - 1, N,
                                                      minsup, sample_rate, ctypes.byref(jid)), "fim_server_submit")
        return jid.value

    def wait(self, job_id: int):
        """Returns (Result, latency seconds, service seconds)."""
        res, lat, svc, _ = self.wait_ex(job_id)
        return res, lat, svc

    def wait_ex(self, job_id: int):
        """fim_server_wait_ex: (Result, latency s, service s, (device start ms, device end ms) from the
        server's creation)."""
        h = ctypes.c_void_p()
        lat, svc, t0, t1 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self._lib, self._lib.fim_server_wait_ex(self._h, job_id, ctypes.byref(h), ctypes.byref(lat),
                                                       ctypes.byref(svc), ctypes.byref(t0), ctypes.byref(t1)),
               "fim_server_wait_ex")
        return Result(self._lib, h.value, None), lat.value, svc.value, (t0.value, t1.value)

    def stats(self):
        a, b, c, d = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
        _check(self._lib, self._lib.fim_server_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                                     ctypes.byref(d)), "fim_server_stats")
        return {"in_use_bytes": a.value, "in_flight": b.value, "peak_in_flight": c.value, "queued": d.value}

    def free(self):
        if self._h:
            self._lib.fim_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
