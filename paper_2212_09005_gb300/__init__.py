"""GPU filters for GB300: the two-choice filter (TCF) and the counting quotient
filter (GQF) of "High-Performance Filters for GPUs" (arXiv 2212.09005).

This module is a thin ctypes binding over the C ABI in include/gpufilter.h:
it marshals torch CUDA tensors (device pointers) and the current CUDA stream
into the library's calls. Every step of every operation runs in the
library's CUDA kernels; there is no CPU fallback. If libgpufilter.so has not
been built, importing works but creating a filter raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = [
    "Filter", "TCF", "GQF", "FilterGroup", "FilterServer", "lib", "build", "FilterError",
    "FILTER_TCF", "FILTER_GQF", "MODE_BULK", "MODE_POINT",
    "KEY_OK", "KEY_FULL", "KEY_NOT_FOUND", "STATUS_FULL", "STATUS_TIMEOUT", "FilterBatch", "BATCH_TCF", "BATCH_GQF",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgpufilter.so")

FILTER_TCF, FILTER_GQF = 1, 2
MODE_BULK, MODE_POINT = 0, 1
KEY_OK, KEY_FULL, KEY_NOT_FOUND = 0, 1, 2
ERR_FULL, ERR_TIMEOUT, ERR_INTERNAL = 4, 5, 7
STATUS_FULL, STATUS_TIMEOUT, STATUS_INTERNAL = 1 << ERR_FULL, 1 << ERR_TIMEOUT, 1 << ERR_INTERNAL

# entry points declared in include/gpufilter.h
EXPORTS = [
    "filter_create", "filter_destroy", "filter_clear", "filter_insert", "filter_query",
    "filter_insert_values", "filter_query_values", "filter_insert_counts",
    "filter_remove", "filter_count", "filter_get_stats", "filter_get_device_view", "filter_export_size",
    "filter_gqf_enumerate", "filter_gqf_keys_of",
    "filter_export", "filter_import", "filter_error_string",
    "filter_trace_enable", "filter_trace_reset", "filter_trace_summary",
    "filter_gqf_insert_noalloc",
    "filter_group_create", "filter_group_destroy", "filter_group_clear", "filter_group_insert",
    "filter_group_remove", "filter_group_query", "filter_group_count", "filter_group_get_stats",
    "filter_group_export_size", "filter_group_export",
    "filter_server_create", "filter_server_submit", "filter_server_wait", "filter_server_get_stats",
    "filter_server_destroy",
    "filter_calibrate_gather",
    "filter_debug_fail_alloc", "filter_debug_live_allocations", "filter_debug_wait_timeout",
    "filter_batch_create", "filter_batch_run", "filter_batch_destroy",
    "filter_set_tuning", "filter_get_tuning", "filter_group_set_tuning",
    "filter_gqf_point_update",
]

TCF_PATH_AUTO, TCF_PATH_BLOCK, TCF_PATH_TILED = 0, 1, 2

BATCH_TCF, BATCH_GQF = 0, 1

OP_INSERT, OP_QUERY, OP_REMOVE, OP_COUNT = 0, 1, 2, 3


class FilterConfig(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("log2_slots", C.c_uint32), ("tag_bits", C.c_uint32),
                ("mode", C.c_uint32), ("hash_seed", C.c_uint64), ("max_batch", C.c_uint64),
                ("value_bits", C.c_uint32), ("block_slots", C.c_uint32)]


class FilterStats(C.Structure):
    _fields_ = [("status_word", C.c_uint64), ("failed_keys", C.c_uint64),
                ("backing_used", C.c_uint64), ("table_bytes", C.c_uint64),
                ("device_bytes", C.c_uint64), ("nslots", C.c_uint64)]


class FilterDeviceView(C.Structure):
    """The filter_device_view of include/gpufilter.h (pass it by value to a
    kernel that includes include/gpufilter_device.cuh)."""
    _fields_ = [("kind", C.c_uint32), ("tag_bits", C.c_uint32), ("q", C.c_uint32), ("mode", C.c_uint32),
                ("seed", C.c_uint64), ("table", C.c_void_p), ("aux", C.c_void_p), ("n_blocks", C.c_uint64),
                ("n_aux", C.c_uint64), ("counters", C.c_void_p), ("value_bits", C.c_uint32),
                ("reserved", C.c_uint32), ("locks", C.c_void_p)]


class FilterRequest(C.Structure):
    _fields_ = [("filter", C.c_uint32), ("op", C.c_uint32), ("host_keys", C.c_void_p), ("n", C.c_uint64),
                ("host_out", C.c_void_p)]


class FilterWork(C.Structure):
    _fields_ = [("group", C.c_uint32), ("member", C.c_uint32), ("op", C.c_uint32), ("reserved", C.c_uint32),
                ("d_keys", C.c_void_p), ("n", C.c_uint64), ("d_out", C.c_void_p)]


class FilterTuning(C.Structure):
    _fields_ = [("tcf_path", C.c_uint32), ("tcf_tile_target", C.c_uint32), ("gqf_region_groups", C.c_uint32),
                ("reserved", C.c_uint32), ("tcf_tiled_min_blocks", C.c_uint64)]


class ServerStats(C.Structure):
    _fields_ = [("batches", C.c_uint64), ("requests", C.c_uint64), ("merged_requests", C.c_uint64),
                ("max_concurrent", C.c_uint64), ("pool_bytes", C.c_uint64), ("pool_peak_bytes", C.c_uint64)]


class TraceEntry(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_uint64), ("units", C.c_uint64),
                ("ms", C.c_double)]


class FilterError(RuntimeError):
    pass


_lib = None


def build(force: bool = False) -> str:
    from . import _build

    return _build.build(force=force)


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FilterError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(paper_2212_09005_gb300.build())")
        L = C.CDLL(LIB_PATH)
        vp, u64, i32 = C.c_void_p, C.c_uint64, C.c_int
        L.filter_create.argtypes = [C.POINTER(FilterConfig), vp, C.POINTER(vp)]
        L.filter_destroy.argtypes = [vp]
        L.filter_clear.argtypes = [vp, vp]
        for name in ("filter_insert", "filter_query", "filter_remove", "filter_count", "filter_query_values"):
            getattr(L, name).argtypes = [vp, vp, u64, vp, vp]
        L.filter_insert_values.argtypes = [vp, vp, vp, u64, vp, vp]
        L.filter_insert_counts.argtypes = [vp, vp, vp, u64, vp, vp]
        L.filter_get_stats.argtypes = [vp, vp, C.POINTER(FilterStats)]
        L.filter_export_size.argtypes = [vp, C.POINTER(u64)]
        L.filter_export.argtypes = [vp, vp, u64, vp]
        L.filter_import.argtypes = [vp, vp, u64, vp]
        L.filter_trace_enable.argtypes = [i32]
        L.filter_trace_reset.argtypes = []
        L.filter_trace_summary.argtypes = [C.c_uint32, C.POINTER(TraceEntry), C.POINTER(C.c_uint32)]
        L.filter_gqf_insert_noalloc.argtypes = [C.c_uint32, C.c_uint32, u64, vp, vp, vp, u64, vp, vp]
        L.filter_group_create.argtypes = [C.POINTER(FilterConfig), C.c_uint32, u64, vp, C.POINTER(vp)]
        L.filter_group_destroy.argtypes = [vp]
        L.filter_group_clear.argtypes = [vp, vp]
        for name in ("filter_group_insert", "filter_group_remove", "filter_group_query", "filter_group_count"):
            getattr(L, name).argtypes = [vp, vp, vp, u64, vp, vp]
        L.filter_group_get_stats.argtypes = [vp, C.c_uint32, vp, C.POINTER(FilterStats)]
        L.filter_group_export_size.argtypes = [vp, C.c_uint32, C.POINTER(u64)]
        L.filter_group_export.argtypes = [vp, C.c_uint32, vp, u64, vp]
        L.filter_server_create.argtypes = [C.POINTER(vp), C.c_uint32, C.c_uint32, u64, C.POINTER(vp)]
        L.filter_server_submit.argtypes = [vp, C.POINTER(FilterRequest), C.POINTER(u64)]
        L.filter_server_wait.argtypes = [vp, u64, C.POINTER(i32), C.POINTER(C.c_double)]
        L.filter_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.filter_batch_create.argtypes = [vp, vp, u64, C.c_uint32, C.POINTER(vp)]
        L.filter_batch_run.argtypes = [vp, C.POINTER(FilterWork), C.c_uint32, vp]
        L.filter_batch_destroy.argtypes = [vp]
        L.filter_debug_fail_alloc.argtypes = [C.c_uint32]
        L.filter_debug_live_allocations.argtypes = [C.POINTER(u64)]
        L.filter_debug_wait_timeout.argtypes = [vp, C.c_uint32, vp]
        L.filter_server_destroy.argtypes = [vp]
        L.filter_set_tuning.argtypes = [vp, C.POINTER(FilterTuning)]
        L.filter_gqf_point_update.argtypes = [vp, vp, u64, i32, vp, vp]
        L.filter_get_tuning.argtypes = [vp, C.POINTER(FilterTuning)]
        L.filter_group_set_tuning.argtypes = [vp, C.POINTER(FilterTuning)]
        L.filter_calibrate_gather.argtypes = [vp, u64, vp, u64, C.c_uint32, vp, vp]
        L.filter_error_string.argtypes = [i32]
        L.filter_error_string.restype = C.c_char_p
        for name in EXPORTS:
            if name != "filter_error_string":
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = lib().filter_error_string(rc).decode()
        raise FilterError(f"{what}: {msg} (code {rc})")


def _stream(stream):
    if stream is None:
        import torch

        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t, dtype_bytes=None):
    """Device pointer of a contiguous CUDA tensor."""
    if t is None:
        return None
    if not t.is_cuda:
        raise FilterError("expected a CUDA tensor (device memory)")
    if not t.is_contiguous():
        raise FilterError("expected a contiguous tensor")
    if dtype_bytes is not None and t.element_size() != dtype_bytes:
        raise FilterError(f"expected {dtype_bytes}-byte elements")
    return C.c_void_p(t.data_ptr())


class Filter:
    """One filter on the current CUDA device."""

    def __init__(self, kind: int, log2_slots: int, tag_bits: int, mode: int = MODE_BULK,
                 seed: int = 0, max_batch: int = 1 << 22, stream=None, value_bits: int = 0, block_slots: int = 0):
        self.cfg = FilterConfig(kind, log2_slots, tag_bits, mode, seed & 0xFFFFFFFFFFFFFFFF,
                                max(1, int(max_batch)), value_bits, int(block_slots))
        h = C.c_void_p()
        _check(lib().filter_create(C.byref(self.cfg), _stream(stream), C.byref(h)), "filter_create")
        self._h = h
        self.kind, self.log2_slots, self.tag_bits, self.mode = kind, log2_slots, tag_bits, mode
        self.seed, self.max_batch, self.value_bits = seed, max(1, int(max_batch)), value_bits
        t = tuning.lookup(kind, log2_slots)
        if t:
            self.set_tuning(**t)

    def point_update(self, keys, remove: bool = False, status=None, stream=None):
        """GQF: locked point inserts (or removes) of the keys, one thread per
        key, asynchronous and graph-capturable; status: uint8, one per key."""
        _check(lib().filter_gqf_point_update(self._h, _dptr(keys, 8), keys.numel(), 1 if remove else 0,
                                             _dptr(status, 1), _stream(stream)), "filter_gqf_point_update")

    def set_tuning(self, **knobs):
        """Kernel choices that never change results: tcf_path (TCF_PATH_*),
        tcf_tile_target, tcf_tiled_min_blocks, gqf_region_groups; 0 = default."""
        _check(lib().filter_set_tuning(self._h, C.byref(tuning.struct(knobs))), "filter_set_tuning")

    def get_tuning(self) -> dict:
        t = FilterTuning()
        _check(lib().filter_get_tuning(self._h, C.byref(t)), "filter_get_tuning")
        return {k: getattr(t, k) for k, _ in FilterTuning._fields_ if k != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            lib().filter_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- batched operations (asynchronous on the stream) ----
    def insert(self, keys, status=None, stream=None, values=None):
        """values (TCF with value_bits > 0): one uint8 per key."""
        if values is not None:
            if values.numel() != keys.numel():
                raise FilterError("one value per key")
            _check(lib().filter_insert_values(self._h, _dptr(keys, 8), _dptr(values, 1), keys.numel(),
                                              _dptr(status, 1), _stream(stream)), "filter_insert_values")
            return
        _check(lib().filter_insert(self._h, _dptr(keys, 8), keys.numel(), _dptr(status, 1),
                                   _stream(stream)), "filter_insert")

    def query(self, keys, found, stream=None):
        _check(lib().filter_query(self._h, _dptr(keys, 8), keys.numel(), _dptr(found, 1),
                                  _stream(stream)), "filter_query")

    def insert_counts(self, keys, counts, status=None, stream=None):
        """GQF: key i counts as counts[i] >= 1 copies (int32 tensor, read as uint32)."""
        if counts.numel() != keys.numel():
            raise FilterError("one count per key")
        _check(lib().filter_insert_counts(self._h, _dptr(keys, 8), _dptr(counts, 4), keys.numel(),
                                          _dptr(status, 1), _stream(stream)), "filter_insert_counts")

    def query_values(self, keys, values, stream=None):
        """TCF with values: smallest stored value per key, 0xFF when absent."""
        _check(lib().filter_query_values(self._h, _dptr(keys, 8), keys.numel(), _dptr(values, 1),
                                         _stream(stream)), "filter_query_values")

    def remove(self, keys, status=None, stream=None):
        _check(lib().filter_remove(self._h, _dptr(keys, 8), keys.numel(), _dptr(status, 1),
                                   _stream(stream)), "filter_remove")

    def count(self, keys, counts, stream=None):
        _check(lib().filter_count(self._h, _dptr(keys, 8), keys.numel(), _dptr(counts, 8),
                                  _stream(stream)), "filter_count")

    def clear(self, stream=None):
        _check(lib().filter_clear(self._h, _stream(stream)), "filter_clear")

    def enumerate(self, stream=None):
        """GQF: (fingerprints, counts) of every group, ascending, as int64 CUDA tensors."""
        import torch

        n = C.c_uint64()
        _check(lib().filter_gqf_enumerate(self._h, None, None, 0, C.byref(n), _stream(stream)), "filter_gqf_enumerate")
        fps = torch.empty(n.value, dtype=torch.int64, device="cuda")
        cnt = torch.empty(n.value, dtype=torch.int64, device="cuda")
        m = C.c_uint64()
        _check(lib().filter_gqf_enumerate(self._h, _dptr(fps, 8), _dptr(cnt, 8), n.value, C.byref(m),
                                          _stream(stream)), "filter_gqf_enumerate")
        return fps, cnt

    def keys_of(self, fingerprints, keys, stream=None):
        """GQF: the keys (below 2^(q + r)) whose fingerprints these are."""
        _check(lib().filter_gqf_keys_of(self._h, _dptr(fingerprints, 8), fingerprints.numel(), _dptr(keys, 8),
                                        _stream(stream)), "filter_gqf_keys_of")

    def device_view(self) -> "FilterDeviceView":
        """Table pointers and geometry for device-side point queries; take it
        again after any update of the filter."""
        v = FilterDeviceView()
        _check(lib().filter_get_device_view(self._h, C.byref(v)), "filter_get_device_view")
        return v

    # ---- synchronous helpers ----
    def stats(self, stream=None) -> dict:
        s = FilterStats()
        _check(lib().filter_get_stats(self._h, _stream(stream), C.byref(s)), "filter_get_stats")
        return {k: int(getattr(s, k)) for k, _ in FilterStats._fields_}

    def export(self, stream=None) -> np.ndarray:
        n = C.c_uint64()
        _check(lib().filter_export_size(self._h, C.byref(n)), "filter_export_size")
        buf = np.zeros(n.value, np.uint8)
        _check(lib().filter_export(self._h, buf.ctypes.data_as(C.c_void_p), n.value, _stream(stream)),
               "filter_export")
        return buf

    def import_(self, image: np.ndarray, stream=None):
        image = np.ascontiguousarray(image, dtype=np.uint8)
        _check(lib().filter_import(self._h, image.ctypes.data_as(C.c_void_p), image.size,
                                   _stream(stream)), "filter_import")


def TCF(log2_slots: int, tag_bits: int = 16, mode: int = MODE_BULK, seed: int = 0,
        max_batch: int = 1 << 22, stream=None, value_bits: int = 0, block_slots: int = 0) -> Filter:
    """block_slots: slots per block (0: one 32-byte sector); other sizes are
    packed bulk-mode geometries with nb the largest power of two such that
    nb * block_slots <= 2^log2_slots."""
    return Filter(FILTER_TCF, log2_slots, tag_bits, mode, seed, max_batch, stream, value_bits, block_slots)


def GQF(q: int, r: int = 8, seed: int = 0, max_batch: int = 1 << 22, stream=None) -> Filter:
    return Filter(FILTER_GQF, q, r, 0, seed, max_batch, stream)


class FilterGroup:
    """Many filters of one kind (all TCF bulk-mode or all GQF, one tag width),
    driven by one set of kernel launches per call. Member i's keys of a call
    are keys[offsets[i]:offsets[i + 1]] (offsets: int64 CUDA tensor of
    n_filters + 1 entries)."""

    def __init__(self, kind: int, log2_slots, tag_bits: int, seeds, max_total: int, stream=None):
        log2_slots = [int(x) for x in log2_slots]
        seeds = [int(x) & 0xFFFFFFFFFFFFFFFF for x in seeds]
        if len(seeds) != len(log2_slots) or not log2_slots:
            raise FilterError("need one seed per member")
        self.n = len(log2_slots)
        cfgs = (FilterConfig * self.n)()
        for i, (lg, sd) in enumerate(zip(log2_slots, seeds)):
            cfgs[i] = FilterConfig(kind, lg, tag_bits, MODE_BULK if kind == FILTER_TCF else 0, sd, 1)
        h = C.c_void_p()
        _check(lib().filter_group_create(cfgs, self.n, max(1, int(max_total)), _stream(stream), C.byref(h)),
               "filter_group_create")
        self._h = h
        self.kind, self.tag_bits, self.log2_slots, self.seeds = kind, tag_bits, log2_slots, seeds
        self.max_total = max(1, int(max_total))
        total = sum(1 << lg for lg in log2_slots)
        t = tuning.lookup(kind, total.bit_length() - 1, group=True)
        if t:
            self.set_tuning(**t)

    def set_tuning(self, **knobs):
        """The same knobs as Filter.set_tuning, for the group and every member."""
        _check(lib().filter_group_set_tuning(self._h, C.byref(tuning.struct(knobs))), "filter_group_set_tuning")

    def close(self):
        if getattr(self, "_h", None):
            lib().filter_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, offsets, keys, out, out_bytes, stream):
        if offsets.numel() != self.n + 1:
            raise FilterError(f"offsets must have {self.n + 1} entries")
        _check(getattr(lib(), name)(self._h, _dptr(offsets, 8), _dptr(keys, 8), keys.numel(),
                                    _dptr(out, out_bytes), _stream(stream)), name)

    def insert(self, offsets, keys, status=None, stream=None):
        self._call("filter_group_insert", offsets, keys, status, 1, stream)

    def remove(self, offsets, keys, status=None, stream=None):
        self._call("filter_group_remove", offsets, keys, status, 1, stream)

    def query(self, offsets, keys, found, stream=None):
        self._call("filter_group_query", offsets, keys, found, 1, stream)

    def count(self, offsets, keys, counts, stream=None):
        self._call("filter_group_count", offsets, keys, counts, 8, stream)

    def clear(self, stream=None):
        _check(lib().filter_group_clear(self._h, _stream(stream)), "filter_group_clear")

    def stats(self, member: int, stream=None) -> dict:
        s = FilterStats()
        _check(lib().filter_group_get_stats(self._h, member, _stream(stream), C.byref(s)),
               "filter_group_get_stats")
        return {k: int(getattr(s, k)) for k, _ in FilterStats._fields_}

    def export_size(self, member: int) -> int:
        n = C.c_uint64()
        _check(lib().filter_group_export_size(self._h, member, C.byref(n)), "filter_group_export_size")
        return n.value

    def export(self, member: int, stream=None) -> np.ndarray:
        n = C.c_uint64()
        _check(lib().filter_group_export_size(self._h, member, C.byref(n)), "filter_group_export_size")
        buf = np.zeros(n.value, np.uint8)
        _check(lib().filter_group_export(self._h, member, buf.ctypes.data_as(C.c_void_p), n.value,
                                         _stream(stream)), "filter_group_export")
        return buf


class FilterBatch:
    """A work list over a TCF group and a GQF group (either may be None): each
    run applies items (group, member, op, keys, out) with one group call per
    (group, operation) class; per group inserts run first, then removes, then
    queries, then counts. Keys and results are CUDA tensors; the list is host
    data, so a run never synchronises and can be captured in a CUDA graph."""

    def __init__(self, tcf_group=None, gqf_group=None, max_keys: int = 1 << 22, max_items: int = 8192):
        self.groups = (tcf_group, gqf_group)  # keeps the groups alive
        h = C.c_void_p()
        _check(lib().filter_batch_create(tcf_group._h if tcf_group else None, gqf_group._h if gqf_group else None,
                                         int(max_keys), int(max_items), C.byref(h)), "filter_batch_create")
        self._h = h

    def run(self, items, stream=None):
        """items: iterable of (group, member, op, keys, out); group BATCH_TCF or
        BATCH_GQF, op OP_*, keys an int64 CUDA tensor, out a uint8 (statuses,
        found flags) or int64 (counts) CUDA tensor of the same length, or None."""
        items = list(items)
        arr = (FilterWork * max(1, len(items)))()
        for k, (g, m, op, keys, out) in enumerate(items):
            arr[k] = FilterWork(g, m, op, 0, _dptr(keys, 8) if keys.numel() else None, keys.numel(),
                                _dptr(out) if out is not None else None)
        self._keep = items
        _check(lib().filter_batch_run(self._h, arr, len(items), _stream(stream)), "filter_batch_run")

    def close(self):
        if getattr(self, "_h", None):
            lib().filter_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FilterServer:
    """Serves batches of host keys for many filters on `workers` CUDA streams
    with continuous batching: any idle worker takes the oldest waiting request
    of a filter with nothing in flight (merged with the queries, counts or GQF
    removes queued right behind it) once its staging fits in the device pool.
    Each filter's requests run in submission order."""

    _OUT_DTYPE = {OP_INSERT: np.uint8, OP_QUERY: np.uint8, OP_REMOVE: np.uint8, OP_COUNT: np.uint64}

    def __init__(self, filters, workers: int = 4, max_keys: int = 1 << 22):
        self.filters = list(filters)  # keeps the filters alive while served
        arr = (C.c_void_p * len(self.filters))(*[f._h.value for f in self.filters])
        h = C.c_void_p()
        _check(lib().filter_server_create(arr, len(self.filters), workers, max(1, int(max_keys)), C.byref(h)),
               "filter_server_create")
        self._h = h
        self._pending = {}

    def submit(self, filter_index: int, op: int, keys: np.ndarray, out: np.ndarray = None,
               want_out: bool = True) -> int:
        """Enqueue a batch; returns a ticket. The arrays are kept until wait().
        `out` (optional) receives the results; page-locked arrays (e.g. numpy
        views of pinned torch tensors) skip the staging copies."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        if out is not None:
            if out.size < keys.size or out.dtype != self._OUT_DTYPE[op] or not out.flags.c_contiguous:
                raise FilterError("out must be a contiguous array of n results of the op's type")
        elif want_out:
            out = np.zeros(keys.size, self._OUT_DTYPE[op])
        req = FilterRequest(filter_index, op, keys.ctypes.data_as(C.c_void_p), keys.size,
                            out.ctypes.data_as(C.c_void_p) if out is not None else None)
        t = C.c_uint64()
        _check(lib().filter_server_submit(self._h, C.byref(req), C.byref(t)), "filter_server_submit")
        self._pending[t.value] = (keys, out)
        return t.value

    def wait(self, ticket: int):
        """Block until the batch is done: (results array or None, latency in seconds)."""
        rc, lat = C.c_int(), C.c_double()
        _check(lib().filter_server_wait(self._h, ticket, C.byref(rc), C.byref(lat)), "filter_server_wait")
        _check(rc.value, "served operation")
        keys, out = self._pending.pop(ticket)
        return out, lat.value

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().filter_server_get_stats(self._h, C.byref(st)), "filter_server_get_stats")
        return {k: int(getattr(st, k)) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().filter_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_fail_alloc(nth: int):
    """Make the nth device allocation of the library from now on fail (0: off)."""
    _check(lib().filter_debug_fail_alloc(nth), "filter_debug_fail_alloc")


def debug_live_allocations() -> int:
    n = C.c_uint64()
    _check(lib().filter_debug_live_allocations(C.byref(n)), "filter_debug_live_allocations")
    return n.value


def debug_wait_timeout(f, spin_limit: int, stream=None):
    """Run the bounded look-back wait against a predecessor that never
    publishes; f's status word then carries STATUS_TIMEOUT."""
    _check(lib().filter_debug_wait_timeout(f._h, spin_limit, _stream(stream)), "filter_debug_wait_timeout")


def trace_enable(on: bool = True):
    """Record CUDA events around every library kernel launch (process-wide)."""
    _check(lib().filter_trace_enable(1 if on else 0), "filter_trace_enable")


def trace_reset():
    _check(lib().filter_trace_reset(), "filter_trace_reset")


def trace_summary() -> dict:
    """{kernel name: {"launches", "units", "ms"}} for the launches recorded so far."""
    n = C.c_uint32()
    _check(lib().filter_trace_summary(0, None, C.byref(n)), "filter_trace_summary")
    arr = (TraceEntry * max(1, n.value))()
    _check(lib().filter_trace_summary(n.value, arr, C.byref(n)), "filter_trace_summary")
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "units": int(arr[i].units),
                                   "ms": float(arr[i].ms)} for i in range(n.value)}


def calibrate_gather(table, keys, out, sectors_per_key: int = 2, stream=None):
    """Random 32-byte gathers over `table` (a CUDA tensor), one result byte per key."""
    _check(lib().filter_calibrate_gather(_dptr(table), table.numel() * table.element_size(), _dptr(keys, 8),
                                         keys.numel(), sectors_per_key, _dptr(out, 1), _stream(stream)),
           "filter_calibrate_gather")


NOALLOC_MAX_KEYS = 65536
NOALLOC_MAX_Q = 20


def gqf_insert_noalloc(q: int, r: int, seed: int, table_in, table_out, keys, status=None, stream=None):
    """GQF bulk insert from the table image `table_in` into `table_out` (uint8 CUDA
    tensors in the filter_export layout) without any device allocation; the
    library's static scratch is used instead (at most NOALLOC_MAX_KEYS keys,
    q <= NOALLOC_MAX_Q)."""
    _check(lib().filter_gqf_insert_noalloc(q, r, seed & 0xFFFFFFFFFFFFFFFF, _dptr(table_in, 1),
                                           _dptr(table_out, 1), _dptr(keys, 8), keys.numel(),
                                           _dptr(status, 1), _stream(stream)),
           "filter_gqf_insert_noalloc")


from . import tuning  # noqa: E402  (uses the classes above)
