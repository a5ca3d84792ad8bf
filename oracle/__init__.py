"""ctypes wrapper over the CPU oracle (oracle/*.c).

TEST INFRASTRUCTURE ONLY: only the test suite, the smoke check and the
benchmark's CPU-baseline leg import this package. It never touches the CUDA
library and the CUDA library never touches it.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


_u64p = C.POINTER(C.c_uint64)
_u32p = C.POINTER(C.c_uint32)
_u8p = C.POINTER(C.c_uint8)


def _declare(L):
    L.or_mix64.restype = C.c_uint64
    L.or_mix64.argtypes = [C.c_uint64]
    L.or_unmix64.restype = C.c_uint64
    L.or_unmix64.argtypes = [C.c_uint64]
    L.or_mix_p.restype = C.c_uint64
    L.or_mix_p.argtypes = [C.c_uint64, C.c_uint]
    L.or_unmix_p.restype = C.c_uint64
    L.or_unmix_p.argtypes = [C.c_uint64, C.c_uint]
    L.or_fold_p.restype = C.c_uint64
    L.or_fold_p.argtypes = [C.c_uint64, C.c_uint]
    L.or_mix64_many.argtypes = [_u64p, _u64p, C.c_uint64]
    L.or_mix_p_many.argtypes = [_u64p, _u64p, C.c_uint64, C.c_uint]

    L.or_tcf_new.restype = C.c_void_p
    L.or_tcf_new.argtypes = [C.c_uint, C.c_uint, C.c_uint64]
    L.or_tcf_new_values.restype = C.c_void_p
    L.or_tcf_new_values.argtypes = [C.c_uint, C.c_uint, C.c_uint, C.c_uint64]
    L.or_tcf_new_geom.restype = C.c_void_p
    L.or_tcf_new_geom.argtypes = [C.c_uint, C.c_uint, C.c_uint, C.c_uint, C.c_uint64]
    L.or_tcf_free.argtypes = [C.c_void_p]
    L.or_tcf_keyinfo.argtypes = [C.c_void_p, _u64p, C.c_uint64, _u64p, _u64p, _u32p]
    L.or_tcf_insert.argtypes = [C.c_void_p, _u64p, C.c_uint64, _u8p, _u8p, _u64p]
    L.or_tcf_query.argtypes = [C.c_void_p, _u64p, C.c_uint64, _u8p]
    L.or_tcf_insert_values.argtypes = [C.c_void_p, _u64p, _u8p, C.c_uint64, _u8p, _u8p, _u64p]
    L.or_tcf_query_values.argtypes = [C.c_void_p, _u64p, C.c_uint64, _u8p]
    L.or_tcf_remove.argtypes = [C.c_void_p, _u64p, C.c_uint64, _u8p]
    L.or_tcf_export_size.restype = C.c_uint64
    L.or_tcf_export_size.argtypes = [C.c_void_p]
    L.or_tcf_export.argtypes = [C.c_void_p, _u8p]
    L.or_tcf_backing_count.restype = C.c_uint64
    L.or_tcf_backing_count.argtypes = [C.c_void_p]
    L.or_tcf_stored_count.restype = C.c_uint64
    L.or_tcf_stored_count.argtypes = [C.c_void_p]
    L.or_tcf_geometry.argtypes = [C.c_void_p, _u64p]

    L.or_gqf_new.restype = C.c_void_p
    L.or_gqf_new.argtypes = [C.c_uint, C.c_uint, C.c_uint64]
    L.or_gqf_free.argtypes = [C.c_void_p]
    L.or_gqf_fingerprints.argtypes = [C.c_void_p, _u64p, C.c_uint64, _u64p]
    L.or_gqf_insert.argtypes = [C.c_void_p, _u64p, C.c_uint64, _u8p]
    L.or_gqf_insert_counts.argtypes = [C.c_void_p, _u64p, _u32p, C.c_uint64, _u8p]
    L.or_gqf_remove.argtypes = [C.c_void_p, _u64p, C.c_uint64, _u8p]
    L.or_gqf_count.argtypes = [C.c_void_p, _u64p, C.c_uint64, _u64p]
    L.or_gqf_insert_groups.restype = C.c_uint64
    L.or_gqf_insert_groups.argtypes = [C.c_void_p, _u64p, _u64p, C.c_uint64]
    L.or_gqf_count_fp.restype = C.c_uint64
    L.or_gqf_count_fp.argtypes = [C.c_void_p, C.c_uint64]
    L.or_gqf_groups.restype = C.c_uint64
    L.or_gqf_groups.argtypes = [C.c_void_p, _u64p, _u64p, C.c_uint64]
    L.or_gqf_export_size.restype = C.c_uint64
    L.or_gqf_export_size.argtypes = [C.c_void_p]
    L.or_gqf_export.argtypes = [C.c_void_p, _u8p]
    L.or_gqf_max_cluster.restype = C.c_uint64
    L.or_gqf_max_cluster.argtypes = [C.c_void_p]
    L.or_gqf_geometry.argtypes = [C.c_void_p, _u64p]
    L.or_gqf_build.restype = C.c_int
    L.or_gqf_build.argtypes = [C.c_uint, C.c_uint, _u64p, _u64p, C.c_uint64, _u8p]
    L.or_gqf_tail_slots.restype = C.c_uint64
    L.or_gqf_tail_slots.argtypes = [C.c_uint]


def _p(a, ty):
    return a.ctypes.data_as(ty)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def mix64(x: int) -> int:
    return lib().or_mix64(x)


def unmix64(x: int) -> int:
    return lib().or_unmix64(x)


def mix_p(x: int, p: int) -> int:
    return lib().or_mix_p(x, p)


def unmix_p(x: int, p: int) -> int:
    return lib().or_unmix_p(x, p)


def fold_p(x: int, p: int) -> int:
    return lib().or_fold_p(x, p)


def mix64_many(a):
    a = _u64(a)
    out = np.empty_like(a)
    lib().or_mix64_many(_p(a, _u64p), _p(out, _u64p), a.size)
    return out


def mix_p_many(a, p: int):
    a = _u64(a)
    out = np.empty_like(a)
    lib().or_mix_p_many(_p(a, _u64p), _p(out, _u64p), a.size, p)
    return out


class TCF:
    """Deterministic bulk two-choice filter (see tcf.c for the specification).
    value_bits > 0 gives each slot a value of that many bits below the tag."""

    def __init__(self, log2_slots: int, tag_bits: int = 16, seed: int = 0, value_bits: int = 0,
                 block_slots: int = 0, log2_blocks: int = 0):
        """Either log2_slots (32-byte blocks of 256 / tag_bits slots) or
        log2_blocks and block_slots (any geometry tcf.c allows)."""
        if block_slots:
            self._h = lib().or_tcf_new_geom(log2_blocks, tag_bits, block_slots, value_bits, seed)
        else:
            self._h = lib().or_tcf_new_values(log2_slots, tag_bits, value_bits, seed)
        if not self._h:
            raise ValueError("bad TCF geometry")
        g = np.zeros(8, dtype=np.uint64)
        lib().or_tcf_geometry(self._h, _p(g, _u64p))
        self.nb, self.B, self.f, self.tsc, self.nbk, self.W, self.v, self.block_bytes = (int(v) for v in g)
        self.log2_slots, self.seed = log2_slots, seed

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_tcf_free(self._h)
            self._h = None

    def keyinfo(self, keys):
        keys = _u64(keys)
        b1 = np.empty(keys.size, np.uint64)
        b2 = np.empty(keys.size, np.uint64)
        t = np.empty(keys.size, np.uint32)
        lib().or_tcf_keyinfo(self._h, _p(keys, _u64p), keys.size, _p(b1, _u64p), _p(b2, _u64p),
                             _p(t, _u32p))
        return b1, b2, t

    def fingerprints(self, keys):
        """Canonical fingerprint id: (min(b1, b2) << f) | tag."""
        b1, b2, t = self.keyinfo(keys)
        return (np.minimum(b1, b2) << np.uint64(self.f)) | t.astype(np.uint64)

    def insert(self, keys, trace: bool = False, values=None):
        keys = _u64(keys)
        st = np.zeros(keys.size, np.uint8)
        vp = None
        if values is not None:
            values = np.ascontiguousarray(values, dtype=np.uint8)
            assert values.size == keys.size
            vp = _p(values, _u8p)
        if trace:
            ph = np.zeros(keys.size, np.uint8)
            wh = np.zeros(keys.size, np.uint64)
            lib().or_tcf_insert_values(self._h, _p(keys, _u64p), vp, keys.size, _p(st, _u8p), _p(ph, _u8p),
                                       _p(wh, _u64p))
            return st, ph, wh
        lib().or_tcf_insert_values(self._h, _p(keys, _u64p), vp, keys.size, _p(st, _u8p), None, None)
        return st

    def query_values(self, keys):
        """Smallest value stored with each key's fingerprint, 0xFF if none."""
        keys = _u64(keys)
        out = np.zeros(keys.size, np.uint8)
        lib().or_tcf_query_values(self._h, _p(keys, _u64p), keys.size, _p(out, _u8p))
        return out

    def query(self, keys):
        keys = _u64(keys)
        out = np.zeros(keys.size, np.uint8)
        lib().or_tcf_query(self._h, _p(keys, _u64p), keys.size, _p(out, _u8p))
        return out

    def remove(self, keys):
        keys = _u64(keys)
        st = np.zeros(keys.size, np.uint8)
        lib().or_tcf_remove(self._h, _p(keys, _u64p), keys.size, _p(st, _u8p))
        return st

    def export(self) -> np.ndarray:
        n = lib().or_tcf_export_size(self._h)
        buf = np.zeros(n, np.uint8)
        lib().or_tcf_export(self._h, _p(buf, _u8p))
        return buf

    def blocks(self) -> np.ndarray:
        """Slots per block, unpacked from the image (nb x B, uint16)."""
        raw = self.export()[: self.nb * self.block_bytes].reshape(self.nb, self.block_bytes)
        bits = np.unpackbits(raw, axis=1, bitorder="little")[:, : self.B * self.f]
        w = (1 << np.arange(self.f)).astype(np.uint32)
        return (bits.reshape(self.nb, self.B, self.f).astype(np.uint32) @ w).astype(np.uint16)

    def buckets(self) -> np.ndarray:
        return self.export()[self.nb * self.block_bytes:].view(np.uint64).reshape(self.nbk, self.W)

    def backing_count(self) -> int:
        return lib().or_tcf_backing_count(self._h)

    def stored_count(self) -> int:
        return lib().or_tcf_stored_count(self._h)


def gqf_tail_slots(q: int) -> int:
    return lib().or_gqf_tail_slots(q)


class GQF:
    """Counting quotient filter (see gqf.c for the specification)."""

    def __init__(self, q: int, r: int = 8, seed: int = 0):
        self._h = lib().or_gqf_new(q, r, seed)
        if not self._h:
            raise ValueError("bad GQF geometry")
        g = np.zeros(5, dtype=np.uint64)
        lib().or_gqf_geometry(self._h, _p(g, _u64p))
        self.N, self.S, self.nslots, self.nblk, self.p = (int(v) for v in g)
        self.q, self.r, self.seed = q, r, seed

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_gqf_free(self._h)
            self._h = None

    def fingerprints(self, keys):
        keys = _u64(keys)
        out = np.empty_like(keys)
        lib().or_gqf_fingerprints(self._h, _p(keys, _u64p), keys.size, _p(out, _u64p))
        return out

    def insert(self, keys):
        keys = _u64(keys)
        st = np.zeros(keys.size, np.uint8)
        lib().or_gqf_insert(self._h, _p(keys, _u64p), keys.size, _p(st, _u8p))
        return st

    def insert_counts(self, keys, counts):
        """Key i counts as counts[i] >= 1 copies."""
        keys = _u64(keys)
        counts = np.ascontiguousarray(counts, dtype=np.uint32)
        assert counts.size == keys.size
        st = np.zeros(keys.size, np.uint8)
        lib().or_gqf_insert_counts(self._h, _p(keys, _u64p), _p(counts, _u32p), keys.size, _p(st, _u8p))
        return st

    def remove(self, keys):
        keys = _u64(keys)
        st = np.zeros(keys.size, np.uint8)
        lib().or_gqf_remove(self._h, _p(keys, _u64p), keys.size, _p(st, _u8p))
        return st

    def count(self, keys):
        keys = _u64(keys)
        out = np.zeros(keys.size, np.uint64)
        lib().or_gqf_count(self._h, _p(keys, _u64p), keys.size, _p(out, _u64p))
        return out

    def insert_groups(self, fps, cnts) -> int:
        fps, cnts = _u64(fps), _u64(cnts)
        return lib().or_gqf_insert_groups(self._h, _p(fps, _u64p), _p(cnts, _u64p), fps.size)

    def count_fp(self, fp: int) -> int:
        return lib().or_gqf_count_fp(self._h, fp)

    def groups(self):
        n = lib().or_gqf_groups(self._h, None, None, 0)
        f = np.zeros(n, np.uint64)
        c = np.zeros(n, np.uint64)
        lib().or_gqf_groups(self._h, _p(f, _u64p), _p(c, _u64p), n)
        return f, c

    def export(self) -> np.ndarray:
        n = lib().or_gqf_export_size(self._h)
        buf = np.zeros(n, np.uint8)
        lib().or_gqf_export(self._h, _p(buf, _u8p))
        return buf

    def max_cluster(self) -> int:
        return lib().or_gqf_max_cluster(self._h)


def gqf_build(q: int, r: int, fps, cnts):
    """Canonical byte image of a sorted distinct group list, or None if it does not fit."""
    fps, cnts = _u64(fps), _u64(cnts)
    N = 1 << q
    S = gqf_tail_slots(q)
    size = (N + S) // 64 * 32 + (N + S) * (r // 8)
    buf = np.zeros(size, np.uint8)
    bad = lib().or_gqf_build(q, r, _p(fps, _u64p), _p(cnts, _u64p), fps.size, _p(buf, _u8p))
    return None if bad else buf
