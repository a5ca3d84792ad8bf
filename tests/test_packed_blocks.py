"""CPU tests of the packed TCF block functions (gf_packed.cuh), built for the
host: slot reads and writes against an independent bit-level reading of the
layout (slot s at bits F s .. F s + F - 1, little-endian, padding 0), and the
sorted-block operations against Python lists."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEOMS = [(16, 16), (8, 32), (12, 21), (12, 42), (16, 8), (16, 64), (16, 128), (8, 64)]


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("packed") / "libpacked.so")
    src = os.path.join(ROOT, "tests", "packed", "packed_shim.cpp")
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                        os.path.join(ROOT, "paper_2212_09005_gb300", "csrc"), "-o", out, src],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = C.CDLL(out)
    u32p = C.POINTER(C.c_uint32)
    lib.packed_op.argtypes = [C.c_int, C.c_int, C.c_int, u32p, C.c_int, C.c_int, u32p, u32p]
    lib.packed_op.restype = C.c_int
    return lib


def words_of(f, B):
    return (f * B + 255) // 256 * 8


class Block:
    def __init__(self, lib, f, B):
        self.lib, self.f, self.B = lib, f, B
        self.w = np.zeros(words_of(f, B), np.uint32)

    def op(self, op, a=0, b=0, nv=(0,)):
        nv = np.ascontiguousarray(nv, dtype=np.uint32)
        out = np.zeros(1, np.uint32)
        p = lambda x: x.ctypes.data_as(C.POINTER(C.c_uint32))
        assert self.lib.packed_op(self.f, self.B, op, p(self.w), a, b, p(nv), p(out)) == self.w.size
        return int(out[0])

    def decode(self):
        x = int.from_bytes(self.w.tobytes(), "little")
        slots = [(x >> (self.f * s)) & ((1 << self.f) - 1) for s in range(self.B)]
        return slots, (x >> (self.f * self.B)) == 0


@pytest.mark.parametrize("f,B", GEOMS)
def test_get_set_follow_the_bit_layout(shim, f, B):
    rng = np.random.default_rng(f * 1000 + B)
    blk = Block(shim, f, B)
    model = [0] * B
    for _ in range(4 * B):
        s = int(rng.integers(0, B))
        v = int(rng.integers(0, 1 << f))
        blk.op(1, s, v)
        model[s] = v
        slots, pad = blk.decode()
        assert slots == model and pad
        t = int(rng.integers(0, B))
        assert blk.op(0, t) == model[t]
    assert blk.op(2) == sum(1 for v in model if v)


@pytest.mark.parametrize("f,B", GEOMS)
def test_sorted_block_operations(shim, f, B):
    rng = np.random.default_rng(f * 7 + B)
    vbits = 4 if f >= 12 else 2
    tmask = ((1 << f) - 1) & ~((1 << vbits) - 1)
    for trial in range(30):
        blk = Block(shim, f, B)
        live = []
        while len(live) < B:
            k = int(rng.integers(1, max(2, B // 3)))
            k = min(k, B - len(live))
            # few distinct tags, so equal tags with different values occur
            new = sorted(int(rng.integers(2, 6)) << vbits | int(rng.integers(0, 1 << vbits)) for _ in range(k))
            blk.op(4, len(live), k, new)
            live = sorted(live + new)
            slots, pad = blk.decode()
            assert slots == live + [0] * (B - len(live)) and pad
            for t in (2 << vbits, 3 << vbits, 6 << vbits):
                exp = next((i for i, x in enumerate(live) if x & tmask == t), -1)
                assert blk.op(3, nv=(t, tmask)) == (exp & 0xFFFFFFFF)
                vals = [x & ~tmask & ((1 << f) - 1) for x in live if x & tmask == t]
                assert blk.op(6, nv=(t, tmask)) == (min(vals) if vals else 1 << f)
            if rng.random() < 0.5 and live:
                s = int(rng.integers(0, len(live)))
                blk.op(5, s, len(live))
                del live[s]
                slots, pad = blk.decode()
                assert slots == live + [0] * (B - len(live)) and pad
