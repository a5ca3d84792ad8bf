"""Reader for the hand-derived GQF fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    spec = {"groups": [], "meta": {}, "slots": {}, "counts": []}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tag, *rest = line.split()
            if tag == "q":
                spec["q"] = int(rest[0])
            elif tag == "r":
                spec["r"] = int(rest[0])
            elif tag == "g":
                spec["groups"].append(tuple(int(v) for v in rest))
            elif tag == "m":
                spec["meta"][int(rest[0])] = (int(rest[1], 16), int(rest[2], 16), int(rest[3]))
            elif tag == "s":
                spec["slots"][int(rest[0])] = int(rest[1])
            elif tag == "c":
                spec["counts"].append(tuple(int(v) for v in rest))
    return spec


def expected_image(spec, nslots, nblk):
    """Byte image (metadata blocks, then remainders) described by a fixture."""
    r = spec["r"]
    buf = np.zeros(nblk * 32 + nslots * (r // 8), np.uint8)
    for j, (occ, rend, off) in spec["meta"].items():
        buf[32 * j:32 * j + 8] = np.frombuffer(np.uint64(occ).tobytes(), np.uint8)
        buf[32 * j + 8:32 * j + 16] = np.frombuffer(np.uint64(rend).tobytes(), np.uint8)
        buf[32 * j + 16:32 * j + 20] = np.frombuffer(np.uint32(off).tobytes(), np.uint8)
    rem = buf[nblk * 32:]
    for s, v in spec["slots"].items():
        if r == 8:
            rem[s] = v
        else:
            rem[2 * s] = v & 0xFF
            rem[2 * s + 1] = v >> 8
    return buf


def group_arrays(spec):
    r = spec["r"]
    fps = np.array([(x << r) | v for x, v, _ in spec["groups"]], np.uint64)
    cnt = np.array([c for _, _, c in spec["groups"]], np.uint64)
    order = np.argsort(fps, kind="stable")
    return fps[order], cnt[order]
