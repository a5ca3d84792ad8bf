"""The oracle TCF against a worked example derived by hand from the paper's
placement rules (tests/golden/tcf_q6_f16_worked.txt): the shortcut limit,
the two-choice target with its tie, the other block, the backing table, the
sorted blocks, and deletes from b1, b2 and the backing table with one copy
per key. Pins the table bytes, not only the answers."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    spec = {"keyinfo": {}}
    for line in open(os.path.join(HERE, "golden", name)):
        line = line.split("#", 1)[0].split()
        if not line:
            continue
        tag, vals = line[0], [int(x) for x in line[1:]]
        if tag == "keyinfo":
            spec["keyinfo"][vals[0]] = tuple(vals[1:])
        elif tag.startswith(("block", "bucket")):
            spec.setdefault(tag, {})[vals[0]] = vals[1:]
        else:
            spec[tag] = vals
    return spec


def expect_rows(rows, nrows, width, dtype):
    out = np.zeros((nrows, width), dtype)
    for r, vals in rows.items():
        out[r, :len(vals)] = vals
    return out


def test_worked_example(oracle):
    spec = load("tcf_q6_f16_worked.txt")
    T = oracle.TCF(6, 16, seed=0)
    assert (T.nb, T.B, T.tsc, T.nbk, T.W) == (4, 16, 12, 8, 8)
    keys = np.array(sorted(spec["keyinfo"]), np.uint64)
    b1, b2, t = T.keyinfo(keys)
    for k, x, y, z in zip(keys.tolist(), b1.tolist(), b2.tolist(), t.tolist()):
        assert spec["keyinfo"][k] == (x, y, z), k

    st, ph, _ = T.insert(np.array(spec["batch1"], np.uint64), trace=True)
    assert (st == 0).all()
    assert ph.tolist() == spec["phase1"]
    assert np.array_equal(T.blocks(), expect_rows(spec["block1"], 4, 16, np.uint16))
    assert not T.buckets().any()

    st, ph, _ = T.insert(np.array(spec["batch2"], np.uint64), trace=True)
    assert (st == 0).all() and ph.tolist() == spec["phase2"]
    assert np.array_equal(T.blocks(), expect_rows(spec["block1"], 4, 16, np.uint16))
    assert np.array_equal(T.buckets(), expect_rows(spec["bucket2"], 8, 8, np.uint64))

    st = T.remove(np.array(spec["delete"], np.uint64))
    assert st.tolist() == spec["delete_status"]
    assert np.array_equal(T.blocks(), expect_rows(spec["block3"], 4, 16, np.uint16))
    assert np.array_equal(T.buckets(), expect_rows(spec["bucket3"], 8, 8, np.uint64))
    stored = [k for k in spec["batch1"] + spec["batch2"] if k not in (3, 64, 201, 5, 36)]
    assert T.query(np.array(stored, np.uint64)).all()
