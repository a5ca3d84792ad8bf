"""Pins for the oracle TCF with values (Sec. 1 and Sec. 4: the TCF associates
small values with items). A slot of f bits holds an (f - v)-bit tag above a
v-bit value. Checked here by brute force over the stored multiset: values
never change where a key goes, a value query answers the smallest value stored
with the key's fingerprint, deletes remove the smallest value of the first
block holding a copy, and the false-positive rate follows the closed form with
f - v tag bits."""
import collections

import numpy as np
import pytest

from paper_2212_09005_gb300.workloads import uniform_keys

V = 4


def masked(T):
    m = np.uint16(0xFFFF ^ ((1 << T.v) - 1))
    return T.blocks() & m, T.buckets() & ~np.uint64((1 << T.v) - 1)


def stored_values(T, tag_to_g):
    """(fingerprint, value) pairs read back from the table, as a multiset."""
    out = collections.Counter()
    vm = (1 << T.v) - 1
    blocks = T.blocks()
    for b, s in zip(*np.nonzero(blocks)):
        x = int(blocks[b, s])
        t = x & ~vm
        b2 = int(b) ^ tag_to_g[t]
        out[((min(int(b), b2) << T.f) | t, x & vm)] += 1
    for e in T.buckets().ravel().tolist():
        if e:
            out[(e & ~vm, e & vm)] += 1
    return out


def tag_g_map(T, keys):
    b1, b2, t = T.keyinfo(keys)
    return {int(a): int(x ^ y) for a, x, y in zip(t, b1, b2)}


def test_geometry_and_tag_width(oracle):
    T = oracle.TCF(12, 16, seed=1, value_bits=V)
    assert (T.f, T.B, T.v) == (16, 16, V)
    _, _, t = T.keyinfo(uniform_keys(80, 50000))
    assert (t & ((1 << V) - 1) == 0).all()  # the value part of a bare key is 0
    tags = t >> V
    assert tags.min() >= 2 and tags.max() < (1 << (16 - V))
    assert len(np.unique(tags)) > 3000  # all 12 bits are used
    with pytest.raises(ValueError):
        oracle.TCF(12, 16, value_bits=8)  # 0xFF must stay free to answer "absent"
    with pytest.raises(ValueError):
        oracle.TCF(12, 8, value_bits=5)


def test_values_never_change_placement(oracle):
    """The same keys with random values and with all values 0: after every
    batch the images agree once the value bits are cleared, and so do the
    statuses (bucket choice and acceptance depend on the tag only)."""
    A = oracle.TCF(13, 16, seed=3, value_bits=V)
    Z = oracle.TCF(13, 16, seed=3, value_bits=V)
    keys = uniform_keys(81, int(0.97 * (1 << 13)))
    keys = np.concatenate([keys, keys[:300]])
    vals = np.random.default_rng(5).integers(0, 16, keys.size).astype(np.uint8)
    for s in range(0, keys.size, 1500):
        st_a = A.insert(keys[s:s + 1500], values=vals[s:s + 1500])
        st_z = Z.insert(keys[s:s + 1500])
        assert np.array_equal(st_a, st_z)
        for x, y in zip(masked(A), masked(Z)):
            assert np.array_equal(x, y)
    assert A.backing_count() > 0
    st_a = A.remove(keys[::3])
    st_z = Z.remove(keys[::3])
    assert np.array_equal(st_a, st_z)
    for x, y in zip(masked(A), masked(Z)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("f,v", [(16, 4), (16, 7), (8, 2)])
def test_value_query_is_min_of_stored_values(oracle, f, v):
    log2 = 12
    T = oracle.TCF(log2, f, seed=7 + v, value_bits=v)
    keys = uniform_keys(82 + v, int(0.92 * (1 << log2)))
    keys = np.concatenate([keys, keys[:400], keys[:100]])  # repeated keys carry other values
    vals = np.random.default_rng(v).integers(0, 1 << v, keys.size).astype(np.uint8)
    gmap = tag_g_map(T, keys)
    want = collections.Counter()
    fps = T.fingerprints(keys).tolist()
    for s in range(0, keys.size, 700):
        st = T.insert(keys[s:s + 700], values=vals[s:s + 700])
        for j in np.nonzero(st == 0)[0]:
            want[(fps[s + j], int(vals[s + j]))] += 1
    assert stored_values(T, gmap) == want
    best = {}
    for (fp, val), c in want.items():
        best[fp] = min(best.get(fp, 0xFF), val)
    probe = np.concatenate([keys[:2500], uniform_keys(90 + v, 5000)])
    exp = np.array([best.get(fp, 0xFF) for fp in T.fingerprints(probe).tolist()], np.uint8)
    assert np.array_equal(T.query_values(probe), exp)
    assert np.array_equal(T.query(probe), (exp != 0xFF).astype(np.uint8))

    # deletes: the stored pairs lose exactly one copy per successful delete,
    # of the deleted key's fingerprint, and the value query follows the table
    gone = keys[1::4]
    st = T.remove(gone)
    after = stored_values(T, gmap)
    lost = want - after
    assert not (after - want)
    per_fp = collections.Counter(fp for (fp, _), c in lost.items() for _ in range(c))
    ok = collections.Counter(np.asarray(T.fingerprints(gone))[st == 0].tolist())
    assert per_fp == ok
    best = {}
    for (fp, val), c in after.items():
        best[fp] = min(best.get(fp, 0xFF), val)
    exp = np.array([best.get(fp, 0xFF) for fp in T.fingerprints(probe).tolist()], np.uint8)
    assert np.array_equal(T.query_values(probe), exp)


def test_delete_takes_the_smallest_value_of_the_first_block(oracle):
    """One key inserted three times with values 7, 3 and 9: all three copies
    go to its first block (shortcut), so deletes remove 3, then 7, then 9."""
    T = oracle.TCF(10, 16, seed=11, value_bits=V)
    k = uniform_keys(91, 1)
    T.insert(np.repeat(k, 3), values=np.array([7, 3, 9], np.uint8))
    seen = [int(T.query_values(k)[0])]
    for _ in range(3):
        assert T.remove(k)[0] == 0
        seen.append(int(T.query_values(k)[0]))
    assert seen == [3, 7, 9, 0xFF]
    assert T.remove(k)[0] == 2


def test_fpr_closed_form_with_values(oracle):
    """Same closed form as for the plain filter, with f - v tag bits:
    2 d (2^(f-v) + 4) / (nb 4^(f-v))."""
    log2 = 16
    T = oracle.TCF(log2, 16, seed=19, value_bits=V)
    keys = uniform_keys(92, int(0.9 * (1 << log2)))
    vals = (keys & np.uint64(15)).astype(np.uint8)
    for s in range(0, keys.size, 1 << 13):
        T.insert(keys[s:s + (1 << 13)], values=vals[s:s + (1 << 13)])
    tb = 16 - V
    d = len(set(T.fingerprints(keys).tolist()))
    eps = 2 * d * (2 ** tb + 4) / (T.nb * 4 ** tb)
    neg = uniform_keys(1092, 1 << 18)
    fpr = T.query(neg).mean()
    sigma = np.sqrt(eps * (1 - eps) / neg.size)
    assert abs(fpr - eps) <= 4 * sigma, (fpr, eps, sigma)
