"""The synthetic k-mer workload (stand-in for the sequencing reads whose
k-mers the paper counts, Sec. 6): canonical k-mers against a string-based
brute force, the fast generator against the read-by-read one."""
import numpy as np

from paper_2212_09005_gb300 import workloads as W

BASES = "ACGT"
COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def pack(s):
    v = 0
    for ch in s:
        v = (v << 2) | BASES.index(ch)
    return v


def canonical_by_strings(read, k):
    out = []
    for i in range(len(read) - k + 1):
        f = read[i:i + k]
        r = "".join(COMP[c] for c in reversed(f))
        out.append(min(pack(f), pack(r)))
    return out


def test_canonical_kmers_equal_string_brute_force():
    reads = W.synthetic_reads(20, seed=11, read_len=40, genome_len=1 << 12, error_rate=0.05)
    for k in (5, 21, 28, 32):
        got = W.kmers_of_reads(reads, k).reshape(len(reads), -1)
        for row, read in zip(got, reads):
            s = "".join(BASES[b] for b in read)
            assert [int(v) for v in row] == canonical_by_strings(s, k)


def test_canonical_form_is_strand_independent():
    reads = W.synthetic_reads(50, seed=12, read_len=60, genome_len=1 << 12)
    rc = (3 - reads[:, ::-1]).astype(np.uint8)
    a = np.sort(W.kmers_of_reads(reads, 25))
    b = np.sort(W.kmers_of_reads(rc, 25))
    assert np.array_equal(a, b)


def test_fast_reverse_complement_equals_the_loop():
    x = W.uniform_keys(13, 20000)
    for k in (1, 7, 21, 28, 31, 32):
        m = np.uint64((1 << (2 * k)) - 1) if k < 32 else np.uint64(0xFFFFFFFFFFFFFFFF)
        v = x & m
        assert np.array_equal(W._revcomp_fast(v, k), W.revcomp_kmer(v, k))


def test_fast_generator_equals_read_by_read():
    """The generator cuts k-mers from the genome and patches the bits of each
    sequencing error; that must equal extracting them from the erroneous reads."""
    for k, rl, err in ((28, 100, 0.005), (21, 50, 0.05), (31, 31, 0.02)):
        n = 30000
        per = rl - k + 1
        got = W.kmer_workload(n, seed=14, k=k, read_len=rl, genome_len=1 << 14, error_rate=err, chunk_reads=97)
        reads = W.synthetic_reads((n + per - 1) // per, seed=14, read_len=rl, genome_len=1 << 14, error_rate=err)
        assert np.array_equal(got, W.kmers_of_reads(reads, k)[:n])


def test_workload_shape_and_repeats():
    x = W.kmer_workload(200000, seed=15, genome_len=1 << 14)
    assert x.dtype == np.uint64 and x.size == 200000
    assert int(x.max()) < (1 << 56)
    u, c = np.unique(x, return_counts=True)
    # about (2^14 - 27) genomic 28-mers at ~20x coverage plus unique error k-mers
    assert c.max() >= 10 and (c == 1).sum() > 0 and u.size < x.size
