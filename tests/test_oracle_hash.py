"""Pins for the oracle's hashing (the fingerprint function of Sec. 5.1 and the
TCF block/tag hash of Sec. 4): bijectivity, inverses and mixing quality."""
import numpy as np
import pytest

from paper_2212_09005_gb300.workloads import splitmix64, uniform_keys


def test_splitmix64_published_outputs():
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0: first three outputs
    # as listed with the reference generator.
    got = [int(x) for x in splitmix64(0, 0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_mix64_inverse_roundtrip(oracle):
    xs = uniform_keys(11, 20000)
    for x in xs[:2000].tolist():
        assert oracle.unmix64(oracle.mix64(x)) == x
        assert oracle.mix64(oracle.unmix64(x)) == x


@pytest.mark.parametrize("p", [14, 20, 28, 36, 44, 63, 64])
def test_mix_p_inverse_roundtrip(oracle, p):
    m = (1 << p) - 1
    for x in uniform_keys(12 + p, 1000).tolist():
        x &= m
        y = oracle.mix_p(x, p)
        assert 0 <= y <= m
        assert oracle.unmix_p(y, p) == x


@pytest.mark.parametrize("p", [8, 12, 16, 20])
def test_mix_p_is_a_permutation_exhaustive(oracle, p):
    xs = np.arange(1 << p, dtype=np.uint64)
    ys = oracle.mix_p_many(xs, p)
    assert ys.max() < (1 << p)
    assert np.unique(ys).size == (1 << p)


def test_mix_p_64_equals_shift32_variant_of_mix64_family(oracle):
    # p = 64 uses shift 32; mix64 uses shift 33: both are bijections but differ.
    xs = uniform_keys(13, 64).tolist()
    assert any(oracle.mix_p(x, 64) != oracle.mix64(x) for x in xs)


def test_fold_identity_below_2p(oracle):
    for p in (20, 28, 36):
        for x in uniform_keys(14, 200).tolist():
            x &= (1 << p) - 1
            assert oracle.fold_p(x, p) == x


def test_fold_xors_chunks(oracle):
    # fold_p(a + b * 2^p) = a xor b for a, b < 2^p and a 2p-bit value
    p = 28
    a, b = 0x0ABCDEF, 0x1234567
    assert oracle.fold_p(a | (b << p), p) == a ^ b
    assert oracle.fold_p(1 << 63, 21) == 1  # bit 63 = chunk 3, bit 0


@pytest.mark.parametrize("which", ["mix64", "mix36"])
def test_avalanche(oracle, which):
    """Flipping one input bit flips about half of the output bits."""
    rng_keys = uniform_keys(15, 400).tolist()
    bits = 64 if which == "mix64" else 36
    f = oracle.mix64 if which == "mix64" else (lambda x: oracle.mix_p(x, 36))
    m = (1 << bits) - 1
    tot, n = 0, 0
    worst = 1.0
    for i in range(bits):
        flips = 0
        for x in rng_keys:
            x &= m
            flips += bin(f(x) ^ f(x ^ (1 << i))).count("1")
        frac = flips / (len(rng_keys) * bits)
        worst = min(worst, frac, 1 - frac)
        tot += flips
        n += len(rng_keys) * bits
    assert abs(tot / n - 0.5) < 0.01
    assert worst > 0.40


def _murmur3_x64_128(data: bytes, seed: int, fmix) -> bytes:
    """MurmurHash3_x64_128 (Appleby, SMHasher), written from the published
    algorithm, with its 64-bit finaliser passed in as `fmix`."""
    M = (1 << 64) - 1

    def rotl(x, r):
        return ((x << r) | (x >> (64 - r))) & M

    c1, c2 = 0x87C37B91114253D5, 0x4CF5AD432745937F
    n = len(data)
    h1 = h2 = seed & 0xFFFFFFFF
    nb = n // 16
    for i in range(nb):
        k1 = int.from_bytes(data[16 * i:16 * i + 8], "little")
        k2 = int.from_bytes(data[16 * i + 8:16 * i + 16], "little")
        h1 ^= (rotl((k1 * c1) & M, 31) * c2) & M
        h1 = (((rotl(h1, 27) + h2) & M) * 5 + 0x52DCE729) & M
        h2 ^= (rotl((k2 * c2) & M, 33) * c1) & M
        h2 = (((rotl(h2, 31) + h1) & M) * 5 + 0x38495AB5) & M
    tail = data[16 * nb:]
    if len(tail) > 8:
        k2 = int.from_bytes(tail[8:], "little")
        h2 ^= (rotl((k2 * c2) & M, 33) * c1) & M
    if tail:
        k1 = int.from_bytes(tail[:8], "little")
        h1 ^= (rotl((k1 * c1) & M, 31) * c2) & M
    h1 ^= n
    h2 ^= n
    h1 = (h1 + h2) & M
    h2 = (h2 + h1) & M
    h1, h2 = fmix(h1), fmix(h2)
    h1 = (h1 + h2) & M
    h2 = (h2 + h1) & M
    return h1.to_bytes(8, "little") + h2.to_bytes(8, "little")


def test_mix64_is_the_murmur3_finaliser_smhasher_verification(oracle):
    """mix64 is MurmurHash3's fmix64. Pinned by SMHasher's published
    verification code of MurmurHash3_x64_128, 0x6384BA69: hash the keys
    {}, {0}, {0,1}, .. {0..254} with seeds 256, 255, .. 1, hash the 256
    concatenated 16-byte results with seed 0, and read the first 4 bytes
    little-endian. A wrong constant, shift or round in mix64 changes it."""
    hashes = b"".join(_murmur3_x64_128(bytes(range(i)), 256 - i, oracle.mix64) for i in range(256))
    final = _murmur3_x64_128(hashes, 0, oracle.mix64)
    assert int.from_bytes(final[:4], "little") == 0x6384BA69
    assert oracle.mix64(0) == 0  # fmix64 fixes 0: the x64_128 hash of no bytes with seed 0 is all zero
