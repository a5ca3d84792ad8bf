"""The Zipf sampler of the counting workload (rejection-inversion, Hörmann
and Derflinger 1996) against the exact distribution P(k) = k^-s / H_{N,s}:
a chi-square test on small universes, the range, and the head ratio
P(1)/P(2) = 2^s; and the workload's documented shape at full scale is
checked on a sample (hottest key near n / H_{2^32,1})."""
import numpy as np
import pytest
from scipy import stats

from paper_2212_09005_gb300 import workloads as W


@pytest.mark.parametrize("s,universe", [(1.0, 50), (1.5, 50), (0.8, 200), (1.0, 5)])
def test_matches_the_exact_pmf(s, universe):
    n = 400_000
    r = W.zipf_ranks(17 + universe, n, s, universe)
    assert r.min() >= 1 and r.max() <= universe
    k = np.arange(1, universe + 1)
    p = k ** -s / (k ** -s).sum()
    obs = np.bincount(r, minlength=universe + 1)[1:]
    chi2, pval = stats.chisquare(obs, n * p)
    assert pval > 1e-4, (chi2, pval)
    ratio = obs[0] / obs[1]
    assert abs(ratio - 2 ** s) < 6 * 2 ** s * np.sqrt(1 / obs[0] + 1 / obs[1])


def test_reproducible_and_seed_dependent():
    a = W.zipf_ranks(5, 10_000, 1.0, 1 << 32)
    assert np.array_equal(a, W.zipf_ranks(5, 10_000, 1.0, 1 << 32))
    assert not np.array_equal(a, W.zipf_ranks(6, 10_000, 1.0, 1 << 32))


def test_head_of_the_full_universe():
    """Over 2^32 ranks with s = 1, P(1) = 1 / H_{2^32} with H_N ~ ln N + 0.5772
    (about 0.0438): the share of rank 1 in a sample matches it."""
    n = 2_000_000
    r = W.zipf_ranks(3, n, 1.0, 1 << 32)
    p1 = 1.0 / (np.log(2.0 ** 32) + 0.5772156649 + 1 / (2 * 2.0 ** 32))
    share = (r == 1).mean()
    assert abs(share - p1) < 5 * np.sqrt(p1 * (1 - p1) / n), (share, p1)
    keys = W.zipf_keys(3, 1000, 1.0, 1 << 32)
    assert keys.dtype == np.uint64 and int(keys.max()) < (1 << 32)
