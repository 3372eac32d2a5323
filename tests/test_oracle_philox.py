"""Pins for the oracle's counter-based sampler (CPU only)."""
import numpy as np
import pytest
import scipy.stats

from oracle import philox


@pytest.mark.parametrize("key,counter", [((1, 2), (0, 0, 0, 0)), ((7, 0), (5, 3, 2, 1 << 32)),
                                         ((2**64 - 1, 12345), (2**64 - 2, 2**64 - 1, 7, 9))])
def test_philox_matches_numpy(key, counter):
    """Philox4x64-10 equals numpy's library generator (which increments its
    counter before each block, so block c+1 of ours is its first output)."""
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(counter, dtype=np.uint64))
    ref = bg.random_raw(8)
    c = list(counter)
    for blk in range(2):
        # increment the 256-bit counter with carry, as the library does
        for w in range(4):
            c[w] = (c[w] + 1) & philox.MASK64
            if c[w] != 0:
                break
        out = philox.philox4x64_10(c, key)
        assert [int(v) for v in ref[4 * blk:4 * blk + 4]] == list(out)


def test_uniform_indices_range_and_chi2():
    I, m = 37, 20000
    idx = philox.uniform_indices(7, m, I, k=2, tau=3)
    assert idx.min() >= 0 and idx.max() < I
    counts = np.bincount(idx, minlength=I)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4


def test_uniform_index_is_multiply_high():
    u = philox.draw_u64(11, 5, 1, 0, philox.PURPOSE_INDEX)
    assert philox.uniform_indices(11, 6, 1000, 1, 0)[5] == (u * 1000) >> 64


def test_weighted_indices_follow_p_and_skip_zeros():
    rng = np.random.default_rng(0)
    p = rng.random(25)
    p[[0, 3, 24]] = 0.0
    p /= p.sum()
    m = 30000
    idx = philox.weighted_indices(3, m, p, k=1, tau=0)
    assert not np.isin(idx, [0, 3, 24]).any()
    counts = np.bincount(idx, minlength=25)
    nz = p > 0
    assert scipy.stats.chisquare(counts[nz], m * p[nz]).pvalue > 1e-4


def test_weighted_index_definition_by_linear_scan():
    rng = np.random.default_rng(1)
    p = rng.random(40)
    idx = philox.weighted_indices(9, 200, p, k=3, tau=4)
    c = 0.0
    cdf = []
    for v in p:
        c = c + v
        cdf.append(c)
    for s in range(200):
        u = philox.draw_u64(9, s, 3, 4, philox.PURPOSE_INDEX)
        target = float(u >> 11) * 2.0 ** -53 * cdf[-1]
        first = next(i for i, ci in enumerate(cdf) if target < ci)
        assert idx[s] == first


def test_signs_balanced():
    d = philox.signs(5, 4000, k=1, tau=2)
    assert set(np.unique(d)) <= {-1.0, 1.0}
    assert abs(d.mean()) < 4 / np.sqrt(4000)


def test_streams_and_steps_are_distinct():
    a = philox.uniform_indices(1, 64, 1 << 20, 1, 1, stream=0)
    b = philox.uniform_indices(1, 64, 1 << 20, 1, 1, stream=1)
    c = philox.uniform_indices(1, 64, 1 << 20, 1, 2, stream=0)
    assert (a != b).sum() > 60 and (a != c).sum() > 60
