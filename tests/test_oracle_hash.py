"""Pins for the counter-based s-hashing draw (Def. 5, Example 1, Def. 8's D)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import hashing

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if l.startswith("0x")]
    for i, want in enumerate(vals):
        assert hashing.splitmix64((i * hashing.SM_GAMMA) & hashing.MASK64) == want


@pytest.mark.parametrize("s,m", [(1, 7), (2, 3), (3, 5), (4, 4), (2, 1000)])
def test_vectorised_table_equals_pure_python(s, m):
    n = 300
    idx, sign = hashing.hash_table(1234567, s, m, n)
    for j in range(n):
        rows, signs = hashing.column_rows_int(1234567, s, m, j)
        assert list(idx[j]) == rows
        assert list(sign[j]) == signs


def test_rows_distinct_in_range_and_signs():
    idx, sign = hashing.hash_table(99, 3, 11, 5000)
    assert idx.min() >= 0 and idx.max() < 11
    srt = np.sort(idx, axis=1)
    assert (srt[:, 1:] != srt[:, :-1]).all()
    assert set(np.unique(sign)) == {-1, 1}


def test_s_equals_m_takes_every_row():
    idx, _ = hashing.hash_table(5, 6, 6, 200)
    assert (np.sort(idx, axis=1) == np.arange(6)).all()


def test_bucket_uniformity_chi_square():
    m = 64
    idx, _ = hashing.hash_table(2021, 1, m, 200_000)
    counts = np.bincount(idx[:, 0], minlength=m)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_uniform_over_subsets_without_replacement():
    # Def. 5 samples s rows without replacement: every s-subset equally likely.
    m, s, n = 5, 2, 100_000
    idx, _ = hashing.hash_table(77, s, m, n)
    code = np.sort(idx, axis=1) @ np.array([m, 1])
    counts = np.unique(code, return_counts=True)[1]
    assert counts.size == math.comb(m, s)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_signs_and_premix_signs_balanced():
    _, sign = hashing.hash_table(3, 2, 50, 100_000)
    for k in range(2):
        p = stats.binomtest(int((sign[:, k] > 0).sum()), sign.shape[0], 0.5).pvalue
        assert p > 1e-4
    D = hashing.premix_signs(3, 100_000)
    assert stats.binomtest(int((D > 0).sum()), D.size, 0.5).pvalue > 1e-4
    assert all(D[j] == hashing.premix_sign_int(3, j) for j in range(50))


def test_example1_birthday_probability():
    # Example 1: for A = [I_r 0; 0 0], rank(SA) = r iff the first r columns of
    # S fall in distinct rows, probability prod_{k<r}(1 - k/m).
    r, m, trials = 8, 40, 4000
    exact = np.prod([1 - k / m for k in range(r)])
    hits = 0
    for seed in range(trials):
        idx, sign = hashing.hash_table(seed, 1, m, r)
        S1 = np.zeros((m, r))
        S1[idx[:, 0], np.arange(r)] = sign[:, 0]
        full = np.linalg.matrix_rank(S1) == r
        assert full == (np.unique(idx[:, 0]).size == r)
        hits += full
    se = math.sqrt(exact * (1 - exact) / trials)
    assert abs(hits / trials - exact) < 4.5 * se
    assert exact <= math.exp(-r * (r - 1) / (2 * m))


def test_norm_preserved_in_expectation():
    # Footnote to Def. 5: the random signs make E ||Sx||^2 = ||x||^2.
    from oracle import sketch
    x = np.random.default_rng(0).standard_normal(60)
    vals = [np.sum(sketch.sketch_rows(seed, 2, 16, x[:, None]) ** 2) for seed in range(3000)]
    mean, se = np.mean(vals), np.std(vals) / math.sqrt(len(vals))
    assert abs(mean - x @ x) < 4.5 * se
