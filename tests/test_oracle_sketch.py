"""Pins for S*A (Algorithm 1 Step 1): brute-force dense S, Def. 5 structure, CSR."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hashing, sketch


@pytest.mark.parametrize("s", [1, 2, 3])
def test_explicit_matrix_structure(s):
    m, n = 13, 400
    S = sketch.s_hashing_matrix(42, s, m, n)
    nz = S != 0
    assert (nz.sum(axis=0) == s).all()
    assert np.allclose(np.abs(S[nz]), 1 / np.sqrt(s), rtol=0, atol=1e-15)
    assert np.allclose(np.linalg.norm(S, axis=0), 1.0, atol=1e-14)


@pytest.mark.parametrize("s,m", [(1, 9), (2, 17), (3, 8)])
def test_rows_sketch_equals_dense_product(s, m):
    g = np.random.default_rng(1)
    A, b = g.standard_normal((257, 11)), g.standard_normal(257)
    S = sketch.s_hashing_matrix(7, s, m, 257)
    out = sketch.sketch_rows(7, s, m, A, b)
    assert np.allclose(out[:, :11], S @ A, rtol=0, atol=1e-13)
    assert np.allclose(out[:, 11], S @ b, rtol=0, atol=1e-13)
    assert np.allclose(sketch.sketch_rows(7, s, m, A), S @ A, rtol=0, atol=1e-13)


def test_csr_sketch_equals_dense():
    g = np.random.default_rng(2)
    A = sp.random(300, 20, density=0.1, random_state=3, format="csr")
    b = g.standard_normal(300)
    dense = sketch.sketch_rows(11, 2, 15, A.toarray(), b)
    assert np.allclose(sketch.sketch_rows(11, 2, 15, A, b), dense, rtol=0, atol=1e-13)


def test_linearity():
    g = np.random.default_rng(3)
    A, B = g.standard_normal((100, 5)), g.standard_normal((100, 5))
    lhs = sketch.sketch_rows(5, 2, 10, 2.0 * A - B)
    rhs = 2.0 * sketch.sketch_rows(5, 2, 10, A) - sketch.sketch_rows(5, 2, 10, B)
    assert np.allclose(lhs, rhs, atol=1e-13)


def test_variant_at_most_s_nonzeros_and_s1_equals_hashing():
    T = sketch.s_hashing_variant_matrix(8, 3, 6, 500)
    assert ((T != 0).sum(axis=0) <= 3).all()
    assert np.allclose(sketch.s_hashing_variant_matrix(8, 1, 6, 50), sketch.s_hashing_matrix(8, 1, 6, 50))


# ---- the s-hashing variant T (Def. 7) and its decomposition (Lemma 5)
def _variant_from_table(seed, s, m, n):
    idx, sign = hashing.variant_table(seed, s, m, n)
    T = np.zeros((m, n))
    for k in range(s):
        np.add.at(T, (idx[:, k], np.arange(n)), sign[:, k] / np.sqrt(s))
    return T


@pytest.mark.parametrize("seed,s,m", [(3, 3, 4), (5, 2, 3), (9, 5, 7), (1, 1, 5)])
def test_variant_scalar_draw_equals_vectorised_table(seed, s, m):
    # the pure-Python per-column draw and the vectorised table build the same T
    assert np.array_equal(sketch.s_hashing_variant_matrix(seed, s, m, 300), _variant_from_table(seed, s, m, 300))


@pytest.mark.parametrize("s,m", [(3, 4), (2, 3), (4, 50)])
def test_variant_lemma5_sum_of_one_hashing_matrices(s, m):
    # Lemma 5: sqrt(s) T = S1 + ... + Ss, each Sk a 1-hashing matrix (one +-1 per column)
    seed, n = 17, 2000
    idx, sign = hashing.variant_table(seed, s, m, n)
    parts = []
    for k in range(s):
        Sk = np.zeros((m, n))
        Sk[idx[:, k], np.arange(n)] = sign[:, k]
        assert ((Sk != 0).sum(axis=0) == 1).all() and set(np.unique(Sk)) <= {-1.0, 0.0, 1.0}
        parts.append(Sk)
    T = sketch.s_hashing_variant_matrix(seed, s, m, n)
    assert np.allclose(np.sqrt(s) * T, sum(parts), rtol=0, atol=1e-13)
    # coinciding draws ADD: with few rows, entries of magnitude 2/sqrt(s) occur
    if m <= 4:
        assert np.isclose(np.abs(T).max(), 2 / np.sqrt(s)) or np.isclose(np.abs(T).max(), s / np.sqrt(s))
    # S1 is the 1-hashing matrix of the same seed (Def. 5 with s = 1)
    assert np.array_equal(parts[0], sketch.s_hashing_matrix(seed, 1, m, n))
    # the Sk are independent: rows agree at rate 1/m, signs at rate 1/2 (binomial, 5 sigma)
    for k in range(1, s):
        agree = np.mean(idx[:, k] == idx[:, 0])
        assert abs(agree - 1 / m) <= 5 * np.sqrt((1 / m) * (1 - 1 / m) / n)
        assert abs(np.mean(sign[:, k] == sign[:, 0]) - 0.5) <= 5 * np.sqrt(0.25 / n)


@pytest.mark.parametrize("s,m", [(2, 5), (3, 8), (4, 20)])
def test_variant_draws_with_replacement_birthday_rate(s, m):
    # Def. 7 samples with replacement: the s draws of a column are all distinct
    # with probability prod_{k<s} (1 - k/m); s-hashing (Def. 5) always has s distinct rows
    n = 40000
    idx, _ = hashing.variant_table(23, s, m, n)
    distinct = np.array([len(set(r)) == s for r in idx.tolist()])
    p = np.prod([1 - k / m for k in range(s)])
    assert abs(distinct.mean() - p) <= 5 * np.sqrt(p * (1 - p) / n)
    hi, _ = hashing.hash_table(23, s, m, 2000)
    assert all(len(set(r)) == s for r in hi.tolist())


def test_variant_column_equals_hashing_column_where_draws_distinct():
    # draw k of the variant is the first (t = 0) candidate of nonzero k of the
    # s-hashing draw; when a column's s draws are distinct nothing is rejected
    seed, s, m, n = 29, 3, 10, 3000
    iv, sv = hashing.variant_table(seed, s, m, n)
    ih, sh = hashing.hash_table(seed, s, m, n)
    same = np.array([len(set(r)) == s for r in iv.tolist()])
    assert 0.5 < same.mean() < 1.0
    assert np.array_equal(iv[same], ih[same]) and np.array_equal(sv[same], sh[same])
    assert not np.array_equal(iv[~same], ih[~same])


def test_variant_isotropic_in_expectation():
    # E[T^T T] = I (each draw is +-1/sqrt(s) with an independent sign): the mean
    # squared column norm is 1, distinct columns are uncorrelated on average
    seed, s, m, n = 31, 4, 6, 30000
    idx, sign = hashing.variant_table(seed, s, m, n)
    T = np.zeros((m, n))
    for k in range(s):
        np.add.at(T, (idx[:, k], np.arange(n)), sign[:, k] / np.sqrt(s))
    sq = (T * T).sum(axis=0)
    assert abs(sq.mean() - 1.0) <= 5 * sq.std() / np.sqrt(n)
    ip = (T[:, 0::2] * T[:, 1::2]).sum(axis=0)
    assert abs(ip.mean()) <= 5 * ip.std() / np.sqrt(ip.size)


@pytest.mark.parametrize("s,m", [(3, 4), (2, 9)])
def test_variant_rows_sketch_equals_dense_product(s, m):
    g = np.random.default_rng(4)
    A, b = g.standard_normal((300, 7)), g.standard_normal(300)
    T = sketch.s_hashing_variant_matrix(13, s, m, 300)
    out = sketch.sketch_rows(13, s, m, A, b, variant=True)
    assert np.allclose(out[:, :7], T @ A, rtol=0, atol=1e-13)
    assert np.allclose(out[:, 7], T @ b, rtol=0, atol=1e-13)
    Ac = sp.random(300, 7, density=0.2, random_state=5, format="csr")
    assert np.allclose(sketch.sketch_rows(13, s, m, Ac, b, variant=True)[:, :7], T @ Ac.toarray(), atol=1e-13)
