"""Pins for S*A (Algorithm 1 Step 1): brute-force dense S, Def. 5 structure, CSR."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import sketch


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
