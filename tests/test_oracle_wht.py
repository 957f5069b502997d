"""Pins for the Walsh-Hadamard premix (Def. 8, Lemma of Tropp)."""
import math

import numpy as np
import pytest
from scipy.linalg import hadamard

from oracle import embedding, hashing, sketch, wht


@pytest.mark.parametrize("n", [1, 2, 8, 64, 1024])
def test_butterflies_equal_sylvester_matrix(n):
    assert np.array_equal(wht.fwht_rows(np.eye(n)), hadamard(n).astype(float))


def test_entries_from_definition():
    # H_ij proportional to (-1)^{<(i-1)_2, (j-1)_2>} (Def. 8), 0-based i, j here.
    n = 32
    H = wht.fwht_rows(np.eye(n))
    for i in range(n):
        for j in range(n):
            assert H[i, j] == (-1) ** bin(i & j).count("1")


def test_involution_and_isometry():
    g = np.random.default_rng(0)
    X = g.standard_normal((256, 3))
    assert np.allclose(wht.fwht_rows(wht.fwht_rows(X)) / 256, X, atol=1e-13)
    A = g.standard_normal((200, 4))
    Y = wht.premix(5, A, 256)
    assert np.isclose(np.linalg.norm(Y), np.linalg.norm(A), rtol=1e-13)


def test_premix_equals_explicit_product():
    g = np.random.default_rng(1)
    A = g.standard_normal((100, 6))
    D = hashing.premix_signs(9, 100).astype(float)
    Apad = np.zeros((128, 6))
    Apad[:100] = D[:, None] * A
    assert np.allclose(wht.premix(9, A, 128), hadamard(128) @ Apad / math.sqrt(128), atol=1e-13)


def test_hrht_sketch_equals_explicit_product():
    g = np.random.default_rng(2)
    A, b = g.standard_normal((50, 4)), g.standard_normal(50)
    S = sketch.s_hashing_matrix(3, 2, 9, 64)
    D = np.diag(np.r_[hashing.premix_signs(3, 50).astype(float), np.ones(14)])
    HD = hadamard(64) @ D / 8.0
    Apad = np.vstack([A, np.zeros((14, 4))])
    bpad = np.r_[b, np.zeros(14)]
    out = wht.hrht_sketch(3, 2, 9, A, b, 64)
    assert np.allclose(out[:, :4], S @ HD @ Apad, atol=1e-13)
    assert np.allclose(out[:, 4], S @ HD @ bpad, atol=1e-13)


def test_tropp_coherence_bound():
    # Lemma (Tropp): mu(HDU) <= sqrt(r/n) + sqrt(8 log(n/delta)/n) w.p. >= 1-delta.
    n, r, delta = 1024, 8, 0.01
    U = np.zeros((n, r))
    U[:r] = np.eye(r)           # maximally coherent, mu = 1
    bound = math.sqrt(r / n) + math.sqrt(8 * math.log(n / delta) / n)
    fails = sum(embedding.coherence(wht.premix(seed, U, n)) > bound for seed in range(20))
    assert fails <= 2
    assert embedding.coherence(U) == pytest.approx(1.0)
