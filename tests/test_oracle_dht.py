"""Pins for the HR-DHT premix of Ski-LLS-dense (Section 6, Eq. HR-DHT)."""
import numpy as np
import pytest

from oracle import dht, embedding, hashing, sketch


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 50, 97])
def test_fft_route_equals_the_definition(n):
    X = np.random.default_rng(n).standard_normal((n, 5))
    assert np.allclose(dht.dht_rows(X), dht.dht_matrix(n) @ X, rtol=0, atol=1e-12)
    assert np.allclose(dht.dht_rows(X[:, 0]), dht.dht_matrix(n) @ X[:, 0], rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [5, 12, 64])
def test_normalized_dht_is_symmetric_orthogonal_and_involutory(n):
    F = dht.dht_matrix(n)
    assert np.allclose(F, F.T, atol=1e-14)
    assert np.allclose(F @ F, np.eye(n), atol=1e-12)          # the DHT is its own inverse
    x = np.random.default_rng(2).standard_normal(n)
    assert np.isclose(np.linalg.norm(dht.dht_rows(x)), np.linalg.norm(x), rtol=1e-13)


def test_small_cases_by_hand():
    # n = 1: F = [1]; n = 2: cas(0) = 1, cas(pi) = -1, F = [[1, 1], [1, -1]] / sqrt(2);
    # n = 4: cas(k pi / 2) for k = 0..3 is 1, 1, -1, -1
    assert np.allclose(dht.dht_matrix(1), [[1.0]])
    assert np.allclose(dht.dht_matrix(2), np.array([[1, 1], [1, -1]]) / np.sqrt(2))
    F4 = np.array([[1, 1, 1, 1], [1, 1, -1, -1], [1, -1, 1, -1], [1, -1, -1, 1]]) / 2.0
    assert np.allclose(dht.dht_matrix(4), F4, atol=1e-15)


def test_premix_applies_the_def8_signs_first():
    n = 33
    A = np.random.default_rng(4).standard_normal((n, 3))
    D = np.diag(hashing.premix_signs(9, n).astype(float))
    assert np.allclose(dht.premix(9, A), dht.dht_matrix(n) @ D @ A, atol=1e-12)


def test_coherence_reduced_to_the_entry_bound():
    # |F_ij| <= sqrt(2/n), so every row of F D [I_d; 0] has norm <= sqrt(2 d / n):
    # the coherence of the fully coherent [I_d; 0] (mu = 1) drops below that bound
    n, d = 1000, 10
    A = np.zeros((n, d))
    A[:d] = np.eye(d)
    assert embedding.coherence(A) == pytest.approx(1.0)
    assert np.max(np.abs(dht.dht_matrix(n))) <= np.sqrt(2.0 / n) + 1e-15
    assert embedding.coherence(dht.premix(5, A)) <= np.sqrt(2.0 * d / n) + 1e-12


def test_ski_lls_with_the_dht_premix():
    # Algorithm 1 with S = S_h F D on a coherent problem reaches the least-squares solution
    from oracle import lsqr
    from paper_2105_11815_gb300 import workloads
    A, b = workloads.dense_high_coherence(3000, 40, seed=2)
    x, info = lsqr.ski_lls(A, b, seed=7, s=1, m=120, premix="dht")
    xr = lsqr.lstsq_reference(A, b)
    assert np.linalg.norm(x - xr) <= 1e-8 * np.linalg.norm(xr)
    assert lsqr.residual_metric(A, b, x) <= 1e-10


def test_sample_rows_uniform_with_replacement():
    c = hashing.sample_rows(3, 200000, 10)
    counts = np.bincount(c, minlength=10)
    chi2 = np.sum((counts - 20000.0) ** 2 / 20000.0)
    assert c.min() >= 0 and c.max() < 10 and chi2 < 33.7          # chi^2_9 at p = 1e-4
    assert len(set(hashing.sample_rows(3, 50, 40).tolist())) < 50   # repeats occur


def test_hashing_preconditions_better_than_sampling():
    # Fig. blen_motivation: on the coherent [I; 0] + 1e-8 J (4000 x 400), the
    # R of a hashed F D A preconditions better than the R of sampled rows of
    # F D A at the same m, and improves with m
    from paper_2105_11815_gb300 import workloads
    n, d = 4000, 400
    A = workloads.coherent_dense(n, d)
    Y = dht.premix(7, A)

    def kappa(SA):
        R = np.linalg.qr(SA, mode="r")
        sv = np.linalg.svd(A @ np.linalg.inv(R), compute_uv=False)
        return sv[0] / sv[-1]
    kh, ks = [], []
    for g in (1.5, 2.0, 3.0):
        m = int(g * d)
        kh.append(kappa(sketch.sketch_rows(1, 1, m, Y)))
        ks.append(kappa(dht.srdht_sketch(7, m, A)))
    assert all(h < s for h, s in zip(kh, ks)), (kh, ks)
    assert kh[0] > kh[1] > kh[2] and kh[1] < 10


def test_hrdht_sketch_equals_explicit_product():
    n, d, m, s = 300, 6, 40, 2
    g = np.random.default_rng(6)
    A, b = g.standard_normal((n, d)), g.standard_normal(n)
    S = sketch.s_hashing_matrix(11, s, m, n) @ dht.dht_matrix(n) @ np.diag(hashing.premix_signs(11, n).astype(float))
    out = dht.hrdht_sketch(11, s, m, A, b)
    assert np.allclose(out, np.column_stack([S @ A, S @ b]), atol=1e-12)


def test_dht_length_is_the_next_13_smooth_integer():
    def smooth(N):
        for p in (2, 3, 5, 7, 11, 13):
            while N % p == 0:
                N //= p
        return N == 1
    # every size of the paper's experiments is already smooth: no padding
    for n in (4000, 4096, 50000, 200000, 1000000, 1, 2, 13):
        assert dht.dht_length(n) == n
    # worked cases: 17 -> 18 = 2 3^2; 1009 (prime) -> 1014 = 2 3 13^2 (1010 = 2 5 101,
    # 1011 = 3 337, 1012 = 2^2 11 23 and 1013 are not smooth); 0 -> 1
    assert dht.dht_length(17) == 18 and dht.dht_length(1009) == 1014 and dht.dht_length(0) == 1
    for n in range(1, 600):
        N = dht.dht_length(n)
        assert N >= n and smooth(N) and not any(smooth(k) for k in range(n, N))


def test_padded_premix_is_the_transform_of_the_zero_padded_rows():
    n, N = 17, 18
    g = np.random.default_rng(8)
    A, b = g.standard_normal((n, 4)), g.standard_normal(n)
    D = hashing.premix_signs(3, n).astype(float)
    X = np.vstack([D[:, None] * A, np.zeros((N - n, 4))])
    assert np.allclose(dht.premix(3, A, N), dht.dht_matrix(N) @ X, atol=1e-12)
    # orthogonal on the padded space: norms are kept
    assert np.isclose(np.linalg.norm(dht.premix(3, b, N)), np.linalg.norm(b), rtol=1e-13)
    with pytest.raises(ValueError):
        dht.premix(3, A, n - 1)


def test_srdht_sketch_picks_sampled_rows_of_the_premixed_matrix():
    # S_s has a single 1 per row (Eq. SR-DHT): row i of S_s F D [A | b] is row
    # c_i of F D [A | b], c_i the i-th sampled row index
    n, N, m = 17, 18, 9
    g = np.random.default_rng(9)
    A, b = g.standard_normal((n, 3)), g.standard_normal(n)
    rows = hashing.sample_rows(4, m, N)
    Ss = np.zeros((m, N))
    Ss[np.arange(m), rows] = 1.0
    F = dht.dht_matrix(N)
    D = hashing.premix_signs(4, n).astype(float)
    X = np.vstack([np.column_stack([D[:, None] * A, D * b]), np.zeros((N - n, 4))])
    assert np.allclose(dht.srdht_sketch(4, m, A, b, n_h=N), Ss @ F @ X, atol=1e-12)
    assert np.allclose(dht.srdht_sketch(4, m, A, n_h=N), (Ss @ F @ X)[:, :3], atol=1e-12)
