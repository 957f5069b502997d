"""Pins for the Householder QR (Step 2), LSQR (Step 4) and Algorithm 1 end to end."""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp
from scipy.linalg import solve_triangular

from oracle import adjoint, embedding, lsqr, qr, sketch, wht
from paper_2105_11815_gb300 import workloads


def _signfix(R):
    return np.sign(np.diag(R))[:, None] * R


def test_householder_matches_lapack():
    g = np.random.default_rng(0)
    B = g.standard_normal((60, 13))
    R, C = qr.householder_qr(B, ncols=12)
    Q, Rl = np.linalg.qr(B[:, :12])
    assert np.allclose(_signfix(R), _signfix(Rl), atol=1e-12)
    assert np.allclose(R.T @ R, B[:, :12].T @ B[:, :12], atol=1e-11)
    # column 12 carries Q^T b (signs follow the rows of R)
    sgn = np.sign(np.diag(R)) * np.sign(np.diag(Rl))
    assert np.allclose(C[:, 0], sgn * (Q.T @ B[:, 12]), atol=1e-12)


def test_numerical_rank():
    g = np.random.default_rng(1)
    B = g.standard_normal((40, 6))
    B[:, 5] = B[:, 0] + B[:, 1]
    R, _ = qr.householder_qr(B)
    assert qr.numerical_rank(R, 1e-12) == 5
    assert qr.numerical_rank(qr.householder_qr(g.standard_normal((40, 6)))[0], 1e-12) == 6


def test_lsqr_matches_lstsq_unpreconditioned():
    g = np.random.default_rng(2)
    A, b = g.standard_normal((200, 20)), g.standard_normal(200)
    y, it, _ = lsqr.lsqr(lambda v: A @ v, lambda u: A.T @ u, b, 20, 1e-14, 500)
    assert np.allclose(y, np.linalg.lstsq(A, b, rcond=None)[0], rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("premix", [False, True])
def test_ski_lls_matches_lstsq(premix):
    A, b, _ = workloads.gaussian_lls(1024, 64, seed=5)
    x, info = lsqr.ski_lls(A, b, seed=17, s=1, m=128, premix=premix)
    xr = lsqr.lstsq_reference(A, b)
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)
    assert lsqr.residual_metric(A, b, x) <= 1e-10
    assert info["iters"] > 0


@pytest.mark.parametrize("premix,s", [(False, 3), (True, 2)])
def test_ski_lls_with_s_hashing_variant(premix, s):
    # Def. 7's variant (Theorems 4-5: an embedding like s-hashing) preconditions
    # Algorithm 1 as well; the accepted x is the least-squares solution
    A, b, _ = workloads.gaussian_lls(1024, 64, seed=8)
    x, info = lsqr.ski_lls(A, b, seed=19, s=s, m=128, premix=premix, variant=True)
    xr = lsqr.lstsq_reference(A, b)
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)
    assert lsqr.residual_metric(A, b, x) <= 1e-10


def test_qrcp_matches_lapack_pivoting():
    # Businger-Golub pivoting: same permutation as LAPACK's dgeqp3 on a
    # generic matrix (distinct norms), the same R up to row signs, a
    # non-increasing |diag R|, and B[:, piv] = Q R through R^T R = B_p^T B_p
    g = np.random.default_rng(21)
    B = g.standard_normal((60, 13)) * np.linspace(0.5, 3.0, 13)
    R, C, piv = qr.householder_qrcp(B, ncols=12)
    _, R2, P2 = scipy.linalg.qr(B[:, :12], pivoting=True, mode="economic")
    assert np.array_equal(piv, P2)
    assert np.allclose(np.abs(R), np.abs(R2), rtol=0, atol=1e-12)
    dg = np.abs(np.diag(R))
    assert np.all(dg[:-1] >= dg[1:])
    Bp = B[:, piv]
    assert np.allclose(R.T @ R, Bp.T @ Bp, rtol=0, atol=1e-10)
    # the extra column is reflected too: ||Q^T b||^2 splits into C and the rest
    assert np.linalg.norm(C[:, 0]) <= np.linalg.norm(B[:, 12]) + 1e-12


def test_pivoting_r_equals_pivoting_sa():
    # SA = Q R with orthonormal Q keeps every column norm (and every partial
    # column norm below a row) of SA in R, so the column-pivoted QR of the d x d
    # R picks the pivots of the column-pivoted QR of the m x d SA and yields the
    # same R' up to row signs: SA P = Q (R P) = (Q Q') R'.  A GPU path can keep
    # its unpivoted QR of SA and pivot only R when the rank rule fails.
    n, d, r = 600, 24, 15
    A, b = workloads.low_rank_lls(n, d, r, seed=12)
    SAb = sketch.sketch_rows(5, 1, 80, A, b)
    R, C = qr.householder_qr(SAb, ncols=d)
    Rp_sa, _, piv_sa = qr.householder_qrcp(SAb[:, :d])
    Rp_r, _, piv_r = qr.householder_qrcp(R)
    p = qr.numerical_rank(Rp_sa, 1e-12)
    assert p == r and qr.numerical_rank(Rp_r, 1e-12) == r
    assert np.array_equal(piv_sa[:p], piv_r[:p])
    # the leading p rows [R11 R12], columns back in their original order (the
    # pivots after p are picked among rounding-level norms and may differ)
    top_sa = np.abs(Rp_sa[:p])[:, np.argsort(piv_sa)]
    top_r = np.abs(Rp_r[:p])[:, np.argsort(piv_r)]
    assert np.allclose(top_sa, top_r, rtol=0, atol=1e-10 * np.abs(Rp_sa[0, 0]))


def test_complete_orthogonal_form():
    g = np.random.default_rng(22)
    Rtop = np.triu(g.standard_normal((7, 11)))
    Rtop[np.arange(7), np.arange(7)] += 3.0
    T, Z1 = qr.complete_orthogonal(Rtop)
    assert np.allclose(T, np.tril(T)) and np.all(np.abs(np.diag(T)) > 0)
    assert np.allclose(Z1.T @ Z1, np.eye(7), atol=1e-13)
    assert np.allclose(T @ Z1.T, Rtop, atol=1e-12)


@pytest.mark.parametrize("factorization", ["qrcp", "cod"])
def test_rank_revealing_forms_agree_on_full_rank(factorization):
    A, b, _ = workloads.gaussian_lls(1024, 64, seed=5)
    x0, _ = lsqr.ski_lls(A, b, seed=17, s=1, m=128)
    x1, info = lsqr.ski_lls(A, b, seed=17, s=1, m=128, factorization=factorization)
    assert info["rank"] == 64
    assert np.linalg.norm(x1 - x0) <= 1e-10 * np.linalg.norm(x0)


def test_rank_deficient_algorithm1():
    # A of rank r = 20 < d = 30.  Lemma 7: under an embedding p = r.  Lemma 6:
    # W = A V1 R11^{-1} has full rank p (here it is well conditioned, Theorem
    # 10).  Theorem 8: x attains the least-squares residual.  Theorem 9: with
    # R12 = 0 (the complete orthogonal form) x is the minimal-norm solution;
    # with R12 != 0 (plain pivoting) it is a different minimiser.
    n, d, r = 1000, 30, 20
    A, b = workloads.low_rank_lls(n, d, r, seed=3)
    xmin = np.linalg.pinv(A) @ b
    rmin = np.linalg.norm(A @ xmin - b)
    sols = {}
    for f in ("qrcp", "cod"):
        x, info = lsqr.ski_lls(A, b, seed=3, s=1, m=120, factorization=f)
        assert info["rank"] == r
        W = A @ info["V1"] @ np.linalg.inv(info["R11"])
        sv = np.linalg.svd(W, compute_uv=False)
        assert sv.size == r and sv[-1] / sv[0] > 0.1
        # the lemma behind Theorem 8: ker(V1^T) and range(A^T) meet only in 0,
        # i.e. their bases (d - p and r vectors) together span R^d
        V1 = info["V1"]
        ker = np.linalg.svd(V1.T)[2][r:].T                    # d x (d - p), V1^T ker = 0
        rowsp = np.linalg.svd(A, full_matrices=False)[2][:r].T  # d x r, range(A^T)
        assert np.allclose(V1.T @ ker, 0, atol=1e-12)
        assert np.linalg.matrix_rank(np.hstack([ker, rowsp]), tol=1e-8) == d
        assert abs(np.linalg.norm(A @ x - b) - rmin) <= 1e-12 * rmin
        assert lsqr.residual_metric(A, b, x) <= 1e-10
        sols[f] = x
    assert np.linalg.norm(sols["cod"] - xmin) <= 1e-9 * np.linalg.norm(xmin)
    assert np.linalg.norm(sols["qrcp"]) > 1.01 * np.linalg.norm(xmin)
    # the plain-QR form refuses a rank-deficient sketch
    with pytest.raises(np.linalg.LinAlgError):
        lsqr.ski_lls(A, b, seed=3, s=1, m=120)


def test_lemma8_rank_deficient():
    # Lemma 8 holds for the rank-revealing x_s: ||A x_s - b|| <= (1+eps)/(1-eps) ||A x* - b||,
    # eps the distortion of S on range([A b])
    n, d, r, m = 2000, 30, 12, 300
    A, b = workloads.low_rank_lls(n, d, r, seed=8)
    rstar = np.linalg.norm(A @ np.linalg.pinv(A) @ b - b)
    U = embedding.orth(np.column_stack([A, b]))
    eps = embedding.distortion(sketch.sketch_rows(4, 2, m, U))
    assert eps < 1
    _, info = lsqr.ski_lls(A, b, seed=4, s=2, m=m, factorization="qrcp", tau_r=1e-6)
    assert np.linalg.norm(A @ info["x_s"] - b) <= (1 + eps) / (1 - eps) * rstar


def test_ski_lls_sparse():
    rp, ci, v, b = workloads.csr_heavy_rows(4000, 100, seed=3, nnz_row=8, heavy_frac=0.005, heavy_nnz=60)
    A = sp.csr_matrix((v, ci, rp), shape=(4000, 100))
    x, info = lsqr.ski_lls(A, b, seed=1, s=2, m=200)
    assert lsqr.residual_metric(A, b, x) <= 1e-10
    xr = lsqr.lstsq_reference(A, b)
    assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)


def test_preconditioned_spectrum_within_embedding_bound():
    # Thm 10 proof, Eq. (Low condition number): kappa(W^T W) <= (1+eps)/(1-eps)
    # for W = A R^{-1} when S is an eps-subspace embedding for A (eps measured
    # by Lemma 2).  With S A R^{-1} = Q orthonormal the embedding inequality
    # gives sigma(W) in [1/sqrt(1+eps), 1/sqrt(1-eps)]; the proof's intermediate
    # [sqrt(1-eps), sqrt(1+eps)] has the two sides exchanged, the ratio is the same.
    A, b, _ = workloads.gaussian_lls(2000, 40, seed=8)
    m = 400
    SAb = sketch.sketch_rows(4, 2, m, A, b)
    R, _ = qr.householder_qr(SAb, ncols=40)
    U = embedding.orth(A)
    eps = embedding.distortion(sketch.sketch_rows(4, 2, m, U))
    assert 0 < eps < 1
    sv = np.linalg.svd(A @ np.linalg.inv(R), compute_uv=False)
    assert sv[0] <= (1 - eps) ** -0.5 * (1 + 1e-12)
    assert sv[-1] >= (1 + eps) ** -0.5 * (1 - 1e-12)
    assert (sv[0] / sv[-1]) ** 2 <= (1 + eps) / (1 - eps) * (1 + 1e-12)


def test_lemma8_and_theorem10_bounds():
    A, b, _ = workloads.gaussian_lls(3000, 30, seed=9, noise=1.0)
    m = 600
    x, info = lsqr.ski_lls(A, b, seed=6, s=2, m=m, tau_r=1e-6)
    xr = lsqr.lstsq_reference(A, b)
    rstar = np.linalg.norm(A @ xr - b)
    U = embedding.orth(np.column_stack([A, b]))
    eps = embedding.distortion(sketch.sketch_rows(6, 2, m, U))
    assert eps < 1
    # Lemma 8: ||A x_s - b|| <= (1+eps)/(1-eps) ||A x* - b||
    assert np.linalg.norm(A @ info["x_s"] - b) <= (1 + eps) / (1 - eps) * rstar
    # Thm 10 (ii) with the energy-norm reduction tau_r reached by LSQR: the final
    # residual is within (1 + 2 eps tau/(1-eps)) of optimal, tau the achieved reduction.
    e0 = np.linalg.norm(A @ (info["x_s"] - xr))
    e1 = np.linalg.norm(A @ (x - xr))
    tau = e1 / e0
    assert np.linalg.norm(A @ x - b) <= (1 + 2 * eps * tau / (1 - eps)) * rstar * (1 + 1e-12)


def test_theorem10_iteration_count():
    # Thm 10 (i): energy-norm error reduced by tau_r within
    # (log 2 + |log tau_r|)/|log eps| iterations.
    A, b, _ = workloads.gaussian_lls(4000, 40, seed=10, noise=1.0)
    m, tau_r = 400, 1e-8
    SAb = sketch.sketch_rows(12, 2, m, A, b)
    R, C = qr.householder_qr(SAb, ncols=40)
    eps = embedding.distortion(sketch.sketch_rows(12, 2, m, embedding.orth(A)))
    xr = lsqr.lstsq_reference(A, b)
    x_s = solve_triangular(R, C[:, 0])
    r0 = b - A @ x_s
    e0 = np.linalg.norm(A @ (x_s - xr))
    bound = (math.log(2) + abs(math.log(tau_r))) / abs(math.log(eps))
    k = math.ceil(bound)
    d, _, _ = lsqr.lsqr(lambda v: A @ solve_triangular(R, v),
                        lambda u: solve_triangular(R, A.T @ u, trans="T"), r0, 40, 0.0, k)
    xk = x_s + solve_triangular(R, d)
    assert np.linalg.norm(A @ (xk - xr)) <= tau_r * e0


def test_premix_lowers_coherence_and_distortion():
    A, _ = workloads.dense_high_coherence(2048, 32, seed=4)
    Y = wht.premix(1, A, 2048)
    assert embedding.coherence(Y) < 0.5 * embedding.coherence(A)


def test_distortion_decreases_with_gamma():
    A, _ = workloads.dense_gaussian(8192, 32, seed=2)
    U = embedding.orth(A)
    eps = [np.median([embedding.distortion(sketch.sketch_rows(sd, 1, int(g * 32), U))
                      for sd in range(5)]) for g in (2, 4, 8)]
    assert eps[0] > eps[1] > eps[2]


def test_s_above_one_preconditions_coherent_input_better():
    # Theorems 3-5: s-hashing (and its variant) relax the coherence needed for
    # an embedding by sqrt(s).  On the semi-coherent D^5 B of the paper's sparse
    # illustration (coherence ~ 0.99), the R of an s = 2 or 3 sketch gives a
    # lower kappa(A R^-1) than s = 1 at the same m, for both kinds of hashing
    n, d = 4000, 40
    A = workloads.semi_coherent_sparse(n, d, seed=3)
    assert embedding.coherence(A) > 0.9

    def kappa(SA):
        R = np.linalg.qr(SA, mode="r")
        sv = np.linalg.svd(A @ np.linalg.inv(R), compute_uv=False)
        return sv[0] / sv[-1]
    for m in (4 * d, 8 * d):
        for variant in (False, True):
            k = {s: np.median([kappa(sketch.sketch_rows(sd, s, m, A, variant=variant)) for sd in range(5)])
                 for s in (1, 2, 3)}
            assert k[2] < k[1] and k[3] < k[1], (m, variant, k)


def test_adjoint_against_finite_differences():
    g = np.random.default_rng(11)
    A, b = g.standard_normal((512, 32)), g.standard_normal(512)
    c = g.standard_normal(32)

    def L(A_, b_):
        return c @ np.linalg.lstsq(A_, b_, rcond=None)[0]

    x = np.linalg.lstsq(A, b, rcond=None)[0]
    dA, db = adjoint.lstsq_grad(A, b, x, c)
    for trial in range(3):
        EA, eb = g.standard_normal(A.shape), g.standard_normal(b.shape)
        h = 1e-6
        fd = (L(A + h * EA, b + h * eb) - L(A - h * EA, b - h * eb)) / (2 * h)
        an = np.sum(dA * EA) + db @ eb
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
