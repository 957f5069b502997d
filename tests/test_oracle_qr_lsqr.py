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


# ---------------------------------------------------------------- the acceptance metric
@pytest.mark.parametrize("sparse", [False, True])
def test_residual_metric_hand_worked(sparse):
    # ||A^T r|| / (||A||_F ||r||), r = b - A x, worked by hand on matrices where
    # the plausible slips give other numbers.
    # (i) A = [1 2 2]^T, x = 1, r = [2 2 1]: A^T r = 8, ||A||_F = 3, ||r|| = 3
    #     -> 8/9 (||b|| = sqrt(34) in place of ||r|| would give 8/(3 sqrt 34))
    A1 = np.array([[1.0], [2.0], [2.0]])
    b1 = np.array([3.0, 4.0, 3.0])
    # (ii) A = [[2 0 0] [1 1 0] [0 0 1]], x = [1 1 1], r = e_1, b = [3 2 1]:
    #     A^T r = [2 0 0] -> 2; ||A||_F = sqrt 7 -> 2 / sqrt 7.  A r = [2 1 0]
    #     (norm sqrt 5), ||A||_2 = sqrt(3 + sqrt 5) and ||b|| = sqrt 14 all differ
    A2 = np.array([[2.0, 0.0, 0.0], [1.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    b2 = np.array([3.0, 2.0, 1.0])
    cases = [(A1, b1, np.array([1.0]), 8.0 / 9.0), (A2, b2, np.ones(3), 2.0 / np.sqrt(7.0))]
    for A, b, x, want in cases:
        M = sp.csr_matrix(A) if sparse else A
        assert lsqr.residual_metric(M, b, x) == pytest.approx(want, rel=1e-15)
    # the slips named above give different values on (ii)
    assert abs(2.0 / np.sqrt(3.0 + np.sqrt(5.0)) - 2.0 / np.sqrt(7.0)) > 0.1
    assert abs(np.sqrt(5.0) / np.sqrt(7.0) - 2.0 / np.sqrt(7.0)) > 0.05
    # an exact least-squares solution has A^T r = 0, an interpolating one r = 0
    assert lsqr.residual_metric(A2, b2, np.linalg.solve(A2, b2)) == 0.0
    xr = np.linalg.lstsq(A1, b1, rcond=None)[0]
    assert lsqr.residual_metric(A1, b1, xr) <= 1e-15


# ---------------------------------------------------------------- LSQR's estimates
def _golub_kahan(W, rhs, k):
    """k steps of Golub-Kahan bidiagonalisation with full reorthogonalisation:
    U (n x k+1), V (d x k), alphas (k), betas (k+1), so that W V_k = U_{k+1} B_k
    with B_k lower bidiagonal (alphas on the diagonal, betas[1:] below it)."""
    n, d = W.shape
    U = np.zeros((n, k + 1))
    V = np.zeros((d, k))
    al = np.zeros(k)
    be = np.zeros(k + 1)
    be[0] = np.linalg.norm(rhs)
    U[:, 0] = rhs / be[0]
    for i in range(k):
        v = W.T @ U[:, i] - (be[i] * V[:, i - 1] if i > 0 else 0.0)
        v -= V[:, :i] @ (V[:, :i].T @ v)
        al[i] = np.linalg.norm(v)
        V[:, i] = v / al[i]
        u = W @ V[:, i] - al[i] * U[:, i]
        u -= U[:, :i + 1] @ (U[:, :i + 1].T @ u)
        be[i + 1] = np.linalg.norm(u)
        U[:, i + 1] = u / be[i + 1]
    return U, V, al, be


def test_lsqr_estimates_match_the_explicit_quantities():
    # Paige & Saunders: after k steps the LSQR iterate is y_k = V_k z_k with
    # z_k = argmin ||beta_1 e_1 - B_k z||, its residual norm is phibar, ||W^T r_k||
    # is phibar * alpha_{k+1} |c_k|, and the running ||W|| estimate is the
    # Frobenius norm of B_k.  Each is compared with the quantity formed
    # explicitly from an independent bidiagonalisation of W.
    g = np.random.default_rng(31)
    n, d = 40, 10
    Q1, _ = np.linalg.qr(g.standard_normal((n, d)))
    Q2, _ = np.linalg.qr(g.standard_normal((d, d)))
    W = Q1 @ np.diag(np.linspace(1.0, 8.0, d)) @ Q2.T
    rhs = g.standard_normal(n)
    seen = {}

    def hist(k, y, rnorm, arnorm, anorm):
        seen[k] = (y, rnorm, arnorm, anorm)

    lsqr.lsqr(lambda v: W @ v, lambda u: W.T @ u, rhs, d, 0.0, d - 1, history=hist)
    assert sorted(seen) == list(range(1, d))
    U, V, al, be = _golub_kahan(W, rhs, d - 1)
    for k in range(1, d):
        y, rnorm, arnorm, anorm = seen[k]
        B = np.zeros((k + 1, k))
        B[np.arange(k), np.arange(k)] = al[:k]
        B[np.arange(1, k + 1), np.arange(k)] = be[1:k + 1]
        e1 = np.zeros(k + 1)
        e1[0] = be[0]
        z = np.linalg.lstsq(B, e1, rcond=None)[0]
        yk = V[:, :k] @ z
        r = rhs - W @ yk
        assert np.allclose(y, yk, rtol=0, atol=1e-10 * np.linalg.norm(yk))
        assert rnorm == pytest.approx(np.linalg.norm(r), rel=1e-9)
        assert arnorm == pytest.approx(np.linalg.norm(W.T @ r), rel=1e-7)
        assert anorm == pytest.approx(np.linalg.norm(B), rel=1e-12)


def test_lsqr_test_value_is_eq_tc_lsqr():
    # the stopping value is ||W^T r|| / (||B_k||_F ||r||): with the estimates
    # pinned above, the trace equals that ratio formed from them
    g = np.random.default_rng(32)
    W = g.standard_normal((30, 6))
    rhs = g.standard_normal(30)
    seen = []
    _, it, trace = lsqr.lsqr(lambda v: W @ v, lambda u: W.T @ u, rhs, 6, 0.0, 5,
                             history=lambda k, y, rn, arn, an: seen.append(arn / (an * rn)))
    assert it == 5 and np.allclose(trace, seen, rtol=1e-15)


# ---------------------------------------------------------------- perturbed back-solve
def test_perturbed_back_solve_hand_worked():
    # R = [[2 1] [0 0]], c = [3 1], perturb 1/2: dividing by r_ii + 1/2,
    # x_2 = 1 / (1/2) = 2 and x_1 = (3 - 2) / (5/2) = 2/5; with R^T (forward
    # substitution) x_1 = 3 / (5/2) = 6/5 and x_2 = (1 - 6/5) / (1/2) = -2/5
    R = np.array([[2.0, 1.0], [0.0, 0.0]])
    c = np.array([3.0, 1.0])
    assert np.allclose(lsqr.perturbed_back_solve(R, c, 0.5), [0.4, 2.0], rtol=0, atol=1e-15)
    assert np.allclose(lsqr.perturbed_back_solve(R, c, 0.5, trans=True), [1.2, -0.4], rtol=0, atol=1e-15)
    # a 3 x 3 case: R = [[1 2 3] [0 4 5] [0 0 0]], c = [1 2 3], perturb 1:
    # x_3 = 3, x_2 = (2 - 15) / 5 = -13/5, x_1 = (1 + 26/5 - 9) / 2 = -7/5
    R3 = np.array([[1.0, 2.0, 3.0], [0.0, 4.0, 5.0], [0.0, 0.0, 0.0]])
    assert np.allclose(lsqr.perturbed_back_solve(R3, np.array([1.0, 2.0, 3.0]), 1.0), [-1.4, -2.6, 3.0],
                       rtol=0, atol=1e-14)
    # perturb = 0 is LAPACK's triangular solve
    g = np.random.default_rng(33)
    Rg = np.triu(g.standard_normal((7, 7))) + 4 * np.eye(7)
    cg = g.standard_normal(7)
    assert np.allclose(lsqr.perturbed_back_solve(Rg, cg, 0.0), solve_triangular(Rg, cg), rtol=1e-13, atol=0)
    assert np.allclose(lsqr.perturbed_back_solve(Rg, cg, 0.0, trans=True), solve_triangular(Rg, cg, trans="T"),
                       rtol=1e-13, atol=0)


def zero_column_lls(n=600, d=12, zero=5, seed=41):
    """A Gaussian LLS whose column ``zero`` is exactly zero (rank d - 1); its
    sketch then has an exactly zero column, and the Householder QR gives
    r_zz = 0 exactly."""
    A, b, _ = workloads.gaussian_lls(n, d, seed=seed)
    A = A.copy()
    A[:, zero] = 0.0
    return A, b


def test_perturbed_ski_lls_solves_the_reduced_problem():
    # With column z of A zero, the rank rule stops at p = z (the leading count)
    # and plain QR cannot continue.  The perturbed back-solve divides by
    # r_zz + perturb = perturb; column z of (R + perturb e_z e_z^T)^{-1} is then
    # e_z / perturb, so the entries of x other than x_z depend only on the other
    # columns: they equal the least-squares solution of A without column z,
    # which is unique, and the residual is the least-squares residual.
    A, b = zero_column_lls()
    z = 5
    with pytest.raises(np.linalg.LinAlgError):
        lsqr.ski_lls(A, b, seed=3, s=1, m=48)
    x, info = lsqr.ski_lls(A, b, seed=3, s=1, m=48, perturb=1e-10)
    assert info["rank"] == z and info["perturb"] == 1e-10
    keep = np.arange(A.shape[1]) != z
    xr = np.linalg.lstsq(A[:, keep], b, rcond=None)[0]
    assert np.linalg.norm(x[keep] - xr) <= 1e-10 * np.linalg.norm(xr)
    assert np.linalg.norm(b - A @ x) == pytest.approx(np.linalg.norm(b - A[:, keep] @ xr), rel=1e-12)
    assert lsqr.residual_metric(A, b, x) <= 1e-10
    assert np.isfinite(x[z])


# ---------------------------------------------------------------- compensated residual
def test_residual_dd_hand_worked_cancellation():
    # row [1e16, 1, -1e16] . [1, 1, 1] = 1 exactly; in FP64 1e16 + 1 rounds
    # to 1e16 and the plain sum is 0.  r = b - A x with b = 0 is -1.
    A = np.array([[1e16, 1.0, -1e16], [3.0, 0.5, 0.25]])
    x = np.ones(3)
    b = np.array([0.0, 4.0])
    assert (b - A @ x)[0] == 0.0                      # the plain residual loses it
    r = lsqr.residual_dd(A, b, x)
    assert r[0] == -1.0 and r[1] == 0.25
    assert np.array_equal(lsqr.residual_dd(sp.csr_matrix(A), b, x), r)


def test_residual_dd_matches_exact_rational_arithmetic():
    # products and sums of doubles done exactly in rationals, then rounded
    # once: Dot2 agrees to within a few units in the last place, on rows
    # built to cancel (terms of 1e8 summing to O(1))
    from fractions import Fraction
    g = np.random.default_rng(51)
    n, d = 40, 25
    A = g.standard_normal((n, d)) * 10.0 ** g.integers(-3, 9, (n, d))
    x = g.standard_normal(d)
    b = A @ x + g.standard_normal(n) * 1e-3
    r = lsqr.residual_dd(A, b, x)
    rs = lsqr.residual_dd(sp.csr_matrix(A), b, x)
    worst = 0.0
    for i in range(n):
        ex = Fraction(b[i]) - sum(Fraction(A[i, j]) * Fraction(x[j]) for j in range(d))
        want = float(ex)
        worst = max(worst, abs(r[i] - want) / abs(want))
        assert abs(rs[i] - want) <= 4 * np.finfo(float).eps * abs(want)
    assert worst <= 4 * np.finfo(float).eps
    # the plain residual is far off on the same rows
    plain = b - A @ x
    assert np.max(np.abs(plain - r) / np.abs(r)) > 1e-6


def test_residual_metric_dd_agrees_when_nothing_cancels():
    A, b, _ = workloads.gaussian_lls(500, 20, seed=3)
    x = np.linalg.lstsq(A, b, rcond=None)[0] + 1e-6
    assert lsqr.residual_metric_dd(A, b, x) == pytest.approx(lsqr.residual_metric(A, b, x), rel=1e-9)
    A2 = np.array([[2.0, 0.0, 0.0], [1.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    assert lsqr.residual_metric_dd(A2, np.array([3.0, 2.0, 1.0]), np.ones(3)) == pytest.approx(2 / np.sqrt(7),
                                                                                              rel=1e-15)


def test_gram_cholesky_hand_worked_and_against_householder():
    # SA = [[3, 1], [4, 2]]: G = [[25, 11], [11, 5]], r11 = 5, r12 = 11/5,
    # r22 = sqrt(5 - 121/25) = 2/5
    R = qr.gram_cholesky(np.array([[3.0, 1.0], [4.0, 2.0]]))
    assert np.allclose(R, [[5.0, 2.2], [0.0, 0.4]], rtol=0, atol=1e-14)
    g = np.random.default_rng(3)
    SA = g.standard_normal((60, 12)) * np.logspace(0, 2, 12)
    Rc = qr.gram_cholesky(SA)
    assert np.allclose(np.triu(Rc), Rc) and np.all(np.diag(Rc) > 0)
    assert np.allclose(Rc.T @ Rc, SA.T @ SA, rtol=1e-12, atol=1e-9)
    Rh, _ = qr.householder_qr(SA)
    Rh = np.sign(np.diag(Rh))[:, None] * Rh          # the unique R with a positive diagonal
    assert np.allclose(Rc, Rh, rtol=1e-10, atol=1e-10)
    with pytest.raises(np.linalg.LinAlgError):
        qr.gram_cholesky(np.column_stack([SA[:, :3], SA[:, 0]]))   # a repeated column


def test_ski_lls_with_the_gram_cholesky_factor():
    import scipy.sparse as sp
    g = np.random.default_rng(4)
    n, d = 3000, 40
    A = sp.random(n, d, density=0.05, random_state=5, format="csr") + sp.eye(n, d, format="csr")
    b = g.standard_normal(n)
    x, info = lsqr.ski_lls(A, b, seed=2, s=2, m=120, factorization="chol")
    xq, iq = lsqr.ski_lls(A, b, seed=2, s=2, m=120)
    xr = np.linalg.lstsq(A.toarray(), b, rcond=None)[0]
    assert np.linalg.norm(x - xr) <= 1e-8 * np.linalg.norm(xr)
    Rq = np.sign(np.diag(iq["R"]))[:, None] * iq["R"]
    assert np.allclose(info["R"], Rq, rtol=1e-9, atol=1e-9)
    assert np.allclose(info["qtsb"], np.sign(np.diag(iq["R"])) * iq["qtsb"], rtol=1e-9, atol=1e-9)
    assert abs(info["iters"] - iq["iters"]) <= 1
