"""LSQR and the whole of Algorithm 1 (Ski-LLS), step by step.

Test infrastructure: see ``oracle/__init__.py`` for who may import this.

Algorithm 1: (1) draw S, form SA and Sb; (2) factor SA = QR; (3) x_s =
R^{-1} Q^T Sb, stop if ||A x_s - b|| <= tau_a; (4) LSQR on min ||W y - b|| with
W = A R^{-1} (Eq. def::W), stopped by the test of Eq. TC-lsqr
||W^T (W y - b)|| / (||W|| ||W y - b||) <= tau_r; (5) x = R^{-1} y.
LSQR starts from y_0 = Q^T Sb (Theorem 10 (ii)): it is run on the residual
problem min ||W delta - (b - W y_0)|| and y = y_0 + delta.
"""
import numpy as np
from scipy.linalg import solve_triangular

from . import dht as _dht
from . import qr as _qr
from . import sketch as _sketch
from . import wht as _wht


def lsqr(Wmul, WTmul, rhs, nvar, tau_r, it_max, history=None):
    """LSQR of Paige & Saunders (ACM TOMS 8, 1982) for min ||W y - rhs||, y_0 = 0.

    Golub-Kahan bidiagonalisation beta_1 u_1 = rhs, alpha_1 v_1 = W^T u_1, then
    per iteration: beta u <- W v - alpha u; alpha v <- W^T u - beta v; a plane
    rotation (rho, c, s) eliminates beta; y and w are updated.  The estimates
    ||r|| = phibar, ||W^T r|| = phibar * alpha * |c| and ||W||_F ~ sqrt(sum of
    alpha^2 + beta^2) give the stopping test of Eq. TC-lsqr.
    history, when given, is called after iteration k as
    history(k, y_k, rnorm, arnorm, anorm) with the estimates of that iterate.
    Returns (y, iterations, list of test values).
    """
    u = np.array(rhs, dtype=np.float64, copy=True)
    beta = np.linalg.norm(u)
    y = np.zeros(nvar)
    if beta == 0.0:
        return y, 0, []
    u /= beta
    v = WTmul(u)
    alpha = np.linalg.norm(v)
    if alpha == 0.0:
        return y, 0, []
    v /= alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    anorm2 = 0.0
    trace = []
    it = 0
    while it < it_max:
        it += 1
        u = Wmul(v) - alpha * u
        beta = np.linalg.norm(u)
        if beta > 0.0:
            u /= beta
        anorm2 += alpha * alpha + beta * beta
        v = WTmul(u) - beta * v
        alpha = np.linalg.norm(v)
        if alpha > 0.0:
            v /= alpha
        rho = np.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        y += (phi / rho) * w
        w = v - (theta / rho) * w
        rnorm = phibar
        arnorm = phibar * alpha * abs(c)
        test = arnorm / (np.sqrt(anorm2) * rnorm) if rnorm > 0 else 0.0
        trace.append(test)
        if history is not None:
            history(it, y.copy(), rnorm, arnorm, np.sqrt(anorm2))
        if test <= tau_r:
            break
    return y, it, trace


def residual_metric(A, b, x):
    """||A^T r|| / (||A||_F ||r||) with r = b - A x, all in FP64."""
    r = b - A @ x
    fro = np.sqrt((A.multiply(A)).sum()) if hasattr(A, "multiply") else np.linalg.norm(A)
    rn = np.linalg.norm(r)
    return float(np.linalg.norm(A.T @ r) / (fro * rn)) if rn > 0 else 0.0


def perturbed_back_solve(R, c, perturb, trans=False):
    """Solve R x = c (R^T x = c when trans) by substitution, dividing by
    r_ii + perturb wherever the diagonal entry r_ii is needed: the perturbed
    back-solve of Ski-LLS-sparse (Section 6, parameter rcond_thres), a safeguard
    for a triangular factor whose rank detection failed.  perturb = 0 is the
    plain back-solve."""
    R = np.asarray(R, dtype=np.float64)
    d = R.shape[0]
    x = np.zeros(d)
    order = range(d) if trans else range(d - 1, -1, -1)
    for i in order:
        if trans:                      # forward substitution with R^T (lower)
            acc = c[i] - R[:i, i] @ x[:i]
        else:                          # back substitution with R (upper)
            acc = c[i] - R[i, i + 1:] @ x[i + 1:]
        x[i] = acc / (R[i, i] + perturb)
    return x


def _two_sum(a, b):
    """Knuth's TwoSum: s + e = a + b exactly, s = fl(a + b)."""
    s = a + b
    z = s - a
    return s, (a - (s - z)) + (b - z)


def _veltkamp(a):
    """Veltkamp's splitting a = hi + lo into 26- and 27-bit halves."""
    c = 134217729.0 * a               # (2^27 + 1) a
    hi = c - (c - a)
    return hi, a - hi


def _two_prod(a, b):
    """Dekker's TwoProduct: p + e = a * b exactly, p = fl(a * b)."""
    p = a * b
    ah, al = _veltkamp(a)
    bh, bl = _veltkamp(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def residual_dd(A, b, x):
    """r = b - A x with every row's A_i x as the compensated dot product Dot2
    of Ogita, Rump & Oishi (SIAM J. Sci. Comput. 26, 2005) -- TwoProduct of
    each term, TwoSum of the running sum, the errors summed beside it -- and
    b_i - (s + c) rounded once: r as if computed in twice the working
    precision.  Vectorised over the rows; the terms of a row are taken in
    column order.  A: dense ndarray or scipy sparse."""
    x = np.asarray(x, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    s = np.zeros(n)
    c = np.zeros(n)
    if hasattr(A, "tocsr"):
        csr = A.tocsr()
        csr.sort_indices()
        cnt = np.diff(csr.indptr)
        for k in range(int(cnt.max()) if n else 0):
            rows = np.flatnonzero(cnt > k)
            idx = csr.indptr[rows] + k
            p, e = _two_prod(csr.data[idx], x[csr.indices[idx]])
            t, te = _two_sum(s[rows], p)
            s[rows] = t
            c[rows] += e + te
    else:
        At = np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)
        for j in range(At.shape[0]):
            p, e = _two_prod(At[j], x[j])
            s, te = _two_sum(s, p)
            c += e + te
    h, he = _two_sum(b, -s)
    return h + (he - c)


def residual_metric_dd(A, b, x):
    """||A^T r|| / (||A||_F ||r||) with r from ``residual_dd``: the acceptance
    metric free of the rounding of b - A x, which dominates the plain FP64
    value when x is large along small singular directions."""
    r = residual_dd(A, b, x)
    fro = np.sqrt((A.multiply(A)).sum()) if hasattr(A, "multiply") else np.linalg.norm(A)
    rn = np.linalg.norm(r)
    return float(np.linalg.norm(A.T @ r) / (fro * rn)) if rn > 0 else 0.0


def ski_lls(A, b, seed, s, m, premix=False, n_pad=None, tau_a=1e-8, tau_r=1e-12,
            it_max=10000, rcond=1e-12, variant=False, factorization="qr", perturb=0.0):
    """Algorithm 1 with an s-hashing (optionally HRHT) sketch and Householder QR.
    variant=True sketches with the s-hashing variant of Def. 7.
    premix: False, True (the Walsh-Hadamard premix H D of Def. 8, padded to
    n_pad) or "dht" (the HR-DHT premix F D of Ski-LLS-dense, of length n, or
    n_pad when given).

    factorization: "qr" (plain QR: when R fails the rank rule it raises, or,
    with perturb > 0, every back-solve with R divides by r_ii + perturb -- the
    perturbed back-solve of Ski-LLS-sparse), "chol" (R the Cholesky factor of
    SA^T SA, ``qr.gram_cholesky``, and Q^T Sb = R^{-T} SA^T Sb; the same rank
    rule and perturbation), or the rank-revealing forms of Step 2 for any rank:
    "qrcp" (column-pivoted QR) or "cod" (complete orthogonal, R12 = 0); see
    ``ski_lls_rank_revealing``.

    A: dense n x d ndarray or scipy sparse; b: length n.
    Returns (x, info) with info = {iters, early_exit, x_s, R, qtsb, rank, trace}.
    """
    n, d = A.shape
    if premix == "dht":
        SAb = _dht.hrdht_sketch(seed, s, m, np.asarray(A), b, variant=variant, n_h=n_pad)
    elif premix:
        SAb = _wht.hrht_sketch(seed, s, m, np.asarray(A), b, n_pad, variant=variant)
    else:
        SAb = _sketch.sketch_rows(seed, s, m, A, b, variant=variant)
    if factorization not in ("qr", "chol"):
        return ski_lls_rank_revealing(A, b, SAb, factorization, tau_a, tau_r, it_max, rcond)
    if factorization == "chol":                                   # Step 2 from the Gram
        R = _qr.gram_cholesky(SAb[:, :d])
        qtsb = solve_triangular(R, SAb[:, :d].T @ SAb[:, d], trans="T")
    else:
        R, C = _qr.householder_qr(SAb, ncols=d)                   # Step 2
        qtsb = C[:, 0]
    p = _qr.numerical_rank(R, rcond)
    pert = 0.0
    if p < d:
        if perturb <= 0.0:
            raise np.linalg.LinAlgError(f"sketch has numerical rank {p} < {d}")
        pert = perturb

    def Rinv(v, trans=False):
        if pert > 0.0:
            return perturbed_back_solve(R, v, pert, trans=trans)
        return solve_triangular(R, v, trans="T" if trans else "N")

    x_s = Rinv(qtsb)                                              # Step 3
    r0 = b - A @ x_s
    info = dict(x_s=x_s, R=R, qtsb=qtsb, rank=p, early_exit=False, iters=0, trace=[], perturb=pert)
    if np.linalg.norm(r0) <= tau_a:
        info["early_exit"] = True
        return x_s, info

    def Wmul(v):
        return A @ Rinv(v)

    def WTmul(u):
        return Rinv(A.T @ u, trans=True)

    delta, iters, trace = lsqr(Wmul, WTmul, r0, d, tau_r, it_max)  # Step 4
    x = x_s + Rinv(delta)                                         # Step 5
    info.update(iters=iters, trace=trace)
    return x, info


def ski_lls_rank_revealing(A, b, SAb, factorization, tau_a, tau_r, it_max, rcond):
    """Steps 2-5 of Algorithm 1 with a rank-revealing factorization of SA.

    Step 2: SA = Q R V^T with R = [R11 R12; 0 0], R11 (p x p) nonsingular.
    "qrcp": column-pivoted Householder QR of [SA | Sb] (pivoting the d columns
    of SA only), p by the rcond rule, the trailing rows of R dropped; V = the
    column permutation, V1 its first p columns, Q1^T Sb the first p entries of
    the reflected Sb.  "cod": the same, then [R11 R12] = T Z1^T
    (``complete_orthogonal``), so R11 becomes T, R12 = 0, and V1 = P Z1.
    Step 3: x_s = V1 R11^{-1} Q1^T Sb; stop if ||A x_s - b|| <= tau_a.
    Step 4: LSQR on W = A V1 R11^{-1} (n x p) from y_0 = Q1^T Sb.
    Step 5: x = V1 R11^{-1} y.
    """
    n, d = A.shape
    R, C, piv = _qr.householder_qrcp(SAb, ncols=d)
    qtsb = C[:, 0]
    p = _qr.numerical_rank(R, rcond)
    if p == 0:
        raise np.linalg.LinAlgError("sketch is zero")
    P1 = np.eye(d)[:, piv[:p]]
    if factorization == "qrcp":
        R11, lower, V1 = R[:p, :p], False, P1
    elif factorization == "cod":
        T, Z1 = _qr.complete_orthogonal(R[:p, :])
        R11, lower, V1 = T, True, np.eye(d)[:, piv] @ Z1
    else:
        raise ValueError("factorization must be qr, qrcp or cod")
    c1 = qtsb[:p]

    def solve(v, trans="N"):
        return solve_triangular(R11, v, lower=lower, trans=trans)

    x_s = V1 @ solve(c1)                                          # Step 3
    r0 = b - A @ x_s
    info = dict(x_s=x_s, R=R, R11=R11, V1=V1, piv=piv, qtsb=qtsb, rank=p, early_exit=False, iters=0, trace=[])
    if np.linalg.norm(r0) <= tau_a:
        info["early_exit"] = True
        return x_s, info

    def Wmul(v):
        return A @ (V1 @ solve(v))

    def WTmul(u):
        return solve(V1.T @ (A.T @ u), trans="T")

    delta, iters, trace = lsqr(Wmul, WTmul, r0, p, tau_r, it_max)  # Step 4
    x = x_s + V1 @ solve(delta)                                   # Step 5
    info.update(iters=iters, trace=trace)
    return x, info


def lstsq_reference(A, b):
    """The exact least-squares minimiser by LAPACK (gelsd), the result oracle."""
    A = A.toarray() if hasattr(A, "toarray") else A
    return np.linalg.lstsq(A, b, rcond=None)[0]
