"""Unblocked Householder QR of the sketch (Algorithm 1, Step 2).

Test infrastructure: see ``oracle/__init__.py`` for who may import this.

Step 2 factors SA = Q R (plain QR when SA has full rank, Remark (i)); Step 3
needs Q_1^T Sb.  Factoring the first d columns of the augmented [SA | Sb] while
applying every reflector to column d as well gives both: R is the leading
d x d upper triangle and Q_1^T Sb the first d entries of column d.

For a possibly rank-deficient SA, Step 2 asks for SA = Q R V^T with
R = [R11 R12; 0 0] and R11 (p x p) nonsingular; Remark (i) names column-pivoted
QR and the complete orthogonal decomposition (R12 = 0) among the allowed
factorizations.  ``householder_qrcp`` is the first (Businger & Golub's column
pivoting), ``complete_orthogonal`` turns its leading p rows into the second.
"""
import numpy as np


def householder_qr(B, ncols=None):
    """Householder QR of the first ``ncols`` columns of B (m x c, m >= ncols).

    For column j: x = B[j:, j]; beta = -sign(x_0) ||x||; v = x - beta e_1;
    B[j:, j:] -= (2 / v^T v) v (v^T B[j:, j:]).  Reflectors are applied to every
    column to the right, including columns beyond ``ncols``.
    Returns (R, C): R (ncols x ncols) upper triangular and C = (Q^T B)[:ncols, ncols:].
    """
    B = np.array(B, dtype=np.float64, copy=True)
    m, c = B.shape
    k = c if ncols is None else ncols
    if m < k:
        raise ValueError("need m >= ncols")
    for j in range(k):
        x = B[j:, j]
        normx = np.sqrt(np.dot(x, x))
        if normx == 0.0:
            continue
        beta = -normx if x[0] >= 0 else normx
        v = x.copy()
        v[0] -= beta
        vtv = np.dot(v, v)
        w = v @ B[j:, j:]
        B[j:, j:] -= np.outer(v, (2.0 / vtv) * w)
        B[j + 1:, j] = 0.0
        B[j, j] = beta
    return np.triu(B[:k, :k]), B[:k, k:]


def householder_qrcp(B, ncols=None):
    """Householder QR with column pivoting of the first ``ncols`` columns of B.

    Step j first swaps into position j the column among j..ncols-1 whose part
    in rows j.. has the largest Euclidean norm (the first such on ties; the
    norms are recomputed from B at every step, not downdated), then reflects
    as ``householder_qr`` does, applying the reflector to every column to the
    right including those beyond ``ncols``.  The diagonal of R is then
    non-increasing in magnitude.
    Returns (R, C, piv): B[:, piv] = Q [R; 0] on the first ncols columns,
    C = (Q^T B)[:ncols, ncols:].
    """
    B = np.array(B, dtype=np.float64, copy=True)
    m, c = B.shape
    k = c if ncols is None else ncols
    if m < k:
        raise ValueError("need m >= ncols")
    piv = np.arange(k)
    for j in range(k):
        norms = np.sqrt(np.sum(B[j:, j:k] ** 2, axis=0))
        q = j + int(np.argmax(norms))
        if q != j:
            B[:, [j, q]] = B[:, [q, j]]
            piv[[j, q]] = piv[[q, j]]
        x = B[j:, j]
        normx = np.sqrt(np.dot(x, x))
        if normx == 0.0:
            continue
        beta = -normx if x[0] >= 0 else normx
        v = x.copy()
        v[0] -= beta
        vtv = np.dot(v, v)
        w = v @ B[j:, j:]
        B[j:, j:] -= np.outer(v, (2.0 / vtv) * w)
        B[j + 1:, j] = 0.0
        B[j, j] = beta
    return np.triu(B[:k, :k]), B[:k, k:], piv


def complete_orthogonal(Rtop):
    """[R11 R12] = [T 0] Z^T for the leading p x d rows of a column-pivoted R.

    The Householder QR of [R11 R12]^T (d x p), Z [T^T; 0], gives T (p x p,
    lower triangular, nonsingular when R11 is) and the first p columns Z1 of the
    orthogonal Z, so that [R11 R12] = T Z1^T.  Returns (T, Z1).
    """
    p, d = Rtop.shape
    X = np.hstack([Rtop.T, np.eye(d)])
    Tt, C = householder_qr(X, ncols=p)
    return Tt.T, C.T


def numerical_rank(R, rcond):
    """p = number of leading diagonal entries with |r_qq| >= rcond * |r_11|.

    The paper's rule ("largest q with r_qq >= rcond", Ski-LLS-dense parameters)
    read relative to |r_11| and on magnitudes, since Householder diagonals carry
    arbitrary signs.
    """
    dg = np.abs(np.diag(R))
    if dg.size == 0 or dg[0] == 0.0:
        return 0
    ok = dg >= rcond * dg[0]
    p = 0
    while p < dg.size and ok[p]:
        p += 1
    return p


def gram_cholesky(SA):
    """R (d x d upper, positive diagonal) with R^T R = SA^T SA: the Cholesky
    factor of the sketch's Gram matrix, written out column by column
    (r_jj = sqrt(g_jj - sum_{k<j} r_kj^2), r_ji = (g_ji - sum_{k<j} r_kj r_ki) / r_jj
    for i > j).  In exact arithmetic it is the R of a QR factorization of SA
    with a positive diagonal -- the factor Ski-LLS-sparse takes from SPQR on a
    sparse SA (Section 6) -- formed from a Gram matrix that a sparse SA gives
    cheaply.  Raises LinAlgError when a pivot is not positive (SA numerically
    rank-deficient in the Gram's precision)."""
    SA = np.asarray(SA, dtype=np.float64)
    G = SA.T @ SA
    d = G.shape[0]
    R = np.zeros((d, d))
    for j in range(d):
        piv = G[j, j] - R[:j, j] @ R[:j, j]
        if not piv > 0.0:
            raise np.linalg.LinAlgError(f"Gram pivot {j} is not positive")
        R[j, j] = np.sqrt(piv)
        R[j, j + 1:] = (G[j, j + 1:] - R[:j, j] @ R[:j, j + 1:]) / R[j, j]
    return R
