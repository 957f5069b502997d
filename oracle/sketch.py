"""The s-hashing sketch S*A and S*b (Algorithm 1, Step 1; Def. 5; Def. 7).

Test infrastructure: see ``oracle/__init__.py`` for who may import this.
"""
import numpy as np

from . import hashing


def s_hashing_matrix(seed, s, m, n):
    """The m x n s-hashing matrix of Def. 5, built column by column (dense).

    Column j holds +-1/sqrt(s) in the s distinct rows drawn for it.  Only for
    small n: this is the brute-force reference for the row-wise sketch.
    """
    S = np.zeros((m, n), dtype=np.float64)
    scale = 1.0 / np.sqrt(s)
    for j in range(n):
        rows, signs = hashing.column_rows_int(seed, s, m, j)
        for i, sg in zip(rows, signs):
            S[i, j] = sg * scale
    return S


def s_hashing_variant_matrix(seed, s, m, n):
    """The m x n s-hashing VARIANT of Def. 7, built column by column (dense).

    For each column j, each of the s draws (with replacement) ADDS +-1/sqrt(s)
    to its row, so a row drawn twice holds the sum.  Only for small n.
    """
    T = np.zeros((m, n), dtype=np.float64)
    scale = 1.0 / np.sqrt(s)
    for j in range(n):
        rows, signs = hashing.variant_column_rows_int(seed, s, m, j)
        for i, sg in zip(rows, signs):
            T[i, j] += sg * scale
    return T


def sketch_rows(seed, s, m, A, b=None, variant=False):
    """S*A (and S*b) for the s-hashing matrix of Def. 5, row by row of A.

    Row j of A is added, with sign sign[j,k]/sqrt(s), to row idx[j,k] of SA for
    each k < s: the product S*A written out over the nonzeros of S (Step 1 of
    Algorithm 1).  A may be dense (n x d ndarray) or a scipy CSR matrix.
    variant=True uses the draws of the s-hashing variant T (Def. 7) instead;
    the same accumulation then adds coinciding draws.
    Returns SA (m x d) or, when b is given, the augmented [SA | Sb] (m x (d+1)).
    """
    n, d = A.shape
    idx, sign = (hashing.variant_table if variant else hashing.hash_table)(seed, s, m, n)
    scale = 1.0 / np.sqrt(s)
    cols = d + (1 if b is not None else 0)
    out = np.zeros((m, cols), dtype=np.float64)
    dense = isinstance(A, np.ndarray)
    for k in range(s):
        coef = sign[:, k].astype(np.float64) * scale
        if dense:
            np.add.at(out[:, :d], idx[:, k], coef[:, None] * A)
        else:
            csr = A.tocsr()
            rows = np.repeat(np.arange(n), np.diff(csr.indptr))
            np.add.at(out, (idx[rows, k], csr.indices), coef[rows] * csr.data)
        if b is not None:
            np.add.at(out[:, d], idx[:, k], coef * b)
    return out
