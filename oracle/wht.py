"""Walsh-Hadamard transform and the HRHT premix S_h H D (Def. 8).

Test infrastructure: see ``oracle/__init__.py`` for who may import this.

Def. 8: H is the n x n matrix with H_ij = n^{-1/2} (-1)^{<(i-1)_2, (j-1)_2>}
(natural, Sylvester order) and D a diagonal of independent +-1.  For a height
that is not a power of two the rows are zero-padded to n_pad = 2^ceil(log2 n),
so that H is n_pad x n_pad and S_h hashes all n_pad rows of H D [A; 0].
"""
import numpy as np

from . import hashing, sketch


def fwht_rows(X):
    """Unnormalised Walsh-Hadamard transform along axis 0, Sylvester order.

    For every bit b of the row index, rows i and i + 2^b (bit b of i clear) are
    replaced by their sum and difference: H_{2h} = [[H_h, H_h], [H_h, -H_h]].
    The height of X must be a power of two.  Returns a new array.
    """
    X = np.array(X, dtype=np.float64, copy=True)
    n = X.shape[0]
    if n & (n - 1):
        raise ValueError("height must be a power of two")
    tail = X.shape[1:]
    h = 1
    while h < n:
        Y = X.reshape((n // (2 * h), 2, h) + tail)
        a = Y[:, 0].copy()
        bb = Y[:, 1].copy()
        Y[:, 0] = a + bb
        Y[:, 1] = a - bb
        X = Y.reshape((n,) + tail)
        h *= 2
    return X


def premix(seed, A, n_pad):
    """H D [A; 0] with H the normalised n_pad x n_pad Walsh-Hadamard matrix (Def. 8).

    A: n x d (or a length-n vector).  The rows of A are multiplied by D_jj,
    padded with zero rows to n_pad, transformed, and scaled by n_pad^{-1/2}.
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if n_pad < n or n_pad & (n_pad - 1):
        raise ValueError("n_pad must be a power of two >= n")
    D = hashing.premix_signs(seed, n).astype(np.float64)
    Y = np.zeros((n_pad,) + A.shape[1:], dtype=np.float64)
    Y[:n] = D.reshape((n,) + (1,) * (A.ndim - 1)) * A
    return fwht_rows(Y) / np.sqrt(n_pad)


def hrht_sketch(seed, s, m, A, b=None, n_pad=None, variant=False):
    """[S_h H D A | S_h H D b] for the HRHT sketch of Def. 8 with an s-hashing S_h
    (the s-hashing variant of Def. 7 when variant=True)."""
    n = A.shape[0]
    if n_pad is None:
        n_pad = 1 << max(0, (n - 1).bit_length())
    Y = premix(seed, A, n_pad)
    yb = premix(seed, b, n_pad) if b is not None else None
    return sketch.sketch_rows(seed, s, m, Y, yb, variant=variant)
