"""The HR-DHT sketch S = S_h F D of Ski-LLS-dense (Section 6, Eq. HR-DHT).

Test infrastructure: see ``oracle/__init__.py`` for who may import this.

F is the normalized discrete Hartley transform, F_ij = N^{-1/2} cas(2 pi i j / N)
with cas = cos + sin and 0-based i, j.  The paper's F has N = n (no padding).
Optionally ``n_h`` = N > n rows: [D A; 0] zero-padded to N rows before F, as
the Walsh-Hadamard premix pads to a power of two (the GPU path transforms
lengths whose prime factors are at most 13 -- n itself for every size the
paper's experiments use -- and pads other n to the next such length, see
``dht_length``).  D is the diagonal of random signs of Def. 8 (the same counter
draw as the Walsh-Hadamard premix), and S_h an s-hashing matrix over the N rows
of F D A.
"""
import numpy as np

from . import hashing, sketch

SMOOTH_PRIMES = (2, 3, 5, 7, 11, 13)


def dht_length(n):
    """The smallest N >= max(n, 1) whose prime factors are all in
    SMOOTH_PRIMES: n itself when n already is such a number."""
    N = max(int(n), 1)
    while True:
        r = N
        for p in SMOOTH_PRIMES:
            while r % p == 0:
                r //= p
        if r == 1:
            return N
        N += 1


def dht_matrix(n):
    """F written out entry by entry from the definition (small n only)."""
    i = np.arange(n)
    theta = 2.0 * np.pi * np.outer(i, i) / n
    return (np.cos(theta) + np.sin(theta)) / np.sqrt(n)


def dht_rows(X):
    """F X for X (n x c or n): the transform applied down every column.

    For real x, sum_j x_j cas(2 pi j k / n) = Re(fft(x))_k - Im(fft(x))_k, since
    the DFT sums x_j (cos - i sin)(2 pi j k / n); the FFT is the library step.
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.fft.fft(X, axis=0)
    return (Y.real - Y.imag) / np.sqrt(X.shape[0])


def premix(seed, A, n_h=None):
    """F D A (or F D b): the signs D of Def. 8, then the normalized DHT of
    length N = n_h (default n) applied to [D A; 0]."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    N = n if n_h is None else int(n_h)
    if N < n:
        raise ValueError("n_h < n")
    D = hashing.premix_signs(seed, n).astype(np.float64)
    X = np.zeros((N,) + A.shape[1:])
    X[:n] = D.reshape((-1,) + (1,) * (A.ndim - 1)) * A
    return dht_rows(X)


def srdht_sketch(seed, m, A, b=None, n_h=None):
    """S_s F D A (Eq. SR-DHT, the sampling sketch the paper compares against):
    m rows of F D A, each chosen uniformly at random with replacement among
    its N rows (``hashing.sample_rows``); with b, [S_s F D A | S_s F D b]."""
    Y = premix(seed, A, n_h)
    rows = hashing.sample_rows(seed, m, Y.shape[0])
    if b is None:
        return Y[rows]
    return np.hstack([Y[rows], premix(seed, b, n_h)[rows, None]])


def hrdht_sketch(seed, s, m, A, b=None, variant=False, n_h=None):
    """[S_h F D A | S_h F D b] with S_h an s-hashing matrix (the variant of
    Def. 7 when variant=True) over the N rows of F D A."""
    Y = premix(seed, A, n_h)
    yb = premix(seed, b, n_h) if b is not None else None
    return sketch.sketch_rows(seed, s, m, Y, yb, variant=variant)
