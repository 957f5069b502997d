"""The HR-DHT sketch S = S_h F D of Ski-LLS-dense (Section 6, Eq. HR-DHT).

Test infrastructure: see ``oracle/__init__.py`` for who may import this.

F is the normalized discrete Hartley transform, F_ij = n^{-1/2} cas(2 pi i j / n)
with cas = cos + sin and 0-based i, j; it needs no padding (any n).  D is the
diagonal of random signs of Def. 8 (the same counter draw as the Walsh-Hadamard
premix), and S_h an s-hashing matrix over the n rows of F D A.
"""
import numpy as np

from . import hashing, sketch


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


def premix(seed, A):
    """F D A (or F D b): the signs D of Def. 8, then the normalized DHT."""
    A = np.asarray(A, dtype=np.float64)
    D = hashing.premix_signs(seed, A.shape[0]).astype(np.float64)
    return dht_rows(D.reshape((-1,) + (1,) * (A.ndim - 1)) * A)


def srdht_sketch(seed, m, A):
    """S_s F D A (Eq. SR-DHT, the sampling sketch the paper compares against):
    m rows of F D A, each chosen uniformly at random with replacement."""
    return premix(seed, A)[hashing.sample_rows(seed, m, np.asarray(A).shape[0])]


def hrdht_sketch(seed, s, m, A, b=None, variant=False):
    """[S_h F D A | S_h F D b] with S_h an s-hashing matrix (the variant of
    Def. 7 when variant=True) over the n rows of F D A."""
    Y = premix(seed, A)
    yb = premix(seed, b) if b is not None else None
    return sketch.sketch_rows(seed, s, m, Y, yb, variant=variant)
