"""Gradient of the least-squares solution x(A, b) = argmin ||A x - b||_2.

Test infrastructure: see ``oracle/__init__.py`` for who may import this.

The paper has no backward pass; this is the closed form the differentiable
solve must reproduce.  Differentiating the normal equations A^T A x = A^T b:
A^T A dx = dA^T r + A^T db - A^T dA x with r = b - A x.  For a loss L with
g = dL/dx and lambda = (A^T A)^{-1} g this gives
dL/db = A lambda and dL/dA = r lambda^T - (A lambda) x^T.
lambda is obtained from LAPACK's QR of A (A^T A = R_A^T R_A).
"""
import numpy as np
from scipy.linalg import solve_triangular


def lstsq_grad(A, b, x, g):
    """(dL/dA, dL/db) for x = argmin ||Ax - b|| and upstream gradient g = dL/dx."""
    A = np.asarray(A, dtype=np.float64)
    Ra = np.linalg.qr(A, mode="r")
    lam = solve_triangular(Ra, solve_triangular(Ra, g, trans="T"))
    r = b - A @ x
    Al = A @ lam
    return np.outer(r, lam) - np.outer(Al, x), Al
