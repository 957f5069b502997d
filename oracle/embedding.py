"""Subspace-embedding distortion (Lemma 2) and coherence (Def. 6).

Test infrastructure: see ``oracle/__init__.py`` for who may import this.
"""
import numpy as np


def orth(A, tol=1e-12):
    """U of the thin SVD A = U Sigma V^T (Eq. thin-SVD), restricted to rank r."""
    U, sv, _ = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    r = int(np.sum(sv > tol * sv[0])) if sv.size and sv[0] > 0 else 0
    return U[:, :r]


def distortion(SU):
    """Smallest eps with (1-eps)||z||^2 <= ||S U z||^2 <= (1+eps)||z||^2 (Lemma 2 (ii)).

    SU is S applied to an orthonormal basis U of range(A): eps is
    max(sigma_max(SU)^2 - 1, 1 - sigma_min(SU)^2).
    """
    sv = np.linalg.svd(SU, compute_uv=False)
    return float(max(sv[0] ** 2 - 1.0, 1.0 - sv[-1] ** 2))


def coherence(A):
    """mu(A) = max_i ||U_i||_2 over the rows of U (Def. 6)."""
    U = orth(A)
    return float(np.max(np.linalg.norm(U, axis=1)))
