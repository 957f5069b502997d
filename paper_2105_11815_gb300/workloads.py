"""Seeded synthetic inputs shaped like the paper's least-squares test sets.

This module holds input generators only -- none of the method's arithmetic --
so that the CUDA path and the CPU oracle are fed identical matrices.  The
paper's Test Sets 1-2 (Section 7.1) are random matrices; the shapes and value
laws below stand in for them:

* ``gaussian_lls``: dense A with i.i.d. N(0,1) entries, b = A x_true + noise.
* ``dense_gaussian`` / ``dense_high_coherence``: dense n x d, b = ones (Section
  7.1 sets b to all ones); the high-coherence variant puts 1e3 * I_d plus
  N(0, (1e-3)^2) in its first d rows (a coherent block as in Test Set 1 (c)).
* ``csr_heavy_rows``: CSR A with ~nnz_row uniformly placed N(0,1) entries per
  row plus a fraction of heavy rows (high coherence), b = ones.
* ``usv``: A = U Sigma V^T with Haar U, V and geometric singular values of a
  given condition number (Test Set 1 (a) with a geometric spectrum).
* ``ragged_batch``: shapes of a ragged batch of problems.
* ``semi_coherent_sparse``: D^5 B (Test Set 2 (b)) with B an incoherent sparse
  pattern of N(0,1) values and D a diagonal of N(0,1) entries, stored dense.
* ``coherent_dense``: [I_d; 0] + 1e-8 J (Section 7.1, Test Set 1 (c)).
* ``low_rank_lls``: dense A = G1 G2 of rank r < d (the rank-deficient problems
  of Test Set 2 and Table 2), b ~ N(0,1).
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(np.uint64(seed))


def gaussian_lls(n, d, seed, noise=1e-3):
    """A n x d i.i.d. N(0,1); b = A x_true + noise * N(0,1); returns (A, b, x_true)."""
    g = rng(seed)
    A = g.standard_normal((n, d))
    x_true = g.standard_normal(d)
    b = A @ x_true + noise * g.standard_normal(n)
    return A, b, x_true


def dense_gaussian(n, d, seed):
    """A n x d i.i.d. N(0,1) and b = ones."""
    g = rng(seed)
    return g.standard_normal((n, d)), np.ones(n)


def dense_high_coherence(n, d, seed, big=1e3, small_sd=1e-3):
    """First d rows big * I_d + N(0, small_sd^2), the rest N(0,1); b = ones."""
    g = rng(seed)
    A = g.standard_normal((n, d))
    A[:d] = big * np.eye(d) + small_sd * g.standard_normal((d, d))
    return A, np.ones(n)


def csr_heavy_rows(n, d, seed, nnz_row=8, heavy_frac=1e-3, heavy_nnz=2000):
    """CSR arrays (rowptr int64, colidx int32, val f64) and b = ones.

    Every row has ``nnz_row`` distinct uniformly placed columns; floor(heavy_frac*n)
    rows chosen uniformly have ``min(heavy_nnz, d)`` instead.  Values N(0,1).
    Column indices within a row are sorted ascending.
    """
    g = rng(seed)
    counts = np.full(n, min(nnz_row, d), dtype=np.int64)
    nheavy = int(np.floor(heavy_frac * n))
    heavy = g.choice(n, size=nheavy, replace=False) if nheavy else np.zeros(0, dtype=np.int64)
    counts[heavy] = min(heavy_nnz, d)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = np.empty(rowptr[-1], dtype=np.int32)
    light = counts == min(nnz_row, d)
    # light rows: rejection-free distinct columns via sorting random keys per row
    lrows = np.nonzero(light)[0]
    k = min(nnz_row, d)
    if lrows.size:
        cols = g.integers(0, d, size=(lrows.size, k))
        # resample rows with duplicate columns until all are distinct
        srt = np.sort(cols, axis=1)
        dup = (srt[:, 1:] == srt[:, :-1]).any(axis=1) if k > 1 else np.zeros(lrows.size, bool)
        while dup.any():
            cols[dup] = g.integers(0, d, size=(int(dup.sum()), k))
            srt = np.sort(cols, axis=1)
            dup = (srt[:, 1:] == srt[:, :-1]).any(axis=1)
        starts = rowptr[lrows]
        colidx[(starts[:, None] + np.arange(k)[None, :]).ravel()] = srt.ravel()
    for r in heavy:
        colidx[rowptr[r]:rowptr[r + 1]] = np.sort(g.choice(d, size=counts[r], replace=False))
    val = g.standard_normal(rowptr[-1])
    return rowptr, colidx, val, np.ones(n)


def haar(n, d, g):
    """n x d matrix with Haar-distributed orthonormal columns (QR of a Gaussian,
    diagonal of R made positive, Mezzadri 2007)."""
    Z = g.standard_normal((n, d))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def usv(n, d, kappa, seed):
    """A = U diag(sigma) V^T, sigma_i = kappa^{-(i-1)/(d-1)}; b = ones."""
    g = rng(seed)
    U = haar(n, d, g)
    V = haar(d, d, g)
    sig = kappa ** (-np.arange(d) / max(d - 1, 1))
    return (U * sig[None, :]) @ V.T, np.ones(n)


def semi_coherent_sparse(n, d, seed, density=0.1, power=5):
    """A = D^power B, B with N(0,1) values at a uniform fraction ``density`` of
    positions, D = diag(N(0,1)) (the row scaling makes a few rows dominate)."""
    g = rng(seed)
    B = g.standard_normal((n, d)) * (g.random((n, d)) < density)
    return (g.standard_normal(n) ** power)[:, None] * B


def coherent_dense(n, d):
    """A = [I_d; 0] + 1e-8 J, J all ones (Test Set 1 (c)): coherence ~ 1."""
    A = np.full((n, d), 1e-8)
    A[np.arange(d), np.arange(d)] += 1.0
    return A


def low_rank_lls(n, d, r, seed):
    """A = G1 G2 with G1 (n x r) and G2 (r x d) i.i.d. N(0,1): rank r; b ~ N(0,1)."""
    g = rng(seed)
    A = g.standard_normal((n, r)) @ g.standard_normal((r, d))
    return A, g.standard_normal(n)


def ragged_batch(count, seed, n_lo=2000, n_hi=60000, d_lo=64, d_hi=1024, ratio=4):
    """List of (n, d): d ~ U{d_lo..d_hi}, then n ~ U{max(n_lo, ratio*d)..n_hi}."""
    g = rng(seed)
    out = []
    for _ in range(count):
        d = int(g.integers(d_lo, d_hi + 1))
        n = int(g.integers(max(n_lo, ratio * d), n_hi + 1))
        out.append((n, d))
    return out


# ---- device-side generators for the full-size measurement workloads --------
# Same distributions as above, drawn with torch's seeded generator on the GPU
# (numpy would take minutes at these sizes).  Used by the benchmark only; the
# parity tests use the numpy generators.

def gaussian_torch(n, d, seed, device):
    """A n x d i.i.d. N(0,1) (FP64, on `device`) and b = ones."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    A = torch.randn(n, d, generator=g, device=device, dtype=torch.float64)
    return A, torch.ones(n, dtype=torch.float64, device=device)


def dense_high_coherence_torch(n, d, seed, device, big=1e3, small_sd=1e-3):
    """`dense_high_coherence` drawn on `device` with torch's seeded generator."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    A = torch.randn(n, d, generator=g, device=device, dtype=torch.float64)
    A[:d] = big * torch.eye(d, device=device, dtype=torch.float64) + small_sd * torch.randn(
        d, d, generator=g, device=device, dtype=torch.float64)
    return A, torch.ones(n, dtype=torch.float64, device=device)


def usv_torch(n, d, kappa, seed, device, rhs="ones"):
    """A = U diag(sigma) V^T with Haar U (n x d), V (d x d) (QR of a Gaussian,
    diag(R) made positive), sigma_i = kappa^{-(i-1)/(d-1)}.
    rhs="ones": b = ones.  rhs="perp": b = A x_true + e with x_true ~ N(0, 1)
    and e orthogonal to range(A) (e = g - U U^T g, g ~ N(0, 1)) scaled to
    ||e|| = ||A x_true||: the solution is x_true, O(1), whatever kappa."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))

    def haar_t(rows, cols):
        Z = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float64)
        Q, R = torch.linalg.qr(Z)
        del Z
        Q *= torch.sign(torch.diagonal(R))[None, :]
        return Q

    U = haar_t(n, d)
    V = haar_t(d, d)
    e = None
    if rhs == "perp":
        e = torch.randn(n, generator=g, device=device, dtype=torch.float64)
        e -= U @ (U.T @ e)
    sig = kappa ** (-torch.arange(d, dtype=torch.float64, device=device) / max(d - 1, 1))
    U *= sig[None, :]
    A = U @ V.T
    del U
    if rhs == "perp":
        xt = torch.randn(d, generator=g, device=device, dtype=torch.float64)
        ax = A @ xt
        return A, ax + e * (torch.linalg.norm(ax) / torch.linalg.norm(e))
    return A, torch.ones(n, dtype=torch.float64, device=device)


def ragged_batch_torch(count, seed, device, **kw):
    """The ragged batch of `ragged_batch` with A_i, b_i i.i.d. N(0,1) on `device`."""
    import torch
    shapes = ragged_batch(count, seed, **kw)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    As = [torch.randn(n, d, generator=g, device=device, dtype=torch.float64) for n, d in shapes]
    bs = [torch.randn(n, generator=g, device=device, dtype=torch.float64) for n, _ in shapes]
    return shapes, As, bs
