"""Counter-based draw of the s-hashing matrix (Def. 5) and the premix signs D (Def. 8).

Test infrastructure: see ``oracle/__init__.py`` for who may import this.

Def. 5 asks, independently for every column j of S (one per row of A), for s
row indices i_1..i_s drawn uniformly WITHOUT replacement from [m], each entry
being +-1/sqrt(s).  The paper fixes no random number generator, so the draw is
a pure function of (seed, j, k, t) -- a counter-based hash -- which both this
oracle and the CUDA library implement independently from one published
definition:

* ``splitmix64(z)``: the output function of the SplitMix64 generator of Steele,
  Lea & Flood (OOPSLA 2014): z += 0x9E3779B97F4A7C15, then two xor-shift-multiply
  rounds with 0xBF58476D1CE4E5B9 (shift 30) and 0x94D049BB133111EB (shift 27),
  then z ^ (z >> 31).  Pinned against the published generator outputs for
  state 0 in ``tests/golden/splitmix64.txt``.
* ``key(seed, tag, j, k, t) = sm(sm(sm(seed ^ (tag << 56)) ^ j) ^ (k << 32 | t))``
  with sm = splitmix64, all arithmetic modulo 2**64.
* bucket draw number t of nonzero k of column j: floor(key(seed, BUCKET, j, k, t) * m / 2**64),
  i.e. the high 64 bits of the 128-bit product (bias below m / 2**64).
* without replacement (s >= 2): nonzero k takes the first draw t = 0, 1, ...
  that differs from the rows already taken by nonzeros 0..k-1 (rejection), so
  the s rows are a uniform s-subset of [m] in draw order.
* with replacement (the s-hashing variant of Def. 7): draw k is the t = 0
  bucket draw of nonzero k, whatever the earlier draws were.
* sign of nonzero k: -1 when the top bit of key(seed, SIGN, j, k, 0) is set, else +1.
* premix sign D_j (Def. 8): -1 when the top bit of key(seed, PREMIX, j, 0, 0) is set.
"""
import numpy as np

MASK64 = (1 << 64) - 1
SM_GAMMA = 0x9E3779B97F4A7C15
SM_MUL1 = 0xBF58476D1CE4E5B9
SM_MUL2 = 0x94D049BB133111EB

TAG_BUCKET = 0xB1
TAG_SIGN = 0x5A
TAG_PREMIX = 0xD3
TAG_SAMPLE = 0x5E


def splitmix64(z):
    """SplitMix64 output function on one Python integer (Steele, Lea & Flood 2014)."""
    z = (z + SM_GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * SM_MUL1) & MASK64
    z = ((z ^ (z >> 27)) * SM_MUL2) & MASK64
    return z ^ (z >> 31)


def key(seed, tag, j, k, t):
    """The 64-bit hash word for (seed, tag, column j, nonzero k, retry t)."""
    base = splitmix64((seed ^ (tag << 56)) & MASK64)
    return splitmix64(splitmix64(base ^ j) ^ (((k & 0xFFFFFFFF) << 32) | (t & 0xFFFFFFFF)))


def column_rows_int(seed, s, m, j):
    """Rows i_1..i_s and signs of column j of an s-hashing matrix (Def. 5), pure Python.

    Used on small cases to cross-check the vectorised ``hash_table``.
    """
    rows, signs = [], []
    for k in range(s):
        t = 0
        while True:
            i = (key(seed, TAG_BUCKET, j, k, t) * m) >> 64
            if i not in rows:
                break
            t += 1
        rows.append(i)
        signs.append(-1 if key(seed, TAG_SIGN, j, k, 0) >> 63 else 1)
    return rows, signs


def variant_column_rows_int(seed, s, m, j):
    """Draws i_1..i_s and signs of column j of the s-hashing variant (Def. 7), pure Python.

    Def. 7 samples the s rows uniformly WITH replacement, so draw k is simply
    the t = 0 bucket draw of nonzero k; rows may repeat.
    """
    rows = [(key(seed, TAG_BUCKET, j, k, 0) * m) >> 64 for k in range(s)]
    signs = [-1 if key(seed, TAG_SIGN, j, k, 0) >> 63 else 1 for k in range(s)]
    return rows, signs


def premix_sign_int(seed, j):
    """D_jj of Def. 8 for one j, pure Python."""
    return -1 if key(seed, TAG_PREMIX, j, 0, 0) >> 63 else 1


# ---------------------------------------------------------------- vectorised
def _sm64_np(z):
    z = z + np.uint64(SM_GAMMA)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(SM_MUL1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(SM_MUL2)
    return z ^ (z >> np.uint64(31))


def _key_np(seed, tag, j, k, t):
    base = np.uint64(splitmix64((seed ^ (tag << 56)) & MASK64))
    ctr = np.uint64(((k & 0xFFFFFFFF) << 32)) | np.asarray(t, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _sm64_np(_sm64_np(base ^ j) ^ ctr)


def _mulhi_np(w, m):
    """floor(w * m / 2**64) for uint64 w and 0 < m < 2**32, in 64-bit pieces."""
    m = np.uint64(m)
    hi = w >> np.uint64(32)
    lo = w & np.uint64(0xFFFFFFFF)
    with np.errstate(over="ignore"):
        return (hi * m + ((lo * m) >> np.uint64(32))) >> np.uint64(32)


def hash_table(seed, s, m, n):
    """Rows idx[j, k] and signs sign[j, k] of the s-hashing matrix S (m x n), Def. 5.

    Column j of S has the entry sign[j, k] / sqrt(s) in row idx[j, k], k < s.
    Returns (idx int64 (n, s), sign int8 (n, s)).
    """
    if not (1 <= s <= m < 2 ** 31):
        raise ValueError("need 1 <= s <= m < 2**31")
    j = np.arange(n, dtype=np.uint64)
    idx = np.empty((n, s), dtype=np.int64)
    sign = np.empty((n, s), dtype=np.int8)
    for k in range(s):
        t = np.zeros(n, dtype=np.uint64)
        cand = _mulhi_np(_key_np(seed, TAG_BUCKET, j, k, t), m).astype(np.int64)
        clash = np.zeros(n, dtype=bool)
        for kk in range(k):
            clash |= cand == idx[:, kk]
        while clash.any():
            t = t + clash.astype(np.uint64)
            redraw = _mulhi_np(_key_np(seed, TAG_BUCKET, j[clash], k, t[clash]), m).astype(np.int64)
            cand[clash] = redraw
            clash = np.zeros(n, dtype=bool)
            for kk in range(k):
                clash |= cand == idx[:, kk]
        idx[:, k] = cand
        w = _key_np(seed, TAG_SIGN, j, k, np.zeros(n, dtype=np.uint64))
        sign[:, k] = np.where((w >> np.uint64(63)) != 0, -1, 1).astype(np.int8)
    return idx, sign


def premix_signs(seed, n):
    """Diagonal of D (Def. 8) for rows 0..n-1, as int8 +-1."""
    j = np.arange(n, dtype=np.uint64)
    w = _key_np(seed, TAG_PREMIX, j, 0, np.zeros(n, dtype=np.uint64))
    return np.where((w >> np.uint64(63)) != 0, -1, 1).astype(np.int8)


def sample_rows(seed, m, n):
    """Columns c_0..c_{m-1} of a sampling matrix S_s (m x n): row i of S_s holds
    a single 1 in column c_i, drawn uniformly from [n] (independently for every
    row, so columns may repeat): c_i = floor(key(seed, SAMPLE, i, 0, 0) n / 2^64)."""
    i = np.arange(m, dtype=np.uint64)
    return _mulhi_np(_key_np(seed, TAG_SAMPLE, i, 0, np.zeros(m, dtype=np.uint64)), n).astype(np.int64)


def variant_table(seed, s, m, n):
    """Rows and signs of the s-hashing VARIANT (Def. 7): s draws WITH replacement.

    Draw k of column j is the t = 0 bucket draw; coinciding rows add up.
    """
    j = np.arange(n, dtype=np.uint64)
    idx = np.empty((n, s), dtype=np.int64)
    sign = np.empty((n, s), dtype=np.int8)
    z = np.zeros(n, dtype=np.uint64)
    for k in range(s):
        idx[:, k] = _mulhi_np(_key_np(seed, TAG_BUCKET, j, k, z), m).astype(np.int64)
        w = _key_np(seed, TAG_SIGN, j, k, z)
        sign[:, k] = np.where((w >> np.uint64(63)) != 0, -1, 1).astype(np.int8)
    return idx, sign
