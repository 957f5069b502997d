"""C ABI: the library builds for sm_103a, loads, exports every declared entry
point, and rejects bad arguments on the host (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "skills.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def lib():
    from paper_2105_11815_gb300 import build
    build.build()
    import paper_2105_11815_gb300 as pkg
    return pkg


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"typedef[^;]*;", "", text)  # types (the all-reduce callback), not entry points
    return sorted(set(re.findall(r"\b(ski_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    h = ctypes.CDLL(lib.lib_path)
    for n in names:
        assert hasattr(h, n), n
    assert set(names) == set(lib._SIGS), set(names) ^ set(lib._SIGS)


def test_host_only_entry_points(lib):
    assert lib.ski_version() == 100
    assert lib.ski_status_string(0) == "SKI_OK"
    assert "workspace" in lib.ski_status_string(2)
    assert lib.ski_status_string(99) == "unknown ski_status"
    o = lib.ski_opts_default(m=10)
    assert (o.s, o.m, o.tau_a, o.tau_r, o.it_max, o.rcond) == (1, 10, 1e-8, 1e-6, 10000, 1e-12)


def test_mixed_lsqr_budget_follows_theorem10(lib):
    # 2.2 x (log 2 + |log tau_r|) / |log eps| with eps = sqrt(d / m), in [150, 4000]
    import math

    def bound(m, d, tau):
        return (math.log(2) - math.log(tau)) / (0.5 * math.log(m / d))
    assert lib.ski_mixed_lsqr_budget(8000, 4000, 1e-10) == 151          # m = 2d: the former fixed 150
    assert lib.ski_mixed_lsqr_budget(8000, 4000, 1e-10) == math.ceil(2.2 * bound(8000, 4000, 1e-10))
    assert lib.ski_mixed_lsqr_budget(4800, 4000, 1e-10) == math.ceil(2.2 * bound(4800, 4000, 1e-10)) > 500
    assert lib.ski_mixed_lsqr_budget(480, 400, 1e-12) == math.ceil(2.2 * bound(480, 400, 1e-12))
    assert lib.ski_mixed_lsqr_budget(40000, 1000, 1e-10) == 150           # large gamma: the floor
    assert lib.ski_mixed_lsqr_budget(4000, 4000, 1e-10) == 4000           # m = d: no embedding bound
    assert lib.ski_mixed_lsqr_budget(4001, 4000, 1e-10) == 4000           # capped
    assert lib.ski_mixed_lsqr_budget(8000, 4000, 0.0) == 150              # tau_r outside (0, 1)
    assert lib.ski_mixed_lsqr_budget(8000, 4000, 1.0) == 150
    # monotone: a smaller sketch is allowed more iterations, a tighter tau_r too
    ms = [4400, 4800, 5600, 6800, 8000]
    b = [lib.ski_mixed_lsqr_budget(m, 4000, 1e-10) for m in ms]
    assert b == sorted(b, reverse=True)
    assert lib.ski_mixed_lsqr_budget(4800, 4000, 1e-12) > lib.ski_mixed_lsqr_budget(4800, 4000, 1e-10)


def _fake_dense(lib, n, d):
    return lib.ski_matrix(kind=lib.SKI_DENSE, n=n, d=d, ld=d, val=0x1000, rowptr=None, colidx=None, nnz=0)


def test_argument_errors_before_launch(lib):
    L = lib.lib()
    # s > m, m >= 2^31, n < 0 rejected without touching the device
    assert L.ski_hash_indices(1, 5, 4, 10, None, None, None) == 1
    assert L.ski_hash_indices(1, 1, 1 << 31, 10, None, None, None) == 1
    assert L.ski_hash_indices(1, 1, 4, -1, None, None, None) == 1
    assert L.ski_hash_indices(1, 1, 4, 0, None, None, None) == 0  # empty: nothing to do
    # the variant (Def. 7) draws with replacement: s > m is valid, s > 64 and m < 1 are not
    assert L.ski_hash_variant_indices(1, 5, 4, 0, None, None, None) == 0
    assert L.ski_hash_variant_indices(1, 5, 4, 10, None, None, None) == 1   # valid sizes, null outputs
    assert L.ski_hash_variant_indices(1, 65, 100, 0, None, None, None) == 1
    assert L.ski_hash_variant_indices(1, 1, 0, 0, None, None, None) == 1
    A_ = _fake_dense(lib, 100, 3)
    for hk, ok_ in ((0, True), (1, True), (2, False), (-1, False)):
        o_ = lib.ski_opts_default(m=20, s=2, hash_kind=hk)
        assert (L.ski_sketch_workspace_size(ctypes.byref(A_), 1, ctypes.byref(o_)) > 0) == ok_
    o_ = lib.ski_opts_default(m=2, s=3, hash_kind=1)    # s > m: only the variant allows it
    assert L.ski_sketch_workspace_size(ctypes.byref(A_), 1, ctypes.byref(o_)) > 0
    o_.hash_kind = 0
    assert L.ski_sketch_workspace_size(ctypes.byref(A_), 1, ctypes.byref(o_)) == 0
    A = _fake_dense(lib, 100, 10)
    bad = lib.ski_opts_default(m=5, s=1)          # m < d
    x = ctypes.c_void_p(0x2000)
    info = lib.ski_info()
    assert L.ski_solve(ctypes.byref(A), x, ctypes.byref(bad), x, None, ctypes.byref(info), None, 0, None) == 1
    ok = lib.ski_opts_default(m=20, s=2)
    need = L.ski_solve_workspace_size(ctypes.byref(A), ctypes.byref(ok))
    assert need > 0
    assert L.ski_solve(ctypes.byref(A), x, ctypes.byref(ok), x, None, ctypes.byref(info), x, need - 1, None) == 2
    assert info.status == 2
    prem = lib.ski_opts_default(m=20, s=1, premix=1, n_pad=96)  # not a power of two
    assert L.ski_sketch_workspace_size(ctypes.byref(A), 1, ctypes.byref(prem)) == 0
    csr = lib.ski_matrix(kind=lib.SKI_CSR, n=100, d=10, ld=0, val=0x1000, rowptr=0x1000, colidx=0x1000, nnz=5)
    prem2 = lib.ski_opts_default(m=20, s=1, premix=1)
    assert L.ski_sketch_workspace_size(ctypes.byref(csr), 1, ctypes.byref(prem2)) == 0  # premix is dense-only
    assert L.ski_precondition(10, 20, 1, x, 21, 0, x, 20, None, None, None, x, 1 << 30, None) == 1  # m < d
    # dense width above the LSQR pass's limit (8192 columns), negative options
    wide = _fake_dense(lib, 20000, 8193)
    ow = lib.ski_opts_default(m=16386, s=1)
    assert L.ski_solve(ctypes.byref(wide), x, ctypes.byref(ow), x, None, ctypes.byref(info), x, 1 << 40, None) == 1
    assert L.ski_solve_adjoint(ctypes.byref(wide), x, x, x, 8193, x, x, 8193, x, ctypes.byref(ow), None, x, 1 << 40,
                               None) == 1
    for field, v in (("premix_slab", -1), ("streams", -1), ("s", 0), ("qr_dtype", 2), ("it_max", -1),
                     ("lsqr_pass", 6), ("lsqr_pass", -1), ("lsqr_ctas", -1), ("graphs", 2), ("batch_lsqr", 2),
                     ("batch_lsqr", -1)):
        o2 = lib.ski_opts_default(m=20, s=1)
        setattr(o2, field, v)
        assert L.ski_solve(ctypes.byref(A), x, ctypes.byref(o2), x, None, ctypes.byref(info), x, 1 << 40, None) == 1, \
            field


def test_workspace_queries_are_consistent(lib):
    L = lib.lib()
    A = _fake_dense(lib, 50000, 4000)
    o = lib.ski_opts_default(m=8000, s=2, premix=1, n_pad=65536)
    sk = L.ski_sketch_workspace_size(ctypes.byref(A), 1, ctypes.byref(o))
    so = L.ski_solve_workspace_size(ctypes.byref(A), ctypes.byref(o))
    assert 0 < sk < so
    # full-width FP64 premix: two int64 planes of n_pad x 4032, handed to the
    # gather as they are (no FP64 copy of the premixed matrix)
    assert 2 * 65536 * 4001 * 8 <= sk < 3 * 65536 * 4001 * 8
    # in column slabs of 64: the same planes 64 columns wide
    slab = lib.ski_opts_default(m=8000, s=2, premix=1, n_pad=65536, premix_slab=64)
    sks = L.ski_sketch_workspace_size(ctypes.byref(A), 1, ctypes.byref(slab))
    assert 3 * 65536 * 64 * 8 <= sks < 3 * 65536 * 65 * 8 + 8 * 65536 * 2 + (64 << 20)
    o32 = lib.ski_opts_default(m=8000, s=2, premix=1, n_pad=65536, sketch_dtype=lib.SKI_F32, qr_dtype=lib.SKI_F32)
    assert L.ski_sketch_workspace_size(ctypes.byref(A), 1, ctypes.byref(o32)) > 0
    bad = lib.ski_opts_default(m=8000, s=2, premix=1, n_pad=65536, premix_slab=-1)
    assert L.ski_sketch_workspace_size(ctypes.byref(A), 1, ctypes.byref(bad)) == 0


def test_gram_step2_workspace_covers_its_scratch(lib):
    # factorization = 2 for dense A: the FP64 slices of SA (11 FP16 slices of
    # d x m at m = 8000) and, for d > 1024, the d x d FP64 panel product come
    # out of the same workspace; the mixed form is sized for its FP64
    # fallback too
    L = lib.lib()
    A = _fake_dense(lib, 50000, 4000)
    sizes = {}
    for f in (0, 2):
        for mixed in (False, True):
            prec = dict(sketch_dtype=lib.SKI_F32, qr_dtype=lib.SKI_F32) if mixed else {}
            o = lib.ski_opts_default(m=8000, s=1, factorization=f, **prec)
            sizes[f, mixed] = L.ski_solve_workspace_size(ctypes.byref(A), ctypes.byref(o))
    assert sizes[2, False] > sizes[0, False] > 0
    assert sizes[2, False] >= 11 * 4000 * 8000 * 2 + 4000 * 4000 * 8
    assert sizes[2, True] >= sizes[2, False]


def test_missing_library_fails_loudly(monkeypatch):
    import paper_2105_11815_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "lib_path", "/nonexistent/libskills.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        pkg.lib()


def test_batched_workspace_scales_with_streams_and_rejects_negative(lib):
    pkg = lib
    mats = [pkg.ski_matrix(kind=0, n=1000 + 10 * i, d=20 + i, ld=20 + i, val=ctypes.c_void_p(4096))
            for i in range(5)]
    one = pkg.ski_opts_default(m=-2000, streams=1)
    four = pkg.ski_opts_default(m=-2000, streams=4)
    auto = pkg.ski_opts_default(m=-2000)
    w1 = pkg.ski_solve_batched_workspace_size(mats, one)
    assert w1 > 0 and w1 % 256 == 0
    assert pkg.ski_solve_batched_workspace_size(mats, four) == 4 * w1
    assert pkg.ski_solve_batched_workspace_size(mats, auto) == 5 * w1   # min(nprob, 8)
    # grouped Step 4 adds the executor's job and work-item lists
    grouped = pkg.ski_solve_batched_workspace_size(mats, pkg.ski_opts_default(m=-2000, streams=4, batch_lsqr=1))
    assert 4 * w1 < grouped < 5 * w1 and grouped % 256 == 0
    assert pkg.ski_solve_batched_workspace_size(mats, pkg.ski_opts_default(m=-2000, batch_lsqr=2)) == 0
    a1 = pkg.ski_solve_adjoint_batched_workspace_size(mats, one)
    assert a1 > 0 and pkg.ski_solve_adjoint_batched_workspace_size(mats, four) == 4 * a1
    bad = pkg.ski_opts_default(m=-2000, streams=-1)
    arr = (pkg.ski_matrix * 5)(*mats)
    ptrs = (ctypes.c_void_p * 5)(*([4096] * 5))
    st = pkg.lib().ski_solve_batched(5, arr, ptrs, ctypes.byref(bad), ptrs, None, None, ctypes.c_void_p(4096),
                                     1 << 40, None)
    assert st == 1  # SKI_EINVAL
    st = pkg.lib().ski_solve_adjoint_batched(5, arr, ptrs, ptrs, ptrs, ptrs, None, ptrs, ctypes.byref(bad), None,
                                             ctypes.c_void_p(4096), 1 << 40, None)
    assert st == 1  # SKI_EINVAL


def test_noalloc_limits_fit_its_fixed_scratch(lib):
    # ski_sketch_hash_noalloc takes rows * s <= 262144 and m <= 32768 into a
    # 4 MiB array: at those limits the bucket-list scratch must fit, for every
    # s it accepts, dense or CSR, with or without b
    pkg = lib
    cap = 4 << 20
    for s in range(1, 65):
        rows = 262144 // s
        dense = pkg.ski_matrix(kind=pkg.SKI_DENSE, n=rows, d=4, ld=4, val=4096)
        csr = pkg.ski_matrix(kind=pkg.SKI_CSR, n=rows, d=4, ld=0, val=4096, rowptr=4096, colidx=4096, nnz=rows)
        for hk in (0, 1):
            o = pkg.ski_opts_default(m=32768, s=s, seed=1, hash_kind=hk)
            for M in (dense, csr):
                for wb in (0, 1):
                    need = pkg.lib().ski_sketch_workspace_size(ctypes.byref(M), wb, ctypes.byref(o))
                    assert 0 < need <= cap, (s, hk, M.kind, wb, need)


def test_hartley_premix_and_sampling_options(lib):
    L = lib.lib()
    A = _fake_dense(lib, 1009, 6)
    ws = lambda **kw: L.ski_sketch_workspace_size(ctypes.byref(A), 1, ctypes.byref(lib.ski_opts_default(m=40, **kw)))
    pm = lambda **kw: L.ski_premix_workspace_size(ctypes.byref(A), 1, ctypes.byref(lib.ski_opts_default(**kw)))
    # F D of Eq. HR-DHT: lengths whose prime factors are <= 13, at least n; 0 = 1014
    assert pm(premix=2) == pm(premix=2, n_pad=1014) > 0
    for bad in (1010, 1013, 1008, 2 * 1009):
        assert pm(premix=2, n_pad=bad) == 0, bad
    # FP64: twiddles (2 x 1014) and four complex planes of 1014 x 8 doubles, at least
    assert pm(premix=2) >= 8 * (2 * 1014 + 4 * 1014 * 8)
    assert ws(premix=2) > 0 and ws(premix=2, n_pad=1010) == 0 and ws(premix=3) == 0
    # the sampling sketch S_s (Eq. SR-DHT): s = 1, with the Hartley premix or none
    assert ws(hash_kind=2) > 0 and ws(hash_kind=2, premix=2) > 0
    assert ws(hash_kind=2, s=2) == 0 and ws(hash_kind=2, premix=1) == 0 and ws(hash_kind=3) == 0
    csr = lib.ski_matrix(kind=lib.SKI_CSR, n=100, d=10, ld=0, val=0x1000, rowptr=0x1000, colidx=0x1000, nnz=5)
    o = lib.ski_opts_default(m=20, hash_kind=2)
    assert L.ski_sketch_workspace_size(ctypes.byref(csr), 1, ctypes.byref(o)) == 0
