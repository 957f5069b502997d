"""GB300-native Ski-LLS hot path (Cartis, Fiala & Shao, arXiv 2105.11815).

Thin Python binding of the C ABI in ``include/skills.h``: each function here
has the name of the C entry point it calls and only marshals arguments
(torch tensors -> device pointers, the current CUDA stream, the workspace).
Every step of the method runs in the CUDA library ``_lib/libskills.so``;
there is no CPU fallback: calling into the library without it raises.

The library is built by ``paper_2105_11815_gb300.build.build()`` (nvcc,
sm_103a) and loaded lazily on first use.
"""
import ctypes
import os

__all__ = [
    "SKI_F64", "SKI_F32", "SKI_BF16", "SKI_DENSE", "SKI_CSR", "SKI_S_HASHING", "SKI_S_HASHING_VARIANT", "SKI_SAMPLING", "SkiError",
    "ski_opts", "ski_info", "ski_matrix", "lib", "lib_path",
    "ski_opts_default", "ski_status_string", "ski_version", "ski_last_cuda_error", "ski_launch_count",
    "ski_selftest_wait_timeout", "ski_mixed_lsqr_budget",
    "ski_hash_indices", "ski_hash_variant_indices", "ski_premix_signs", "ski_premix_workspace_size", "ski_premix",
    "ski_sketch_workspace_size", "ski_sketch_hash", "ski_sketch_hash_noalloc",
    "ski_precondition_workspace_size", "ski_precondition",
    "ski_gemm_tc_f32", "ski_trinv_workspace_size", "ski_trinv",
    "ski_solve_workspace_size", "ski_solve",
    "ski_solve_batched_workspace_size", "ski_solve_batched",
    "ski_solve_adjoint_workspace_size", "ski_solve_adjoint",
    "ski_solve_adjoint_batched_workspace_size", "ski_solve_adjoint_batched",
    "dense_matrix", "csr_matrix",
]

SKI_F64, SKI_F32, SKI_BF16, SKI_TF32 = 0, 1, 2, 3
SKI_DENSE, SKI_CSR = 0, 1
SKI_S_HASHING, SKI_S_HASHING_VARIANT, SKI_SAMPLING = 0, 1, 2
STATUS = ["SKI_OK", "SKI_EINVAL", "SKI_ENOMEM", "SKI_ECUDA", "SKI_ENONFINITE",
          "SKI_ESINGULAR", "SKI_ENOCONV", "SKI_ETIMEOUT"]

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "_lib", "libskills.so")


class SkiError(RuntimeError):
    def __init__(self, status, where):
        self.status = int(status)
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{where}: {name}")


class ski_matrix(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("n", ctypes.c_int64), ("d", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("val", ctypes.c_void_p), ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p),
                ("nnz", ctypes.c_int64)]


class ski_opts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("s", ctypes.c_int32), ("premix", ctypes.c_int32),
                ("m", ctypes.c_int64), ("n_pad", ctypes.c_int64),
                ("sketch_dtype", ctypes.c_int32), ("qr_dtype", ctypes.c_int32),
                ("tau_a", ctypes.c_double), ("tau_r", ctypes.c_double), ("tol", ctypes.c_double),
                ("rcond", ctypes.c_double), ("perturb", ctypes.c_double), ("it_max", ctypes.c_int64),
                ("streams", ctypes.c_int32), ("premix_slab", ctypes.c_int32),
                ("lsqr_pass", ctypes.c_int32), ("lsqr_ctas", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("hash_kind", ctypes.c_int32), ("factorization", ctypes.c_int32), ("batch_lsqr", ctypes.c_int32),
                ("row_offset", ctypes.c_int64)]


class ski_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("restarts", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("early_exit", ctypes.c_int32), ("status", ctypes.c_int32),
                ("metric", ctypes.c_double), ("resid_norm", ctypes.c_double),
                ("anorm_f", ctypes.c_double), ("lsqr_test", ctypes.c_double),
                ("ms_sketch", ctypes.c_float), ("ms_qr", ctypes.c_float), ("ms_trinv", ctypes.c_float),
                ("ms_lsqr", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("ms_premix", ctypes.c_float), ("ms_gather", ctypes.c_float), ("ms_qr_gemm", ctypes.c_float),
                ("qr_fallback", ctypes.c_int32), ("inv_dtype", ctypes.c_int32), ("rdiag_ratio", ctypes.c_double),
                ("pivoted", ctypes.c_int32), ("gram", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# ski_allreduce_fn: (buf, count, dtype, ctx, stream) -> ski_status
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_void_p)


_lib = None
_P, _I32, _I64, _U64, _SZ, _D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_size_t, ctypes.c_double)
_MP, _OP, _IP = ctypes.POINTER(ski_matrix), ctypes.POINTER(ski_opts), ctypes.POINTER(ski_info)

_SIGS = {
    "ski_opts_default": (None, [_OP]),
    "ski_status_string": (ctypes.c_char_p, [_I32]),
    "ski_version": (_I32, []),
    "ski_last_cuda_error": (_I32, []),
    "ski_launch_count": (_I64, []),
    "ski_mixed_lsqr_budget": (_I64, [_I64, _I64, _D]),
    "ski_selftest_wait_timeout": (_I32, [_I64, _P, _SZ, _P]),
    "ski_hash_indices": (_I32, [_U64, _I32, _I64, _I64, _P, _P, _P]),
    "ski_hash_variant_indices": (_I32, [_U64, _I32, _I64, _I64, _P, _P, _P]),
    "ski_premix_signs": (_I32, [_U64, _I64, _P, _P]),
    "ski_premix_workspace_size": (_SZ, [_MP, _I32, _OP]),
    "ski_premix": (_I32, [_MP, _P, _OP, _P, _I64, _P, _SZ, _P]),
    "ski_sketch_workspace_size": (_SZ, [_MP, _I32, _OP]),
    "ski_sketch_hash": (_I32, [_MP, _P, _OP, _P, _I64, _P, _SZ, _P]),
    "ski_sketch_hash_noalloc": (_I32, [_MP, _P, _OP, _P, _I64, _P]),
    "ski_precondition_workspace_size": (_SZ, [_I64, _I64, _I32, _I32]),
    "ski_precondition": (_I32, [_I64, _I64, _I32, _P, _I64, _I32, _P, _I64, _P, _P, _OP, _P, _SZ, _P]),
    "ski_gemm_tc_f32": (_I32, [_I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _I32, _I32, _P, _SZ, _P]),
    "ski_trinv_workspace_size": (_SZ, [_I64, _I32]),
    "ski_trinv": (_I32, [_I64, _P, _I64, _P, _P, _I64, _I32, _D, _P, _SZ, _P]),
    "ski_solve_workspace_size": (_SZ, [_MP, _OP]),
    "ski_solve": (_I32, [_MP, _P, _OP, _P, _P, _IP, _P, _SZ, _P]),
    "ski_solve_rowblock": (_I32, [_MP, _P, _OP, _P, _P, _IP, _P, _SZ, _P, ALLREDUCE_FN, _P]),
    "ski_solve_batched_workspace_size": (_SZ, [_I32, _MP, _OP]),
    "ski_solve_batched": (_I32, [_I32, _MP, _P, _OP, _P, _P, _IP, _P, _SZ, _P]),
    "ski_solve_adjoint_workspace_size": (_SZ, [_MP, _OP]),
    "ski_solve_adjoint": (_I32, [_MP, _P, _P, _P, _I64, _P, _P, _I64, _P, _OP, _IP, _P, _SZ, _P]),
    "ski_solve_adjoint_batched_workspace_size": (_SZ, [_I32, _MP, _OP]),
    "ski_solve_adjoint_batched": (_I32, [_I32, _MP, _P, _P, _P, _P, _P, _P, _OP, _IP, _P, _SZ, _P]),
}


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(lib_path):
            raise RuntimeError(
                "CUDA library %s is missing: build it with "
                "paper_2105_11815_gb300.build.build() (there is no CPU fallback)" % lib_path)
        h = ctypes.CDLL(lib_path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def _check(st, where):
    if st != 0:
        raise SkiError(st, where)
    return st


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ws(nbytes, device, ws):
    import torch
    if ws is not None:
        if ws.numel() * ws.element_size() < nbytes:
            raise ValueError("workspace smaller than the size query (%d bytes)" % nbytes)
        return ws
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------- marshalling
def dense_matrix(A):
    """ski_matrix for a row-major FP64 CUDA tensor A (n x d, unit column stride)."""
    import torch
    if A.dtype != torch.float64 or not A.is_cuda or A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a 2-D float64 CUDA tensor with unit column stride")
    m = ski_matrix(kind=SKI_DENSE, n=A.shape[0], d=A.shape[1], ld=A.stride(0), val=A.data_ptr(),
                   rowptr=None, colidx=None, nnz=0)
    m._keep = (A,)  # the device memory must outlive the descriptor
    return m


def csr_matrix(rowptr, colidx, val, n, d):
    """ski_matrix for CSR CUDA tensors (int64 rowptr, int32 colidx, float64 val)."""
    import torch
    if rowptr.dtype != torch.int64 or colidx.dtype != torch.int32 or val.dtype != torch.float64:
        raise ValueError("CSR arrays must be int64 rowptr, int32 colidx, float64 val")
    m = ski_matrix(kind=SKI_CSR, n=n, d=d, ld=0, val=val.data_ptr(), rowptr=rowptr.data_ptr(),
                   colidx=colidx.data_ptr(), nnz=val.numel())
    m._keep = (rowptr, colidx, val)
    return m


def ski_opts_default(**kw):
    """ski_opts with the library defaults, then the given fields overridden."""
    o = ski_opts()
    lib().ski_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def ski_status_string(status):
    return lib().ski_status_string(int(status)).decode()


def ski_version():
    return lib().ski_version()


def ski_last_cuda_error():
    return lib().ski_last_cuda_error()


def ski_launch_count():
    return lib().ski_launch_count()


def ski_mixed_lsqr_budget(m, d, tau_r):
    return lib().ski_mixed_lsqr_budget(m, d, tau_r)


def ski_selftest_wait_timeout(spin_limit, ws=None, stream=None):
    """Returns the status of the bounded-wait self-test (SKI_ETIMEOUT = 7 expected)."""
    import torch
    w = ws if ws is not None else torch.zeros(16, dtype=torch.uint8, device="cuda")
    return lib().ski_selftest_wait_timeout(int(spin_limit), _ptr(w), 16, _stream(stream))


# ---------------------------------------------------------------- entry points
def ski_hash_indices(seed, s, m, n, idx, sign, stream=None):
    return _check(lib().ski_hash_indices(seed, s, m, n, _ptr(idx), _ptr(sign), _stream(stream)), "ski_hash_indices")


def ski_hash_variant_indices(seed, s, m, n, idx, sign, stream=None):
    return _check(lib().ski_hash_variant_indices(seed, s, m, n, _ptr(idx), _ptr(sign), _stream(stream)),
                  "ski_hash_variant_indices")


def ski_premix_signs(seed, n, D, stream=None):
    return _check(lib().ski_premix_signs(seed, n, _ptr(D), _stream(stream)), "ski_premix_signs")


def ski_premix_workspace_size(A, with_b, opts):
    return lib().ski_premix_workspace_size(ctypes.byref(A), int(with_b), ctypes.byref(opts))


def ski_premix(A, b, opts, Y, ld_y, ws=None, stream=None):
    nb = ski_premix_workspace_size(A, b is not None, opts)
    w = _ws(nb, Y.device, ws)
    return _check(lib().ski_premix(ctypes.byref(A), _ptr(b), ctypes.byref(opts), _ptr(Y), ld_y, _ptr(w), nb,
                                   _stream(stream)), "ski_premix")


def ski_sketch_workspace_size(A, with_b, opts):
    return lib().ski_sketch_workspace_size(ctypes.byref(A), int(with_b), ctypes.byref(opts))


def ski_sketch_hash(A, b, opts, SA, ld_sa, ws=None, stream=None):
    nb = ski_sketch_workspace_size(A, b is not None, opts)
    w = _ws(nb, SA.device, ws)
    return _check(lib().ski_sketch_hash(ctypes.byref(A), _ptr(b), ctypes.byref(opts), _ptr(SA), ld_sa, _ptr(w), nb,
                                        _stream(stream)), "ski_sketch_hash")


def ski_sketch_hash_noalloc(A, b, opts, SA, ld_sa, stream=None):
    """ski_sketch_hash with the library's own fixed scratch (no workspace)."""
    return _check(lib().ski_sketch_hash_noalloc(ctypes.byref(A), _ptr(b), ctypes.byref(opts), _ptr(SA), ld_sa,
                                                _stream(stream)), "ski_sketch_hash_noalloc")


def ski_precondition_workspace_size(m, d, with_rhs, sa_dtype):
    return lib().ski_precondition_workspace_size(m, d, int(with_rhs), sa_dtype)


def ski_precondition(m, d, with_rhs, SA, ld_sa, sa_dtype, R, ldr, qtsb=None, want_rank=True, opts=None,
                     ws=None, stream=None):
    """Returns the numerical rank (when want_rank) else None."""
    nb = ski_precondition_workspace_size(m, d, with_rhs, sa_dtype)
    w = _ws(nb, SA.device, ws)
    rank = ctypes.c_int32(-1)
    o = opts if opts is not None else ski_opts_default()
    _check(lib().ski_precondition(m, d, int(with_rhs), _ptr(SA), ld_sa, sa_dtype, _ptr(R), ldr, _ptr(qtsb),
                                  ctypes.byref(rank) if want_rank else None, ctypes.byref(o), _ptr(w), nb,
                                  _stream(stream)), "ski_precondition")
    return rank.value if want_rank else None


def ski_gemm_tc_f32(M, N, K, A, lda, B, ldb, C, ldc, subtract=False, passes=1, ws=None, stream=None):
    """C = A B^T (or C -= A B^T) on the TF32 tensor cores (1 or 3 passes)."""
    import torch
    w = ws if ws is not None else torch.zeros(16, dtype=torch.uint8, device=C.device)
    return _check(lib().ski_gemm_tc_f32(M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, int(subtract),
                                        int(passes), _ptr(w), 16, _stream(stream)), "ski_gemm_tc_f32")


def ski_trinv_workspace_size(d, dtype):
    return lib().ski_trinv_workspace_size(d, dtype)


def ski_trinv(d, R, ldr, M, Mt, ldm, dtype=SKI_F64, perturb=0.0, ws=None, stream=None):
    nb = ski_trinv_workspace_size(d, dtype)
    w = _ws(nb, R.device, ws)
    return _check(lib().ski_trinv(d, _ptr(R), ldr, _ptr(M), _ptr(Mt), ldm, dtype, perturb, _ptr(w), nb,
                                  _stream(stream)), "ski_trinv")


def ski_solve_workspace_size(A, opts):
    return lib().ski_solve_workspace_size(ctypes.byref(A), ctypes.byref(opts))


def ski_solve(A, b, opts, x, R_out=None, ws=None, stream=None, check=True):
    """Algorithm 1 end to end; returns the ski_info record."""
    nb = ski_solve_workspace_size(A, opts)
    if nb == 0:
        raise SkiError(1, "ski_solve_workspace_size")
    w = _ws(nb, x.device, ws)
    info = ski_info()
    st = lib().ski_solve(ctypes.byref(A), _ptr(b), ctypes.byref(opts), _ptr(x), _ptr(R_out), ctypes.byref(info),
                         _ptr(w), nb, _stream(stream))
    if check:
        _check(st, "ski_solve")
    return info


def ski_solve_rowblock(A, b, opts, x, allreduce, R_out=None, ws=None, stream=None, check=True):
    """Algorithm 1 on this process's row block of A (opts.row_offset: the
    global index of its first row).  allreduce(ptr, count, dtype, stream_ptr)
    sums `count` elements of ski_dtype `dtype` at device address `ptr` over the
    processes, in place and in the order of the CUDA stream `stream_ptr`.
    Returns the ski_info record."""
    nb = ski_solve_workspace_size(A, opts)
    if nb == 0:
        raise SkiError(1, "ski_solve_workspace_size")
    w = _ws(nb, x.device, ws)
    info = ski_info()
    failed = []

    def _cb(buf, count, dtype, ctx, st):
        try:
            allreduce(buf, count, dtype, st)
            return 0
        except Exception as e:  # the status ends the solve; the exception is re-raised below
            failed.append(e)
            return STATUS.index("SKI_ECUDA")

    cb = ALLREDUCE_FN(_cb)
    st = lib().ski_solve_rowblock(ctypes.byref(A), _ptr(b), ctypes.byref(opts), _ptr(x), _ptr(R_out),
                                  ctypes.byref(info), _ptr(w), nb, _stream(stream), cb, None)
    if failed:
        raise failed[0]
    if check:
        _check(st, "ski_solve_rowblock")
    return info


def ski_solve_batched_workspace_size(mats, opts):
    arr = (ski_matrix * len(mats))(*mats)
    return lib().ski_solve_batched_workspace_size(len(mats), arr, ctypes.byref(opts))


def ski_solve_batched(mats, bs, opts, xs, R_outs=None, ws=None, stream=None, check=True):
    """nprob independent solves; returns the list of ski_info records."""
    k = len(mats)
    arr = (ski_matrix * k)(*mats)
    nb = lib().ski_solve_batched_workspace_size(k, arr, ctypes.byref(opts))
    w = _ws(nb, xs[0].device, ws)
    bp = (ctypes.c_void_p * k)(*[b.data_ptr() for b in bs])
    xp = (ctypes.c_void_p * k)(*[x.data_ptr() for x in xs])
    rp = (ctypes.c_void_p * k)(*[r.data_ptr() for r in R_outs]) if R_outs is not None else None
    infos = (ski_info * k)()
    st = lib().ski_solve_batched(k, arr, bp, ctypes.byref(opts), xp, rp, infos, _ptr(w), nb, _stream(stream))
    if check:
        _check(st, "ski_solve_batched")
    return list(infos)


def _ptr_array(ts):
    if ts is None:
        return None
    return (ctypes.c_void_p * len(ts))(*[(t.data_ptr() if t is not None else None) for t in ts])


def ski_solve_adjoint_batched_workspace_size(mats, opts):
    arr = (ski_matrix * len(mats))(*mats)
    return lib().ski_solve_adjoint_batched_workspace_size(len(mats), arr, ctypes.byref(opts))


def ski_solve_adjoint_batched(mats, bs, xs, Rs, gs, dAs, dbs, opts, ws=None, stream=None, check=True):
    """nprob independent adjoint solves (R[i] d_i x d_i, dA[i] n_i x d_i, both
    contiguous); dAs may be None. Returns the list of ski_info records."""
    k = len(mats)
    arr = (ski_matrix * k)(*mats)
    nb = lib().ski_solve_adjoint_batched_workspace_size(k, arr, ctypes.byref(opts))
    w = _ws(nb, xs[0].device, ws)
    infos = (ski_info * k)()
    st = lib().ski_solve_adjoint_batched(k, arr, _ptr_array(bs), _ptr_array(xs), _ptr_array(Rs), _ptr_array(gs),
                                         _ptr_array(dAs), _ptr_array(dbs), ctypes.byref(opts), infos, _ptr(w), nb,
                                         _stream(stream))
    if check:
        _check(st, "ski_solve_adjoint_batched")
    return list(infos)


def ski_solve_adjoint_workspace_size(A, opts):
    return lib().ski_solve_adjoint_workspace_size(ctypes.byref(A), ctypes.byref(opts))


def ski_solve_adjoint(A, b, x, R, ldr, g, dA, ld_da, db, opts, ws=None, stream=None, check=True):
    nb = ski_solve_adjoint_workspace_size(A, opts)
    w = _ws(nb, x.device, ws)
    info = ski_info()
    st = lib().ski_solve_adjoint(ctypes.byref(A), _ptr(b), _ptr(x), _ptr(R), ldr, _ptr(g), _ptr(dA), ld_da,
                                 _ptr(db), ctypes.byref(opts), ctypes.byref(info), _ptr(w), nb, _stream(stream))
    if check:
        _check(st, "ski_solve_adjoint")
    return info
