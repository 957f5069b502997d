"""Row-block sharding of the hot path over processes, one GPU each.

A is split by rows: process k holds rows [r_k, r_k + n_k) of A and b.  The
s-hashing matrix S of Def. 5 draws each column from its global row index, so
every process sketches its own rows with its own columns of S -- nothing of S
is exchanged -- and

    S A = sum over row blocks k of S[:, rows_k] A[rows_k, :]

is one all-reduce of the m x (d + 1) partial sketches.  Steps 2-3 then run on
every process on the same sketch.  Each LSQR iteration needs the sum of
A_k^T t_k (d values) and ||t_k||^2; the residual passes sum A_k^T r_k,
||r_k||^2 and ||A_k||_F^2.  The library does all of this in
``ski_solve_rowblock`` and calls back for each sum; this module supplies the
sum through ``torch.distributed`` (NCCL between GPUs, gloo on the host).

The premix H D mixes every row of A, so it does not shard by rows; the
row-block form takes S = S_h alone.
"""
import ctypes
import copy

import numpy as np

from . import (SKI_BF16, SKI_F32, SKI_F64, dense_matrix, ski_opts_default, ski_sketch_hash,
               ski_sketch_workspace_size, ski_solve_rowblock)

_NP = {SKI_F64: np.float64, SKI_F32: np.float32}


def row_blocks(n, world):
    """(start, count) of each process's rows: n split as evenly as possible,
    the first n % world processes taking one row more."""
    base, extra = divmod(int(n), int(world))
    out, start = [], 0
    for k in range(int(world)):
        cnt = base + (1 if k < extra else 0)
        out.append((start, cnt))
        start += cnt
    return out


def _tensor_at(ptr, count, dtype, device):
    """A torch tensor over `count` elements of ski_dtype `dtype` at address
    `ptr` (device memory of the current CUDA device, or host memory)."""
    import torch
    if device == "cpu":
        if dtype not in _NP:
            raise ValueError("host buffers: FP64 or FP32 only")
        buf = (ctypes.c_char * (int(count) * np.dtype(_NP[dtype]).itemsize)).from_address(int(ptr))
        return torch.from_numpy(np.frombuffer(buf, dtype=_NP[dtype], count=int(count)))

    class _Cuda:
        pass

    typestr = {SKI_F64: "<f8", SKI_F32: "<f4", SKI_BF16: "<V2"}[dtype]
    obj = _Cuda()
    obj.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                    "version": 3, "strides": None}
    t = torch.as_tensor(obj, device="cuda")
    if dtype == SKI_BF16:
        t = t.view(torch.bfloat16)
    return t


class TorchAllreduce:
    """The library's all-reduce callback through torch.distributed: the sum,
    in place, over the processes of `group`, enqueued on the library's CUDA
    stream (NCCL), or on host memory with device="cpu" (gloo)."""

    def __init__(self, group=None, device="cuda"):
        self.group = group
        self.device = device

    def __call__(self, ptr, count, dtype, stream):
        import torch
        import torch.distributed as dist
        t = _tensor_at(ptr, count, dtype, self.device)
        if not dist.is_initialized() or dist.get_world_size(self.group) == 1:
            return
        if self.device == "cpu":
            dist.all_reduce(t, group=self.group)
            return
        with torch.cuda.stream(torch.cuda.ExternalStream(int(stream) if stream else 0)):
            dist.all_reduce(t, group=self.group)


def sketch_rowblock(A_local, b_local, row_offset, opts, SA_out, allreduce=None, stream=None):
    """[S A | S b] of the whole row-sharded A on every process: this
    process's partial sketch (its rows, its columns of S) summed over the
    processes.  A_local: ski_matrix of the local rows; b_local: device tensor
    or None; SA_out: device tensor m x (d + 1) (m x d without b) of the sketch
    dtype, overwritten."""
    import torch
    o = copy.copy(opts)
    o.row_offset = int(row_offset)
    if o.premix:
        raise ValueError("the premix mixes every row of A: it does not shard by rows")
    ld = SA_out.stride(0)
    ws = torch.empty(max(1, ski_sketch_workspace_size(A_local, 1 if b_local is not None else 0, o)),
                     dtype=torch.uint8, device=SA_out.device)
    ski_sketch_hash(A_local, b_local, o, SA_out, ld, ws=ws, stream=stream)
    st = torch.cuda.current_stream() if stream is None else stream
    (allreduce or TorchAllreduce())(SA_out.data_ptr(), SA_out.shape[0] * ld, o.sketch_dtype, st.cuda_stream)
    return SA_out


def solve_rowblock(A_local, b_local, row_offset, opts, x, allreduce=None, R_out=None, ws=None, stream=None,
                   check=True):
    """Algorithm 1 on the row-sharded A (see the module docstring); x (device
    FP64 [d]) receives the whole solution on every process.  Returns the
    ski_info record, the same on every process."""
    o = copy.copy(opts)
    o.row_offset = int(row_offset)
    return ski_solve_rowblock(A_local, b_local, o, x, allreduce or TorchAllreduce(), R_out=R_out, ws=ws,
                              stream=stream, check=check)


def local_block(A, b, rank, world):
    """This process's rows of a dense device matrix A and vector b:
    (ski_matrix, b view, row offset)."""
    start, cnt = row_blocks(A.shape[0], world)[rank]
    Ab = A[start:start + cnt]
    return dense_matrix(Ab), b[start:start + cnt], start


__all__ = ["row_blocks", "TorchAllreduce", "sketch_rowblock", "solve_rowblock", "local_block",
           "ski_opts_default"]
