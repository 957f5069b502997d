// Batched entry points: many independent least-squares problems (ragged
// n_i x d_i), each solved by the single-problem path of Algorithm 1 (or its
// adjoint), several at a time.
//
// A problem's control flow has host decisions that depend on device results
// (the rank rule after Step 2, the LSQR convergence poll of Step 4, the
// restarts of the acceptance test), so one problem is one sequence of launches
// on one stream.  Throughput comes from running W such sequences at once: W
// host workers, each owning a non-blocking stream and one workspace slice,
// pull problems from a shared counter in longest-first order (a list schedule
// that bounds the idle tail by the cost of one problem).  The kernels a problem
// runs, and so its results, are the same whichever worker solves it.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kMaxStreams = 32;
constexpr int kAutoStreams = 8;

void batched_opts(const ski_opts* o, const ski_matrix* A, int32_t i, ski_opts* oi) {
  *oi = *o;
  if (o->m <= 0) {
    const double gamma = (o->m < 0 ? -(double)o->m : 2000.0) / 1000.0;
    oi->m = (int64_t)ceil(gamma * (double)A->d);
    if (oi->m < A->d) oi->m = A->d;
  }
  oi->seed = o->seed + (uint64_t)i;
}

// Problems in flight.  o->streams > 0 fixes it; 0 picks min(nprob, 8): with
// the fused LSQR pass filling the GPU at about one CTA per SM, eight streams
// keep every SM busy while the latency-bound pieces of the others (QR panels,
// trmv, the host poll) are in flight.
int stream_count(int32_t nprob, const ski_opts* o) {
  int w = o->streams > 0 ? o->streams : kAutoStreams;
  w = std::min(w, kMaxStreams);
  w = (int)std::min<int64_t>(w, nprob);
  return std::max(w, 1);
}

// Longest-first order by a cost model of one solve: the LSQR passes read
// n d values each (tens of passes), the QR of the m x (d+1) sketch costs
// 2 m d^2 flops on the FP64 pipe.
std::vector<int32_t> lpt_order(int32_t nprob, const ski_matrix* A, const std::vector<int64_t>& m) {
  std::vector<double> cost(nprob);
  for (int32_t i = 0; i < nprob; ++i) {
    const double n = (double)A[i].n, d = (double)A[i].d;
    const double nnz = A[i].kind == SKI_DENSE ? n * d : (double)A[i].nnz;
    cost[i] = 57.0 * nnz + (double)m[i] * d * d;
  }
  std::vector<int32_t> ord(nprob);
  for (int32_t i = 0; i < nprob; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  return ord;
}

// Runs solve_one(i, slice, slice_bytes, stream) for every problem on W workers.
// Work on the worker streams is ordered after the work already queued on the
// caller's stream, and the caller's stream is ordered after all of it.
// Returns the status of the lowest-numbered problem that failed.
template <class F>
ski_status run_pool(int32_t nprob, int W, const std::vector<int32_t>& order, char* ws, size_t slice,
                    cudaStream_t caller, F&& solve_one) {
  std::vector<int32_t> status(nprob, SKI_OK);
  if (W <= 1) {
    for (int32_t k = 0; k < nprob; ++k) {
      const int32_t i = order[k];
      status[i] = solve_one(i, ws, slice, caller);
      if (status[i] == SKI_ECUDA) break;
    }
  } else {
    int dev = 0;
    SKI_CUDA_TRY(cudaGetDevice(&dev));
    cudaEvent_t start;
    SKI_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    if (cudaEventRecord(start, caller) != cudaSuccess) {
      cudaEventDestroy(start);
      return SKI_ECUDA;
    }
    std::atomic<int32_t> next{0};
    std::atomic<bool> abort{false};
    std::vector<int32_t> cuda_err(W, 0);
    std::vector<cudaEvent_t> done(W, nullptr);
    auto worker = [&](int w) {
      if (cudaSetDevice(dev) != cudaSuccess) {
        abort = true;
        cuda_err[w] = ski_last_cuda_error();
        return;
      }
      cudaStream_t s = nullptr;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamWaitEvent(s, start, 0) != cudaSuccess) {
        if (s) cudaStreamDestroy(s);
        abort = true;
        return;
      }
      char* mine = ws + (size_t)w * slice;
      for (;;) {
        if (abort.load()) break;
        const int32_t k = next.fetch_add(1);
        if (k >= nprob) break;
        const int32_t i = order[k];
        status[i] = solve_one(i, mine, slice, s);
        if (status[i] == SKI_ECUDA) {
          cuda_err[w] = ski_last_cuda_error();
          abort = true;
        }
      }
      if (cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventRecord(done[w], s) != cudaSuccess)
        abort = true;
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    };
    std::vector<std::thread> th;
    th.reserve(W - 1);
    for (int w = 0; w < W - 1; ++w) {
      try {
        th.emplace_back(worker, w);
      } catch (...) {
        break;  // fewer threads: the remaining workers take their problems
      }
    }
    worker(W - 1);
    for (auto& t : th) t.join();
    cudaEventDestroy(start);
    bool ecuda = abort.load();
    for (int w = 0; w < W; ++w) {
      if (done[w]) {
        if (cudaStreamWaitEvent(caller, done[w], 0) != cudaSuccess) ecuda = true;
        cudaEventDestroy(done[w]);
      }
      if (cuda_err[w]) ski_note_cuda_error((cudaError_t)cuda_err[w]);
    }
    if (ecuda) {
      for (int32_t i = 0; i < nprob; ++i)
        if (status[i] != SKI_OK) return (ski_status)status[i];
      return SKI_ECUDA;
    }
  }
  for (int32_t i = 0; i < nprob; ++i)
    if (status[i] != SKI_OK) return (ski_status)status[i];
  return SKI_OK;
}

size_t slice_round(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" size_t ski_solve_batched_workspace_size(int32_t nprob, const ski_matrix* A, const ski_opts* o) {
  if (nprob < 0 || (nprob > 0 && (!A || !o))) return 0;
  if (nprob == 0) return 0;
  size_t mx = 0;
  for (int32_t i = 0; i < nprob; ++i) {
    ski_opts oi;
    batched_opts(o, &A[i], i, &oi);
    const size_t b = ski_solve_workspace_size(&A[i], &oi);
    if (b == 0) return 0;
    mx = std::max(mx, b);
  }
  return slice_round(mx) * (size_t)stream_count(nprob, o);
}

extern "C" ski_status ski_solve_batched(int32_t nprob, const ski_matrix* A, const double* const* b, const ski_opts* o,
                                        double* const* x, double* const* R_out, ski_info* info, void* ws,
                                        size_t ws_bytes, void* stream) {
  if (nprob < 0 || (nprob > 0 && (!A || !b || !x || !o))) return SKI_EINVAL;
  if (o && (o->streams < 0)) return SKI_EINVAL;
  if (nprob == 0) return SKI_OK;
  const size_t need = ski_solve_batched_workspace_size(nprob, A, o);
  if (need == 0) return SKI_EINVAL;
  if (!ws || ws_bytes < need) return SKI_ENOMEM;
  const int W = stream_count(nprob, o);
  const size_t slice = need / (size_t)W;
  std::vector<ski_opts> oi(nprob);
  std::vector<int64_t> m(nprob);
  for (int32_t i = 0; i < nprob; ++i) {
    batched_opts(o, &A[i], i, &oi[i]);
    m[i] = oi[i].m;
  }
  const std::vector<int32_t> order = lpt_order(nprob, A, m);
  return run_pool(nprob, W, order, (char*)ws, slice, ski_stream(stream),
                  [&](int32_t i, char* w, size_t wb, cudaStream_t s) -> ski_status {
                    return ski_solve(&A[i], b[i], &oi[i], x[i], R_out ? R_out[i] : nullptr, info ? &info[i] : nullptr,
                                     w, wb, (void*)s);
                  });
}

extern "C" size_t ski_solve_adjoint_batched_workspace_size(int32_t nprob, const ski_matrix* A, const ski_opts* o) {
  if (nprob <= 0 || !A || !o) return 0;
  size_t mx = 0;
  for (int32_t i = 0; i < nprob; ++i) {
    const size_t b = ski_solve_adjoint_workspace_size(&A[i], o);
    if (b == 0) return 0;
    mx = std::max(mx, b);
  }
  return slice_round(mx) * (size_t)stream_count(nprob, o);
}

extern "C" ski_status ski_solve_adjoint_batched(int32_t nprob, const ski_matrix* A, const double* const* b,
                                                const double* const* x, const double* const* R, const double* const* g,
                                                double* const* dA, double* const* db, const ski_opts* o,
                                                ski_info* info, void* ws, size_t ws_bytes, void* stream) {
  if (nprob < 0 || (nprob > 0 && (!A || !b || !x || !R || !g || !db || !o))) return SKI_EINVAL;
  if (o && (o->streams < 0)) return SKI_EINVAL;
  if (nprob == 0) return SKI_OK;
  const size_t need = ski_solve_adjoint_batched_workspace_size(nprob, A, o);
  if (need == 0) return SKI_EINVAL;
  if (!ws || ws_bytes < need) return SKI_ENOMEM;
  const int W = stream_count(nprob, o);
  const size_t slice = need / (size_t)W;
  std::vector<int64_t> m(nprob, 0);
  const std::vector<int32_t> order = lpt_order(nprob, A, m);
  return run_pool(nprob, W, order, (char*)ws, slice, ski_stream(stream),
                  [&](int32_t i, char* w, size_t wb, cudaStream_t s) -> ski_status {
                    return ski_solve_adjoint(&A[i], b[i], x[i], R[i], A[i].d, g[i], dA ? dA[i] : nullptr, A[i].d,
                                             db[i], o, info ? &info[i] : nullptr, w, wb, (void*)s);
                  });
}
