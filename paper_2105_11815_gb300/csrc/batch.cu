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
// that bounds the idle tail by the cost of one problem).
//
// Step 4 of the dense problems can be grouped (ski_opts.batch_lsqr = 1): a
// problem's LSQR pass alone fills every SM with one 512-thread CTA each, so
// the passes of problems on different streams cannot overlap, and a small
// problem's iteration is bound by launch and barrier latency.  Instead, a
// worker whose problem reaches Step 4 hands it to one executor thread and
// waits; the executor runs every iteration of all problems in flight as one
// launch per kernel over a list of (problem, block) work items, polls all
// their scalars with one copy every chunk of iterations, and releases each
// problem when its own loop would have stopped.  Problems join and leave the
// group between chunks while the other workers' sketches and QRs proceed on
// their streams.  Each problem's results depend only on its own kernels' row
// blocks, not on the group it ran in.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "lsqr_impl.cuh"

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

size_t slice_round(size_t b) { return (b + 255) & ~(size_t)255; }

// ---- grouped Step 4
int64_t group_items(const ski_matrix* A, const ski_opts* oi) {
  const int64_t d = A->d;
  return (int64_t)ski_lsqr_ctas(A->n, oi) + std::max<int64_t>(1, ski_cdiv(d, 32)) + ski_vv_blocks(d);
}
bool grouped_mode(const ski_opts* o) { return o->batch_lsqr == 1; }

// Device area of the executor: jobs [W], work items, scalars [W].
struct GroupArea {
  size_t jobs_off, items_off, sc_off, bytes;
  int64_t cap_items;
};
GroupArea group_area(int W, int64_t cap_items) {
  GroupArea g{};
  g.cap_items = cap_items;
  g.jobs_off = 0;
  g.items_off = slice_round(sizeof(LsqrGroupJob) * (size_t)W);
  g.sc_off = g.items_off + slice_round(sizeof(LsqrGroupItem) * (size_t)cap_items);
  g.bytes = g.sc_off + slice_round(sizeof(LsqrScalars) * (size_t)W);
  return g;
}

class GroupExec final : public LsqrGroupHook {
 public:
  GroupExec(int W, char* area, const GroupArea& g)
      : workers_(W), cap_jobs_(W), cap_items_(g.cap_items),
        djobs_((LsqrGroupJob*)(area + g.jobs_off)), ditems_((LsqrGroupItem*)(area + g.items_off)),
        dsc_((LsqrScalars*)(area + g.sc_off)) {}

  ski_status run(LsqrGroupTask& t) override {
    Entry e;
    e.task = &t;
    if (cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming) != cudaSuccess) return SKI_ECUDA;
    if (cudaEventRecord(e.ready, t.st) != cudaSuccess) {
      cudaEventDestroy(e.ready);
      return SKI_ECUDA;
    }
    {
      std::unique_lock<std::mutex> lk(mu_);
      if (failed_ != SKI_OK) {
        e.status = failed_;
        e.done = true;
      } else {
        pending_.push_back(&e);
        cv_exec_.notify_one();
        cv_done_.wait(lk, [&] { return e.done; });
      }
    }
    cudaEventDestroy(e.ready);  // the executor's stream waited on it before e.done
    return e.status;
  }

  // a worker has no problem left
  void worker_left() {
    std::lock_guard<std::mutex> lk(mu_);
    --workers_;
    cv_exec_.notify_one();
  }

  // the executor thread
  void loop() {
    if (cudaSetDevice(dev_) != cudaSuccess) fail_all(SKI_ECUDA);
    std::vector<Entry*> active, fresh;
    bool dirty = false;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_exec_.wait(lk, [&] { return !pending_.empty() || !active.empty() || workers_ <= 0; });
        if (pending_.empty() && active.empty() && workers_ <= 0) break;
        fresh.swap(pending_);
      }
      ski_status s = SKI_OK;
      for (Entry* e : fresh) {
        if (cudaStreamWaitEvent(st_, e->ready, 0) != cudaSuccess) s = SKI_ECUDA;
        active.push_back(e);
        dirty = true;
      }
      fresh.clear();
      if (s == SKI_OK && dirty) {
        s = layout(active);
        dirty = false;
      }
      const int chunk = active.empty() ? 0 : active[0]->task->chunk;
      for (int k = 0; k < chunk && s == SKI_OK; ++k) s = iterate();
      const int nj = (int)active.size();
      hsc_.resize(nj);
      if (s == SKI_OK) s = ski_group_scalars_launch(djobs_, nj, dsc_, st_);
      if (s == SKI_OK && nj > 0 &&
          cudaMemcpyAsync(hsc_.data(), dsc_, sizeof(LsqrScalars) * (size_t)nj, cudaMemcpyDeviceToHost, st_) !=
              cudaSuccess)
        s = SKI_ECUDA;
      if (s == SKI_OK && cudaStreamSynchronize(st_) != cudaSuccess) s = SKI_ECUDA;
      std::lock_guard<std::mutex> lk(mu_);
      if (s != SKI_OK) {
        if (s == SKI_ECUDA) ski_note_cuda_error(cudaGetLastError());
        failed_ = s;
        for (Entry* e : active) {
          e->status = s;
          e->done = true;
        }
        active.clear();
        cv_done_.notify_all();
        continue;
      }
      size_t keep = 0;
      bool released = false;
      for (int j = 0; j < nj; ++j) {
        Entry* e = active[j];
        LsqrGroupTask& t = *e->task;
        const LsqrScalars& h = hsc_[j];
        e->polled += t.chunk;
        const bool stop = h.flag_a || e->polled > t.it_max + t.chunk ||
                          (t.budgeted && ski_weak_preconditioner(h.test, h.iters, t.tau_r, t.budget));
        if (stop) {
          t.hs = h;
          e->status = SKI_OK;
          e->done = true;
          released = true;
        } else {
          active[keep++] = e;
        }
      }
      active.resize(keep);
      if (released) {
        dirty = true;
        cv_done_.notify_all();
      }
    }
  }

  void set_device(int dev) { dev_ = dev; }
  void set_stream(cudaStream_t st) { st_ = st; }

 private:
  struct Entry {
    LsqrGroupTask* task = nullptr;
    cudaEvent_t ready = nullptr;
    int64_t polled = 0;
    bool done = false;
    ski_status status = SKI_OK;
  };

  void fail_all(ski_status s) {
    std::lock_guard<std::mutex> lk(mu_);
    failed_ = s;
  }

  // Work items of the problems in flight: K2 blocks by template class, then
  // K3 column blocks, then the K4 / K1 row blocks.
  ski_status layout(const std::vector<Entry*>& active) {
    const int nj = (int)active.size();
    if (nj > cap_jobs_) return SKI_EINVAL;
    hjobs_.resize(nj);
    items_.clear();
    for (int j = 0; j < nj; ++j) hjobs_[j] = active[j]->task->job;
    for (int c = 0; c < kDfGroupClasses; ++c) {
      cls_begin_[c] = (int)items_.size();
      cls_smem_[c] = 0;
      for (int j = 0; j < nj; ++j) {
        const LsqrGroupTask& t = *active[j]->task;
        if (t.cls != c) continue;
        cls_smem_[c] = std::max(cls_smem_[c], t.smem);
        for (int b = 0; b < t.job.df.nblk; ++b) items_.push_back({j, b});
      }
    }
    cls_begin_[kDfGroupClasses] = (int)items_.size();
    red_begin_ = (int)items_.size();
    for (int j = 0; j < nj; ++j) {
      const int64_t nb = std::max<int64_t>(1, ski_cdiv(hjobs_[j].d, 32));
      for (int64_t b = 0; b < nb; ++b) items_.push_back({j, (int32_t)b});
    }
    trmv_begin_ = (int)items_.size();
    for (int j = 0; j < nj; ++j)
      for (int b = 0; b < hjobs_[j].nvv; ++b) items_.push_back({j, b});
    if ((int64_t)items_.size() > cap_items_) return SKI_EINVAL;
    if (nj > 0) {
      SKI_CUDA_TRY(cudaMemcpyAsync(djobs_, hjobs_.data(), sizeof(LsqrGroupJob) * (size_t)nj, cudaMemcpyHostToDevice,
                                   st_));
      SKI_CUDA_TRY(cudaMemcpyAsync(ditems_, items_.data(), sizeof(LsqrGroupItem) * items_.size(),
                                   cudaMemcpyHostToDevice, st_));
    }
    return SKI_OK;
  }

  // one LSQR iteration of every problem in flight
  ski_status iterate() {
    for (int c = 0; c < kDfGroupClasses; ++c)
      SKI_TRY(ski_group_df_launch(c, djobs_, ditems_ + cls_begin_[c], cls_begin_[c + 1] - cls_begin_[c],
                                  cls_smem_[c], st_));
    SKI_TRY(ski_group_reduce_launch(djobs_, ditems_ + red_begin_, trmv_begin_ - red_begin_, st_));
    SKI_TRY(ski_group_trmv_launch(djobs_, ditems_ + trmv_begin_, (int)items_.size() - trmv_begin_, st_));
    return SKI_OK;
  }

  std::mutex mu_;
  std::condition_variable cv_exec_, cv_done_;
  std::vector<Entry*> pending_;
  int workers_;
  ski_status failed_ = SKI_OK;
  int dev_ = 0;
  const int cap_jobs_;
  const int64_t cap_items_;
  cudaStream_t st_ = nullptr;
  LsqrGroupJob* djobs_;
  LsqrGroupItem* ditems_;
  LsqrScalars* dsc_;
  std::vector<LsqrGroupJob> hjobs_;
  std::vector<LsqrGroupItem> items_;
  std::vector<LsqrScalars> hsc_;
  int cls_begin_[kDfGroupClasses + 1] = {};
  size_t cls_smem_[kDfGroupClasses] = {};
  int red_begin_ = 0, trmv_begin_ = 0;
};

// Runs solve_one(i, slice, slice_bytes, stream) for every problem on W workers.
// Work on the worker streams is ordered after the work already queued on the
// caller's stream, and the caller's stream is ordered after all of it.
// Returns the status of the lowest-numbered problem that failed.
// gx (W > 1 only): the grouped Step 4 executor, run on its own thread and
// stream for as long as any worker is.
template <class F>
ski_status run_pool(int32_t nprob, int W, const std::vector<int32_t>& order, char* ws, size_t slice,
                    cudaStream_t caller, F&& solve_one, GroupExec* gx = nullptr) {
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
    cudaStream_t gst = nullptr;
    std::thread gth;
    if (gx) {
      if (cudaStreamCreateWithFlags(&gst, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamWaitEvent(gst, start, 0) != cudaSuccess) {
        if (gst) cudaStreamDestroy(gst);
        cudaEventDestroy(start);
        return SKI_ECUDA;
      }
      gx->set_stream(gst);
      gx->set_device(dev);
      try {
        gth = std::thread([gx] { gx->loop(); });
      } catch (...) {
        cudaStreamDestroy(gst);
        cudaEventDestroy(start);
        return SKI_ENOMEM;
      }
    }
    struct Leave {  // every worker leaves the executor's count once, however it ends
      GroupExec* g;
      ~Leave() {
        if (g) g->worker_left();
      }
    };
    auto worker = [&](int w) {
      Leave leave{gx};
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
        // fewer threads: the remaining workers take their problems
        if (gx)
          for (int u = w; u < W - 1; ++u) gx->worker_left();
        break;
      }
    }
    worker(W - 1);
    for (auto& t : th) t.join();
    cudaEventDestroy(start);
    bool ecuda = abort.load();
    if (gx) {
      gth.join();
      cudaEvent_t gdone = nullptr;
      if (cudaEventCreateWithFlags(&gdone, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventRecord(gdone, gst) != cudaSuccess || cudaStreamWaitEvent(caller, gdone, 0) != cudaSuccess)
        ecuda = true;
      if (gdone) cudaEventDestroy(gdone);
      cudaStreamDestroy(gst);
    }
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


}  // namespace

namespace {
// Workspace of ski_solve_batched: W slices of the largest problem's need,
// then (grouped Step 4) the executor's area.
struct BatchLayout {
  int W = 0;
  size_t slice = 0, total = 0;
  bool grouped = false;
  GroupArea g{};
};
bool batch_layout(int32_t nprob, const ski_matrix* A, const ski_opts* o, BatchLayout* L) {
  size_t mx = 0;
  int64_t items = 0;
  bool dense = false;
  for (int32_t i = 0; i < nprob; ++i) {
    ski_opts oi;
    batched_opts(o, &A[i], i, &oi);
    const size_t b = ski_solve_workspace_size(&A[i], &oi);
    if (b == 0) return false;
    mx = std::max(mx, b);
    if (A[i].kind == SKI_DENSE) {
      dense = true;
      items = std::max(items, group_items(&A[i], &oi));
    }
  }
  L->W = stream_count(nprob, o);
  L->slice = slice_round(mx);
  L->total = L->slice * (size_t)L->W;
  L->grouped = grouped_mode(o) && dense && L->W > 1;
  if (L->grouped) {
    L->g = group_area(L->W, items * L->W);
    L->total += L->g.bytes;
  }
  return true;
}
}  // namespace

extern "C" size_t ski_solve_batched_workspace_size(int32_t nprob, const ski_matrix* A, const ski_opts* o) {
  if (nprob < 0 || (nprob > 0 && (!A || !o))) return 0;
  if (nprob == 0) return 0;
  BatchLayout L;
  return batch_layout(nprob, A, o, &L) ? L.total : 0;
}

extern "C" ski_status ski_solve_batched(int32_t nprob, const ski_matrix* A, const double* const* b, const ski_opts* o,
                                        double* const* x, double* const* R_out, ski_info* info, void* ws,
                                        size_t ws_bytes, void* stream) {
  if (nprob < 0 || (nprob > 0 && (!A || !b || !x || !o))) return SKI_EINVAL;
  if (o && (o->streams < 0)) return SKI_EINVAL;
  if (nprob == 0) return SKI_OK;
  if (o->batch_lsqr != 0 && o->batch_lsqr != 1) return SKI_EINVAL;
  BatchLayout L;
  if (!batch_layout(nprob, A, o, &L)) return SKI_EINVAL;
  if (!ws || ws_bytes < L.total) return SKI_ENOMEM;
  std::vector<ski_opts> oi(nprob);
  std::vector<int64_t> m(nprob);
  for (int32_t i = 0; i < nprob; ++i) {
    batched_opts(o, &A[i], i, &oi[i]);
    m[i] = oi[i].m;
  }
  const std::vector<int32_t> order = lpt_order(nprob, A, m);
  if (L.grouped) {
    GroupExec gx(L.W, (char*)ws + L.slice * (size_t)L.W, L.g);
    return run_pool(
        nprob, L.W, order, (char*)ws, L.slice, ski_stream(stream),
        [&](int32_t i, char* w, size_t wb, cudaStream_t s) -> ski_status {
          return ski_solve_grouped(&A[i], b[i], &oi[i], x[i], R_out ? R_out[i] : nullptr, info ? &info[i] : nullptr,
                                   w, wb, (void*)s, &gx);
        },
        &gx);
  }
  return run_pool(nprob, L.W, order, (char*)ws, L.slice, ski_stream(stream),
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
