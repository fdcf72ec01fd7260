// Batched solves and the serving loop.  Both run BKS solves of independent
// jobs on several CUDA streams at once, one host worker thread per stream,
// so that the many small, latency-bound kernels of different jobs overlap
// on the GPU.  The server adds a FIFO queue with admission by predicted
// device memory (continuous batching: a job joins as soon as a slot and its
// memory are free) and keeps every running job's state on the device.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace bks {

int solve_impl(const bks_tensor* t, const bks_params* prm, const double* U0, const double* W0,
               double* U, double* W, double* F, bks_info* info, cudaStream_t stream,
               const std::atomic<int>* cancel);
int autotune_tensor(bks_tensor* t, cudaStream_t s, int* tile, int* split);
int set_tiles(bks_tensor* t, int tile, int split, cudaStream_t s);

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int size_class(int64_t nnz) {
  int c = 0;
  while ((int64_t(1) << (c + 1)) <= std::max<int64_t>(nnz, 1)) ++c;
  return c;
}

// Work-tile choices per size class, shared by the workers of one batch or
// server.  The first job of a class is tuned; later ones reuse its choice.
struct TileCache {
  std::mutex mu;
  std::map<int, std::pair<int, int>> best;
  int apply(bks_tensor* t, cudaStream_t s) {
    const int c = size_class(t->nnz);
    {
      std::lock_guard<std::mutex> lock(mu);
      auto it = best.find(c);
      if (it != best.end()) return set_tiles(t, it->second.first, it->second.second, s);
    }
    int tile = 0, split = 0;
    BKS_TRY(autotune_tensor(t, s, &tile, &split));
    std::lock_guard<std::mutex> lock(mu);
    best[c] = {tile, split};
    return BKS_OK;
  }
};

}  // namespace
}  // namespace bks

using namespace bks;

// ---------------------------------------------------------------------------
extern "C" int bks_batch_solve(int njobs, bks_tensor* const* T, const bks_params* P,
                               const double* const* U0, const double* const* W0,
                               double* const* U, double* const* W, double* const* F,
                               bks_info* info, int* status, int nstreams, int flags,
                               void* stream) {
  if (njobs < 0 || (njobs > 0 && (!T || !P || !U || !W || !F)))
    return fail(BKS_EINVAL, "batch: null arrays");
  if (njobs == 0) return BKS_OK;
  for (int q = 0; q < njobs; ++q) BKS_TRY(require_symmetric(T[q]));
  nstreams = std::max(1, std::min(nstreams, njobs));
  int dev = 0;
  BKS_CUDA_TRY(cudaGetDevice(&dev));
  // the jobs start after the work the caller queued on `stream` (their
  // inputs may still be in flight there)
  cudaEvent_t ready = nullptr;
  BKS_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  const cudaError_t rec = cudaEventRecord(ready, (cudaStream_t)stream);
  if (rec != cudaSuccess) {
    cudaEventDestroy(ready);
    return fail(BKS_ECUDA, std::string("batch: ") + cudaGetErrorString(rec));
  }
  std::vector<int> rc(njobs, BKS_OK);
  std::atomic<int> next{0};
  TileCache cache;
  std::vector<cudaEvent_t> done(nstreams);
  std::vector<std::string> errs(njobs);
  auto worker = [&](int w) {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(st, ready, 0) != cudaSuccess) {
      if (st) cudaStreamDestroy(st);
      for (int q; (q = next.fetch_add(1)) < njobs;) rc[q] = fail(BKS_ECUDA, "batch: stream");
      return;
    }
    for (int q; (q = next.fetch_add(1)) < njobs;) {
      int r = BKS_OK;
      if (flags & BKS_BATCH_AUTOTUNE) r = cache.apply(T[q], st);
      if (r == BKS_OK)
        r = solve_impl(T[q], &P[q], U0 ? U0[q] : nullptr, W0 ? W0[q] : nullptr, U[q], W[q], F[q],
                       info ? &info[q] : nullptr, st, nullptr);
      rc[q] = r;
      if (r != BKS_OK) errs[q] = bks_last_error_string();
    }
    cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming);
    cudaEventRecord(done[w], st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> th;
  for (int w = 0; w < nstreams; ++w) th.emplace_back(worker, w);
  for (auto& x : th) x.join();
  cudaEventDestroy(ready);
  for (int w = 0; w < nstreams; ++w) {
    if (done[w]) {
      cudaStreamWaitEvent((cudaStream_t)stream, done[w], 0);
      cudaEventDestroy(done[w]);
    }
  }
  int first = BKS_OK;
  for (int q = 0; q < njobs; ++q) {
    if (status) status[q] = rc[q];
    if (rc[q] != BKS_OK && first == BKS_OK) {
      first = rc[q];
      set_error("batch job " + std::to_string(q) + ": " + errs[q]);
    }
  }
  return first;
}

// ---------------------------------------------------------------------------
namespace bks {
namespace {

struct Job {
  uint64_t ticket = 0;
  int64_t m = 0, n = 0, nnz = 0;
  std::vector<int32_t> i, j, k;
  std::vector<unsigned char> v;
  int vdtype = BKS_F64, coo_flags = 0;
  bks_params prm{};
  size_t pred = 0;
  std::atomic<int> cancel{0};
  bool running = false, done = false;
  int status = BKS_EPENDING;
  std::string err;
  std::vector<double> U, W, F;
  bks_info info{};
  double t_submit = 0, t_done = 0;
};

size_t predicted_bytes(int64_t m, int64_t n, int64_t nnz) {
  return (size_t)96 * (size_t)nnz + (size_t)8 * (size_t)(m + n) * 168 + ((size_t)64 << 20);
}

}  // namespace
}  // namespace bks

struct bks_server {
  size_t budget = 0;
  int max_slots = 1;
  int flags = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<bks::Job>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<bks::Job>> jobs;
  size_t resident = 0;
  int running = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::vector<std::thread> workers;
  bks::TileCache tiles;

  void run_job(bks::Job& J, cudaStream_t st) {
    bks_tensor* T = nullptr;
    int rc = bks_tensor_create_coo(J.m, J.n, J.nnz, J.i.data(), J.j.data(), J.k.data(),
                                   J.v.data(), J.vdtype, J.coo_flags, st, &T);
    double *U = nullptr, *W = nullptr, *F = nullptr;
    const size_t nu = (size_t)J.m * J.prm.r1, nw = (size_t)J.n * J.prm.r3,
                 nf = (size_t)J.prm.r1 * J.prm.r1 * J.prm.r3;
    if (rc == BKS_OK && (flags & BKS_SERVE_AUTOTUNE)) rc = tiles.apply(T, st);
    if (rc == BKS_OK) {
      if (cudaMallocAsync(&U, sizeof(double) * nu, st) != cudaSuccess ||
          cudaMallocAsync(&W, sizeof(double) * nw, st) != cudaSuccess ||
          cudaMallocAsync(&F, sizeof(double) * nf, st) != cudaSuccess)
        rc = bks::fail(BKS_ENOMEM, "server: result buffers");
    }
    if (rc == BKS_OK) {
      rc = bks::solve_impl(T, &J.prm, nullptr, nullptr, U, W, F, &J.info, st, &J.cancel);
      if (rc == BKS_OK || rc == BKS_ENOTCONV) {
        J.U.resize(nu);
        J.W.resize(nw);
        J.F.resize(nf);
        cudaMemcpyAsync(J.U.data(), U, sizeof(double) * nu, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(J.W.data(), W, sizeof(double) * nw, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(J.F.data(), F, sizeof(double) * nf, cudaMemcpyDeviceToHost, st);
      }
    }
    if (rc != BKS_OK) J.err = bks_last_error_string();
    if (U) cudaFreeAsync(U, st);
    if (W) cudaFreeAsync(W, st);
    if (F) cudaFreeAsync(F, st);
    cudaStreamSynchronize(st);
    if (T) bks_tensor_destroy(T);
    J.status = rc;
  }

  void worker_loop() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
      std::shared_ptr<bks::Job> J;
      {
        std::unique_lock<std::mutex> lock(mu);
        cv_work.wait(lock, [&] {
          return stop || (!queue.empty() && resident + queue.front()->pred <= budget);
        });
        if (stop) break;
        J = queue.front();
        queue.pop_front();
        resident += J->pred;
        ++running;
        J->running = true;
      }
      run_job(*J, st);
      {
        std::lock_guard<std::mutex> lock(mu);
        resident -= J->pred;
        --running;
        J->running = false;
        J->done = true;
        J->t_done = bks::now_s();
      }
      cv_work.notify_all();
      cv_done.notify_all();
    }
    cudaStreamDestroy(st);
  }
};

extern "C" bks_server* bks_server_create(size_t hbm_budget, int max_slots, int flags) {
  if (max_slots < 1 || hbm_budget == 0) {
    fail(BKS_EINVAL, "server: need max_slots >= 1 and a budget");
    return nullptr;
  }
  auto* S = new bks_server();
  S->budget = hbm_budget;
  S->max_slots = max_slots;
  S->flags = flags;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    fail(BKS_ECUDA, "server: no device");
    delete S;
    return nullptr;
  }
  for (int w = 0; w < max_slots; ++w) S->workers.emplace_back([S] { S->worker_loop(); });
  return S;
}

extern "C" int bks_server_submit(bks_server* S, int64_t m, int64_t n, int64_t nnz,
                                 const int32_t* i, const int32_t* j, const int32_t* k,
                                 const void* v, int vdtype, int coo_flags, const bks_params* prm,
                                 uint64_t* ticket) {
  if (!S || !prm || !ticket) return fail(BKS_EINVAL, "server: null argument");
  if (m < 1 || n < 1 || nnz < 0 || (nnz > 0 && (!i || !j || !k || !v)))
    return fail(BKS_EINVAL, "server: bad tensor arguments");
  if (vdtype != BKS_F32 && vdtype != BKS_F64) return fail(BKS_EINVAL, "server: bad vdtype");
  if (coo_flags & BKS_INPUT_ON_DEVICE)
    return fail(BKS_EINVAL, "server: submissions take host arrays");
  if (prm->r1 < 1 || prm->r3 < 1 || prm->r1 > m || prm->r3 > n)
    return fail(BKS_EINVAL, "server: bad ranks");
  auto J = std::make_shared<bks::Job>();
  J->m = m;
  J->n = n;
  J->nnz = nnz;
  J->pred = bks::predicted_bytes(m, n, nnz);
  if (J->pred > S->budget) return fail(BKS_EBUDGET, "server: job exceeds the device-memory budget");
  J->i.assign(i, i + nnz);
  J->j.assign(j, j + nnz);
  J->k.assign(k, k + nnz);
  const size_t vs = vdtype == BKS_F64 ? 8 : 4;
  J->v.resize(vs * nnz);
  if (nnz) std::memcpy(J->v.data(), v, vs * nnz);
  J->vdtype = vdtype;
  J->coo_flags = coo_flags;
  J->prm = *prm;
  J->t_submit = bks::now_s();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    J->ticket = S->next_ticket++;
    S->jobs[J->ticket] = J;
    S->queue.push_back(J);
    *ticket = J->ticket;
  }
  S->cv_work.notify_all();
  return BKS_OK;
}

extern "C" int bks_server_poll(bks_server* S, uint64_t ticket, int wait, double* U, double* W,
                               double* F, bks_info* info, int* job_status, double* latency_s) {
  if (!S) return fail(BKS_EINVAL, "server: null");
  std::shared_ptr<bks::Job> J;
  {
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return fail(BKS_EINVAL, "server: unknown ticket");
    J = it->second;
    if (!J->done) {
      if (!wait) return BKS_EPENDING;
      S->cv_done.wait(lock, [&] { return J->done; });
    }
    S->jobs.erase(ticket);
  }
  if (job_status) *job_status = J->status;
  if (latency_s) *latency_s = J->t_done - J->t_submit;
  if (info) {
    double* h = info->history;
    int cap = info->history_cap;
    *info = J->info;
    info->history = h;
    info->history_cap = cap;
    info->history_len = 0;
  }
  if (!J->U.empty()) {
    if (U) std::memcpy(U, J->U.data(), sizeof(double) * J->U.size());
    if (W) std::memcpy(W, J->W.data(), sizeof(double) * J->W.size());
    if (F) std::memcpy(F, J->F.data(), sizeof(double) * J->F.size());
  }
  if (J->status != BKS_OK) set_error(J->err);
  return BKS_OK;
}

extern "C" int bks_server_cancel(bks_server* S, uint64_t ticket) {
  if (!S) return fail(BKS_EINVAL, "server: null");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return fail(BKS_EINVAL, "server: unknown ticket");
  auto J = it->second;
  if (J->done) return BKS_OK;
  J->cancel.store(1);
  if (!J->running) {
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
      if ((*q)->ticket == ticket) {
        S->queue.erase(q);
        break;
      }
    J->status = BKS_ECANCELED;
    J->err = "cancelled before it started";
    J->done = true;
    J->t_done = bks::now_s();
    S->cv_done.notify_all();
  }
  return BKS_OK;
}

extern "C" int bks_server_stats(bks_server* S, int* queued, int* running, int* finished,
                                size_t* resident_bytes) {
  if (!S) return fail(BKS_EINVAL, "server: null");
  std::lock_guard<std::mutex> lock(S->mu);
  if (queued) *queued = (int)S->queue.size();
  if (running) *running = S->running;
  if (finished) {
    int f = 0;
    for (auto& kv : S->jobs) f += kv.second->done ? 1 : 0;
    *finished = f;
  }
  if (resident_bytes) *resident_bytes = S->resident;
  return BKS_OK;
}

extern "C" void bks_server_destroy(bks_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    for (auto& kv : S->jobs) kv.second->cancel.store(1);
    for (auto& J : S->queue) {
      J->status = BKS_ECANCELED;
      J->err = "server destroyed before the job started";
      J->done = true;
    }
    S->queue.clear();
    S->stop = true;
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  for (auto& w : S->workers) w.join();
  delete S;
}
