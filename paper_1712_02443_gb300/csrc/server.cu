// Solve server: a request loop over the public C API (include/macroaim.h).
//
// Requests (an array description, incidences, tolerance) are queued; a request
// is admitted when its estimated device footprint fits in the budget left by
// the requests in flight (FIFO; the first waiting request that fits goes).
// Each admitted request runs on one of the worker threads, each with its own
// context and CUDA stream, so the products and Krylov iterations of requests
// that are in flight at the same time overlap on the device, and a request that
// arrives while others run starts as soon as a worker and memory are free.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <complex>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "macroaim.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t id = 0;
  std::vector<const mm_type*> types;
  std::vector<double> offsets;
  mm_aim_opts aim{};
  int32_t nrhs = 1;
  std::vector<double> th, ph;
  std::vector<int32_t> pol;
  mm_solve_opts opts{};
  size_t est = 0;
  int64_t n = 0;
  // results
  bool done = false;
  mm_status status = MM_OK;
  std::string err;
  std::vector<double> E;   // complex128 interleaved, N^ x nrhs
  mm_solve_stats stats{};
  double t_submit = 0, t_start = 0, t_setup = 0, t_end = 0;
};

}  // namespace

struct mm_server {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  std::deque<Req*> queue;
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t next_id = 1;
  int64_t completed = 0;
};

namespace {

void run_request(int device, mm_ctx* ctx, cudaStream_t st, Req* r) {
  mm_array* arr = nullptr;
  void* V = nullptr;
  void* E = nullptr;
  auto finish = [&](mm_status s, const std::string& msg) {
    r->status = s;
    if (s != MM_OK) r->err = msg.empty() ? std::string(mm_last_error(ctx)) : msg;
  };
  r->t_start = now_s();
  mm_status s = mm_array_create(ctx, (int64_t)r->types.size(), r->types.data(), r->offsets.data(), &r->aim, &arr);
  r->t_setup = now_s();
  if (s != MM_OK) return finish(s, "");
  mm_array_info info{};
  mm_array_info_get(arr, &info);
  r->n = info.n_unknowns;
  const size_t bytes = sizeof(double) * 2 * (size_t)r->n * r->nrhs;
  cudaSetDevice(device);
  if (cudaMallocAsync(&V, bytes, st) != cudaSuccess || cudaMallocAsync(&E, bytes, st) != cudaSuccess) {
    mm_array_destroy(arr);
    if (V) cudaFreeAsync(V, st);
    return finish(MM_ENOMEM, "device allocation for the request failed");
  }
  s = mm_rhs_planewave(arr, r->nrhs, r->th.data(), r->ph.data(), r->pol.data(), V, MM_C128, st);
  if (s == MM_OK) s = mm_solve(arr, r->nrhs, V, E, &r->opts, &r->stats, st);
  if (s == MM_OK || s == MM_ENOCONV) {
    r->E.resize(2 * (size_t)r->n * r->nrhs);
    if (cudaMemcpyAsync(r->E.data(), E, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = MM_ECUDA;
  }
  const mm_status s_final = s;
  const std::string msg = s != MM_OK ? std::string(mm_last_error(ctx)) : std::string();
  cudaFreeAsync(V, st);
  cudaFreeAsync(E, st);
  cudaStreamSynchronize(st);
  mm_array_destroy(arr);
  finish(s_final, msg);
}

void worker_main(mm_server* sv) {
  mm_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  const bool ok = mm_ctx_create(sv->device, &ctx) == MM_OK &&
                  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_work.wait(lk, [&] {
        if (sv->stop) return true;
        for (Req* q : sv->queue)
          if (sv->in_use == 0 || sv->in_use + q->est <= sv->budget) return true;
        return false;
      });
      if (sv->stop && sv->queue.empty()) break;
      for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it)
        if (sv->in_use == 0 || sv->in_use + (*it)->est <= sv->budget) {
          r = *it;
          sv->queue.erase(it);
          break;
        }
      if (!r) continue;
      sv->in_use += r->est;
    }
    if (ok)
      run_request(sv->device, ctx, st, r);
    else {
      r->status = MM_ECUDA;
      r->err = "worker could not create its context or stream";
    }
    r->t_end = now_s();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->in_use -= r->est;
      r->done = true;
      ++sv->completed;
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
  if (st) cudaStreamDestroy(st);
  if (ctx) mm_ctx_destroy(ctx);
}

}  // namespace

extern "C" {

mm_status mm_server_create(int device, int32_t workers, size_t hbm_budget_bytes, mm_server** out) {
  if (!out || workers < 1 || workers > 64 || device < 0) return MM_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device >= n) return MM_ECUDA;
  auto sv = std::make_unique<mm_server>();
  sv->device = device;
  if (hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaSetDevice(device);
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return MM_ECUDA;
    hbm_budget_bytes = fr / 10 * 8;
  }
  sv->budget = hbm_budget_bytes;
  for (int i = 0; i < workers; ++i) sv->workers.emplace_back(worker_main, sv.get());
  *out = sv.release();
  return MM_OK;
}

mm_status mm_server_submit(mm_server* sv, const mm_request* q, uint64_t* ticket) {
  if (!sv || !q || !ticket || q->n_elem < 1 || !q->types || !q->offsets_xyz || q->nrhs < 1 || !q->theta ||
      !q->phi || !q->pol)
    return MM_EINVAL;
  auto r = std::make_unique<Req>();
  int64_t nh = 0, ns = 0;
  for (int64_t e = 0; e < q->n_elem; ++e) {
    if (!q->types[e]) return MM_EINVAL;
    int64_t a = 0, b = 0;
    if (mm_type_info(q->types[e], &a, &b) != MM_OK) return MM_EINVAL;
    ns += a;
    nh += b;
    r->types.push_back(q->types[e]);
  }
  r->offsets.assign(q->offsets_xyz, q->offsets_xyz + 3 * q->n_elem);
  r->aim = q->aim;
  r->nrhs = q->nrhs;
  r->th.assign(q->theta, q->theta + q->nrhs);
  r->ph.assign(q->phi, q->phi + q->nrhs);
  r->pol.assign(q->pol, q->pol + q->nrhs);
  r->opts = q->solve;
  // footprint estimate: Krylov basis and work vectors, grids, the near-field
  // blocks and, when the array assembles it (moderate sizes), the near-field
  // CSR (~650 entries per row, values of both precisions and columns)
  const size_t csr = std::min<size_t>((size_t)nh * 650 * 36, (size_t)8 << 30);
  r->est = csr + (size_t)nh * q->nrhs * 16 * (q->solve.restart + 8) + (size_t)nh * q->nrhs * 256 + (size_t)ns * 64 +
           ((size_t)64 << 20);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->id = sv->next_id++;
    *ticket = r->id;
    sv->queue.push_back(r.get());
    sv->reqs[r->id] = std::move(r);
  }
  sv->cv_work.notify_all();
  return MM_OK;
}

mm_status mm_server_poll(mm_server* sv, uint64_t ticket, int32_t wait, mm_result* res, double* E_host,
                         int64_t E_count) {
  if (!sv || !res) return MM_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return MM_EINVAL;
  Req* r = it->second.get();
  if (wait) sv->cv_done.wait(lk, [&] { return r->done; });
  res->done = r->done ? 1 : 0;
  if (!r->done) return MM_EBUSY;
  res->status = r->status;
  res->stats = r->stats;
  res->n_unknowns = r->n;
  res->queue_s = r->t_start - r->t_submit;
  res->setup_s = r->t_setup - r->t_start;
  res->solve_s = r->t_end - r->t_setup;
  res->latency_s = r->t_end - r->t_submit;
  std::snprintf(res->message, sizeof(res->message), "%s", r->err.c_str());
  if (E_host) {
    if (E_count < 2 * r->n * r->nrhs) return MM_EINVAL;
    std::copy(r->E.begin(), r->E.end(), E_host);
  }
  return MM_OK;
}

mm_status mm_server_release(mm_server* sv, uint64_t ticket) {
  if (!sv) return MM_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end() || !it->second->done) return MM_EINVAL;
  sv->reqs.erase(it);
  return MM_OK;
}

void mm_server_destroy(mm_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->workers) t.join();
  delete sv;
}

}  // extern "C"
