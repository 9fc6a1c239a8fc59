// Solve server: a request loop over the public C API (include/macroaim.h).
//
// Requests (an array description, incidences, tolerance) are queued; a request
// is admitted when its estimated device footprint fits in the budget left by
// the requests in flight (FIFO; the first waiting request that fits goes).
// Each admitted request runs on one of the worker threads, each with its own
// context and CUDA stream, so the products and Krylov iterations of requests
// that are in flight at the same time overlap on the device, and a request that
// arrives while others run starts as soon as a worker and memory are free.
// When a worker takes a request, the waiting requests with the same geometry
// and solve options join it: their incidences become further columns of one
// batched solve (one product and one Arnoldi step per iteration for all of
// them), and each request receives its own columns of the solution.  Green's
// spectra are shared across arrays of equal grid size (the set-up cache), the
// near-field blocks across arrays of the same element types.
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

constexpr int kMaxMergedRhs = 64;   // columns of one merged solve

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
  size_t est = 0;           // device footprint estimate of the request solved alone
  size_t est_per_rhs = 0;   // its part that grows with the number of columns
  int64_t n = 0;
  // results
  bool done = false;
  mm_status status = MM_OK;
  std::string err;
  std::vector<double> E;   // complex128 interleaved, N^ x nrhs
  mm_solve_stats stats{};
  double t_submit = 0, t_start = 0, t_setup = 0, t_end = 0;
  int group_requests = 1, group_columns = 0;   // the solve this request was part of
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
  int64_t merged = 0;   // requests that joined another request's solve
};

namespace {

bool same_geometry(const Req* a, const Req* b) {
  return a->types == b->types && a->offsets == b->offsets && a->aim.h == b->aim.h && a->aim.order == b->aim.order &&
         a->aim.n_nf == b->aim.n_nf && a->aim.near_csr == b->aim.near_csr && a->aim.phase[0] == b->aim.phase[0] &&
         a->aim.phase[1] == b->aim.phase[1] && a->aim.phase[2] == b->aim.phase[2] && a->opts.tol == b->opts.tol &&
         a->opts.restart == b->opts.restart && a->opts.max_iter == b->opts.max_iter &&
         a->opts.precision == b->opts.precision && a->opts.refine == b->opts.refine &&
         a->opts.inner_tol == b->opts.inner_tol && a->opts.orth == b->opts.orth && a->opts.precond == b->opts.precond;
}

// One solve for a group of requests of the same geometry and options: their
// incidences become the columns of one batched solve (every product and
// Arnoldi step covers all of them), and each request receives its columns.
void run_group(int device, mm_ctx* ctx, cudaStream_t st, const std::vector<Req*>& g) {
  mm_array* arr = nullptr;
  void* V = nullptr;
  void* E = nullptr;
  Req* r = g[0];
  int nrhs = 0;
  std::vector<double> th, ph;
  std::vector<int32_t> pol;
  for (Req* q : g) {
    th.insert(th.end(), q->th.begin(), q->th.end());
    ph.insert(ph.end(), q->ph.begin(), q->ph.end());
    pol.insert(pol.end(), q->pol.begin(), q->pol.end());
    nrhs += q->nrhs;
  }
  auto finish = [&](mm_status s, const std::string& msg) {
    for (Req* q : g) {
      q->status = s;
      if (s != MM_OK) q->err = msg.empty() ? std::string(mm_last_error(ctx)) : msg;
    }
  };
  const double t_start = now_s();
  for (Req* q : g) q->t_start = t_start;
  mm_status s = mm_array_create(ctx, (int64_t)r->types.size(), r->types.data(), r->offsets.data(), &r->aim, &arr);
  const double t_setup = now_s();
  for (Req* q : g) q->t_setup = t_setup;
  if (s != MM_OK) return finish(s, "");
  mm_array_info info{};
  mm_array_info_get(arr, &info);
  for (Req* q : g) q->n = info.n_unknowns;
  const int64_t n = info.n_unknowns;
  const size_t bytes = sizeof(double) * 2 * (size_t)n * nrhs;
  cudaSetDevice(device);
  if (cudaMallocAsync(&V, bytes, st) != cudaSuccess || cudaMallocAsync(&E, bytes, st) != cudaSuccess) {
    mm_array_destroy(arr);
    if (V) cudaFreeAsync(V, st);
    return finish(MM_ENOMEM, "device allocation for the request failed");
  }
  mm_solve_stats stats{};
  s = mm_rhs_planewave(arr, nrhs, th.data(), ph.data(), pol.data(), V, MM_C128, st);
  if (s == MM_OK) s = mm_solve(arr, nrhs, V, E, &r->opts, &stats, st);
  std::vector<double> Eall;
  if (s == MM_OK || s == MM_ENOCONV) {
    Eall.resize(2 * (size_t)n * nrhs);
    if (cudaMemcpyAsync(Eall.data(), E, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = MM_ECUDA;
  }
  const mm_status s_final = s;
  const std::string msg = s != MM_OK ? std::string(mm_last_error(ctx)) : std::string();
  cudaFreeAsync(V, st);
  cudaFreeAsync(E, st);
  cudaStreamSynchronize(st);
  mm_array_destroy(arr);
  // each request's columns of E (rows of nrhs interleaved complex entries)
  int c0 = 0;
  for (Req* q : g) {
    q->stats = stats;
    q->group_requests = (int)g.size();
    q->group_columns = nrhs;
    if (!Eall.empty()) {
      q->E.resize(2 * (size_t)n * q->nrhs);
      for (int64_t i = 0; i < n; ++i)
        std::copy(Eall.begin() + 2 * (i * nrhs + c0), Eall.begin() + 2 * (i * nrhs + c0 + q->nrhs),
                  q->E.begin() + 2 * i * q->nrhs);
    }
    c0 += q->nrhs;
  }
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
    // waiting requests of the same geometry and options join this solve as
    // further columns (up to kMaxMergedRhs columns); the merged request's
    // extra columns cost its per-column share of the footprint
    std::vector<Req*> group{r};
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      int cols = r->nrhs;
      for (auto it = sv->queue.begin(); it != sv->queue.end();) {
        Req* q = *it;
        if (cols + q->nrhs <= kMaxMergedRhs && same_geometry(r, q) &&
            sv->in_use + q->est_per_rhs * q->nrhs <= sv->budget) {
          group.push_back(q);
          cols += q->nrhs;
          sv->in_use += q->est_per_rhs * q->nrhs;
          it = sv->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    if (ok)
      run_group(sv->device, ctx, st, group);
    else
      for (Req* q : group) {
        q->status = MM_ECUDA;
        q->err = "worker could not create its context or stream";
      }
    const double t_end = now_s();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->in_use -= r->est;
      for (size_t i = 1; i < group.size(); ++i) sv->in_use -= group[i]->est_per_rhs * group[i]->nrhs;
      for (Req* q : group) {
        q->t_end = t_end;
        q->done = true;
        ++sv->completed;
      }
      sv->merged += (int64_t)group.size() - 1;
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
  r->est_per_rhs = (size_t)nh * 16 * (q->solve.restart + 8) + (size_t)nh * 256;
  r->est = (q->aim.near_csr == 2 ? 0 : csr) + r->est_per_rhs * q->nrhs + (size_t)ns * 64 + ((size_t)64 << 20);
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
  res->group_requests = r->group_requests;
  res->group_columns = r->group_columns;
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
