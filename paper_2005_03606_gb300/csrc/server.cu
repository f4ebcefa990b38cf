// Serving loop: requests are admitted while the HBM budget and the slot
// count allow, each admitted request runs its delayed-assembly solve on its
// own pair of CUDA streams (so the work of different requests overlaps on the
// device), and results are kept per ticket until polled.
//
// Admission is first-come first-served: the head of the queue waits until its
// footprint estimate fits, later requests do not overtake it.
#include "mg_internal.cuh"
#include "mg.h"

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace mg {
void problem_use_graphs(mg_problem* P, bool on);
}

using namespace mg;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  mg_problem_desc desc{};
  double* dst = nullptr;
  size_t est = 0;
  mg_result res{};
  bool done = false;
  Clock::time_point t_submit, t_admit, t_done;
};

// Upper bound of the device bytes of one problem (vectors of all levels,
// worst-case FP32 surplus records, scratch, coarse storage).
size_t estimate_bytes(const mg_problem_desc& d) {
  const int D = d.dim;
  double nv = 1, nc = 1;
  for (int a = 0; a < D; ++a) {
    nv *= d.n_cells + 1;
    nc *= d.n_cells;
  }
  const bool mixed = d.path == MG_PATH_MIXED_DELAYED || d.path == MG_PATH_MIXED_PLAIN;
  const int NP = D == 3 ? 28 : 6;
  double bytes = nv * 8 * 5;                        // u f r p q
  bytes += nv * (mixed ? 4 : 8) * 3 * 1.05;         // V-cycle vectors, all levels
  bytes += nc * (mixed ? 4 : 8);                    // eps_c
  const double per_cell = mixed ? (D == 3 ? 113.0 : 33.0) : 8.0 * NP;
  bytes += nc * per_cell * 2.0;                     // published + one in-flight accuracy
  if (mixed) bytes += nc * (D == 3 ? 112.0 : 32.0) / 9.0 + nc * 1.1;   // scratch (one chunk) + classes
  bytes += nc / (D == 3 ? 27.0 : 9.0) * NP * (mixed ? 4 : 8) * 1.05;   // coarse levels
  const double ns = D == 3 ? 14.0 : 5.0;                                 // vertex stencils (symmetric)
  bytes += (mixed ? 0.0 : nv * ns * 8) + nv / (D == 3 ? 27.0 : 9.0) * ns * (mixed ? 4 : 8) * 1.05;
  if (mixed && D == 3) bytes += nv * 5 + (nv / 4) * 27 * 4;   // touched list, flags, stencil table
  if (mixed && D == 3) {
    bytes += nv * 4 * 8 + nc * 8 * 1.01;   // FP64 bulk pass in vertex form: vertex and edge weights, scaled eps
    bytes += nc * 12 + nv * 4;             // exact FP64 operator: eps64, list positions, touched vertices
  }
  bytes += 64ull << 20;                             // partials, tables, pool slack
  return (size_t)bytes;
}

}  // namespace

struct mg_server {
  mg_server_desc desc{};
  size_t budget = 0, in_use = 0;
  int active = 0;
  int device = 0;
  uint64_t next_id = 1;
  uint64_t admissions = 0;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> all;
  std::vector<std::thread> workers;
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

void run_request(mg_server* S, Request* R) {
  mg_problem* P = nullptr;
  mg_status st = MG_OK;
  bool injected = false;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->admissions++;
    if (S->desc.inject_fail_every > 0 && S->admissions % (uint64_t)S->desc.inject_fail_every == 0) injected = true;
  }
  if (injected) {
    st = MG_ERR_INJECTED;
  } else {
    st = mg_create_problem(&R->desc, nullptr, &P);
    if (st == MG_OK) problem_use_graphs(P, S->desc.use_graphs != 0);
  }
  mg_solve_info info{};
  if (st == MG_OK) st = mg_solve(P, &info);
  if (st == MG_OK && R->dst) {
    double nv = 1;
    for (int a = 0; a < R->desc.dim; ++a) nv *= R->desc.n_cells + 1;
    st = mg_get_solution(P, R->dst, (size_t)nv);
  }
  if (st != MG_OK && getenv("MG_TRACE"))   // diagnostics: the worker thread's message
    fprintf(stderr, "mg: request %llu failed (status %d): %s\n", (unsigned long long)R->id, (int)st, mg_last_error());
  if (P) mg_destroy_problem(P);
  R->t_done = Clock::now();
  R->res.status = st;
  R->res.cycles = info.cycles;
  R->res.publishes = info.publishes;
  R->res.rel_residual = info.rel_residual;
  R->res.queue_ms = ms_between(R->t_submit, R->t_admit);
  R->res.solve_ms = ms_between(R->t_admit, R->t_done);
  R->res.total_ms = ms_between(R->t_submit, R->t_done);
}

void worker_loop(mg_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    Request* R = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] {
        if (S->stop) return true;
        if (S->queue.empty()) return false;
        Request* h = S->queue.front();
        return S->in_use + h->est <= S->budget || S->active == 0;
      });
      if (S->stop) return;
      R = S->queue.front();
      S->queue.pop_front();
      S->in_use += R->est;
      S->active++;
      R->t_admit = Clock::now();
    }
    run_request(S, R);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->in_use -= R->est;
      S->active--;
      R->done = true;
    }
    S->cv.notify_all();
  }
}

}  // namespace

extern "C" {

mg_status mg_server_create(const mg_server_desc* desc, mg_server** out) {
  if (!out) {
    set_error("null output pointer");
    return MG_ERR_INVALID;
  }
  mg_server* S = new mg_server();
  if (desc) S->desc = *desc;
  if (S->desc.max_active <= 0) S->desc.max_active = 8;
  if (cudaGetDevice(&S->device) != cudaSuccess) S->device = 0;
  if (S->desc.hbm_budget_bytes > 0) {
    S->budget = (size_t)S->desc.hbm_budget_bytes;
  } else {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete S;
      set_error("cudaMemGetInfo failed");
      return MG_ERR_CUDA;
    }
    S->budget = fr > (4ull << 30) ? fr - (4ull << 30) : fr / 2;
  }
  for (int i = 0; i < S->desc.max_active; ++i) S->workers.emplace_back(worker_loop, S);
  *out = S;
  return MG_OK;
}

mg_status mg_submit(mg_server* S, const mg_problem_desc* desc, double* solution_dst, uint64_t* ticket) {
  if (!S || !desc || !ticket) {
    set_error("bad arguments");
    return MG_ERR_INVALID;
  }
  Request* R = new Request();
  R->desc = *desc;
  R->desc.u0 = nullptr;
  R->dst = solution_dst;
  R->est = estimate_bytes(*desc);
  R->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete R;
      set_error("server stopped");
      return MG_ERR_CANCELLED;
    }
    if (R->est > S->budget) {
      delete R;
      set_error("request needs %zu bytes, budget is %zu", estimate_bytes(*desc), S->budget);
      return MG_ERR_OOM;
    }
    R->id = S->next_id++;
    S->all[R->id] = R;
    S->queue.push_back(R);
    *ticket = R->id;
  }
  S->cv.notify_all();
  return MG_OK;
}

mg_status mg_poll(mg_server* S, uint64_t ticket, mg_result* result) {
  if (!S) {
    set_error("null server");
    return MG_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) {
    set_error("unknown ticket");
    return MG_ERR_INVALID;
  }
  if (!it->second->done) return MG_ERR_PENDING;
  if (result) *result = it->second->res;
  return (mg_status)it->second->res.status;
}

mg_status mg_server_drain(mg_server* S, double timeout_ms) {
  if (!S) {
    set_error("null server");
    return MG_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto pred = [&] {
    if (!S->queue.empty() || S->active > 0) return false;
    return true;
  };
  if (timeout_ms <= 0) {
    S->cv.wait(lk, pred);
    return MG_OK;
  }
  if (!S->cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred)) {
    set_error("drain timed out");
    return MG_ERR_TIMEOUT;
  }
  return MG_OK;
}

mg_status mg_server_destroy(mg_server* S) {
  if (!S) return MG_OK;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    for (Request* R : S->queue) {
      R->res.status = MG_ERR_CANCELLED;
      R->done = true;
    }
    S->queue.clear();
    S->cv.wait(lk, [&] { return S->active == 0; });
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->all) delete kv.second;
  delete S;
  return MG_OK;
}

}  // extern "C"
