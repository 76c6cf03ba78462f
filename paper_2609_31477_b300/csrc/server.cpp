// Serving loop for parameter sweeps of cylinder cases: continuous admission
// by predicted device memory, concurrent cases on their own streams, per-step
// latency accounting.
//
// A scheduler thread moves requests whose arrival time has come into a FIFO
// queue and admits them while the sum of predicted device bytes stays within
// the budget and a slot is free.  Each admitted case runs in a worker thread
// on its own CUDA stream, so the kernels of different cases overlap on the
// GPU; when it finishes, its memory is released and the next request is
// admitted.  A failing case records its status and does not affect others.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "viv_internal.h"

extern "C" vivStatus viv_internal_case_create(vivMesh* mesh, const vivParams* prm, const double* u0, void* s,
                                             vivCase** out);

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  int64_t id;
  vivRequest r;
  std::vector<double> u0;
  size_t bytes;
};

struct Done {
  vivResult res;
  std::vector<double> state;   // u(Dn) p(n) x(Dn) lam(Dn) delta(2)
  int dim = 2;
};

}  // namespace

struct vivServer {
  size_t budget = 0, used = 0, peak_used = 0;
  int max_active = 1, active = 0, peak_active = 0;
  int device = 0;
  int64_t next_id = 1;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::vector<Req> incoming;        // not yet arrived
  std::deque<Req> pending;          // arrived, waiting for admission
  std::vector<std::thread> workers;
  std::map<int64_t, Done> finished;
  std::deque<int64_t> unpolled;
  std::vector<double> step_ms;
  std::vector<double> steady_ms;    // without each case's first two (graph-capturing) steps
  int64_t steps_total = 0, cases_done = 0;
  bool stop = false;
  std::thread sched;
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void run_case(vivServer* S, Req q, double admit_s) {
  Done d{};
  vivResult& R = d.res;
  R.id = q.id;
  R.submit_s = q.r.arrival_time;
  R.admit_s = admit_s;
  R.status = VIV_OK;
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  vivCase* c = nullptr;
  std::vector<double> lat;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    R.status = VIV_ERR_CUDA;
  } else {
    R.status = viv_internal_case_create(q.r.mesh, &q.r.params, q.u0.data(), st, &c);
  }
  for (int s = 0; R.status == VIV_OK && s < q.r.n_steps; ++s) {
    vivStepInfo info{};
    auto a = Clock::now();
    R.status = viv_step(c, &info);
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - a).count();
    if (R.status != VIV_OK) break;
    lat.push_back(ms);
    R.steps_done = s + 1;
    R.t = info.t;
    R.newton_total += info.newton_iters;
    std::memcpy(R.delta, info.delta, sizeof R.delta);
    std::memcpy(R.force, info.force, sizeof R.force);
  }
  if (R.status != VIV_OK) {
    std::strncpy(R.message, viv_last_error(), sizeof R.message - 1);
  }
  if (c) {
    const int64_t n = q.r.mesh->m.n_nodes, D = q.r.mesh->m.dim;
    d.dim = (int)D;
    d.state.assign(3 * D * n + n + 2, 0.0);
    double* b = d.state.data();
    if (viv_get_state(c, 0, b, b + D * n, b + D * n + n, b + 2 * D * n + n, b + 3 * D * n + n, nullptr) != VIV_OK &&
        R.status == VIV_OK)
      R.status = VIV_ERR_CUDA;
    viv_case_destroy(c);
  }
  if (st) cudaStreamDestroy(st);
  R.finish_s = S->now();
  if (!lat.empty()) {
    double sum = 0, mx = 0;
    for (double v : lat) {
      sum += v;
      mx = std::max(mx, v);
    }
    R.step_ms_mean = sum / lat.size();
    R.step_ms_max = mx;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->used -= q.bytes;
  S->active -= 1;
  S->step_ms.insert(S->step_ms.end(), lat.begin(), lat.end());
  if (lat.size() > 2) S->steady_ms.insert(S->steady_ms.end(), lat.begin() + 2, lat.end());
  S->steps_total += (int64_t)lat.size();
  S->cases_done += 1;
  S->finished[q.id] = std::move(d);
  S->unpolled.push_back(q.id);
  S->cv_sched.notify_all();
  S->cv_done.notify_all();
}

void scheduler(vivServer* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    const double t = S->now();
    double next_arrival = 1e300;
    // arrivals, in arrival order
    std::sort(S->incoming.begin(), S->incoming.end(),
              [](const Req& a, const Req& b) { return a.r.arrival_time < b.r.arrival_time; });
    size_t k = 0;
    while (k < S->incoming.size() && S->incoming[k].r.arrival_time <= t) {
      S->pending.push_back(std::move(S->incoming[k]));
      ++k;
    }
    S->incoming.erase(S->incoming.begin(), S->incoming.begin() + k);
    if (!S->incoming.empty()) next_arrival = S->incoming.front().r.arrival_time;
    // admission: FIFO while memory and slots allow
    while (!S->pending.empty() && S->active < S->max_active && S->used + S->pending.front().bytes <= S->budget) {
      Req q = std::move(S->pending.front());
      S->pending.pop_front();
      S->used += q.bytes;
      S->active += 1;
      S->peak_used = std::max(S->peak_used, S->used);
      S->peak_active = std::max(S->peak_active, S->active);
      S->workers.emplace_back(run_case, S, std::move(q), t);
    }
    if (S->stop && S->incoming.empty() && S->pending.empty()) break;
    if (next_arrival < 1e300)
      S->cv_sched.wait_for(lk, std::chrono::duration<double>(std::max(0.0, next_arrival - S->now())));
    else
      S->cv_sched.wait(lk);
  }
}

}  // namespace

extern "C" {

vivStatus viv_server_create(size_t mem_budget, int32_t max_active, vivServer** out) {
  if (!out || mem_budget == 0 || max_active <= 0) {
    viv::set_error("viv_server_create: bad arguments");
    return VIV_ERR_ARG;
  }
  vivServer* S = new vivServer();
  S->budget = mem_budget;
  S->max_active = max_active;
  cudaGetDevice(&S->device);
  S->t0 = Clock::now();
  S->sched = std::thread(scheduler, S);
  *out = S;
  return VIV_OK;
}

vivStatus viv_server_submit(vivServer* S, const vivRequest* r, int64_t* id) {
  if (!S || !r || !r->mesh || !r->u0 || r->n_steps < 0) {
    viv::set_error("viv_server_submit: bad arguments");
    return VIV_ERR_ARG;
  }
  if (!r->mesh->m.on_device) {
    viv::set_error("viv_server_submit: mesh was analysed on the host only");
    return VIV_ERR_STATE;
  }
  vivMeshInfo info{};
  viv_mesh_info(r->mesh, &info);
  const size_t bytes = r->params.precision == VIV_MIXED ? info.device_bytes_mixed : info.device_bytes_fp64;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) {
    viv::set_error("viv_server_submit: server is draining");
    return VIV_ERR_STATE;
  }
  const int64_t nid = S->next_id++;
  if (id) *id = nid;
  if (bytes > S->budget) {
    // can never be admitted: finish it at once with an admission error
    Done d{};
    d.res.id = nid;
    d.res.status = VIV_ERR_ADMISSION;
    d.res.submit_s = r->arrival_time;
    d.res.finish_s = S->now();
    std::snprintf(d.res.message, sizeof d.res.message, "needs %zu bytes, budget is %zu", bytes, S->budget);
    S->finished[nid] = std::move(d);
    S->unpolled.push_back(nid);
    S->cv_done.notify_all();
    return VIV_OK;
  }
  Req q;
  q.id = nid;
  q.r = *r;
  q.r.u0 = nullptr;
  q.u0.assign(r->u0, r->u0 + r->mesh->m.dim * r->mesh->m.n_nodes);
  q.bytes = bytes;
  S->incoming.push_back(std::move(q));
  S->cv_sched.notify_all();
  return VIV_OK;
}

vivStatus viv_server_poll(vivServer* S, vivResult* out, int32_t max, int32_t* n, int32_t wait_ms) {
  if (!S || !n || (max > 0 && !out)) {
    viv::set_error("viv_server_poll: bad arguments");
    return VIV_ERR_ARG;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->unpolled.empty() && wait_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->unpolled.empty(); });
  int32_t k = 0;
  while (k < max && !S->unpolled.empty()) {
    out[k++] = S->finished[S->unpolled.front()].res;
    S->unpolled.pop_front();
  }
  *n = k;
  return VIV_OK;
}

vivStatus viv_server_state(vivServer* S, int64_t id, double* u, double* p, double* x, double* lam, double* delta) {
  if (!S) {
    viv::set_error("viv_server_state: NULL server");
    return VIV_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->finished.find(id);
  if (it == S->finished.end() || it->second.state.empty()) {
    viv::set_error("viv_server_state: no final state for this id");
    return VIV_ERR_STATE;
  }
  const std::vector<double>& st = it->second.state;
  const size_t D = it->second.dim, n = (st.size() - 2) / (3 * D + 1);
  if (u) std::memcpy(u, st.data(), D * n * sizeof(double));
  if (p) std::memcpy(p, st.data() + D * n, n * sizeof(double));
  if (x) std::memcpy(x, st.data() + D * n + n, D * n * sizeof(double));
  if (lam) std::memcpy(lam, st.data() + 2 * D * n + n, D * n * sizeof(double));
  if (delta) std::memcpy(delta, st.data() + 3 * D * n + n, 2 * sizeof(double));
  return VIV_OK;
}

vivStatus viv_server_stats(vivServer* S, vivServerStats* out) {
  if (!S || !out) {
    viv::set_error("viv_server_stats: bad arguments");
    return VIV_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto pct = [](std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))];
  };
  out->step_ms_p50 = pct(S->step_ms, 0.50);
  out->step_ms_p99 = pct(S->step_ms, 0.99);
  out->steady_ms_p50 = pct(S->steady_ms, 0.50);
  out->steady_ms_p99 = pct(S->steady_ms, 0.99);
  out->steps = S->steps_total;
  out->cases_done = S->cases_done;
  out->elapsed_s = S->now();
  out->peak_active = S->peak_active;
  out->peak_bytes = S->peak_used;
  out->active = S->active;
  out->pending = (int32_t)(S->pending.size() + S->incoming.size());
  return VIV_OK;
}

vivStatus viv_server_destroy(vivServer* S) {
  if (!S) return VIV_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_sched.notify_all();
  }
  if (S->sched.joinable()) S->sched.join();
  for (auto& w : S->workers)
    if (w.joinable()) w.join();
  delete S;
  return VIV_OK;
}

}  // extern "C"
