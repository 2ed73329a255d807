// Request server: queued ALI solves on worker threads, admitted by estimated
// device footprint, each on its own grid and CUDA stream (see rt_sc.h); in the
// shared mode the Jacobi solves of the admitted requests run in lock-step, one
// set per size class on its own scheduler thread, their sweeps merged into
// shared launches (rt_lockstep.h), while the workers set grids up and take
// results back.  Host code only.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "rt_lockstep.h"
#include "rt_sc.h"

rt_status rt_internal_error(rt_status st, const char *msg);   // rt_api.cu

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  long long id = 0;
  rt_grid_desc desc{};
  int interp = RT_INTERP_LINEAR;
  int iteration = RT_ITER_JACOBI;
  std::vector<double> chi, eps, B, fw;
  double tol = 1e-6;
  int max_iter = 1000;
  long long footprint = 0;
  int state = RT_REQ_QUEUED;
  int status = RT_OK;
  int iters = 0;
  double resid = 0.0;
  Clock::time_point t_submit, t_start, t_done;
  std::vector<double> J, S, Q;
  std::string message;       // the solve's error message (worker thread's rt_last_error)
  rt_grid g = nullptr;       // shared mode: the grid while it is set up, solved and read
  int lane = 0;              // shared mode: the lock-step set it joins
};

// Shared mode: requests are sorted into lock-step sets by the work of one of
// their iterations (cells x rays x frequencies), each set iterating on its own
// thread and stream, so that a small grid is not held to the pace of the largest
// grid's sweep: below 2^22, below 2^26, and above.
constexpr int kLanes = 3;
int lane_of(const rt_grid_desc &d) {
  const long long na = (long long)d.n_mu * (d.n_mu + 2) / (d.nz == 1 ? 2 : 1);
  const long long u = (long long)d.nx * d.ny * d.nz * na * d.nfreq;
  return u < (1LL << 22) ? 0 : (u < (1LL << 26) ? 1 : 2);
}

}  // namespace

struct rt_server_s {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request *> queue;
  std::unordered_map<long long, Request *> reqs;
  long long budget = 0;
  long long resident = 0;   // footprints of the running solves
  int device = 0;
  bool stop = false;
  long long next_id = 1;
  std::vector<std::thread> workers;
  // shared mode (cluster > 0): grids set up by the workers wait in `ready` for
  // the scheduler, which moves solved ones to `solved` for a worker to read back
  int cluster = 0;
  std::deque<Request *> ready[kLanes], solved;
  std::vector<Request *> in_lockstep[kLanes];
  long long shared_launches[kLanes] = {0, 0, 0};
  std::vector<std::thread> schedulers;
};

namespace {

// One solve, on the calling worker thread (its grid has its own stream).
void run_solve(Request *r, int device) {
  cudaSetDevice(device);
  rt_grid g = nullptr;
  rt_status st = rt_create_grid(&r->desc, &g);
  if (st == RT_OK && r->interp != RT_INTERP_LINEAR) st = rt_set_interpolation(g, r->interp);
  if (st == RT_OK && r->iteration != RT_ITER_JACOBI) st = rt_set_iteration(g, r->iteration);
  if (st == RT_OK)
    st = rt_set_opacity_source(g, r->chi.data(), r->eps.data(), r->B.data(), r->fw.data(), 0);
  int iters = 0;
  double resid = 0.0;
  if (st == RT_OK) {
    rt_solve_opts o{};
    o.tol = r->tol;
    o.max_iter = r->max_iter;
    st = rt_ali_solve(g, nullptr, 0, &o, &iters, &resid);
  }
  if (st == RT_OK || st == RT_ERR_NOT_CONVERGED) {
    const size_t N = r->chi.size(), C = N / (size_t)r->desc.nfreq;
    r->J.resize(N);
    r->S.resize(N);
    r->Q.resize(C);
    rt_status s2 = rt_moments(g, r->J.data(), nullptr, nullptr, nullptr, r->Q.data(), 0, nullptr);
    if (s2 == RT_OK) s2 = rt_get_S(g, r->S.data(), 0, nullptr);
    if (s2 != RT_OK) st = s2;
  }
  if (st != RT_OK) r->message = rt_last_error();
  if (g) rt_destroy_grid(g);
  r->status = st;
  r->iters = iters;
  r->resid = resid;
}

// Shared mode: the request's grid, planned with the server's cluster size where
// that plan fits (else the grid's own plan: it then shares launches only with
// grids that ended up with the same one), with its medium set.  Grids of the
// largest size class keep their own plan: they fill the GPU by themselves, and
// the common cluster size would slow their sweeps.
rt_status prepare_grid(Request *r, int device, int cluster) {
  cudaSetDevice(device);
  rt_status st = rt_create_grid(&r->desc, &r->g);
  if (st != RT_OK) return st;
  if (r->lane == kLanes - 1 || rt_set_sweep_config(r->g, 0, cluster, 0, 3) != RT_OK)
    st = rt_set_sweep_config(r->g, 0, 0, 0, 0);
  if (st == RT_OK)
    st = rt_set_opacity_source(r->g, r->chi.data(), r->eps.data(), r->B.data(), r->fw.data(), 0);
  return st;
}

// Shared mode: J, S and Q of a solved request back to host memory; the grid freed.
void read_back(Request *r, int device) {
  cudaSetDevice(device);
  rt_status st = (rt_status)r->status;
  if (r->g && (st == RT_OK || st == RT_ERR_NOT_CONVERGED)) {
    const size_t N = r->chi.size(), C = N / (size_t)r->desc.nfreq;
    r->J.resize(N);
    r->S.resize(N);
    r->Q.resize(C);
    rt_status s2 = rt_moments(r->g, r->J.data(), nullptr, nullptr, nullptr, r->Q.data(), 0, nullptr);
    if (s2 == RT_OK) s2 = rt_get_S(r->g, r->S.data(), 0, nullptr);
    if (s2 != RT_OK) {
      st = s2;
      r->message = rt_last_error();
    }
  }
  if (r->g) rt_destroy_grid(r->g);
  r->g = nullptr;
  r->status = st;
}

void finish_request(rt_server s, Request *r) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->resident -= r->footprint;
    r->state = RT_REQ_DONE;
    r->t_done = Clock::now();
  }
  s->cv.notify_all();
}

bool shareable(const rt_server_s *s, const Request *r) {
  return s->cluster > 0 && r->iteration == RT_ITER_JACOBI && r->interp == RT_INTERP_LINEAR;
}

void worker_loop(rt_server s) {
  for (;;) {
    Request *r = nullptr;
    bool readback = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] {
        if (s->stop) return true;
        if (!s->solved.empty()) return true;
        if (s->queue.empty()) return false;
        const long long fp = s->queue.front()->footprint;
        return s->resident == 0 || s->resident + fp <= s->budget;
      });
      if (s->stop) return;
      if (!s->solved.empty()) {   // results first: they free device memory
        r = s->solved.front();
        s->solved.pop_front();
        readback = true;
      } else {
        r = s->queue.front();
        s->queue.pop_front();
        s->resident += r->footprint;
        r->state = RT_REQ_RUNNING;
        r->t_start = Clock::now();
      }
    }
    if (readback) {
      read_back(r, s->device);
      finish_request(s, r);
    } else if (shareable(s, r)) {
      const rt_status st = prepare_grid(r, s->device, s->cluster);
      if (st != RT_OK) {
        r->status = st;
        r->message = rt_last_error();
        read_back(r, s->device);
        finish_request(s, r);
      } else {
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->ready[r->lane].push_back(r);
        }
        s->cv.notify_all();
      }
    } else {
      run_solve(r, s->device);
      finish_request(s, r);
    }
  }
}

// Shared mode: the Jacobi solves of one lane's admitted requests in lock-step on
// this thread's stream; ready grids join at each step, solved ones go to `solved`.
void scheduler_loop(rt_server s, int lane) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  rt_lockstep L = nullptr;
  ls_create(st, &L);
  std::vector<LsResult> done;
  for (;;) {
    std::vector<Request *> join;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || !s->ready[lane].empty() || ls_size(L) > 0; });
      if (s->stop) break;
      join.assign(s->ready[lane].begin(), s->ready[lane].end());
      s->ready[lane].clear();
    }
    std::vector<Request *> out;
    for (Request *r : join) {
      rt_solve_opts o{};
      o.tol = r->tol;
      o.max_iter = r->max_iter;
      const rt_status e = ls_add(L, r->g, &o, r);
      if (e != RT_OK) {
        r->status = e;
        r->message = rt_last_error();
        out.push_back(r);
      } else {
        std::lock_guard<std::mutex> lk(s->mu);
        s->in_lockstep[lane].push_back(r);
      }
    }
    done.clear();
    rt_status e = ls_size(L) > 0 ? ls_step(L, &done) : RT_OK;
    if (e != RT_OK) {   // a shared launch out: every member fails with it
      const std::string msg = rt_last_error();
      std::lock_guard<std::mutex> lk(s->mu);
      for (Request *r : s->in_lockstep[lane]) {
        r->status = e;
        r->message = msg;
        out.push_back(r);
      }
      s->in_lockstep[lane].clear();
      ls_destroy(L);
      ls_create(st, &L);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (const LsResult &d : done) {
        Request *r = (Request *)d.tag;
        r->status = d.status;
        r->iters = d.iters;
        r->resid = d.resid;
        r->message = d.message;
        out.push_back(r);
        auto &v = s->in_lockstep[lane];
        for (size_t i = 0; i < v.size(); ++i)
          if (v[i] == r) {
            v.erase(v.begin() + i);
            break;
          }
      }
      for (Request *r : out) s->solved.push_back(r);
      s->shared_launches[lane] += ls_shared_launches(L);
      ls_reset_shared(L);
    }
    if (!out.empty()) s->cv.notify_all();
  }
  // stopping: grids still in the set are freed with their requests
  ls_destroy(L);
  cudaStreamSynchronize(st);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Request *r : s->in_lockstep[lane])
      if (r->g) {
        rt_destroy_grid(r->g);
        r->g = nullptr;
      }
    s->in_lockstep[lane].clear();
  }
  cudaStreamDestroy(st);
}

void fill_info(const Request *r, rt_request_info *info) {
  if (!info) return;
  info->state = r->state;
  info->status = r->status;
  info->iters = r->iters;
  info->resid = r->resid;
  const Clock::time_point now = Clock::now();
  info->queue_ms = ms_between(r->t_submit, r->state == RT_REQ_QUEUED ? now : r->t_start);
  info->solve_ms = r->state == RT_REQ_QUEUED ? 0.0 : ms_between(r->t_start, r->state == RT_REQ_DONE ? r->t_done : now);
  info->footprint = r->footprint;
}

}  // namespace

extern "C" {

rt_status rt_server_create(const rt_server_opts *opts, rt_server *out) {
  if (!opts || !out || opts->workers < 1) return rt_internal_error(RT_ERR_ARG, "rt_server_create: NULL argument or workers < 1");
  *out = nullptr;
  rt_server s = new rt_server_s();
  cudaGetDevice(&s->device);
  s->budget = opts->device_bytes;
  if (s->budget <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return rt_internal_error(RT_ERR_CUDA, "rt_server_create: cudaMemGetInfo failed");
    }
    s->budget = (long long)(0.8 * (double)fr);
  }
  if (opts->shared_cluster < 0 || opts->shared_cluster > 16) {
    delete s;
    return rt_internal_error(RT_ERR_ARG, "rt_server_create: shared_cluster must be in 0..16");
  }
  s->cluster = opts->shared_cluster;
  for (int i = 0; i < opts->workers; ++i) s->workers.emplace_back(worker_loop, s);
  if (s->cluster > 0)
    for (int l = 0; l < kLanes; ++l) s->schedulers.emplace_back(scheduler_loop, s, l);
  *out = s;
  return RT_OK;
}

rt_status rt_server_shared_launches(rt_server s, long long *n) {
  if (!s || !n) return rt_internal_error(RT_ERR_ARG, "rt_server_shared_launches: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *n = s->shared_launches[0] + s->shared_launches[1] + s->shared_launches[2];
  return RT_OK;
}

rt_status rt_server_destroy(rt_server s) {
  if (!s) return rt_internal_error(RT_ERR_ARG, "rt_server_destroy: NULL server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  for (auto &t : s->workers) t.join();
  for (auto &t : s->schedulers) t.join();
  for (auto &q : s->ready)
    for (Request *r : q)
      if (r->g) rt_destroy_grid(r->g);
  for (Request *r : s->solved)
    if (r->g) rt_destroy_grid(r->g);
  for (auto &kv : s->reqs) delete kv.second;
  delete s;
  return RT_OK;
}

rt_status rt_submit(rt_server s, const rt_request *req, long long *id_out) {
  if (!s || !req || !id_out || !req->chi || !req->eps || !req->B)
    return rt_internal_error(RT_ERR_ARG, "rt_submit: NULL argument");
  long long fp = 0;
  rt_status st = rt_grid_footprint(&req->desc, &fp);
  if (st != RT_OK) return st;
  if (req->interp != 0 && req->interp != RT_INTERP_LINEAR && req->interp != RT_INTERP_QUADRATIC)
    return rt_internal_error(RT_ERR_ARG, "rt_submit: interp must be 0, 1 or 2");
  if (req->iteration != RT_ITER_JACOBI && req->iteration != RT_ITER_GAUSS_SEIDEL)
    return rt_internal_error(RT_ERR_ARG, "rt_submit: iteration must be 0 or 1");
  if (req->iteration == RT_ITER_GAUSS_SEIDEL && req->interp == RT_INTERP_QUADRATIC)
    return rt_internal_error(RT_ERR_ARG, "rt_submit: the Gauss-Seidel iteration takes linear interpolation");
  Request *r = new Request();
  r->desc = req->desc;
  r->interp = req->interp == 0 ? RT_INTERP_LINEAR : req->interp;
  const size_t N = (size_t)req->desc.nx * req->desc.ny * req->desc.nz * req->desc.nfreq;
  r->chi.assign(req->chi, req->chi + N);
  r->eps.assign(req->eps, req->eps + N);
  r->B.assign(req->B, req->B + N);
  if (req->freq_w) r->fw.assign(req->freq_w, req->freq_w + req->desc.nfreq);
  else r->fw.assign((size_t)req->desc.nfreq, 1.0);
  r->tol = req->tol;
  r->max_iter = req->max_iter;
  r->iteration = req->iteration;
  r->footprint = fp;
  r->lane = lane_of(r->desc);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *id_out = r->id;
  }
  s->cv.notify_all();
  return RT_OK;
}

rt_status rt_poll(rt_server s, long long id, rt_request_info *info) {
  if (!s) return rt_internal_error(RT_ERR_ARG, "rt_poll: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return rt_internal_error(RT_ERR_ARG, "rt_poll: unknown request id");
  fill_info(it->second, info);
  return RT_OK;
}

rt_status rt_wait(rt_server s, long long id, double timeout_s, rt_request_info *info) {
  if (!s) return rt_internal_error(RT_ERR_ARG, "rt_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return rt_internal_error(RT_ERR_ARG, "rt_wait: unknown request id");
  Request *r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
  const bool done = s->cv.wait_until(lk, deadline, [&] { return r->state == RT_REQ_DONE; });
  fill_info(r, info);
  return done ? RT_OK : rt_internal_error(RT_ERR_TIMEOUT, "rt_wait: the request is not done yet");
}

rt_status rt_fetch(rt_server s, long long id, double *J, double *S, double *Q) {
  if (!s) return rt_internal_error(RT_ERR_ARG, "rt_fetch: NULL server");
  Request *r = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return rt_internal_error(RT_ERR_ARG, "rt_fetch: unknown request id");
    r = it->second;
    if (r->state != RT_REQ_DONE) return rt_internal_error(RT_ERR_STATE, "rt_fetch: the request is not done");
    s->reqs.erase(it);
  }
  if (J && !r->J.empty()) std::memcpy(J, r->J.data(), r->J.size() * sizeof(double));
  if (S && !r->S.empty()) std::memcpy(S, r->S.data(), r->S.size() * sizeof(double));
  if (Q && !r->Q.empty()) std::memcpy(Q, r->Q.data(), r->Q.size() * sizeof(double));
  const rt_status st = (rt_status)r->status;
  const std::string msg = r->message;
  delete r;
  return st == RT_OK ? st : rt_internal_error(st, msg.c_str());
}

}  // extern "C"
