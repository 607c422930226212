// Continuous-batching RT-TDA server (include/rttda_server.h).
//
// One scheduler thread owns every admitted request's handle.  Per loop it
//   1. admits pending requests in arrival order while their estimated
//      footprint fits the budget and an active slot is free (a request that
//      needs its own handle is handed to the creator thread, which casts its
//      factors and plans its contraction while the scheduler keeps stepping
//      the others, and hands it back once the handle exists);
//   2. enqueues the next chunk of RK4 steps of every idle active request on
//      that request's own stream (the chunks of different requests overlap
//      on the GPU);
//   3. retires finished chunks (polled CUDA events); a request whose last
//      chunk finished gets its spectrum computed on the GPU, copied out, and
//      its memory released.
// Host waits are bounded; device waits inside the kernels are bounded too
// (a timeout fails only the request it happened in).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rttda.h"
#include "../../include/rttda_server.h"
#include "engine_internal.h"
#include "group_internal.h"

namespace {

using clk = std::chrono::steady_clock;

double seconds_since(clk::time_point t0) {
  return std::chrono::duration<double>(clk::now() - t0).count();
}

struct Request {
  long id = 0;
  rttda_request req{};
  std::vector<double> eps_o, eps_v, Bov, Boo, Bvv, moo, mvv, m0;  // owned copies until admission
  int state = RTTDA_REQ_PENDING;
  std::atomic<bool> cancel{false};  // written by rttda_server_cancel, read by the scheduler thread
  double t_submit = 0.0, t_done = 0.0;
  rttda_t h = nullptr;
  rttda::GroupReq* g = nullptr;  // grouped request (small BF16): no handle
  double* dev = nullptr;  // handle: [dip nsteps+1][nrm nsteps+1][omega nfreq][S nfreq]; grouped: [omega][S]
  size_t bytes = 0;
  double gwork = 0.0;  // grouped: its share of the group's work (nocc nvirt^2 naux)
  long done_steps = 0, inflight = 0;
  cudaEvent_t ev = nullptr;
  std::vector<double> spectrum, omega, dipole;
  std::string error;
};

}  // namespace

struct rttda_server {
  int device = 0;
  size_t budget = 0;
  int max_active = 1;
  long chunk = 256;
  clk::time_point t0;

  std::mutex mu;
  std::condition_variable cv;       // wakes the scheduler (new work)
  std::condition_variable done_cv;  // wakes waiters (a request finished)
  std::deque<long> pending;
  std::map<long, std::unique_ptr<Request>> reqs;
  std::vector<Request*> active;  // touched by the scheduler only
  size_t used = 0;
  long next_id = 1;
  std::atomic<bool> stop{false};
  std::thread worker;

  // handle creation (seconds for a large molecule: factor casts, the tile
  // plan's timed candidates) runs on its own thread so that the scheduler
  // keeps launching the other requests' chunks meanwhile
  std::thread creator;
  std::condition_variable create_cv;
  std::deque<Request*> to_create;  // admitted, handle not created yet (under mu)
  std::vector<Request*> created;   // handle ready, not yet taken by the scheduler (under mu)
  int creating = 0;                // requests admitted but not yet active (under mu)

  // grouped step of the small BF16 requests (one persistent kernel per chunk
  // for all of them); touched by the scheduler only, except `grouping`
  rttda::GroupRunner grp;
  std::atomic<int> grouping{1};  // rttda_server_set_grouping mode: 0 off, 1 by work, 2 every eligible request
  bool grp_ready = false, grp_busy = false;
  double grp_work = 0.0;  // summed work of the admitted grouped requests (under mu)
  std::vector<Request*> grp_batch;

  // statistics
  long submitted = 0, completed = 0, failed = 0, cancelled = 0, grouped = 0;
  int max_concurrent = 0;
  double traj_steps = 0.0, first_submit = -1.0, last_done = 0.0;
  std::vector<double> latencies;

  void run();
  bool admit_one();
  void create_loop();
  rttda_status create_handle(Request* r);
  void release(Request* r, int final_state);
};

// Free a request's device resources and record its final state.
void rttda_server::release(Request* r, int final_state) {
  // stream-ordered frees: releasing one request does not wait for the others
  if (r->g) {
    if (r->dev) cudaFreeAsync(r->dev, grp.stream);
    r->dev = nullptr;
    rttda::group_release(r->g, grp.stream);
    r->g = nullptr;
  }
  if (r->h) {
    cudaStream_t hs = rttda::handle_stream(r->h);
    if (r->dev) cudaFreeAsync(r->dev, hs);
    r->dev = nullptr;
    cudaStreamSynchronize(hs);
    rttda_destroy(r->h);
    r->h = nullptr;
  }
  if (r->dev) cudaFree(r->dev);
  r->dev = nullptr;
  if (r->ev) cudaEventDestroy(r->ev);
  r->ev = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  used -= r->bytes;
  r->bytes = 0;
  grp_work -= r->gwork;
  r->gwork = 0.0;
  r->state = final_state;
  r->t_done = seconds_since(t0);
  if (final_state == RTTDA_REQ_DONE) {
    ++completed;
    latencies.push_back(r->t_done - r->t_submit);
    last_done = r->t_done;
  } else if (final_state == RTTDA_REQ_FAILED) {
    ++failed;
  } else if (final_state == RTTDA_REQ_CANCELLED) {
    ++cancelled;
  }
  done_cv.notify_all();
}

// Admit the request at the head of the queue if it fits; true if admitted
// (or removed because it was cancelled / can never fit).
bool rttda_server::admit_one() {
  Request* r = nullptr;
  bool to_group = false;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (pending.empty() || (int)active.size() + creating >= max_active) return false;
    r = reqs[pending.front()].get();
    if (r->cancel) {
      pending.pop_front();
      r->state = RTTDA_REQ_CANCELLED;
      ++cancelled;
      done_cv.notify_all();
      return true;
    }
    const rttda_request& q = r->req;
    const int gm = grouping.load();
    if (gm != 0 && rttda::group_eligible(q)) {
      const double w = rttda::group_work(q);
      to_group = gm == 2 || (w <= rttda::grp::kAutoWork && grp_work + w <= rttda::grp::kMaxGroupWork);
    }
    const size_t need = to_group ? rttda::group_estimate_bytes(q)
                                : rttda::estimate_bytes(q.nocc, q.nvirt, q.naux, 1, q.prec, q.nsteps);
    if (used + need > budget) {
      // wait for memory to free up, unless nothing else holds any
      if (!active.empty() || creating > 0) return false;
      pending.pop_front();
      r->state = RTTDA_REQ_FAILED;
      r->error = "request footprint " + std::to_string(need) + " B exceeds the server budget";
      ++failed;
      done_cv.notify_all();
      return true;
    }
    pending.pop_front();
    used += need;
    r->bytes = need;
    if (to_group) {
      r->gwork = rttda::group_work(q);
      grp_work += r->gwork;
    }
    // the state stays PENDING until the molecule has been copied: a caller
    // with device factors may free them once the request leaves PENDING
    if (!to_group) {
      ++creating;
      to_create.push_back(r);
    }
  }
  if (!to_group) {
    create_cv.notify_one();
    return true;
  }
  const rttda_request& q = r->req;
  rttda_status st = RTTDA_OK;
  {
    // small BF16 request: stepped with the others in the grouped kernel
    if (!grp_ready) {
      st = rttda::group_runner_init(&grp);
      grp_ready = st == RTTDA_OK;
    }
    // r->req points at the owned host copies, or at the caller's device arrays
    // uploads on the group's admission stream (group_admit synchronises it),
    // so admitting never waits for the chunk running on the group stream
    if (st == RTTDA_OK) st = rttda::group_admit(q, grp.upload, &r->g);
    if (st == RTTDA_OK && (cudaMallocAsync((void**)&r->dev, 2 * (size_t)q.nfreq * sizeof(double), grp.upload) !=
                               cudaSuccess ||
                           cudaStreamSynchronize(grp.upload) != cudaSuccess))
      st = RTTDA_E_OOM;
    if (st != RTTDA_OK) {
      r->error = rttda_last_error();
      release(r, RTTDA_REQ_FAILED);
      return true;
    }
    std::vector<double>().swap(r->Bov);
    std::vector<double>().swap(r->Boo);
    std::vector<double>().swap(r->Bvv);
    active.push_back(r);
    {
      std::lock_guard<std::mutex> lk(mu);
      max_concurrent = std::max(max_concurrent, (int)active.size());
      r->state = RTTDA_REQ_ACTIVE;  // group_admit has copied the molecule
      ++grouped;
    }
    return true;
  }
}

// The request's own handle, its field, its trace buffer and its event
// (creator thread).  The molecule is copied from the owned host copies or
// from the caller's device arrays (the copies inside accept both).
rttda_status rttda_server::create_handle(Request* r) {
  const rttda_request& q = r->req;
  rttda_status st = rttda_create(q.nocc, q.nvirt, q.naux, q.eps_occ, q.eps_virt, q.B_ov, q.B_oo, q.B_vv, q.mu_oo,
                                 q.mu_vv, q.mu_0ov, q.c_x, q.prec, &r->h);
  if (st == RTTDA_OK) st = rttda_set_field(r->h, &q.pulse, 1);
  if (st == RTTDA_OK) {
    const size_t n = 2 * (size_t)(q.nsteps + 1) + 2 * (size_t)q.nfreq;
    cudaStream_t hs = rttda::handle_stream(r->h);
    if (cudaMallocAsync((void**)&r->dev, n * sizeof(double), hs) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamSynchronize(hs) != cudaSuccess)
      st = RTTDA_E_OOM;
  }
  if (st != RTTDA_OK) return st;
  // the factors now live on the device (rttda_set_field synchronised the
  // handle's stream, so every copy from the caller's arrays has completed)
  std::vector<double>().swap(r->Bov);
  std::vector<double>().swap(r->Boo);
  std::vector<double>().swap(r->Bvv);
  return RTTDA_OK;
}

// Creator thread: builds the handles of admitted requests in admission
// order.  A request cancelled before its turn (or left at shutdown) is
// released without a handle; a finished one is handed to the scheduler.
void rttda_server::create_loop() {
  cudaSetDevice(device);
  while (true) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      create_cv.wait(lk, [&] { return stop.load() || !to_create.empty(); });
      if (to_create.empty()) return;  // stopping, nothing left
      r = to_create.front();
      to_create.pop_front();
    }
    rttda_status st = RTTDA_OK;
    const bool skip = r->cancel || stop.load();
    if (!skip) st = create_handle(r);
    if (skip || st != RTTDA_OK) {
      if (!skip) r->error = rttda_last_error();
      release(r, skip ? RTTDA_REQ_CANCELLED : RTTDA_REQ_FAILED);
      std::lock_guard<std::mutex> lk(mu);
      --creating;
      continue;
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      r->state = RTTDA_REQ_ACTIVE;
      created.push_back(r);
    }
    cv.notify_all();
  }
}

void rttda_server::run() {
  cudaSetDevice(device);
  while (!stop.load()) {
    bool progressed = false;
    {
      // requests whose handles the creator thread has finished
      std::lock_guard<std::mutex> lk(mu);
      if (!created.empty()) {
        active.insert(active.end(), created.begin(), created.end());
        creating -= (int)created.size();
        created.clear();
        max_concurrent = std::max(max_concurrent, (int)active.size());
        progressed = true;
      }
    }
    while (admit_one()) progressed = true;
    // enqueue the next chunk of every idle request
    for (Request* r : active) {
      if (r->g || r->inflight || r->cancel) continue;
      const rttda_request& q = r->req;
      const long n = std::min(chunk, q.nsteps - r->done_steps);
      cudaStream_t s = rttda::handle_stream(r->h);
      double* dip = r->dev;
      double* nrm = r->dev + (q.nsteps + 1);
      rttda_status st = rttda::advance(r->h, r->done_steps == 0, q.dt, n, dip, nrm, q.nsteps + 1, r->done_steps, s);
      if (st == RTTDA_OK && cudaEventRecord(r->ev, s) != cudaSuccess) st = RTTDA_E_CUDA;
      if (st != RTTDA_OK) {
        std::lock_guard<std::mutex> lk(mu);
        r->error = rttda_last_error();
        r->cancel = true;  // retired below as failed
        r->state = RTTDA_REQ_FAILED;
        continue;
      }
      r->inflight = n;
      progressed = true;
    }
    // one chunk of the grouped step for every idle grouped request
    if (grp_ready && !grp_busy) {
      std::vector<rttda::GroupReq*> gs;
      std::vector<long> n, done;
      std::vector<int> fresh;
      grp_batch.clear();
      for (Request* r : active) {
        if (!r->g || r->inflight || r->cancel) continue;
        if ((int)grp_batch.size() >= rttda::grp::kMaxGroup) break;
        grp_batch.push_back(r);
        gs.push_back(r->g);
        n.push_back(std::min(chunk, r->req.nsteps - r->done_steps));
        done.push_back(r->done_steps);
        fresh.push_back(r->done_steps == 0);
      }
      if (!grp_batch.empty()) {
        const rttda_status st = rttda::group_launch(&grp, gs, n, done, fresh);
        for (size_t k = 0; k < grp_batch.size(); ++k) {
          Request* r = grp_batch[k];
          if (st == RTTDA_OK) {
            r->inflight = n[k];
          } else {
            std::lock_guard<std::mutex> lk(mu);
            r->error = rttda_last_error();
            r->cancel = true;
            r->state = RTTDA_REQ_FAILED;
          }
        }
        grp_busy = st == RTTDA_OK;
        progressed = true;
      }
    }
    bool grp_done = false;
    rttda_status grp_st = RTTDA_OK;
    std::string grp_err;
    if (grp_busy && cudaEventQuery(grp.ev) == cudaSuccess) {
      grp_done = true;
      grp_busy = false;
      grp_st = rttda::group_status(&grp);
      if (grp_st != RTTDA_OK) grp_err = rttda_last_error();
    }
    // retire finished chunks
    for (size_t k = 0; k < active.size();) {
      Request* r = active[k];
      bool remove = false;
      int final_state = RTTDA_REQ_DONE;
      if (r->g && r->inflight && grp_done) {
        progressed = true;
        if (grp_st != RTTDA_OK) {
          r->error = grp_err;
          remove = true;
          final_state = RTTDA_REQ_FAILED;
        } else {
          r->done_steps += r->inflight;
          {
            std::lock_guard<std::mutex> lk(mu);
            traj_steps += (double)r->inflight;
          }
          r->inflight = 0;
          if (r->done_steps >= r->req.nsteps && !r->cancel) {
            const rttda_request& q = r->req;
            cudaStream_t s = grp.stream;
            const double* dip = r->g->trace;
            double* om = r->dev;
            double* S = om + q.nfreq;
            rttda_status st = rttda::spectrum_device(dip, 1, q.nsteps + 1, q.dt, q.pulse.E0, q.gamma, q.wmin,
                                                     q.wmax, q.nfreq, om, S, s);
            r->spectrum.resize(q.nfreq);
            r->omega.resize(q.nfreq);
            r->dipole.resize(q.nsteps + 1);
            if (st == RTTDA_OK &&
                (cudaMemcpyAsync(r->spectrum.data(), S, q.nfreq * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaMemcpyAsync(r->omega.data(), om, q.nfreq * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaMemcpyAsync(r->dipole.data(), dip, (q.nsteps + 1) * 8, cudaMemcpyDeviceToHost, s) !=
                     cudaSuccess ||
                 cudaStreamSynchronize(s) != cudaSuccess))
              st = RTTDA_E_CUDA;
            remove = true;
            if (st != RTTDA_OK) {
              r->error = rttda_last_error();
              final_state = RTTDA_REQ_FAILED;
            }
          }
        }
      } else if (!r->g && r->inflight && cudaEventQuery(r->ev) == cudaSuccess) {
        progressed = true;
        rttda_status st = rttda::device_error(r->h);
        if (st != RTTDA_OK) {
          r->error = rttda_last_error();
          remove = true;
          final_state = RTTDA_REQ_FAILED;
        } else {
          r->done_steps += r->inflight;
          {
            std::lock_guard<std::mutex> lk(mu);
            traj_steps += (double)r->inflight;
          }
          r->inflight = 0;
          if (r->done_steps >= r->req.nsteps && !r->cancel) {
            const rttda_request& q = r->req;
            cudaStream_t s = rttda::handle_stream(r->h);
            double* dip = r->dev;
            double* om = r->dev + 2 * (q.nsteps + 1);
            double* S = om + q.nfreq;
            st = rttda::spectrum_device(dip, 1, q.nsteps + 1, q.dt, q.pulse.E0, q.gamma, q.wmin, q.wmax, q.nfreq, om,
                                        S, s);
            r->spectrum.resize(q.nfreq);
            r->omega.resize(q.nfreq);
            r->dipole.resize(q.nsteps + 1);
            if (st == RTTDA_OK &&
                (cudaMemcpyAsync(r->spectrum.data(), S, q.nfreq * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaMemcpyAsync(r->omega.data(), om, q.nfreq * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaMemcpyAsync(r->dipole.data(), dip, (q.nsteps + 1) * 8, cudaMemcpyDeviceToHost, s) !=
                     cudaSuccess ||
                 cudaStreamSynchronize(s) != cudaSuccess))
              st = RTTDA_E_CUDA;
            remove = true;
            if (st != RTTDA_OK) {
              r->error = rttda_last_error();
              final_state = RTTDA_REQ_FAILED;
            }
          }
        }
      }
      if (!r->inflight && r->cancel) {
        remove = true;
        final_state = r->state == RTTDA_REQ_FAILED ? RTTDA_REQ_FAILED : RTTDA_REQ_CANCELLED;
      }
      if (remove) {
        active.erase(active.begin() + k);
        release(r, final_state);
      } else {
        ++k;
      }
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait_for(lk, std::chrono::microseconds(200));
    }
  }
  // shutdown: cancel whatever is still on the GPU
  if (grp_ready) cudaStreamSynchronize(grp.stream);
  for (Request* r : active) release(r, RTTDA_REQ_CANCELLED);
  active.clear();
  if (grp_ready) rttda::group_runner_free(&grp);
}

extern "C" {

rttda_status rttda_server_create(size_t hbm_budget, int max_active, long chunk_steps, rttda_server_t* out) {
  rttda::g_last_error.clear();
  if (!out) return rttda::set_error(RTTDA_E_ARG, "rttda_server_create: out is NULL");
  *out = nullptr;
  if (hbm_budget == 0 || max_active < 1 || chunk_steps < 1)
    return rttda::set_error(RTTDA_E_ARG, "rttda_server_create: budget, max_active and chunk_steps must be positive");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rttda::set_error(RTTDA_E_CUDA, std::string("rttda_server_create: ") + cudaGetErrorString(e));
  rttda_server* s = new rttda_server();
  s->device = dev;
  s->budget = hbm_budget;
  s->max_active = max_active;
  s->chunk = chunk_steps;
  s->t0 = clk::now();
  s->worker = std::thread([s] { s->run(); });
  s->creator = std::thread([s] { s->create_loop(); });
  *out = s;
  return RTTDA_OK;
}

rttda_status rttda_server_submit(rttda_server_t s, const rttda_request* q, long* id) {
  rttda::g_last_error.clear();
  if (!s || !q || !id) return rttda::set_error(RTTDA_E_ARG, "rttda_server_submit: NULL argument");
  if (q->nocc < 1 || q->nvirt < 1 || q->naux < 1 || !q->eps_occ || !q->eps_virt || !q->B_ov || !q->B_oo ||
      !q->B_vv || !q->mu_oo || !q->mu_vv || !q->mu_0ov)
    return rttda::set_error(RTTDA_E_ARG, "rttda_server_submit: bad molecule");
  if (!(q->dt > 0.0) || q->nsteps < 1 || q->nfreq < 1 || !(q->gamma >= 0.0) || q->pulse.E0 == 0.0)
    return rttda::set_error(RTTDA_E_ARG, "rttda_server_submit: bad time grid, spectrum or zero E0");
  if (q->pulse.kind < RTTDA_KICK || q->pulse.kind > RTTDA_SIN2)
    return rttda::set_error(RTTDA_E_ARG, "rttda_server_submit: unknown pulse kind");
  auto r = std::make_unique<Request>();
  const size_t o = q->nocc, v = q->nvirt, P = q->naux;
  r->req = *q;
  if (!q->factors_on_device) {
    // host arrays: owned copies until admission
    r->eps_o.assign(q->eps_occ, q->eps_occ + o);
    r->eps_v.assign(q->eps_virt, q->eps_virt + v);
    r->Bov.assign(q->B_ov, q->B_ov + P * o * v);
    r->Boo.assign(q->B_oo, q->B_oo + P * o * o);
    r->Bvv.assign(q->B_vv, q->B_vv + P * v * v);
    r->moo.assign(q->mu_oo, q->mu_oo + 3 * o * o);
    r->mvv.assign(q->mu_vv, q->mu_vv + 3 * v * v);
    r->m0.assign(q->mu_0ov, q->mu_0ov + 3 * o * v);
    r->req.eps_occ = r->eps_o.data();
    r->req.eps_virt = r->eps_v.data();
    r->req.B_ov = r->Bov.data();
    r->req.B_oo = r->Boo.data();
    r->req.B_vv = r->Bvv.data();
    r->req.mu_oo = r->moo.data();
    r->req.mu_vv = r->mvv.data();
    r->req.mu_0ov = r->m0.data();
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->t_submit = seconds_since(s->t0);
    if (s->first_submit < 0) s->first_submit = r->t_submit;
    *id = r->id;
    s->pending.push_back(r->id);
    s->reqs[r->id] = std::move(r);
    ++s->submitted;
  }
  s->cv.notify_all();
  return RTTDA_OK;
}

rttda_status rttda_server_poll(rttda_server_t s, long id, int* state, double* spectrum, double* omega, double* dipole,
                               double* latency_s) {
  rttda::g_last_error.clear();
  if (!s || !state) return rttda::set_error(RTTDA_E_ARG, "rttda_server_poll: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return rttda::set_error(RTTDA_E_ARG, "rttda_server_poll: unknown id");
  Request* r = it->second.get();
  *state = r->state;
  if (r->state == RTTDA_REQ_DONE) {
    if (spectrum) std::copy(r->spectrum.begin(), r->spectrum.end(), spectrum);
    if (omega) std::copy(r->omega.begin(), r->omega.end(), omega);
    if (dipole) std::copy(r->dipole.begin(), r->dipole.end(), dipole);
    if (latency_s) *latency_s = r->t_done - r->t_submit;
  } else if (r->state == RTTDA_REQ_FAILED) {
    rttda::g_last_error = r->error;
  }
  return RTTDA_OK;
}

rttda_status rttda_server_wait(rttda_server_t s, long id, double timeout_s) {
  rttda::g_last_error.clear();
  if (!s || !(timeout_s >= 0.0)) return rttda::set_error(RTTDA_E_ARG, "rttda_server_wait: bad argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return rttda::set_error(RTTDA_E_ARG, "rttda_server_wait: unknown id");
  Request* r = it->second.get();
  const auto until = clk::now() + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(timeout_s));
  while (r->state == RTTDA_REQ_PENDING || r->state == RTTDA_REQ_ACTIVE) {
    if (s->done_cv.wait_until(lk, until) == std::cv_status::timeout &&
        (r->state == RTTDA_REQ_PENDING || r->state == RTTDA_REQ_ACTIVE))
      return rttda::set_error(RTTDA_E_TIMEOUT, "rttda_server_wait: request still running");
  }
  return RTTDA_OK;
}

rttda_status rttda_server_cancel(rttda_server_t s, long id) {
  rttda::g_last_error.clear();
  if (!s) return rttda::set_error(RTTDA_E_ARG, "rttda_server_cancel: NULL server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return rttda::set_error(RTTDA_E_ARG, "rttda_server_cancel: unknown id");
    it->second->cancel = true;
  }
  s->cv.notify_all();
  return RTTDA_OK;
}

rttda_status rttda_server_set_grouping(rttda_server_t s, int enable) {
  rttda::g_last_error.clear();
  if (!s) return rttda::set_error(RTTDA_E_ARG, "rttda_server_set_grouping: NULL server");
  if (enable < 0 || enable > 2) return rttda::set_error(RTTDA_E_ARG, "rttda_server_set_grouping: mode must be 0, 1 or 2");
  s->grouping.store(enable);
  return RTTDA_OK;
}

rttda_status rttda_server_stats_get(rttda_server_t s, rttda_server_stats* st) {
  rttda::g_last_error.clear();
  if (!s || !st) return rttda::set_error(RTTDA_E_ARG, "rttda_server_stats_get: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *st = rttda_server_stats{};
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->cancelled = s->cancelled;
  st->pending = (long)s->pending.size();
  long act = 0;
  for (auto& kv : s->reqs) act += kv.second->state == RTTDA_REQ_ACTIVE;
  st->active = act;
  st->max_concurrent = s->max_concurrent;
  st->trajectory_steps = s->traj_steps;
  if (!s->latencies.empty()) {
    std::vector<double> l = s->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
      const double x = p * (double)(l.size() - 1);
      const size_t a = (size_t)std::floor(x), b = std::min(a + 1, l.size() - 1);
      return l[a] + (x - (double)a) * (l[b] - l[a]);
    };
    st->p50_latency_s = pct(0.50);
    st->p99_latency_s = pct(0.99);
    double sum = 0.0;
    for (double x : l) sum += x;
    st->mean_latency_s = sum / (double)l.size();
  }
  st->busy_seconds = s->first_submit >= 0 ? s->last_done - s->first_submit : 0.0;
  st->bytes_in_use = s->used;
  st->bytes_budget = s->budget;
  st->grouped = s->grouped;
  return RTTDA_OK;
}

void rttda_server_destroy(rttda_server_t s) {
  if (!s) return;
  s->stop.store(true);
  s->cv.notify_all();
  s->create_cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->creator.joinable()) s->creator.join();
  // handles finished after the scheduler stopped
  for (Request* r : s->created) s->release(r, RTTDA_REQ_CANCELLED);
  s->created.clear();
  delete s;
}

}  // extern "C"
