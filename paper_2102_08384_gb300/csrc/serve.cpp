// Serving loop: continuous batching of estimator requests on one GPU.
//
// n worker slots, each owning an engine (its own stream, cuFFT plans and work
// area, geometry caches); the JIT kernel cache and the device memory pool are
// shared.  A slot that becomes free takes the first queued request whose
// projected footprint fits the remaining HBM budget, so requests arriving
// while others run are admitted as memory frees up, and work of different
// slots overlaps on the device.  Waits poll nothing on the GPU: completion is
// the worker returning from its synchronous request.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"

namespace bym {

namespace {
double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}
}  // namespace

struct ReqRec {
  uint64_t ticket = 0;
  bym_request req{};
  bym_result out{};
  bym_params p{};
  std::vector<double> kedges, redges;
  bym_bins kb{}, rb{};
  size_t footprint = 0;
  int status = 1;
  bool done = false;
  double t_submit = 0, t_start = 0, t_end = 0;
};

struct Server {
  bym_ctx *parent = nullptr;
  size_t budget = 0, in_use = 0, peak = 0;
  std::vector<bym_ctx *> engines;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<ReqRec>> queue;
  std::map<uint64_t, std::shared_ptr<ReqRec>> live;
  uint64_t next = 1;
  int running = 0;
  bool stopping = false;
  std::vector<double> lat_total, lat_run, lat_queue;

  void worker(int slot) {
    bym_ctx *eng = engines[slot];
    for (;;) {
      std::shared_ptr<ReqRec> r;
      {
        std::unique_lock<std::mutex> lock(mu);
        for (;;) {
          auto it = std::find_if(queue.begin(), queue.end(),
                                 [&](const std::shared_ptr<ReqRec> &q) { return in_use + q->footprint <= budget; });
          if (it != queue.end()) {
            r = *it;
            queue.erase(it);
            in_use += r->footprint;
            peak = std::max(peak, in_use);
            ++running;
            r->t_start = now_s();
            break;
          }
          if (stopping && queue.empty()) return;
          cv_work.wait(lock);
        }
      }
      Request rq{&r->req.gal,
                 r->req.ran.n > 0 ? &r->req.ran : nullptr,
                 &r->p,
                 r->kb.nbins > 0 ? &r->kb : nullptr,
                 r->rb.nbins > 0 ? &r->rb : nullptr,
                 r->out.pk,
                 r->out.k_mean,
                 r->out.n_modes,
                 r->out.xi,
                 r->out.r_mean,
                 r->out.n_cells};
      int rc;
      {
        std::lock_guard<std::mutex> elock(eng->mu);
        rc = run_request(eng, rq, eng->stream);
      }
      {
        std::lock_guard<std::mutex> lock(mu);
        in_use -= r->footprint;
        --running;
        r->status = rc;
        r->done = true;
        r->t_end = now_s();
        lat_total.push_back(r->t_end - r->t_submit);
        lat_run.push_back(r->t_end - r->t_start);
        lat_queue.push_back(r->t_start - r->t_submit);
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

void shutdown_serving(bym_ctx *c) {
  Server *s = c->server;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  for (bym_ctx *e : s->engines) bym_destroy(e);
  delete s;
  c->server = nullptr;
}

}  // namespace bym

using namespace bym;

static int serve_fail(bym_ctx *c, int code, const char *msg) {
  if (c) c->err = msg;
  return code;
}

extern "C" {

int bym_serve_start(bym_ctx *c, int n_slots, size_t budget) {
  if (!c) return BYM_E_INVAL;
  if (n_slots < 1 || n_slots > 16) return serve_fail(c, BYM_E_INVAL, "n_slots must be in 1..16");
  if (c->server) return serve_fail(c, BYM_E_BUSY, "a serving loop is already running");
  if (cudaSetDevice(c->device) != cudaSuccess) return serve_fail(c, BYM_E_CUDA, "cudaSetDevice failed");
  if (!budget) {   // 90 % of what requests can take: free memory and what the memory pool holds unused
    budget = (size_t)(0.9 * (double)device_available(c, 0));
    if (!budget) return serve_fail(c, BYM_E_CUDA, "no device memory available for serving");
  }
  auto *s = new Server();
  s->parent = c;
  s->budget = budget;
  for (int i = 0; i < n_slots; ++i) {
    bym_ctx *e = nullptr;
    if (bym_create(&e, c->device, 0) != BYM_OK) {
      for (bym_ctx *x : s->engines) bym_destroy(x);
      delete s;
      return serve_fail(c, BYM_E_CUDA, "could not create a serving slot");
    }
    // a slot runs requests exactly as the parent context would: its FFT backend, field ranges
    // and measured launch shapes
    e->fft_mode = c->fft_mode;
    e->field_chunk = c->field_chunk;
    {
      std::lock_guard<std::mutex> lock(c->mu);
      e->tune = c->tune;
    }
    s->engines.push_back(e);
  }
  c->server = s;
  for (int i = 0; i < n_slots; ++i) s->workers.emplace_back([s, i] {
    cudaSetDevice(s->parent->device);
    s->worker(i);
  });
  return BYM_OK;
}

int bym_serve_stop(bym_ctx *c) {
  if (!c) return BYM_E_INVAL;
  if (!c->server) return serve_fail(c, BYM_E_INVAL, "no serving loop");
  shutdown_serving(c);
  return BYM_OK;
}

int bym_submit(bym_ctx *c, const bym_request *req, const bym_result *out, uint64_t *ticket) {
  if (!c || !req || !out || !ticket) return BYM_E_INVAL;
  Server *s = c->server;
  if (!s) return serve_fail(c, BYM_E_INVAL, "no serving loop: call bym_serve_start");
  auto r = std::make_shared<ReqRec>();
  r->req = *req;
  r->out = *out;
  r->p = req->params;
  const bool want_pk = req->kbins.nbins > 0, want_xi = req->rbins.nbins > 0;
  if (want_pk) {
    if (!req->kbins.edges || !out->pk) return serve_fail(c, BYM_E_INVAL, "kbins without edges or pk output");
    r->kedges.assign(req->kbins.edges, req->kbins.edges + req->kbins.nbins + 1);
    r->kb = {r->kedges.data(), req->kbins.nbins};
  }
  if (want_xi) {
    if (!req->rbins.edges || !out->xi) return serve_fail(c, BYM_E_INVAL, "rbins without edges or xi output");
    r->redges.assign(req->rbins.edges, req->rbins.edges + req->rbins.nbins + 1);
    r->rb = {r->redges.data(), req->rbins.nbins};
  }
  if (!want_pk && !want_xi) return serve_fail(c, BYM_E_INVAL, "request asks for neither P nor xi");
  int rc = validate(c, &r->req.gal, r->req.ran.n > 0 ? &r->req.ran : nullptr, &r->p, want_pk ? &r->kb : nullptr,
                    want_xi ? &r->rb : nullptr);
  if (rc) return rc;
  r->footprint = footprint_bytes(&r->p, req->gal.n, req->ran.n, want_pk, want_xi,
                                 req->gal.on_device && (req->ran.n == 0 || req->ran.on_device));
  if (r->footprint > s->budget) return serve_fail(c, BYM_E_NOMEM, "request footprint exceeds the serving budget");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    r->ticket = s->next++;
    r->t_submit = now_s();
    s->queue.push_back(r);
    s->live[r->ticket] = r;
  }
  s->cv_work.notify_one();
  *ticket = r->ticket;
  return BYM_OK;
}

int bym_poll(bym_ctx *c, uint64_t ticket, int *done) {
  if (!c || !done || !c->server) return BYM_E_INVAL;
  Server *s = c->server;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->live.find(ticket);
  if (it == s->live.end()) return serve_fail(c, BYM_E_INVAL, "unknown ticket");
  *done = it->second->done ? 1 : 0;
  return BYM_OK;
}

int bym_wait(bym_ctx *c, uint64_t ticket, double timeout_s, int *status) {
  if (!c || !status || !c->server) return BYM_E_INVAL;
  Server *s = c->server;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->live.find(ticket);
  if (it == s->live.end()) return serve_fail(c, BYM_E_INVAL, "unknown ticket");
  std::shared_ptr<ReqRec> r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_s < 0)
    s->cv_done.wait(lock, pred);
  else if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), pred))
    return BYM_E_TIMEOUT;
  *status = r->status;
  if (r->status < 0) {
    std::lock_guard<std::mutex> elock(c->mu);
    c->err = "request " + std::to_string(ticket) + " failed with code " + std::to_string(r->status);
  }
  s->live.erase(ticket);
  return BYM_OK;
}

int bym_serve_stats(bym_ctx *c, double stats[7]) {
  if (!c || !stats || !c->server) return BYM_E_INVAL;
  Server *s = c->server;
  std::lock_guard<std::mutex> lock(s->mu);
  stats[0] = (double)s->lat_total.size();
  stats[1] = percentile(s->lat_total, 0.50);
  stats[2] = percentile(s->lat_total, 0.99);
  stats[3] = percentile(s->lat_run, 0.50);
  stats[4] = percentile(s->lat_run, 0.99);
  double q = 0.0;
  for (double v : s->lat_queue) q += v;
  stats[5] = s->lat_queue.empty() ? 0.0 : q / s->lat_queue.size();
  stats[6] = (double)s->peak;
  return BYM_OK;
}

int bym_serve_reset_stats(bym_ctx *c) {
  if (!c || !c->server) return BYM_E_INVAL;
  Server *s = c->server;
  std::lock_guard<std::mutex> lock(s->mu);
  s->lat_total.clear();
  s->lat_run.clear();
  s->lat_queue.clear();
  s->peak = s->in_use;
  return BYM_OK;
}

int bym_batch_run(bym_ctx *c, int n, const bym_request *reqs, const bym_result *outs, int *status) {
  if (!c || n < 0 || (n > 0 && (!reqs || !outs || !status))) return BYM_E_INVAL;
  const bool temporary = c->server == nullptr;
  if (temporary) {
    const int rc = bym_serve_start(c, 4, 0);
    if (rc) return rc;
  }
  std::vector<uint64_t> tickets(n, 0);
  int first_err = BYM_OK;
  for (int i = 0; i < n; ++i) {
    const int rc = bym_submit(c, &reqs[i], &outs[i], &tickets[i]);
    if (rc) {
      status[i] = rc;
      tickets[i] = 0;
      if (!first_err) first_err = rc;
    }
  }
  for (int i = 0; i < n; ++i)
    if (tickets[i]) {
      bym_wait(c, tickets[i], -1.0, &status[i]);
      if (status[i] && !first_err) first_err = status[i];
    }
  if (temporary) bym_serve_stop(c);
  return first_err;
}

}  // extern "C"
