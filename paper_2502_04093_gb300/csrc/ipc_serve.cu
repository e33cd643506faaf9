// Continuous-batching retrieval server of libipcomp (host runtime).
//
// Compressed fields stay resident on the device. Clients submit retrieve /
// refine / release requests; a worker thread admits them in arrival order
// while output memory (and free HBM) allows, groups everything admitted
// since the last launch into one batched reconstruction (one launch per
// interpolation level over all requests of an element type), and issues it
// on the next of its streams, so batches that arrive while others run
// overlap on the device. Completion is observed through CUDA events; each
// request's latency runs from submit to the moment its batch is seen done.
// A refine waits while its view has work in flight; its reconstruction is
// bitwise equal to a fresh retrieval of the same planes.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ipc.h"
#include "ipc_internal.h"
#include "ipc_serve_internal.h"

using Clock = std::chrono::steady_clock;

namespace {

const uint32_t kServerTag = 0x53435049u;

double us_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::micro>(b - a).count();
}

struct SView {
  ipc_field* f = nullptr;
  void* out = nullptr;
  uint64_t out_bytes = 0;
  std::vector<int> b;
  uint64_t bytes = 0;
  double bound = 0;
  int busy = 0;  // batches in flight that write `out`
  ipc_view* hv = nullptr;  // incremental servers: the view that refines `out`
};

// What a request's completion applies to its view: the new selection of a
// refine (taken only once its batch has finished without error).
struct NewSel {
  bool refine = false;
  bool incremental = false;  // refined through the view's own increment path
  ipc_target target{};
  std::vector<int> b;
  uint64_t bytes = 0;
  double bound = 0;
};

struct Pending {
  uint64_t ticket;
  ipc_request req;
  Clock::time_point t_submit;
};

struct Flight {
  cudaEvent_t done;
  std::vector<void*> tabs;  // device entry tables (freed when done)
  int stream;
  std::vector<Pending> reqs;
  std::vector<uint64_t> views;  // view of each request (0 if none)
  std::vector<NewSel> nsel;     // per request
  std::vector<int> status;
  Clock::time_point t_launch;
};

}  // namespace

struct ipc_server {
  uint32_t tag;
  int device;
  ipc_server_cfg cfg;
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  std::mutex mu;
  std::condition_variable cv_in, cv_out;
  std::deque<Pending> incoming;
  std::deque<ipc_completion> done;
  std::deque<Pending> pending;  // worker-owned
  std::deque<Flight> flights;   // worker-owned
  std::map<uint64_t, SView> views;
  uint64_t next_ticket = 1, next_view = 1;
  uint64_t mem_used = 0;
  std::atomic<bool> stop{false};
  std::thread worker;
  uint64_t batches = 0, launched_requests = 0;
};

namespace {

void complete(ipc_server* s, const Pending& p, int status, uint64_t view, const SView* v,
              Clock::time_point t_launch, Clock::time_point now) {
  ipc_completion c{};
  c.ticket = p.ticket;
  c.user_tag = p.req.user_tag;
  c.status = status;
  c.view_id = view;
  c.d_out = v ? v->out : nullptr;
  c.bytes = v ? v->bytes : 0;
  c.bound = v ? v->bound : 0;
  c.latency_us = us_since(p.t_submit, now);
  c.queue_us = us_since(p.t_submit, t_launch);
  std::lock_guard<std::mutex> lk(s->mu);
  s->done.push_back(c);
  s->cv_out.notify_all();
}

// Harvests finished batches, each as soon as it is done (batches on
// different streams finish out of launch order: a small batch behind a large
// one on another stream completes first).
void reap(ipc_server* s) {
  for (auto fit = s->flights.begin(); fit != s->flights.end();) {
    Flight& fl = *fit;
    const cudaError_t q = cudaEventQuery(fl.done);
    if (q == cudaErrorNotReady) {
      ++fit;
      continue;
    }
    const Clock::time_point now = Clock::now();
    for (size_t i = 0; i < fl.reqs.size(); ++i) {
      auto it = s->views.find(fl.views[i]);
      SView* v = it == s->views.end() ? nullptr : &it->second;
      const int st = q == cudaSuccess ? fl.status[i] : IPC_ECUDA;
      if (v) {
        v->busy -= 1;
        const NewSel& ns = fl.nsel[i];
        if (ns.refine && st == IPC_OK) {
          if (ns.incremental) {
            ipc_internal_view_selection(v->hv, &v->b, &v->bytes, &v->bound);
          } else {
            v->b = ns.b;
            v->bytes = ns.bytes;
            v->bound = ns.bound;
          }
        } else if (ns.refine && ns.incremental) {
          // the output and the view's state may be half updated: the next
          // refinement reconstructs (and records the state again)
          ipc_view_set_refine_mode(v->hv, IPC_REFINE_CANONICAL);
          ipc_view_set_refine_mode(v->hv, IPC_REFINE_INCREMENTAL);
        }
      }
      complete(s, fl.reqs[i], st, fl.views[i], v, fl.t_launch, now);
    }
    for (void* t : fl.tabs) cudaFreeAsync(t, s->streams[fl.stream]);
    cudaEventDestroy(fl.done);
    fit = s->flights.erase(fit);
  }
}

// The stream of the next batch: one with no batch in flight, the round-robin
// one first (a batch queued behind another on the same stream would wait
// for it); the round-robin one when every stream is busy.
int pick_stream(const ipc_server* s) {
  const int n = (int)s->streams.size();
  for (int k = 0; k < n; ++k) {
    const int c = (s->next_stream + k) % n;
    bool busy = false;
    for (const Flight& fl : s->flights) busy |= fl.stream == c;
    if (!busy) return c;
  }
  return s->next_stream;
}

// Admits pending requests (arrival order) and launches one batch.
void admit_and_launch(ipc_server* s) {
  if (s->pending.empty()) return;
  if ((int)s->flights.size() >= s->cfg.max_inflight) return;
  const int maxb = s->cfg.max_batch > 0 ? s->cfg.max_batch : 1 << 30;
  std::vector<Pending> take;
  std::vector<uint64_t> vid;
  std::vector<std::vector<int>> sel;
  std::vector<NewSel> nsel;
  std::vector<int> status;
  std::deque<Pending> keep;
  bool blocked = false;
  uint64_t values = 0;  // output elements of the batch so far
  const uint64_t maxv = s->cfg.max_batch_values;
  std::vector<uint64_t> touched;
  const int sidx = pick_stream(s);  // output buffers are allocated on the batch's stream
  size_t free_hbm = 0, total_hbm = 0;
  cudaMemGetInfo(&free_hbm, &total_hbm);
  while (!s->pending.empty()) {
    Pending p = s->pending.front();
    s->pending.pop_front();
    // memory waits block only later requests that need memory: releases
    // (which free it) and refines (which reuse their buffer) go on
    if ((blocked && p.req.kind == IPC_REQ_RETRIEVE) || (int)take.size() >= maxb) {
      keep.push_back(p);
      continue;
    }
    // the batch's size limit: a request that would pass it waits (and keeps
    // its place) for the next batch; the first request of a batch always goes
    if (maxv && !take.empty() && p.req.kind != IPC_REQ_RELEASE) {
      uint64_t nv = 0;
      int dt = 0;
      if (p.req.kind == IPC_REQ_RETRIEVE && p.req.field) ipc_internal_field_shape(p.req.field, &nv, &dt);
      if (p.req.kind == IPC_REQ_REFINE) {
        auto it = s->views.find(p.req.view_id);
        if (it != s->views.end()) ipc_internal_field_shape(it->second.f, &nv, &dt);
      }
      if (values + nv > maxv) {
        blocked = true;  // later retrieves keep arrival order behind it
        keep.push_back(p);
        continue;
      }
    }
    const Clock::time_point now = Clock::now();
    const ipc_request& r = p.req;
    if (r.kind == IPC_REQ_RELEASE) {
      auto it = s->views.find(r.view_id);
      if (it == s->views.end()) {
        complete(s, p, IPC_EINVAL, 0, nullptr, now, now);
        continue;
      }
      if (it->second.busy || std::find(touched.begin(), touched.end(), r.view_id) != touched.end()) {
        keep.push_back(p);  // wait for the view's work
        continue;
      }
      if (it->second.out) cudaFreeAsync(it->second.out, s->streams[0]);
      if (it->second.hv) ipc_free(it->second.hv);
      s->mem_used -= it->second.out_bytes;
      s->views.erase(it);
      complete(s, p, IPC_OK, r.view_id, nullptr, now, now);
      continue;
    }
    if (r.kind == IPC_REQ_REFINE) {
      auto it = s->views.find(r.view_id);
      if (it == s->views.end()) {
        complete(s, p, IPC_EINVAL, 0, nullptr, now, now);
        continue;
      }
      SView& v = it->second;
      if (v.busy || std::find(touched.begin(), touched.end(), r.view_id) != touched.end()) {
        keep.push_back(p);  // in arrival order per view: later work waits too
        continue;
      }
      std::vector<int> nb;
      uint64_t nbytes = 0;
      double nbound = 0;
      int rc = ipc_internal_select(v.f, r.target, &v.b, &nb, &nbytes, &nbound);
      if (rc == IPC_EBUDGET && r.target.kind == IPC_TARGET_BITRATE) {
        complete(s, p, IPC_OK, r.view_id, &v, now, now);  // already beyond the budget
        continue;
      }
      if (rc) {
        complete(s, p, rc, r.view_id, &v, now, now);
        continue;
      }
      if (nb == v.b) {
        complete(s, p, IPC_OK, r.view_id, &v, now, now);  // target already met
        continue;
      }
      NewSel ns;  // applied when the batch is done
      ns.refine = true;
      ns.incremental = v.hv != nullptr;
      ns.target = r.target;
      ns.b = nb;
      ns.bytes = nbytes;
      ns.bound = nbound;
      nsel.push_back(ns);
      {
        uint64_t nv = 0;
        int dt = 0;
        ipc_internal_field_shape(v.f, &nv, &dt);
        values += nv;
      }
      take.push_back(p);
      vid.push_back(r.view_id);
      sel.push_back(nb);
      status.push_back(IPC_OK);
      touched.push_back(r.view_id);
      continue;
    }
    // retrieve: a new view with its own output buffer
    if (!r.field) {
      complete(s, p, IPC_EINVAL, 0, nullptr, now, now);
      continue;
    }
    uint64_t n = 1;
    int dtype = 0;
    ipc_internal_field_shape(r.field, &n, &dtype);
    const uint64_t need = ((n * (dtype == 0 ? 4 : 8) + 255) / 256) * 256;
    if (need > s->cfg.mem_budget) {
      complete(s, p, IPC_ENOMEM, 0, nullptr, now, now);  // can never fit
      continue;
    }
    const uint64_t reserve = s->cfg.hbm_reserve;
    if (s->mem_used + need > s->cfg.mem_budget || need + reserve > free_hbm) {
      blocked = true;  // head of line waits for memory
      keep.push_back(p);
      continue;
    }
    std::vector<int> nb;
    uint64_t nbytes = 0;
    double nbound = 0;
    uint64_t rparts[2] = {0, 0};
    int rc = ipc_internal_select(r.field, r.target, nullptr, &nb, &nbytes, &nbound, rparts);
    if (rc) {
      complete(s, p, rc, 0, nullptr, now, now);
      continue;
    }
    ipc_view* hv = nullptr;
    if (ipc_internal_refine_mode(r.field, s->cfg.refine_mode) == IPC_REFINE_INCREMENTAL) {
      hv = ipc_internal_view_make(r.field, nb, nbytes, nbound, rparts[0], IPC_REFINE_INCREMENTAL);
      if (!hv) {
        complete(s, p, IPC_ENOMEM, 0, nullptr, now, now);
        continue;
      }
    }
    void* out = nullptr;
    if (cudaMallocAsync(&out, need, s->streams[sidx]) != cudaSuccess) {
      cudaGetLastError();
      if (hv) ipc_free(hv);
      blocked = true;
      keep.push_back(p);
      continue;
    }
    free_hbm = free_hbm > need ? free_hbm - need : 0;
    s->mem_used += need;
    const uint64_t id = s->next_view++;
    SView v;
    v.f = r.field;
    v.out = out;
    v.out_bytes = need;
    v.b = nb;
    v.bytes = nbytes;
    v.bound = nbound;
    v.hv = hv;
    s->views[id] = v;
    take.push_back(p);
    vid.push_back(id);
    sel.push_back(nb);
    nsel.push_back(NewSel());
    status.push_back(IPC_OK);
    touched.push_back(id);
    values += n;
  }
  s->pending = std::move(keep);
  if (take.empty()) return;
  s->next_stream = (sidx + 1) % (int)s->streams.size();
  cudaStream_t st = s->streams[sidx];
  Flight fl;
  fl.stream = sidx;
  fl.reqs = take;
  fl.views = vid;
  fl.status = status;
  fl.t_launch = Clock::now();
  std::vector<ipc_field*> fs;
  std::vector<void*> outs;
  std::vector<std::vector<int>> bsel;
  std::vector<size_t> inc;  // refines of incremental views: through the view
  for (size_t i = 0; i < take.size(); ++i) {
    SView& v = s->views[vid[i]];
    v.busy += 1;
    if (nsel[i].incremental) {
      inc.push_back(i);
      continue;
    }
    fs.push_back(v.f);
    outs.push_back(v.out);
    bsel.push_back(sel[i]);
  }
  int rc = IPC_OK;
  // a batch of one takes the single-field path (no entry table to upload)
  if (!fs.empty()) {
    if (s->cfg.plain || fs.size() == 1) rc = ipc_internal_reconstruct_each(fs, bsel, outs, st);
    else rc = ipc_internal_reconstruct_batch(fs, bsel, outs, st, &fl.tabs);
  }
  if (rc)
    for (size_t i = 0; i < take.size(); ++i)
      if (!nsel[i].incremental) fl.status[i] = rc;
  for (size_t i : inc) {
    // the same constrained selection; the increment when its bound allows,
    // else a reconstruction that records the view's state
    SView& v = s->views[vid[i]];
    fl.status[i] = ipc_refine(v.hv, nsel[i].target, v.out, st);
  }
  fl.nsel = std::move(nsel);
  cudaEventCreateWithFlags(&fl.done, cudaEventDisableTiming);
  cudaEventRecord(fl.done, st);
  s->batches += 1;
  s->launched_requests += take.size();
  s->flights.push_back(std::move(fl));
}

void worker_main(ipc_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->incoming.empty() && s->pending.empty() && s->flights.empty()) {
        if (s->stop.load()) break;
        s->cv_in.wait_for(lk, std::chrono::microseconds(200));
      }
      while (!s->incoming.empty()) {
        s->pending.push_back(s->incoming.front());
        s->incoming.pop_front();
      }
    }
    reap(s);
    admit_and_launch(s);
    if (!s->flights.empty() && (s->pending.empty() || (int)s->flights.size() >= s->cfg.max_inflight))
      std::this_thread::yield();
    if (s->stop.load() && s->flights.empty()) {
      // shutting down: what cannot be admitted any more is cancelled
      {
        std::lock_guard<std::mutex> lk(s->mu);
        while (!s->incoming.empty()) {
          s->pending.push_back(s->incoming.front());
          s->incoming.pop_front();
        }
      }
      admit_and_launch(s);
      if (!s->flights.empty()) continue;
      const Clock::time_point now = Clock::now();
      while (!s->pending.empty()) {
        complete(s, s->pending.front(), IPC_EBUSY, 0, nullptr, now, now);
        s->pending.pop_front();
      }
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->incoming.empty()) break;
    }
  }
}

}  // namespace

extern "C" {

int ipc_server_create(const ipc_server_cfg* cfg, ipc_server** out) {
  if (!cfg || !out || cfg->nstreams < 1 || cfg->nstreams > 16 || cfg->max_inflight < 1 ||
      cfg->refine_mode < IPC_REFINE_CANONICAL || cfg->refine_mode > IPC_REFINE_AUTO)
    return IPC_EINVAL;
  ipc_server* s = new (std::nothrow) ipc_server();
  if (!s) return IPC_ENOMEM;
  s->tag = kServerTag;
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  for (int i = 0; i < cfg->nstreams; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (auto x : s->streams) cudaStreamDestroy(x);
      delete s;
      return IPC_ECUDA;
    }
    s->streams.push_back(st);
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return IPC_OK;
}

int ipc_server_submit(ipc_server* s, const ipc_request* r, uint64_t* ticket) {
  if (!s || s->tag != kServerTag || !r) return IPC_EINVAL;
  if (r->kind != IPC_REQ_RETRIEVE && r->kind != IPC_REQ_REFINE && r->kind != IPC_REQ_RELEASE)
    return IPC_EINVAL;
  if (s->stop.load()) return IPC_EBUSY;
  Pending p;
  p.req = *r;
  p.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    p.ticket = s->next_ticket++;
    s->incoming.push_back(p);
  }
  s->cv_in.notify_one();
  if (ticket) *ticket = p.ticket;
  return IPC_OK;
}

int ipc_server_poll(ipc_server* s, ipc_completion* out, int max, int* n, int timeout_us) {
  if (!s || s->tag != kServerTag || !n || (max > 0 && !out)) return IPC_EINVAL;
  *n = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && timeout_us > 0)
    s->cv_out.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !s->done.empty(); });
  while (*n < max && !s->done.empty()) {
    out[(*n)++] = s->done.front();
    s->done.pop_front();
  }
  return (*n == 0 && timeout_us > 0) ? IPC_ETIMEOUT : IPC_OK;
}

int ipc_server_stats(ipc_server* s, uint64_t* batches, uint64_t* requests, uint64_t* mem_used) {
  if (!s || s->tag != kServerTag) return IPC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->batches;
  if (requests) *requests = s->launched_requests;
  if (mem_used) *mem_used = s->mem_used;
  return IPC_OK;
}

int ipc_server_stop(ipc_server* s) {
  if (!s || s->tag != kServerTag) return IPC_EINVAL;
  s->stop.store(true);
  s->cv_in.notify_all();
  if (s->worker.joinable()) s->worker.join();
  return IPC_OK;
}

int ipc_server_destroy(ipc_server* s) {
  if (!s) return IPC_OK;
  if (s->tag != kServerTag) return IPC_EINVAL;
  ipc_server_stop(s);
  for (auto st : s->streams) cudaStreamSynchronize(st);
  for (auto& kv : s->views) {
    if (kv.second.out) cudaFreeAsync(kv.second.out, s->streams[0]);
    if (kv.second.hv) ipc_free(kv.second.hv);
  }
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  s->tag = 0;
  delete s;
  return IPC_OK;
}

}  // extern "C"
