// Request server (include/hps_serve.h): resident operators, batched solves
// on a pool of CUDA streams, builds on a separate host thread, admission of
// builds by planned device footprint.
//
// Threads.  The scheduler thread owns the slots and the streams: it moves
// submitted requests into per-slot FIFOs, completes finished batches
// (cudaEventQuery), and dispatches the head of every idle slot: a run of up
// to max_batch solve requests (all with or all without a new source) becomes
// one hps_solve_batched on a free stream; a build is handed to the builder
// thread.  Only one batch or build per slot is in flight, which keeps each
// handle single-threaded, as hps.h requires.  Each builder thread runs
// hps_build on its own stream and releases the slot's previous operator
// (hps_free waits for that operator's last work, so that wait is kept off
// the scheduler);
// with several builders a small rebuild does not wait behind a large one.
// Handle memory and staging buffers are stream-ordered (devmem.h), so builds,
// frees and buffer growth never wait for the solves on other streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "devmem.h"
#include "hps.h"
#include "hps_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  int64_t id = 0;
  int kind = 0;  // 0 solve, 1 build
  int slot = 0;
  // solve
  const void* g = nullptr;
  const void* f = nullptr;
  void* u = nullptr;
  // build
  hps_tree tree{};
  int p = 0, q = 0;
  hps_coeffs cf{};
  const void* fb = nullptr;
  hps_options opts{};
  bool has_opts = false;
  // result
  int status = HPS_PENDING;
  int batch = 0;
  double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
};

struct Slot {
  hps_handle* h = nullptr;
  bool iti = false;
  int64_t n_root = 0, n_pts = 0;  // g entries, u / f entries
  int64_t bytes = 0;
  std::deque<Req*> q;
  bool busy = false;
};

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct StreamCtx {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  DevBuf dg, df, du;  // device
  DevBuf hg, hf, hu;  // pinned host
  std::vector<Req*> batch;     // requests in flight, in staging order
  std::vector<size_t> uoff;    // byte offset of each request's u in hu
  std::vector<size_t> ubytes;  // its size
  std::vector<int> slots;      // slots whose work is in flight here
  bool busy = false;
};

// Device staging buffers of a stream: allocated and freed in that stream's
// order (a regrowth does not wait for the other streams).
bool grow_dev(DevBuf& b, size_t bytes, cudaStream_t st) {
  if (b.cap >= bytes) return true;
  if (b.p) hps::dev_free(b.p, st);
  b.p = nullptr;
  b.cap = 0;
  if (hps::dev_malloc(&b.p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return false;
  }
  // A stream-ordered allocation is mapped when its stream reaches it; until
  // then a pointer query (the solve entry points' device-pointer check) may
  // not recognise it.  The stream is idle here (it is the free stream a
  // dispatch picked), so waiting for it costs next to nothing.
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    hps::dev_free(b.p, st);
    b.p = nullptr;
    return false;
  }
  b.cap = bytes;
  return true;
}

bool grow_host(DevBuf& b, size_t bytes) {
  if (b.cap >= bytes) return true;
  if (b.p) cudaFreeHost(b.p);
  b.p = nullptr;
  b.cap = 0;
  if (cudaHostAlloc(&b.p, bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  b.cap = bytes;
  return true;
}

}  // namespace

struct hps_server {
  hps_server_options opts{};
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done, cv_build;
  std::deque<Req*> incoming;
  std::unordered_map<int64_t, Req*> reqs;
  int64_t next_id = 1;
  std::vector<Slot> slots;
  std::vector<StreamCtx> streams;
  std::thread sched;
  bool stop = false;          // destroy: the scheduler drains, then exits
  bool builder_stop = false;  // set once the scheduler has exited
  int64_t outstanding = 0;    // submitted, not yet finished
  // builder hand-off (under mu)
  struct BuildJob {
    Req* r = nullptr;
    hps_handle* old = nullptr;  // the slot's operator while the build runs
    bool free_first = false;    // old released before building (memory)
    int64_t need = 0;           // reserved bytes
    hps_handle* out = nullptr;
    hps_status status = HPS_OK;
  };
  std::deque<BuildJob*> build_queue;
  std::vector<BuildJob*> build_done_list;
  int active_builds = 0;
  std::vector<std::thread> builders;
  // accounting
  int64_t resident = 0;
  hps_server_stats stats{};

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }
};

namespace {

void finish(hps_server* s, Req* r, int status) {
  std::lock_guard<std::mutex> lk(s->mu);
  r->status = status;
  r->t_done = s->now_ms();
  --s->outstanding;
  if (r->kind == 0 && status == HPS_OK) ++s->stats.solves;
  if (r->kind == 1 && status == HPS_OK) ++s->stats.builds;
  s->cv_done.notify_all();
}

// Dispatch a batch of solve requests of one slot onto a free stream.
void dispatch_solves(hps_server* s, int si, StreamCtx& sc) {
  Slot& sl = s->slots[si];
  const bool with_f = sl.q.front()->f != nullptr;
  std::vector<Req*> b;
  while (!sl.q.empty() && (int)b.size() < s->opts.max_batch) {
    Req* r = sl.q.front();
    if (r->kind != 0 || (r->f != nullptr) != with_f) break;
    b.push_back(r);
    sl.q.pop_front();
  }
  const size_t es = sl.iti ? 16 : 8;
  const size_t gb = (size_t)sl.n_root * es, ub = (size_t)sl.n_pts * es;
  const int nb = (int)b.size();
  bool ok = grow_dev(sc.dg, gb * nb, sc.s) && grow_dev(sc.du, ub * nb, sc.s) && grow_host(sc.hg, gb * nb) &&
            grow_host(sc.hu, ub * nb);
  if (ok && with_f) ok = grow_dev(sc.df, ub * nb, sc.s) && grow_host(sc.hf, ub * nb);
  hps_status st = ok ? HPS_OK : HPS_ERR_OOM;
  const double t = s->now_ms();
  if (st == HPS_OK) {
    for (int i = 0; i < nb; ++i) {
      std::memcpy((char*)sc.hg.p + i * gb, b[i]->g, gb);
      if (with_f) std::memcpy((char*)sc.hf.p + i * ub, b[i]->f, ub);
      b[i]->t_start = t;
      b[i]->batch = nb;
    }
    if (cudaMemcpyAsync(sc.dg.p, sc.hg.p, gb * nb, cudaMemcpyHostToDevice, sc.s) != cudaSuccess ||
        (with_f && cudaMemcpyAsync(sc.df.p, sc.hf.p, ub * nb, cudaMemcpyHostToDevice, sc.s) != cudaSuccess))
      st = HPS_ERR_CUDA;
  }
  if (st == HPS_OK)
    st = hps_solve_batched(sl.h, nb, sc.dg.p, with_f ? sc.df.p : nullptr, sc.du.p, sc.s);
  if (st == HPS_OK &&
      (cudaMemcpyAsync(sc.hu.p, sc.du.p, ub * nb, cudaMemcpyDeviceToHost, sc.s) != cudaSuccess ||
       cudaEventRecord(sc.ev, sc.s) != cudaSuccess))
    st = HPS_ERR_CUDA;
  if (st != HPS_OK) {
    cudaGetLastError();
    for (Req* r : b) finish(s, r, st);
    return;
  }
  sc.uoff.clear();
  sc.ubytes.clear();
  for (int i = 0; i < nb; ++i) {
    sc.uoff.push_back((size_t)i * ub);
    sc.ubytes.push_back(ub);
  }
  sc.batch = std::move(b);
  sc.slots.assign(1, si);
  sc.busy = true;
  sl.busy = true;
  std::lock_guard<std::mutex> lk(s->mu);
  ++s->stats.batches;
  s->stats.max_batch_seen = std::max<int64_t>(s->stats.max_batch_seen, nb);
}

// Dispatch the apply-only solves (build-time source) waiting at the heads of
// several slots as one hps_solve_multi on a free stream: up to max_batch
// requests per slot, up to max_group slots, whatever their depths, orders
// and kinds.  The operators' downward passes then share their launches.
void dispatch_group(hps_server* s, const std::vector<int>& cand, StreamCtx& sc) {
  std::vector<int> gs;
  std::vector<std::vector<Req*>> reqs;
  for (int si : cand) {
    if ((int)gs.size() >= s->opts.max_group) break;
    Slot& sl = s->slots[si];
    std::vector<Req*> b;
    while (!sl.q.empty() && (int)b.size() < s->opts.max_batch) {
      Req* r = sl.q.front();
      if (r->kind != 0 || r->f != nullptr) break;
      b.push_back(r);
      sl.q.pop_front();
    }
    if (b.empty()) continue;
    gs.push_back(si);
    reqs.push_back(std::move(b));
  }
  const int n = (int)gs.size();
  if (n == 0) return;
  // staging layout: per slot its requests' g (and u) back to back
  std::vector<size_t> goff(n), uoff_slot(n);
  size_t gtot = 0, utot = 0;
  for (int k = 0; k < n; ++k) {
    const Slot& sl = s->slots[gs[k]];
    const size_t es = sl.iti ? 16 : 8;
    goff[k] = gtot;
    uoff_slot[k] = utot;
    gtot += (size_t)sl.n_root * es * reqs[k].size();
    utot += (size_t)sl.n_pts * es * reqs[k].size();
  }
  bool ok = grow_dev(sc.dg, gtot, sc.s) && grow_dev(sc.du, utot, sc.s) && grow_host(sc.hg, gtot) &&
            grow_host(sc.hu, utot);
  hps_status st = ok ? HPS_OK : HPS_ERR_OOM;
  const double t = s->now_ms();
  std::vector<hps_handle*> hs(n);
  std::vector<int> nrhs(n);
  std::vector<const void*> gp(n);
  std::vector<void*> up(n);
  sc.batch.clear();
  sc.uoff.clear();
  sc.ubytes.clear();
  int nreq = 0;
  for (int k = 0; k < n; ++k) {
    const Slot& sl = s->slots[gs[k]];
    const size_t es = sl.iti ? 16 : 8;
    const size_t gb = (size_t)sl.n_root * es, ub = (size_t)sl.n_pts * es;
    for (size_t i = 0; i < reqs[k].size(); ++i) {
      Req* r = reqs[k][i];
      if (st == HPS_OK) std::memcpy((char*)sc.hg.p + goff[k] + i * gb, r->g, gb);
      r->t_start = t;
      r->batch = (int)reqs[k].size();
      sc.batch.push_back(r);
      sc.uoff.push_back(uoff_slot[k] + i * ub);
      sc.ubytes.push_back(ub);
      ++nreq;
    }
    hs[k] = sl.h;
    nrhs[k] = (int)reqs[k].size();
    gp[k] = (const char*)sc.dg.p + goff[k];
    up[k] = (char*)sc.du.p + uoff_slot[k];
  }
  if (st == HPS_OK && cudaMemcpyAsync(sc.dg.p, sc.hg.p, gtot, cudaMemcpyHostToDevice, sc.s) != cudaSuccess)
    st = HPS_ERR_CUDA;
  if (st == HPS_OK) st = hps_solve_multi(n, hs.data(), nrhs.data(), gp.data(), up.data(), sc.s);
  if (st == HPS_OK && (cudaMemcpyAsync(sc.hu.p, sc.du.p, utot, cudaMemcpyDeviceToHost, sc.s) != cudaSuccess ||
                       cudaEventRecord(sc.ev, sc.s) != cudaSuccess))
    st = HPS_ERR_CUDA;
  if (st != HPS_OK) {
    cudaGetLastError();
    std::vector<Req*> b = std::move(sc.batch);
    sc.batch.clear();
    for (Req* r : b) finish(s, r, st);
    return;
  }
  sc.slots = gs;
  sc.busy = true;
  for (int si : gs) s->slots[si].busy = true;
  std::lock_guard<std::mutex> lk(s->mu);
  ++s->stats.batches;
  if (n > 1) ++s->stats.multi_batches;
  s->stats.max_batch_seen = std::max<int64_t>(s->stats.max_batch_seen, nreq);
  s->stats.max_group_seen = std::max<int64_t>(s->stats.max_group_seen, n);
}

void complete_batch(hps_server* s, StreamCtx& sc) {
  const cudaError_t e = cudaEventQuery(sc.ev);
  if (e == cudaErrorNotReady) return;
  const int st = e == cudaSuccess ? HPS_OK : HPS_ERR_CUDA;
  if (e != cudaSuccess) cudaGetLastError();
  for (size_t i = 0; i < sc.batch.size(); ++i) {
    Req* r = sc.batch[i];
    if (st == HPS_OK) std::memcpy(r->u, (const char*)sc.hu.p + sc.uoff[i], sc.ubytes[i]);
    finish(s, r, st);
  }
  sc.batch.clear();
  for (int si : sc.slots) s->slots[si].busy = false;
  sc.slots.clear();
  sc.busy = false;
}

// Hand the build at the head of slot si to a builder, if memory admits it.
// Returns false when nothing changed (every builder busy, or waiting for
// memory that builds in flight still hold).
bool dispatch_build(hps_server* s, int si) {
  Slot& sl = s->slots[si];
  Req* r = sl.q.front();
  int64_t need = 0;
  hps_status st = hps_plan_bytes(&r->tree, r->p, r->q, r->cf.kind, &need);
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->active_builds >= s->opts.n_builders) return false;
  if (st != HPS_OK) {
    sl.q.pop_front();
    lk.unlock();
    finish(s, r, st);
    return true;
  }
  bool free_first = false;
  if (s->resident + need > s->opts.hbm_budget) {
    if (sl.h && s->resident - sl.bytes + need <= s->opts.hbm_budget) {
      free_first = true;
    } else if (s->active_builds > 0) {
      return false;  // memory reserved by builds in flight comes back when they end
    } else {
      sl.q.pop_front();
      lk.unlock();
      finish(s, r, HPS_ERR_OOM);
      return true;
    }
  }
  sl.q.pop_front();
  r->t_start = s->now_ms();
  hps_server::BuildJob* job = new hps_server::BuildJob();
  job->r = r;
  job->old = sl.h;
  job->free_first = free_first;
  job->need = need;
  if (free_first) {
    s->resident -= sl.bytes;
    sl.h = nullptr;
    sl.bytes = 0;
  }
  s->resident += need;  // reserved until the build reports its real size
  sl.busy = true;
  ++s->active_builds;
  s->build_queue.push_back(job);
  s->cv_build.notify_one();
  return true;
}

void complete_builds(hps_server* s) {
  std::vector<hps_server::BuildJob*> done;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    done.swap(s->build_done_list);
    for (hps_server::BuildJob* job : done) {
      Req* r = job->r;
      --s->active_builds;
      s->resident -= job->need;
      Slot& sl = s->slots[r->slot];
      if (job->status == HPS_OK) {
        if (!job->free_first && job->old) {  // the builder released it after building
          s->resident -= sl.bytes;
          sl.h = nullptr;
          sl.bytes = 0;
        }
        sl.h = job->out;
        sl.bytes = hps_device_bytes(job->out);
        sl.iti = r->cf.kind == HPS_ITI;
        int64_t nl = 0, ppl = 0, nr = 0;
        hps_sizes(&r->tree, r->p, r->q, &nl, &ppl, &nr);
        sl.n_root = nr;
        sl.n_pts = nl * ppl;
        s->resident += sl.bytes;
      }
      sl.busy = false;
    }
  }
  for (hps_server::BuildJob* job : done) {
    finish(s, job->r, job->status);
    delete job;
  }
}

void builder_main(hps_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t bs = nullptr;
  cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
  for (;;) {
    hps_server::BuildJob* job = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_build.wait(lk, [&] { return s->builder_stop || !s->build_queue.empty(); });
      if (s->build_queue.empty()) break;  // builder_stop
      job = s->build_queue.front();
      s->build_queue.pop_front();
    }
    Req* r = job->r;
    if (job->free_first && job->old) hps_free(job->old);
    hps_options o{};
    const hps_options* op = nullptr;
    if (r->has_opts) {
      op = &r->opts;
    } else {
      o.version = 1;
      o.lazy_root = s->opts.lazy_root;
      op = &o;
    }
    hps_handle* h = nullptr;
    hps_status st = hps_build(&r->tree, r->p, r->q, &r->cf, r->fb, op, bs, &h);
    if (st == HPS_ERR_SINGULAR && h) {
      hps_free(h);
      h = nullptr;
    }
    // on success the old operator goes; on failure the slot keeps it
    if (!job->free_first && job->old && st == HPS_OK) hps_free(job->old);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      job->out = h;
      job->status = st;
      s->build_done_list.push_back(job);
    }
    s->cv_sched.notify_all();
  }
  if (bs) cudaStreamDestroy(bs);
}

void sched_main(hps_server* s) {
  cudaSetDevice(s->device);
  size_t rr = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (!s->incoming.empty()) {
        Req* r = s->incoming.front();
        s->incoming.pop_front();
        s->slots[r->slot].q.push_back(r);
      }
      if (s->stop && s->outstanding == 0) break;
    }
    bool progress = false;
    bool inflight = false;
    for (StreamCtx& sc : s->streams) {
      if (!sc.busy) continue;
      complete_batch(s, sc);
      if (!sc.busy) progress = true;
      else inflight = true;
    }
    {
      bool bd;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        bd = !s->build_done_list.empty();
        inflight = inflight || s->active_builds > 0;
      }
      if (bd) {
        complete_builds(s);
        progress = true;
      }
    }
    const size_t ns = s->slots.size();
    auto free_stream = [&]() -> StreamCtx* {
      for (StreamCtx& sc : s->streams)
        if (!sc.busy) return &sc;
      return nullptr;
    };
    std::vector<int> apply_only;  // idle slots whose head is a solve with the build-time source
    for (size_t k = 0; k < ns; ++k) {
      const int si = (int)((rr + k) % ns);
      Slot& sl = s->slots[si];
      if (sl.busy || sl.q.empty()) continue;
      Req* head = sl.q.front();
      if (head->kind == 1) {
        if (dispatch_build(s, si)) progress = true;
        continue;
      }
      if (!sl.h) {
        sl.q.pop_front();
        finish(s, head, HPS_ERR_INVALID);
        progress = true;
        continue;
      }
      if (head->f == nullptr && s->opts.max_group > 1) {
        apply_only.push_back(si);
        continue;
      }
      StreamCtx* free_sc = free_stream();
      if (!free_sc) break;
      dispatch_solves(s, si, *free_sc);
      progress = true;
      inflight = true;
      rr = (size_t)si + 1;
    }
    if (!apply_only.empty()) {
      StreamCtx* free_sc = free_stream();
      if (free_sc) {
        dispatch_group(s, apply_only, *free_sc);
        progress = true;
        inflight = true;
        rr = (size_t)apply_only.back() + 1;
      }
    }
    if (!progress) {
      std::unique_lock<std::mutex> lk(s->mu);
      if (inflight)
        s->cv_sched.wait_for(lk, std::chrono::microseconds(20));
      else
        s->cv_sched.wait(lk, [&] { return s->stop || !s->incoming.empty() || !s->build_done_list.empty(); });
    }
  }
}

int64_t submit(hps_server* s, Req* r) {
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  r->t_submit = s->now_ms();
  s->reqs[r->id] = r;
  s->incoming.push_back(r);
  ++s->outstanding;
  s->cv_sched.notify_all();
  return r->id;
}

hps_status take(hps_server* s, int64_t ticket, hps_ticket_info* info, bool block) {
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return HPS_ERR_INVALID;
  Req* r = it->second;
  if (block) s->cv_done.wait(lk, [&] { return r->status != HPS_PENDING; });
  if (r->status == HPS_PENDING) return HPS_PENDING;
  if (info) {
    info->status = r->status;
    info->kind = r->kind;
    info->slot = r->slot;
    info->batch = r->batch;
    info->t_submit_ms = r->t_submit;
    info->t_start_ms = r->t_start;
    info->t_done_ms = r->t_done;
  }
  const hps_status st = (hps_status)r->status;
  s->reqs.erase(it);
  delete r;
  return st;
}

}  // namespace

extern "C" {

hps_status hps_server_create(const hps_server_options* opts, hps_server** out) {
  if (!out) return HPS_ERR_INVALID;
  *out = nullptr;
  hps_server_options o{};
  if (opts) o = *opts;
  else o.version = 1;
  if (o.version != 1) return HPS_ERR_INVALID;
  if (o.n_slots == 0) o.n_slots = 16;
  if (o.n_streams == 0) o.n_streams = 4;
  if (o.max_batch == 0) o.max_batch = 8;
  if (o.n_builders == 0) o.n_builders = 2;
  if (o.max_group == 0) o.max_group = 8;
  if (o.n_slots < 1 || o.n_slots > 1024 || o.n_streams < 1 || o.n_streams > 64 || o.max_batch < 1 ||
      o.max_batch > 256 || o.hbm_budget < 0 || o.n_builders < 1 || o.n_builders > 8 || o.max_group < 1 ||
      o.max_group > 24)
    return HPS_ERR_INVALID;
  hps_server* s = new (std::nothrow) hps_server();
  if (!s) return HPS_ERR_OOM;
  s->t0 = Clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return HPS_ERR_CUDA;
  }
  if (o.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return HPS_ERR_CUDA;
    }
    o.hbm_budget = (int64_t)(0.85 * (double)fr);
  }
  s->opts = o;
  s->stats.hbm_budget = o.hbm_budget;
  s->slots.resize((size_t)o.n_slots);
  s->streams.resize((size_t)o.n_streams);
  for (StreamCtx& sc : s->streams) {
    if (cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sc.ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (StreamCtx& c : s->streams) {
        if (c.s) cudaStreamDestroy(c.s);
        if (c.ev) cudaEventDestroy(c.ev);
      }
      delete s;
      return HPS_ERR_CUDA;
    }
  }
  s->sched = std::thread(sched_main, s);
  for (int i = 0; i < o.n_builders; ++i) s->builders.emplace_back(builder_main, s);
  *out = s;
  return HPS_OK;
}

void hps_server_destroy(hps_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  s->cv_build.notify_all();
  if (s->sched.joinable()) s->sched.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->builder_stop = true;
  }
  s->cv_build.notify_all();
  for (std::thread& b : s->builders)
    if (b.joinable()) b.join();
  cudaSetDevice(s->device);
  for (StreamCtx& sc : s->streams) {
    if (sc.s) cudaStreamSynchronize(sc.s);
    for (DevBuf* b : {&sc.dg, &sc.df, &sc.du})
      if (b->p) hps::dev_free(b->p, sc.s);
    if (sc.s) cudaStreamSynchronize(sc.s);
    for (DevBuf* b : {&sc.hg, &sc.hf, &sc.hu})
      if (b->p) cudaFreeHost(b->p);
    if (sc.ev) cudaEventDestroy(sc.ev);
    if (sc.s) cudaStreamDestroy(sc.s);
  }
  for (Slot& sl : s->slots) hps_free(sl.h);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
}

hps_status hps_server_submit_build(hps_server* s, int slot, const hps_tree* tree, int p, int q,
                                   const hps_coeffs* coeffs, const void* f, const hps_options* opts,
                                   int64_t* ticket) {
  if (!s || !tree || !coeffs || !ticket || slot < 0 || slot >= s->opts.n_slots) return HPS_ERR_INVALID;
  if (tree->uniform_depth < 0) return HPS_ERR_INVALID;
  Req* r = new (std::nothrow) Req();
  if (!r) return HPS_ERR_OOM;
  r->kind = 1;
  r->slot = slot;
  r->tree = *tree;
  r->p = p;
  r->q = q;
  r->cf = *coeffs;
  r->fb = f;
  if (opts) {
    r->opts = *opts;
    r->has_opts = true;
  }
  *ticket = submit(s, r);
  return HPS_OK;
}

hps_status hps_server_submit_solve(hps_server* s, int slot, const void* g, const void* f, void* u,
                                   int64_t* ticket) {
  if (!s || !g || !u || !ticket || slot < 0 || slot >= s->opts.n_slots) return HPS_ERR_INVALID;
  Req* r = new (std::nothrow) Req();
  if (!r) return HPS_ERR_OOM;
  r->kind = 0;
  r->slot = slot;
  r->g = g;
  r->f = f;
  r->u = u;
  *ticket = submit(s, r);
  return HPS_OK;
}

hps_status hps_server_wait(hps_server* s, int64_t ticket, hps_ticket_info* info) {
  if (!s) return HPS_ERR_INVALID;
  return take(s, ticket, info, true);
}

hps_status hps_server_poll(hps_server* s, int64_t ticket, hps_ticket_info* info) {
  if (!s) return HPS_ERR_INVALID;
  return take(s, ticket, info, false);
}

hps_status hps_server_get_stats(hps_server* s, hps_server_stats* out) {
  if (!s || !out) return HPS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->resident_bytes = s->resident;
  return HPS_OK;
}

hps_status hps_server_operator(hps_server* s, int slot, hps_handle** h) {
  if (!s || !h || slot < 0 || slot >= s->opts.n_slots) return HPS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  *h = s->slots[(size_t)slot].h;
  return HPS_OK;
}

}  // extern "C"
