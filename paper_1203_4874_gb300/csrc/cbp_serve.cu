// A9: serving engine -- continuous batching of independent deblurring
// requests (one frame pair each, any supported shape).
//
// Section 2 and 3 describe a camera that re-draws its pair of kernels for
// every frame; a server of many such cameras sees a stream of independent
// pairs of a few shapes.  The engine:
//   - takes requests from any thread (cbp_stream_submit copies the
//     descriptor and returns a ticket);
//   - groups pending requests by shape bucket (everything but the data
//     addresses agrees), oldest request first, up to kMaxBatch per batch;
//   - admits a batch when its workspace fits the context's HBM budget,
//     evicting idle cached batches first and halving the batch if it still
//     does not fit; a request that cannot fit even alone fails with
//     CBP_ERR_BUDGET;
//   - runs each batch on one of kSlots streams as a CUDA graph captured once
//     per (slot, bucket, batch size): the graph owns a fixed workspace and
//     reads the per-pair addresses from device tables that are refreshed
//     before each replay;
//   - notices completion by event polling, records per-request latency
//     (submit to completion) and wakes pollers.
// The kernels treat every pair of a batch independently, so a request's
// results do not depend on what it was batched with.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include "cbp_nvtx.h"
#include "cbp_serve.h"

namespace cbp {
namespace serve {

constexpr int kSlots = 4;          // concurrent batches, one stream each
constexpr int kMaxBatch = 16;      // requests per batch
constexpr int kCachePerSlot = 8;   // captured batches kept per slot
constexpr int kTables = 5;         // b1, b2, k1, k2, latent addresses
using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  cbp_frames b1{}, b2{};
  cbp_params prm{};
  void* k1 = nullptr;
  void* k2 = nullptr;
  void* lat = nullptr;
  Clock::time_point t0;
  bool done = false;
  cbp_status status = CBP_OK;
  cbp_diag diag{};
};

// Requests batch together when all of this agrees (zero-filled, compared
// bytewise).
struct Bucket {
  int64_t rs1, cs1, rs2, cs2;
  double eps, accept_rho;
  int32_t c, h1, w1, h2, w2, dtype;
  int32_t t1, t2, m, path, pad_h, pad_w, flags, deblur;
};
bool same(const Bucket& a, const Bucket& b) { return std::memcmp(&a, &b, sizeof(Bucket)) == 0; }

Bucket bucket_of(const Request& r) {
  Bucket k;
  std::memset(&k, 0, sizeof(k));
  auto strides = [](const cbp_frames& f, int64_t* rs, int64_t* cs) {
    *rs = f.row_stride ? f.row_stride : f.w;
    *cs = f.chan_stride ? f.chan_stride : (int64_t)f.h * *rs;
  };
  strides(r.b1, &k.rs1, &k.cs1);
  strides(r.b2, &k.rs2, &k.cs2);
  k.eps = r.prm.eps;
  k.accept_rho = r.prm.accept_rho;
  k.c = r.b1.c;
  k.h1 = r.b1.h;
  k.w1 = r.b1.w;
  k.h2 = r.b2.h;
  k.w2 = r.b2.w;
  k.dtype = r.b1.dtype;
  k.t1 = r.prm.t1;
  k.t2 = r.prm.t2;
  k.m = r.prm.m;
  k.path = r.prm.path;
  k.pad_h = r.prm.pad_h;
  k.pad_w = r.prm.pad_w;
  k.flags = r.prm.flags;
  k.deblur = r.lat != nullptr;
  return k;
}

// One captured batch: its workspace, the device address tables and the graph.
struct Entry {
  Bucket key;
  int B = 0;
  Plan plan;
  char* mem = nullptr;        // workspace followed by the tables
  size_t bytes = 0;
  uint64_t* tab = nullptr;    // device [kTables][B]
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;   // timing: the batch's start and end on the device
  uint64_t* tab_host = nullptr;   // pinned [kTables][kMaxBatch]
  cbp_diag* diag_host = nullptr;  // pinned [kMaxBatch]
  std::vector<Request*> batch;
  Entry* cur = nullptr;
  bool busy = false;
  std::vector<Entry*> cache;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace serve

using namespace serve;

struct ServeState {
  Ctx* ctx = nullptr;
  std::mutex mu;
  std::condition_variable wake;     // scheduler: new work or stop
  std::condition_variable done_cv;  // pollers: a request finished
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> tickets;
  uint64_t next_ticket = 1, tick = 0;
  Slot slots[kSlots];
  bool stop = false, ready = false;
  cbp_status init_status = CBP_OK;
  std::vector<double> lat_ms;
  uint64_t completed = 0;
  std::thread th;
  cudaEvent_t ref = nullptr;        // the engine's start on the device (batch timestamps)

  void finish(Request* r, cbp_status s, const cbp_diag* d, Clock::time_point now) {
    r->status = s;
    if (d) r->diag = *d;
    r->diag.status = s;
    r->done = true;
    lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t0).count());
    ++completed;
  }

  void free_entry(Slot& s, Entry* e) {
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->mem) cudaFreeAsync(e->mem, s.st);
    ctx->release(e->bytes);
    delete e;
  }

  // Free idle cached batches, least recently used first, until `bytes` more
  // would fit the budget (or nothing idle is left).
  void evict_for(size_t bytes) {
    for (;;) {
      {
        std::lock_guard<std::mutex> g(ctx->mem_mu);
        if (ctx->used + bytes <= ctx->budget) return;
      }
      Slot* bs = nullptr;
      size_t bi = 0;
      for (Slot& s : slots)
        for (size_t i = 0; i < s.cache.size(); ++i) {
          Entry* e = s.cache[i];
          if (s.busy && e == s.cur) continue;
          if (!bs || e->last_use < bs->cache[bi]->last_use) {
            bs = &s;
            bi = i;
          }
        }
      if (!bs) return;
      Entry* e = bs->cache[bi];
      bs->cache.erase(bs->cache.begin() + bi);
      free_entry(*bs, e);
    }
  }

  // Workspace + tables + captured graph for B requests shaped like r0.
  // Returns nullptr with *st == CBP_OK when the memory is not available now.
  Entry* create_entry(Slot& s, const Bucket& key, int B, const Request& r0, cbp_status* st) {
    *st = CBP_OK;
    cbp_frames f1 = r0.b1, f2 = r0.b2;
    f1.n = f2.n = B;
    f1.frame_stride = f2.frame_stride = 0;
    Plan p;
    cbp_status ps = make_plan(&f1, &f2, &r0.prm, &p);
    if (ps != CBP_OK) {
      *st = ps;
      return nullptr;
    }
    const size_t bytes = align256(p.total) + align256((size_t)kTables * B * sizeof(uint64_t));
    if (!ctx->reserve(bytes)) {
      evict_for(bytes);
      if (!ctx->reserve(bytes)) return nullptr;
    }
    Entry* e = new Entry();
    e->key = key;
    e->B = B;
    e->plan = p;
    e->bytes = bytes;
    if (cudaMallocAsync((void**)&e->mem, bytes, s.st) != cudaSuccess) {
      cudaGetLastError();
      e->mem = nullptr;
      ctx->release(bytes);
      delete e;
      return nullptr;
    }
    e->tab = (uint64_t*)(e->mem + align256(p.total));
    PtrTables t;
    t.b1 = e->tab;
    t.b2 = e->tab + B;
    t.k1 = e->tab + 2 * B;
    t.k2 = e->tab + 3 * B;
    t.lat = r0.lat ? e->tab + 4 * B : nullptr;
    cudaGraph_t g = nullptr;
    cbp_status rs = CBP_ERR_CUDA;
    if (cudaStreamBeginCapture(s.st, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      // the data addresses come from the tables; non-null placeholders
      // satisfy the argument checks
      rs = run_plan(p, &f1, &f2, &r0.prm, r0.k1, r0.k2, r0.lat, r0.lat != nullptr, e->mem, s.st,
                    nullptr, &t, ctx->cnn_w);
      if (cudaStreamEndCapture(s.st, &g) != cudaSuccess) rs = CBP_ERR_CUDA;
    }
    if (rs == CBP_OK && (!g || cudaGraphInstantiate(&e->exec, g, 0) != cudaSuccess)) rs = CBP_ERR_CUDA;
    if (g) cudaGraphDestroy(g);
    if (rs != CBP_OK) {
      cudaGetLastError();
      e->exec = nullptr;
      free_entry(s, e);
      *st = rs;
      return nullptr;
    }
    if ((int)s.cache.size() >= kCachePerSlot) {
      auto it = std::min_element(s.cache.begin(), s.cache.end(),
                                 [](Entry* a, Entry* b) { return a->last_use < b->last_use; });
      Entry* old = *it;
      s.cache.erase(it);
      free_entry(s, old);
    }
    s.cache.push_back(e);
    return e;
  }

  bool any_busy() const {
    for (const Slot& s : slots)
      if (s.busy) return true;
    return false;
  }

  void launch(Slot& s, Entry* e, std::vector<Request*>& batch) {
    NvtxScope range("cbp.serve_batch");
    const int B = e->B;
    for (int i = 0; i < B; ++i) {
      const Request* r = batch[i];
      s.tab_host[0 * B + i] = (uint64_t)r->b1.data;
      s.tab_host[1 * B + i] = (uint64_t)r->b2.data;
      s.tab_host[2 * B + i] = (uint64_t)r->k1;
      s.tab_host[3 * B + i] = (uint64_t)r->k2;
      s.tab_host[4 * B + i] = (uint64_t)r->lat;
    }
    bool ok = cudaEventRecord(s.t0, s.st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(e->tab, s.tab_host, (size_t)kTables * B * sizeof(uint64_t),
                               cudaMemcpyHostToDevice, s.st) == cudaSuccess;
    ok = ok && cudaGraphLaunch(e->exec, s.st) == cudaSuccess;
    ok = ok && cudaEventRecord(s.t1, s.st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(s.diag_host, e->mem + e->plan.off_diag, (size_t)B * sizeof(cbp_diag),
                               cudaMemcpyDeviceToHost, s.st) == cudaSuccess;
    ok = ok && cudaEventRecord(s.ev, s.st) == cudaSuccess;
    e->last_use = ++tick;
    s.batch = batch;
    s.cur = e;
    s.busy = true;
    if (!ok) {
      cudaGetLastError();
      cudaStreamSynchronize(s.st);
      const auto now = Clock::now();
      for (Request* r : s.batch) finish(r, CBP_ERR_CUDA, nullptr, now);
      s.batch.clear();
      s.busy = false;
      done_cv.notify_all();
    }
  }

  // Admit and launch pending batches while a slot is free.
  void schedule() {
    while (!pending.empty()) {
      Slot* s = nullptr;
      for (Slot& x : slots)
        if (!x.busy) {
          s = &x;
          break;
        }
      if (!s) return;
      Request* r0 = pending.front();
      const Bucket key = bucket_of(*r0);
      std::vector<Request*> batch;
      for (Request* r : pending)
        if (same(bucket_of(*r), key)) {
          batch.push_back(r);
          if ((int)batch.size() == kMaxBatch) break;
        }
      // a cached graph of exactly this size, else a new one; when memory is
      // short, the largest cached one that fits, else halve
      auto cached = [&](int maxB, bool exact) {
        Entry* best = nullptr;
        for (Entry* c : s->cache)
          if (same(c->key, key) && (exact ? c->B == maxB : c->B <= maxB) && (!best || c->B > best->B))
            best = c;
        return best;
      };
      const int want = (int)batch.size();
      cbp_status st = CBP_OK;
      Entry* e = cached(want, true);
      if (!e) e = create_entry(*s, key, want, *r0, &st);
      if (!e && st == CBP_OK) e = cached(want, false);
      for (int B = want / 2; B >= 1 && !e && st == CBP_OK; B /= 2) e = create_entry(*s, key, B, *r0, &st);
      if (!e) {
        if (st == CBP_OK && any_busy()) return;   // wait for memory to come back
        // cannot run even alone (or cannot be planned / captured): fail it
        pending.pop_front();
        finish(r0, st == CBP_OK ? CBP_ERR_BUDGET : st, nullptr, Clock::now());
        done_cv.notify_all();
        continue;
      }
      batch.resize(e->B);
      for (Request* r : batch) pending.erase(std::find(pending.begin(), pending.end(), r));
      launch(*s, e, batch);
    }
  }

  // Collect finished batches.
  void reap() {
    for (Slot& s : slots) {
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.ev);
      if (q == cudaErrorNotReady) continue;
      const auto now = Clock::now();
      if (q != cudaSuccess) cudaGetLastError();
      float a_ms = 0.f, b_ms = 0.f;
      if (q == cudaSuccess && (cudaEventElapsedTime(&a_ms, ref, s.t0) != cudaSuccess ||
                               cudaEventElapsedTime(&b_ms, ref, s.t1) != cudaSuccess)) {
        cudaGetLastError();
        a_ms = b_ms = 0.f;
      }
      for (size_t i = 0; i < s.batch.size(); ++i) {
        cbp_diag d = s.diag_host[i];
        d.gpu_start_ms = a_ms;
        d.gpu_end_ms = b_ms;
        finish(s.batch[i], q == cudaSuccess ? (cbp_status)d.status : CBP_ERR_CUDA, &d, now);
      }
      s.batch.clear();
      s.busy = false;
      done_cv.notify_all();
    }
  }

  void run() {
    cudaSetDevice(ctx->device);
    cbp_status is = CBP_OK;
    for (Slot& s : slots) {
      if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreate(&s.t0) != cudaSuccess || cudaEventCreate(&s.t1) != cudaSuccess ||
          cudaMallocHost((void**)&s.tab_host, sizeof(uint64_t) * kTables * kMaxBatch) != cudaSuccess ||
          cudaMallocHost((void**)&s.diag_host, sizeof(cbp_diag) * kMaxBatch) != cudaSuccess)
        is = CBP_ERR_CUDA;
    }
    if (is == CBP_OK && (cudaEventCreate(&ref) != cudaSuccess || cudaEventRecord(ref, slots[0].st) != cudaSuccess ||
                         cudaEventSynchronize(ref) != cudaSuccess))
      is = CBP_ERR_CUDA;
    std::unique_lock<std::mutex> lk(mu);
    init_status = is;
    ready = true;
    done_cv.notify_all();
    if (is == CBP_OK) {
      for (;;) {
        reap();
        schedule();
        const bool busy = any_busy();
        if (stop && pending.empty() && !busy) break;
        if (busy) wake.wait_for(lk, std::chrono::microseconds(50));
        else wake.wait(lk, [&] { return stop || !pending.empty(); });
      }
    }
    for (Slot& s : slots) {
      for (Entry* e : s.cache) free_entry(s, e);
      s.cache.clear();
      if (s.st) cudaStreamSynchronize(s.st);
      if (s.ev) cudaEventDestroy(s.ev);
      if (s.t0) cudaEventDestroy(s.t0);
      if (s.t1) cudaEventDestroy(s.t1);
      if (s.st) cudaStreamDestroy(s.st);
      if (s.tab_host) cudaFreeHost(s.tab_host);
      if (s.diag_host) cudaFreeHost(s.diag_host);
    }
    if (ref) cudaEventDestroy(ref);
  }
};

namespace {

// The context's engine, started on first use.
cbp_status engine(Ctx* c, ServeState** out) {
  std::lock_guard<std::mutex> g(c->serve_mu);
  if (!c->serve) {
    ServeState* s = new (std::nothrow) ServeState();
    if (!s) return CBP_ERR_OOM;
    s->ctx = c;
    s->th = std::thread([s] { s->run(); });
    std::unique_lock<std::mutex> lk(s->mu);
    s->done_cv.wait(lk, [&] { return s->ready; });
    if (s->init_status != CBP_OK) {
      const cbp_status st = s->init_status;
      s->stop = true;
      lk.unlock();
      s->th.join();
      delete s;
      return st;
    }
    c->serve = s;
  }
  *out = c->serve;
  return CBP_OK;
}

}  // namespace

void serve_shutdown(Ctx* c) {
  ServeState* s = nullptr;
  {
    std::lock_guard<std::mutex> g(c->serve_mu);
    s = c->serve;
    c->serve = nullptr;
  }
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->wake.notify_all();
  s->th.join();
  for (auto& kv : s->tickets) delete kv.second;
  delete s;
}

}  // namespace cbp

using cbp::Ctx;
using cbp::ServeState;

extern "C" {

cbp_status cbp_stream_submit(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                             const cbp_params* params, void* k1, void* k2, void* latent,
                             uint64_t* ticket) {
  cbp::NvtxScope range("cbp_stream_submit");
  if (!ctx || !b1 || !b2 || !params || !ticket || !k1 || !k2) return CBP_ERR_INVALID_ARG;
  if (b1->n != 1 || b2->n != 1 || !b1->data || !b2->data) return CBP_ERR_INVALID_ARG;
  if (params->flags & cbp::kServeRejectFlags) return CBP_ERR_INVALID_ARG;
  cbp::Plan p;
  const cbp_status ps = cbp::make_plan(b1, b2, params, &p);
  if (ps != CBP_OK) return ps;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  ServeState* s = nullptr;
  const cbp_status es = cbp::engine(c, &s);
  if (es != CBP_OK) return es;
  auto* r = new (std::nothrow) cbp::serve::Request();
  if (!r) return CBP_ERR_OOM;
  r->b1 = *b1;
  r->b2 = *b2;
  r->prm = *params;
  r->k1 = k1;
  r->k2 = k2;
  r->lat = latent;
  r->t0 = cbp::serve::Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      return CBP_ERR_INVALID_ARG;
    }
    r->ticket = s->next_ticket++;
    s->tickets[r->ticket] = r;
    s->pending.push_back(r);
  }
  s->wake.notify_one();
  *ticket = r->ticket;
  return CBP_OK;
}

cbp_status cbp_stream_poll(cbp_ctx* ctx, uint64_t ticket, int32_t timeout_us, cbp_diag* diag) {
  if (!ctx) return CBP_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  ServeState* s = nullptr;
  {
    std::lock_guard<std::mutex> g(c->serve_mu);
    s = c->serve;
  }
  if (!s) return CBP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return CBP_ERR_INVALID_ARG;
  cbp::serve::Request* r = it->second;
  if (!r->done) {
    if (timeout_us == 0) return CBP_ERR_BUSY;
    if (timeout_us < 0) {
      s->done_cv.wait(lk, [&] { return r->done; });
    } else {
      const auto deadline = cbp::serve::Clock::now() + std::chrono::microseconds(timeout_us);
      if (!s->done_cv.wait_until(lk, deadline, [&] { return r->done; })) return CBP_ERR_TIMEOUT;
    }
  }
  const cbp_status st = r->status;
  if (diag) *diag = r->diag;
  s->tickets.erase(it);
  delete r;
  return st;
}

cbp_status cbp_stream_stats(cbp_ctx* ctx, uint64_t* completed, double* p50_ms, double* p99_ms,
                            int32_t reset) {
  if (!ctx) return CBP_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  ServeState* s = nullptr;
  {
    std::lock_guard<std::mutex> g(c->serve_mu);
    s = c->serve;
  }
  if (completed) *completed = 0;
  if (p50_ms) *p50_ms = 0;
  if (p99_ms) *p99_ms = 0;
  if (!s) return CBP_OK;
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[(size_t)(f * (double)(v.size() - 1) + 0.5)]; };
    if (p50_ms) *p50_ms = q(0.50);
    if (p99_ms) *p99_ms = q(0.99);
  }
  if (reset) {
    s->lat_ms.clear();
    s->completed = 0;
  }
  return CBP_OK;
}

}  // extern "C"
