// Serving loop: continuous batching of encode / decode requests.
//
// A dispatcher thread admits requests in arrival order whenever a stream slot
// is free and the request's buffers fit in the device-memory arena (the
// admission budget); admitted requests run concurrently on their own streams,
// so work that arrives while others are on the GPU overlaps with it.  Plans
// (one per (n, k)), their twiddle tables and the per-pattern locator tables
// (steps 1-3 of Sec. II.B) stay resident; pattern tables live in an LRU pool
// with reference counts so that a table in use is never recycled, and a
// request whose pattern is still being built by another stream waits on the
// builder's event.  Each request's input is generated on the device from its
// seed (uniform 16-bit source symbols for encode, uniform values in
// [0, 65536] for decode), so host-device copies stay out of the loop.
//
// Locking.  Client calls (submit, poll, release, stats) take only `mu`, which
// guards the hand-over queues and the published request state; they never
// wait behind a kernel launch.  The dispatcher owns the arena, the plans, the
// pattern pools and the stream slots, and launches under `wmu`, a lock that
// only it and the rare plan-level calls (preplan, destroy) take.  A pattern
// table whose pinned upload buffer may still be in flight is skipped (its
// event is queried, never waited on); when no table is free the request stays
// pending and the dispatcher retries on its next pass.
//
// Latency is measured from a request's arrival: the moment submit is called,
// or for fnt_rs_server_replay the scheduled arrival time t0 + arrival_s[i]
// (so a submit that runs late still counts from when the request was due), to
// the moment the dispatcher sees its completion event.  fnt_rs_baseline_replay
// runs the same trace one request at a time with a plan and pattern built per
// request, the plain one-launch-per-request path, on the same clock.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "field.cuh"
#include "internal.h"

namespace fntrs {

void count_launch();

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// input of a request: 16-bit symbols (encode) or values in [0, 65536] (decode)
__global__ void k_gen_input(void* buf, size_t count, uint64_t seed, int is_u16) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const uint64_t h = mix64(seed * 0x100000001B3ull + i);
    if (is_u16)
      static_cast<uint16_t*>(buf)[i] = (uint16_t)h;
    else
      static_cast<uint32_t*>(buf)[i] = (uint32_t)((h >> 16) % 65537u);
  }
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

void launch_gen_input(void* buf, size_t count, uint64_t seed, int is_u16, cudaStream_t st) {
  const unsigned blocks = (unsigned)std::min<size_t>(2048, (count + 255) / 256);
  k_gen_input<<<std::max(1u, blocks), 256, 0, st>>>(buf, count, seed, is_u16);
  count_launch();
}

// First-fit allocator over one device arena (256-byte granules).
class Arena {
 public:
  bool init(size_t bytes) {
    if (cudaMalloc(&base_, bytes) != cudaSuccess) return false;
    size_ = bytes;
    free_[0] = bytes;
    return true;
  }
  ~Arena() {
    if (base_) cudaFree(base_);
  }
  char* alloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_ += bytes;
        return base_ + off;
      }
    }
    return nullptr;
  }
  void release(char* p, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    size_t off = (size_t)(p - base_);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }
  size_t used() const { return used_; }

 private:
  char* base_ = nullptr;
  size_t size_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct PatEntry {
  PatternSlot tab;
  std::vector<uint32_t> key;
  int refs = 0;
  cudaEvent_t built = nullptr;  // recorded after the build on its stream
  bool valid = false;
};

struct PlanRes {
  fnt_rs_plan_s* plan = nullptr;
  std::list<PatEntry*> lru;  // front = most recent
  std::vector<PatEntry*> pool;
};

struct Request {
  uint64_t ticket = 0;
  fnt_rs_request r{};
  std::vector<uint32_t> positions;
  double t_arrival = 0, t_start = 0, t_done = 0;
  int status = 0;  // 0 pending, 1 running, 2 done, <0 error
  char* in = nullptr;
  char* out = nullptr;
  size_t in_bytes = 0, out_bytes = 0;
  int stream = -1;
  PatEntry* pat = nullptr;
  PlanRes* pr = nullptr;
  cudaEvent_t done_ev = nullptr;
};

}  // namespace fntrs

using namespace fntrs;

struct fnt_rs_server_s {
  int dev = 0;
  Arena arena;
  uint32_t nstreams = 0;
  int keep_results = 1;
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_busy;
  std::vector<void*> ws;        // split-transform workspace per stream
  std::vector<uint32_t*> pscr;  // pattern-build scratch per stream
  size_t ws_bytes_per = 0, pscr_words = 0;
  uint32_t pats_per_plan = 64;
  std::map<std::pair<uint32_t, uint32_t>, PlanRes*> plans;
  std::mutex mu;   // clients: incoming, all, to_release, published request state
  std::mutex wmu;  // dispatcher state: arena, plans, pools, stream slots
  std::condition_variable cv;
  std::deque<Request*> incoming;
  std::vector<Request*> to_release;  // released by the client, freed by the dispatcher
  std::deque<Request*> pending;      // dispatcher only
  std::vector<Request*> running;     // dispatcher only
  std::unordered_map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  std::thread worker;
  uint64_t completed = 0, rejected = 0;
  double busy_bytes = 0;
  std::vector<std::pair<uint64_t, double>> done_log;  // (ticket, latency ms) for replays
  bool log_done = false;
};

namespace fntrs {

static const size_t kServerMaxN = 65536;

static int get_plan(fnt_rs_server_s* s, uint32_t n, uint32_t k, PlanRes** out) {
  auto key = std::make_pair(n, k);
  auto it = s->plans.find(key);
  if (it != s->plans.end()) {
    *out = it->second;
    return FNT_RS_OK;
  }
  auto* pr = new PlanRes();
  fnt_rs_plan h = nullptr;
  int rc = fnt_rs_plan_create(&h, n, k, FNT_RS_P, 0, nullptr);
  if (rc) {
    delete pr;
    return rc;
  }
  pr->plan = h;
  for (uint32_t i = 0; i < s->pats_per_plan; ++i) {
    auto* e = new PatEntry();
    if (alloc_pattern_tables(e->tab, n, true) != FNT_RS_OK ||
        cudaEventCreateWithFlags(&e->built, cudaEventDisableTiming) != cudaSuccess)
      return FNT_RS_E_CUDA;
    pr->pool.push_back(e);
  }
  s->plans[key] = pr;
  *out = pr;
  return FNT_RS_OK;
}

// Pattern tables for r on stream si: cached (maybe still building) or built now.
static int get_pattern(fnt_rs_server_s* s, Request* r, int si) {
  PlanRes* pr = r->pr;
  fnt_rs_plan_s* p = pr->plan;
  std::vector<uint32_t> key(r->positions.begin(), r->positions.begin() + p->k);
  for (auto it = pr->lru.begin(); it != pr->lru.end(); ++it) {
    PatEntry* e = *it;
    if (e->valid && e->key == key) {
      pr->lru.splice(pr->lru.begin(), pr->lru, it);
      e->refs++;
      r->pat = e;
      // the table may still be under construction on another stream
      return cudaStreamWaitEvent(s->streams[si], e->built, 0) == cudaSuccess ? FNT_RS_OK
                                                                            : FNT_RS_E_CUDA;
    }
  }
  // A free table is reusable once its previous build (whose upload reads the
  // pinned staging buffer) has finished; that is queried, never waited on.
  auto staged = [](PatEntry* c) {
    const cudaError_t q = cudaEventQuery(c->built);
    if (q == cudaErrorNotReady) return false;
    return q == cudaSuccess;
  };
  PatEntry* e = nullptr;
  for (auto* c : pr->pool)
    if (!c->valid && c->refs == 0 && staged(c)) {
      e = c;
      break;
    }
  if (!e) {
    for (auto it = pr->lru.rbegin(); it != pr->lru.rend(); ++it)
      if ((*it)->refs == 0 && staged(*it)) {
        e = *it;
        break;
      }
    if (!e) return 1;  // every table in use or still staging: try later
    pr->lru.remove(e);
    e->valid = false;
  }
  std::memcpy(e->tab.pos_h, key.data(), key.size() * 4);
  cudaStream_t st = s->streams[si];
  if (cudaMemcpyAsync(e->tab.pos_d, e->tab.pos_h, key.size() * 4, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return FNT_RS_E_CUDA;
  int rc = build_pattern_log(p, e->tab, st, s->pscr[si]);
  if (rc) return rc;
  cudaEventRecord(e->built, st);
  e->key.swap(key);
  e->valid = true;
  e->refs = 1;
  pr->lru.push_front(e);
  r->pat = e;
  return FNT_RS_OK;
}

static size_t req_in_bytes(const fnt_rs_request& q) {
  return q.op == FNT_RS_OP_ENCODE ? (size_t)q.k * q.W * 2 : (size_t)q.k * q.W * 4;
}
static size_t req_out_bytes(const fnt_rs_request& q) {
  return q.op == FNT_RS_OP_ENCODE ? (size_t)q.n * q.W * 4 : (size_t)q.k * q.W * 2;
}

// Sets a request's visible status (1 running, 2 done, < 0 error) under mu.
static void publish(fnt_rs_server_s* s, Request* r, int status, double t_done = 0) {
  std::lock_guard<std::mutex> lk(s->mu);
  r->status = status;
  if (status == 2 || status < 0) {
    r->t_done = t_done > 0 ? t_done : now_s();
    s->completed += status == 2 ? 1 : 0;
    if (s->log_done) s->done_log.push_back({r->ticket, (r->t_done - r->t_arrival) * 1e3});
  }
}

// Admission: stream slot + arena space.  Returns true if r was started (or
// failed; its error is then published).  Dispatcher only, under wmu.
static bool try_start(fnt_rs_server_s* s, Request* r) {
  int si = -1;
  for (uint32_t i = 0; i < s->nstreams; ++i)
    if (!s->stream_busy[i]) {
      si = (int)i;
      break;
    }
  if (si < 0) return false;
  if (!r->pr && get_plan(s, r->r.n, r->r.k, &r->pr) != FNT_RS_OK) {
    publish(s, r, FNT_RS_E_CUDA);
    return true;
  }
  r->in_bytes = req_in_bytes(r->r);
  r->out_bytes = req_out_bytes(r->r);
  r->in = s->arena.alloc(r->in_bytes);
  if (!r->in) return false;
  r->out = s->arena.alloc(r->out_bytes);
  if (!r->out) {
    s->arena.release(r->in, r->in_bytes);
    r->in = nullptr;
    return false;
  }
  cudaStream_t st = s->streams[si];
  fnt_rs_plan_s* p = r->pr->plan;
  if (r->r.op == FNT_RS_OP_DECODE) {
    const int rc = get_pattern(s, r, si);
    if (rc == 1) {  // all pattern tables busy
      s->arena.release(r->out, r->out_bytes);
      s->arena.release(r->in, r->in_bytes);
      r->in = r->out = nullptr;
      return false;
    }
    if (rc) {
      publish(s, r, rc);
      return true;
    }
  }
  r->stream = si;
  s->stream_busy[si] = 1;
  r->t_start = now_s();
  const bool enc = r->r.op == FNT_RS_OP_ENCODE;
  launch_gen_input(r->in, (size_t)r->r.k * r->r.W, r->r.seed, enc ? 1 : 0, st);
  int rc;
  if (enc)
    rc = do_encode(p, reinterpret_cast<uint16_t*>(r->in), r->r.W,
                   reinterpret_cast<uint32_t*>(r->out), r->r.W, r->r.W, s->ws[si], st);
  else
    rc = do_decode_tables(p, r->pat->tab, reinterpret_cast<uint32_t*>(r->in), r->r.W,
                          reinterpret_cast<uint16_t*>(r->out), r->r.W, r->r.W, s->ws[si], st, 0);
  cudaEventRecord(r->done_ev, st);
  publish(s, r, rc ? rc : 1);
  s->busy_bytes += (double)r->r.k * r->r.W * 2;
  return true;
}

// Completion seen at t_done: frees the slot and pattern reference (and, without
// kept results, the buffers), then publishes the result.  Dispatcher only.
static void finish(fnt_rs_server_s* s, Request* r, double t_done) {
  if (r->stream >= 0) s->stream_busy[r->stream] = 0;
  if (r->pat) {
    r->pat->refs--;
    r->pat = nullptr;
  }
  char* in = nullptr;
  char* out = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->keep_results) {
      in = r->in;
      out = r->out;
      r->in = r->out = nullptr;
    }
  }
  if (in) {
    s->arena.release(out, r->out_bytes);
    s->arena.release(in, r->in_bytes);
  }
  publish(s, r, 2, t_done);
}

// Frees what the client released (buffers back to the arena, the record).
static void reclaim(fnt_rs_server_s* s, std::vector<Request*>& rel) {
  for (Request* r : rel) {
    if (r->in) {
      s->arena.release(r->out, r->out_bytes);
      s->arena.release(r->in, r->in_bytes);
    }
    cudaEventDestroy(r->done_ev);
    delete r;
  }
  rel.clear();
}

static void worker_loop(fnt_rs_server_s* s) {
  cudaSetDevice(s->dev);
  std::vector<Request*> rel;
  while (true) {
    bool stopping = false;
    // Lock order everywhere: wmu before mu.  pending and running belong to
    // this thread alone, so reading them here needs neither lock.
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->incoming.empty() && s->to_release.empty() && s->pending.empty() &&
          s->running.empty()) {
        if (s->stop) break;
        s->cv.wait_for(lk, std::chrono::microseconds(200));
      }
      while (!s->incoming.empty()) {
        s->pending.push_back(s->incoming.front());
        s->incoming.pop_front();
      }
      rel.swap(s->to_release);
      stopping = s->stop;
    }
    {
      std::lock_guard<std::mutex> wl(s->wmu);
      reclaim(s, rel);
      // completions (each is timed when seen)
      for (size_t i = 0; i < s->running.size();) {
        Request* r = s->running[i];
        if (cudaEventQuery(r->done_ev) == cudaSuccess) {
          finish(s, r, now_s());
          s->running[i] = s->running.back();
          s->running.pop_back();
        } else {
          ++i;
        }
      }
      // admissions, in arrival order; launches run outside mu
      while (!s->pending.empty()) {
        Request* r = s->pending.front();
        if (!try_start(s, r)) break;
        s->pending.pop_front();
        if (r->status < 0) continue;
        s->running.push_back(r);
      }
      if (stopping && s->pending.empty() && s->running.empty()) {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->incoming.empty()) break;
      }
    }
    std::this_thread::yield();
  }
}

}  // namespace fntrs

extern "C" {

int fnt_rs_server_create(fnt_rs_server* out, size_t budget_bytes, uint32_t nstreams,
                         int keep_results) {
  if (!out || budget_bytes == 0) return FNT_RS_E_ARG;
  *out = nullptr;
  auto* s = new fnt_rs_server_s();
  cudaGetDevice(&s->dev);
  s->nstreams = std::max<uint32_t>(1, std::min<uint32_t>(nstreams, 64));
  s->keep_results = keep_results;
  if (!s->arena.init(budget_bytes)) {
    delete s;
    return FNT_RS_E_CUDA;
  }
  // worst-case split workspace (decode, k > n/2: 4 buffers of one chunk) and pattern scratch
  s->ws_bytes_per = kChunkBudget + (1u << 20);
  s->pscr_words = pattern_scratch_words(kServerMaxN, kServerMaxN);
  s->streams.resize(s->nstreams);
  s->stream_busy.assign(s->nstreams, 0);
  s->ws.assign(s->nstreams, nullptr);
  s->pscr.assign(s->nstreams, nullptr);
  for (uint32_t i = 0; i < s->nstreams; ++i) {
    if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&s->ws[i], s->ws_bytes_per) != cudaSuccess ||
        cudaMalloc(&s->pscr[i], s->pscr_words * 4) != cudaSuccess) {
      fnt_rs_server_destroy(s);
      return FNT_RS_E_CUDA;
    }
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return FNT_RS_OK;
}

int fnt_rs_server_preplan(fnt_rs_server s, uint32_t n, uint32_t k) {
  if (!s) return FNT_RS_E_ARG;
  std::lock_guard<std::mutex> lk(s->wmu);
  PlanRes* pr = nullptr;
  return get_plan(s, n, k, &pr);
}

static int submit_at(fnt_rs_server s, const fnt_rs_request* req, double t_arrival,
                     uint64_t* ticket);

int fnt_rs_server_submit(fnt_rs_server s, const fnt_rs_request* req, uint64_t* ticket) {
  return submit_at(s, req, now_s(), ticket);
}

// Queues a request that arrived at t_arrival (now_s clock).
static int submit_at(fnt_rs_server s, const fnt_rs_request* req, double t_arrival,
                     uint64_t* ticket) {
  if (!s || !req || !ticket) return FNT_RS_E_ARG;
  const fnt_rs_request& q = *req;
  if (q.n < 2 || q.n > kServerMaxN || (q.n & (q.n - 1)) || q.k < 1 || q.k > q.n || q.W == 0 ||
      (q.op != FNT_RS_OP_ENCODE && q.op != FNT_RS_OP_DECODE))
    return FNT_RS_E_ARG;
  if (req_in_bytes(q) + req_out_bytes(q) + 512 > s->arena.size()) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->rejected++;
    return FNT_RS_E_BUDGET;
  }
  auto* r = new Request();
  r->r = q;
  if (q.op == FNT_RS_OP_DECODE) {
    if (!q.positions || q.npos < q.k) {
      delete r;
      return FNT_RS_E_POSITIONS;
    }
    r->positions.assign(q.positions, q.positions + q.npos);
    std::vector<uint8_t> seen(q.n, 0);
    for (uint32_t i = 0; i < q.npos; ++i) {
      if (r->positions[i] >= q.n || seen[r->positions[i]]) {
        delete r;
        return FNT_RS_E_POSITIONS;
      }
      seen[r->positions[i]] = 1;
    }
  }
  r->r.positions = nullptr;
  if (cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming) != cudaSuccess) {
    delete r;
    return FNT_RS_E_CUDA;
  }
  r->t_arrival = t_arrival;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    s->all[r->ticket] = r;
    s->incoming.push_back(r);
  }
  s->cv.notify_one();
  *ticket = r->ticket;
  return FNT_RS_OK;
}

// 1 = done, 0 = pending or running, negative = error of that request.
int fnt_rs_server_poll(fnt_rs_server s, uint64_t ticket, double* latency_ms) {
  if (!s) return FNT_RS_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return FNT_RS_E_ARG;
  Request* r = it->second;
  if (r->status < 0) return r->status;
  if (r->status != 2) return 0;
  if (latency_ms) *latency_ms = (r->t_done - r->t_arrival) * 1e3;
  return 1;
}

int fnt_rs_server_drain(fnt_rs_server s) {
  if (!s) return FNT_RS_E_ARG;
  while (true) {
    {
      std::lock_guard<std::mutex> wl(s->wmu);
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->incoming.empty() && s->pending.empty() && s->running.empty()) return FNT_RS_OK;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

// Copies a finished request's input and output to host memory (either may be NULL).
int fnt_rs_server_fetch(fnt_rs_server s, uint64_t ticket, void* h_in, void* h_out) {
  if (!s) return FNT_RS_E_ARG;
  Request* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return FNT_RS_E_ARG;
    r = it->second;
    if (r->status != 2 || !r->in) return FNT_RS_E_ARG;
  }
  if (h_in && cudaMemcpy(h_in, r->in, r->in_bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
    return FNT_RS_E_CUDA;
  if (h_out && cudaMemcpy(h_out, r->out, r->out_bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
    return FNT_RS_E_CUDA;
  return FNT_RS_OK;
}

// Frees a finished request's buffers and record (the dispatcher returns the
// buffers to the arena on its next pass; the ticket is gone at once).
int fnt_rs_server_release(fnt_rs_server s, uint64_t ticket) {
  if (!s) return FNT_RS_E_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return FNT_RS_E_ARG;
    Request* r = it->second;
    if (r->status == 0 || r->status == 1) return FNT_RS_E_ARG;
    s->all.erase(it);
    s->to_release.push_back(r);
  }
  s->cv.notify_one();
  return FNT_RS_OK;
}

// {completed, rejected, arena bytes used, arena bytes, plans resident}
int fnt_rs_server_stats(fnt_rs_server s, double* out, int cap) {
  if (!s || !out) return 0;
  std::lock_guard<std::mutex> wl(s->wmu);
  std::lock_guard<std::mutex> lk(s->mu);
  const double v[5] = {(double)s->completed, (double)s->rejected, (double)s->arena.used(),
                       (double)s->arena.size(), (double)s->plans.size()};
  const int m = std::min(cap, 5);
  for (int i = 0; i < m; ++i) out[i] = v[i];
  return m;
}

void fnt_rs_server_destroy(fnt_rs_server s) {
  if (!s) return;
  if (s->worker.joinable()) {
    s->stop = true;
    s->cv.notify_all();
    s->worker.join();
  }
  cudaDeviceSynchronize();
  for (auto& kv : s->all) {
    cudaEventDestroy(kv.second->done_ev);
    delete kv.second;
  }
  for (Request* r : s->to_release) {
    cudaEventDestroy(r->done_ev);
    delete r;
  }
  for (auto& kv : s->plans) {
    for (auto* e : kv.second->pool) {
      free_pattern_tables(e->tab);
      if (e->built) cudaEventDestroy(e->built);
      delete e;
    }
    fnt_rs_plan_destroy(kv.second->plan);
    delete kv.second;
  }
  for (uint32_t i = 0; i < s->streams.size(); ++i) {
    if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
    cudaFree(s->ws[i]);
    cudaFree(s->pscr[i]);
  }
  delete s;
}

// Replays a trace: request i is due at t0 + arrival_s[i] (real time, t0 =
// the start of the replay) and submitted by this thread once that time has
// come; latency_ms[i] receives its latency counted from the due time, queueing
// and any late submission included (negative: rejected).  Returns the wall
// time of the whole replay in *wall_s.  Results are released as they complete.
int fnt_rs_server_replay(fnt_rs_server s, const fnt_rs_request* reqs, const double* arrival_s,
                         uint32_t count, double* latency_ms, double* wall_s) {
  if (!s || (!reqs && count)) return FNT_RS_E_ARG;
  std::unordered_map<uint64_t, uint32_t> index;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->log_done = true;
    s->done_log.clear();
  }
  const double t0 = now_s();
  uint32_t next = 0, done = 0;
  std::vector<std::pair<uint64_t, double>> batch;
  while (done < count) {
    const double t = now_s() - t0;
    while (next < count && arrival_s[next] <= t) {
      uint64_t tk = 0;
      const int rc = submit_at(s, &reqs[next], t0 + arrival_s[next], &tk);
      if (rc) {
        latency_ms[next] = -1.0;
        ++done;
      } else {
        index[tk] = next;
      }
      ++next;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      batch.swap(s->done_log);
    }
    for (auto& d : batch) {
      auto it = index.find(d.first);
      if (it == index.end()) continue;
      latency_ms[it->second] = d.second;
      index.erase(it);
      fnt_rs_server_release(s, d.first);
      ++done;
    }
    batch.clear();
    if (next < count) {
      const double wait = arrival_s[next] - (now_s() - t0);
      if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::microseconds(100));
    } else {
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
  if (wall_s) *wall_s = now_s() - t0;
  std::lock_guard<std::mutex> lk(s->mu);
  s->log_done = false;
  return FNT_RS_OK;
}

// The plain path on the same trace: one request at a time on `stream`, plan
// and pattern built for each request, input generated as in the server.
int fnt_rs_baseline_replay(const fnt_rs_request* reqs, const double* arrival_s, uint32_t count,
                           double* latency_ms, double* wall_s, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  size_t max_in = 0, max_out = 0, max_ws = 0;
  for (uint32_t i = 0; i < count; ++i) {
    max_in = std::max(max_in, req_in_bytes(reqs[i]));
    max_out = std::max(max_out, req_out_bytes(reqs[i]));
  }
  max_ws = kChunkBudget + (1u << 20);
  void *din = nullptr, *dout = nullptr, *dws = nullptr;
  if (cudaMalloc(&din, max_in + 256) != cudaSuccess || cudaMalloc(&dout, max_out + 256) != cudaSuccess ||
      cudaMalloc(&dws, max_ws) != cudaSuccess) {
    cudaFree(din);
    cudaFree(dout);
    return FNT_RS_E_CUDA;
  }
  const double t0 = now_s();
  int rc = FNT_RS_OK;
  for (uint32_t i = 0; i < count && !rc; ++i) {
    while (now_s() - t0 < arrival_s[i]) std::this_thread::sleep_for(std::chrono::microseconds(50));
    const fnt_rs_request& q = reqs[i];
    fnt_rs_plan h = nullptr;
    rc = fnt_rs_plan_create(&h, q.n, q.k, FNT_RS_P, 0, stream);
    if (rc) break;
    const bool enc = q.op == FNT_RS_OP_ENCODE;
    launch_gen_input(din, (size_t)q.k * q.W, q.seed, enc ? 1 : 0, st);
    if (enc)
      rc = fnt_rs_encode(h, (const uint16_t*)din, q.W, (uint32_t*)dout, q.W, q.W, dws, stream);
    else
      rc = fnt_rs_decode(h, (const uint32_t*)din, q.W, q.positions, q.npos, (uint16_t*)dout, q.W,
                         q.W, dws, stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = FNT_RS_E_CUDA;
    latency_ms[i] = (now_s() - t0 - arrival_s[i]) * 1e3;
    fnt_rs_plan_destroy(h);
  }
  if (wall_s) *wall_s = now_s() - t0;
  cudaFree(din);
  cudaFree(dout);
  cudaFree(dws);
  return rc;
}

}  // extern "C"
