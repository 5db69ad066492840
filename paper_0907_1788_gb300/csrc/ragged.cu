// Ragged batches: many groups of codewords, each with its own (n, k, W,
// erasure pattern), run by one CUDA graph launch.
//
// Every group is a full round trip: encode its source (Sec. II.B, e = FNT of
// the zero-padded source), build its pattern tables (steps 1-3), decode every
// codeword from the encoded matrix used as the receiver's slot buffer
// (steps 4-6).  Groups with n >= 256 and the default root (every length of
// the seeded ragged workload, 256 to 65536) all run in one launch of the ragged
// persistent kernel (ragged_kernel.cu), each with its own pattern tables and
// build scratch; the split-transform work items of the longest codes use a
// scratch area per CTA.  Other groups (n < 256, another root, or the
// product-tree pattern route) keep per-group launches: groups sharing (n, k)
// share one plan and run in order on one stream, and plan classes are spread
// over several streams by estimated work.  The persistent kernel's stream and
// the others are captured into a single graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "internal.h"
#include "ragged_dev.h"
#include "sched.h"

namespace fntrs {

struct RaggedGroup {
  fnt_rs_group g{};
  fnt_rs_plan_s* plan = nullptr;
  PatternSlot tab;  // decode groups only
  int stream = 0;
  bool persistent = false;    // runs in the ragged persistent kernel
  uint32_t* scratch = nullptr;  // its own pattern-build scratch (persistent decode groups)
};

// Words of a persistent decode group's pattern-build scratch: the one-launch
// build's digit convolutions and tail buffers, or for a long code (n >= 32768)
// indicator, spectrum, per-digit products, convolutions and tail buffers.
inline size_t ragged_plan_scratch_words(size_t n, size_t D) {
  return ragged_long_plan((int)n) ? (2 * D + 8) * n : n * D + 6 * n;
}

}  // namespace fntrs

using namespace fntrs;

struct fnt_rs_ragged_s {
  int dev = 0;
  std::map<std::pair<uint32_t, uint32_t>, fnt_rs_plan_s*> plans;
  std::vector<RaggedGroup> groups;
  std::vector<cudaStream_t> streams;
  std::vector<void*> ws;
  cudaStream_t cap = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // ragged persistent kernel
  RaggedArgs ra{};
  RaggedGroupDev* d_groups = nullptr;
  RaggedItem* d_items = nullptr;
  unsigned* d_counters = nullptr;  // next, enc_done[G], plan_done[G]
  size_t counter_bytes = 0;
  int grid = 0;
  int npersistent = 0;
  uint32_t* cta_scratch = nullptr;  // split-transform buffers of the persistent CTAs
  int tuned = 0;  // plans whose schedules the autotuner picked
};

namespace fntrs {

// The work of one group on stream st.
static int run_group(RaggedGroup& rg, void* ws, cudaStream_t st) {
  fnt_rs_plan_s* p = rg.plan;
  const fnt_rs_group& g = rg.g;
  int rc = do_encode(p, g.src, g.ld_src, g.enc, g.ld_enc, g.W, ws, st);
  if (rc || !g.positions) return rc;
  if ((rc = p->plan_tree ? build_pattern(p, rg.tab, st) : build_pattern_log(p, rg.tab, st)))
    return rc;
  return do_decode_tables(p, rg.tab, g.enc, g.ld_enc, g.out, g.ld_out, g.W, ws, st, 1);
}

static void free_group(RaggedGroup& rg) {
  free_pattern_tables(rg.tab);
  cudaFree(rg.scratch);
}

static bool persistent_eligible(const fnt_rs_plan_s* p) {
  if (p->n < (uint32_t)kRaggedMinL || p->n > (uint32_t)kRaggedMaxL || p->u != 1 || p->plan_tree)
    return false;
  // short codes: the one-launch pattern build's digit items
  return ragged_long_plan((int)p->n) || tile_ops((int)p->n).plan_fused != nullptr;
}

// Words of split-transform scratch one persistent CTA needs for this group.
static size_t cta_scratch_words(const RaggedGroup& rg) {
  const fnt_rs_plan_s* p = rg.plan;
  const int n = (int)p->n;
  size_t w = 0;
  if (ragged_split_enc(n)) w = std::max(w, (size_t)n * kRaggedSplitWT);
  if (rg.g.positions) {
    if (ragged_split_dec(n, p->blocked))
      w = std::max(w, (size_t)(p->blocked ? 4 : 2) * n * kRaggedSplitWT);
    if (ragged_long_plan(n) && n > kTileMaxL) w = std::max(w, (size_t)2 * n);
  }
  return w;
}

// Device group record of a persistent group (same arguments as the per-group
// generic encode, one-launch pattern build and generic decode).
static RaggedGroupDev make_dev_group(const RaggedGroup& rg) {
  const fnt_rs_plan_s* p = rg.plan;
  const fnt_rs_group& g = rg.g;
  const int n = (int)p->n, k = (int)p->k;
  RaggedGroupDev d{};
  d.L = n;
  d.blocked = p->blocked ? 1 : 0;
  d.has_plan = g.positions ? 1 : 0;
  d.enc_tiles = (int)((g.W + ragged_wt_enc(n) - 1) / ragged_wt_enc(n));
  d.enc_need = d.enc_tiles;
  d.split_enc = ragged_split_enc(n) ? 1 : 0;
  d.split_dec = ragged_split_dec(n, p->blocked) ? 1 : 0;
  d.long_plan = ragged_long_plan(n) ? 1 : 0;
  d.C = n > kLocalL ? n / kLocalL : 1;
  KArgs& e = d.enc;
  e.in = g.src;
  e.ld_in = g.ld_src;
  e.out = g.enc;
  e.ld_out = g.ld_enc;
  e.W = (int)g.W;
  e.n = n;
  e.k = k;
  e.L = n;
  e.C = 1;
  e.twf = p->tn.twf;
  e.twi = p->tn.twi;
  e.powf = p->tn.powf;
  e.row_mul = p->uinv;
  e.status = p->status;
  if (d.split_enc) {
    KArgs& x = d.xenc;  // the split encode's cross and local passes
    x.n = n;
    x.k = k;
    x.L = kLocalL;
    x.C = d.C;
    x.powf = p->tn.powf;
    x.powi = p->tn.powi;
    x.twf = p->tl.twf;
    x.twi = p->tl.twi;
    x.status = p->status;
  }
  if (!g.positions) return d;
  KArgs& a = d.dec;
  a.slots = 1;
  a.in = g.enc;
  a.ld_in = g.ld_enc;
  a.out = g.out;
  a.ld_out = g.ld_out;
  a.n = n;
  a.k = k;
  a.h = n / 2;
  a.pat = rg.tab.pat;
  a.ahat = rg.tab.ahat;
  a.ahat2 = rg.tab.ahat2;
  a.status = p->status;
  a.W = (int)g.W;
  a.L = n;
  a.C = 1;
  a.twf = p->tn.twf;
  a.twi = p->tn.twi;
  if (d.split_dec) {
    KArgs& x = d.xdec;  // the split decode's passes (received rows = the slot buffer)
    x = a;
    x.L = kLocalL;
    x.C = d.C;
    x.powf = p->tn.powf;
    x.powi = p->tn.powi;
    x.twf = p->tl.twf;
    x.twi = p->tl.twi;
  }
  if (d.long_plan) {
    // scratch: ind [n] | spec [n] | prod [D][n] | conv [n][D] | aval | coef [n] | M2, E2 [n][2]
    const size_t D = (size_t)p->lg_D;
    LongPlanDev& lp = d.lp;
    lp.ind = rg.scratch;
    lp.spec = lp.ind + n;
    lp.prod = lp.spec + n;
    uint32_t* conv = lp.prod + D * n;
    lp.aval = conv + D * n;
    lp.coef = lp.aval + n;
    lp.M2 = lp.coef + n;
    lp.E2 = lp.M2 + 2 * (size_t)n;
    for (KArgs* c : {&d.colf, &d.coli}) {  // one-column transforms of length n
      c->n = n;
      c->C = 1;
      c->status = p->status;
      if (n <= kTileMaxL) {
        c->L = n;
        c->twf = p->tn.twf;
        c->twi = p->tn.twi;
      } else {
        c->L = kLocalL;
        c->C = d.C;
        c->powf = p->tn.powf;
        c->powi = p->tn.powi;
        c->twf = p->tl.twf;
        c->twi = p->tl.twi;
      }
    }
    PlanArgs& pa = d.plan;
    pa.k = k;
    pa.D = p->lg_D;
    pa.b = p->lg_b;
    pa.ninv = p->ninv;
    pa.pos = rg.tab.pos_d;
    pa.ghat = p->ghat;
    pa.exp3 = p->exp3;
    pa.conv = conv;
    pa.pat = rg.tab.pat;
    pa.pat32 = rg.tab.pat32;
    pa.rowtab = rg.tab.rowtab;
    pa.aval = p->blocked ? lp.aval : nullptr;
    pa.ahat = p->blocked ? nullptr : rg.tab.ahat;
    pa.done = rg.tab.done;
    pa.status = p->status;
    return d;
  }
  // scratch: conv [n][D] | aval [n] | coef [n] | halves [n][2] | E [n][2]
  uint32_t* conv = rg.scratch;
  uint32_t* aval = conv + (size_t)n * p->lg_D;
  uint32_t* coef = aval + n;
  uint32_t* halves = coef + n;
  uint32_t* E = halves + 2 * (size_t)n;
  PlanArgs& pa = d.plan;
  pa.k = k;
  pa.D = p->lg_D;
  pa.b = p->lg_b;
  pa.ninv = p->ninv;
  pa.twf = p->tn.twf;
  pa.twi = p->tn.twi;
  pa.pos = rg.tab.pos_d;
  pa.ghat = p->ghat;
  pa.exp3 = p->exp3;
  pa.conv = conv;
  pa.pat = rg.tab.pat;
  pa.pat32 = rg.tab.pat32;
  pa.rowtab = rg.tab.rowtab;
  pa.aval = p->blocked ? aval : nullptr;
  pa.ahat = p->blocked ? nullptr : rg.tab.ahat;
  pa.done = rg.tab.done;
  pa.status = p->status;
  d.halves = halves;
  KArgs& ti = d.tail_inv;
  ti.in = aval;
  ti.ld_in = 1;
  ti.out = coef;
  ti.ld_out = 1;
  ti.W = 1;
  ti.n = n;
  ti.L = n;
  ti.C = 1;
  ti.scale = p->ninv;
  ti.twf = p->tn.twf;
  ti.twi = p->tn.twi;
  KArgs& tf = d.tail_fwd;
  tf.in = halves;
  tf.ld_in = 2;
  tf.out = E;
  tf.ld_out = 2;
  tf.W = 2;
  tf.n = n;
  tf.L = n;
  tf.C = 1;
  tf.twf = p->tn.twf;
  tf.twi = p->tn.twi;
  return d;
}

// The persistent part of one run: reset the counters, one launch.
static int run_persistent(fnt_rs_ragged_s* r, cudaStream_t st) {
  if (!r->npersistent) return FNT_RS_OK;
  if (cudaMemsetAsync(r->d_counters, 0, r->counter_bytes, st) != cudaSuccess)
    return FNT_RS_E_CUDA;
  if (launch_ragged(r->ra, r->grid, st) != 0) return FNT_RS_E_CUDA;
  return cuda_ok(cudaGetLastError());
}

}  // namespace fntrs

extern "C" {

void fnt_rs_ragged_destroy(fnt_rs_ragged r) {
  if (!r) return;
  cudaDeviceSynchronize();
  if (r->exec) cudaGraphExecDestroy(r->exec);
  if (r->graph) cudaGraphDestroy(r->graph);
  for (auto& g : r->groups) free_group(g);
  cudaFree(r->d_groups);
  cudaFree(r->d_items);
  cudaFree(r->d_counters);
  cudaFree(r->cta_scratch);
  for (void* w : r->ws) cudaFree(w);
  for (auto s : r->streams) cudaStreamDestroy(s);
  for (auto e : r->joins) cudaEventDestroy(e);
  if (r->fork) cudaEventDestroy(r->fork);
  if (r->cap) cudaStreamDestroy(r->cap);
  for (auto& kv : r->plans) fnt_rs_plan_destroy(kv.second);
  delete r;
}

int fnt_rs_ragged_create(fnt_rs_ragged* out, const fnt_rs_group* groups, uint32_t ngroups,
                         uint32_t nstreams, void* stream) {
  if (!out || (!groups && ngroups)) return FNT_RS_E_ARG;
  *out = nullptr;
  if (nstreams == 0) nstreams = 8;
  nstreams = std::min<uint32_t>(nstreams, 64);
  auto* r = new fnt_rs_ragged_s();
  cudaGetDevice(&r->dev);
  auto fail = [&](int rc) {
    fnt_rs_ragged_destroy(r);
    return rc;
  };
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  r->groups.resize(ngroups);
  // plans, shared per (n, k)
  for (uint32_t i = 0; i < ngroups; ++i) {
    const fnt_rs_group& g = groups[i];
    if (!g.src || !g.enc || g.ld_src < g.W || g.ld_enc < g.W) return fail(FNT_RS_E_ARG);
    if (g.positions && (!g.out || g.ld_out < g.W)) return fail(FNT_RS_E_ARG);
    auto key = std::make_pair(g.n, g.k);
    if (!r->plans.count(key)) {
      fnt_rs_plan h = nullptr;
      const int rc = fnt_rs_plan_create(&h, g.n, g.k, FNT_RS_P, 0, stream);
      if (rc) return fail(rc);
      r->plans[key] = h;
    }
    r->groups[i].g = g;
    r->groups[i].plan = r->plans[key];
  }
  // pattern tables and positions of decode groups
  for (auto& rg : r->groups) {
    if (!rg.g.positions) continue;
    fnt_rs_plan_s* p = rg.plan;
    int rc = validate_positions(p, rg.g.positions, rg.g.npos);
    if (rc) return fail(rc);
    if ((rc = alloc_pattern_tables(rg.tab, p->n, false))) return fail(rc);
    if (cudaMemcpy(rg.tab.pos_d, rg.g.positions, (size_t)p->k * 4, cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return fail(FNT_RS_E_CUDA);
  }
  // groups of the persistent kernel: own build scratch, device records, work list
  std::vector<int> pers;
  for (int i = 0; i < (int)r->groups.size(); ++i) {
    RaggedGroup& rg = r->groups[i];
    rg.persistent = persistent_eligible(rg.plan);
    if (!rg.persistent) continue;
    pers.push_back(i);
    if (rg.g.positions) {
      const size_t words = ragged_plan_scratch_words(rg.plan->n, (size_t)rg.plan->lg_D);
      if (cudaMalloc(&rg.scratch, words * 4) != cudaSuccess) return fail(FNT_RS_E_CUDA);
    }
  }
  if (!pers.empty()) {
    auto cost = [&](int i) {
      const double n = r->groups[i].plan->n;
      return (double)r->groups[i].g.W * n * std::log2(n);
    };
    std::stable_sort(pers.begin(), pers.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<RaggedGroupDev> dg;
    std::vector<RaggedItem> items;
    // Failure-detection test hook: FNTRS_TEST_STALL_GROUP=g makes the decode
    // items of group g wait for one encode tile more than the group has (a
    // producer that never finishes).  Their bounded waits give up, raise
    // FNT_RS_E_TIMEOUT in the group's status and skip its decode; every other
    // item runs as usual and the launch ends.
    const char* stall_env = std::getenv("FNTRS_TEST_STALL_GROUP");
    const int stall = stall_env ? std::atoi(stall_env) : -1;
    for (int gi = 0; gi < (int)pers.size(); ++gi) {
      dg.push_back(make_dev_group(r->groups[pers[gi]]));
      if (pers[gi] == stall) dg.back().enc_need += 1;
    }
    // Order: the long codes' spectrum items (they wait on nothing), every
    // encode tile, every pattern item, every decode tile.  The encode tiles
    // between the spectra and the digit items that read them give the spectra
    // time to finish, so digit items seldom wait.
    for (int gi = 0; gi < (int)pers.size(); ++gi)
      if (dg[gi].has_plan && dg[gi].long_plan) items.push_back({RI_SPEC, gi, 0});
    for (int gi = 0; gi < (int)pers.size(); ++gi)
      for (int t = 0; t < dg[gi].enc_tiles; ++t) items.push_back({RI_ENC, gi, t});
    for (int gi = 0; gi < (int)pers.size(); ++gi)
      if (dg[gi].has_plan)
        for (int t = 0; t < dg[gi].plan.D; ++t) items.push_back({RI_PLAN, gi, t});
    for (int gi = 0; gi < (int)pers.size(); ++gi) {
      if (!dg[gi].has_plan) continue;
      const int wt = ragged_wt_dec(dg[gi].L, dg[gi].blocked != 0);
      const int tiles = (dg[gi].dec.W + wt - 1) / wt;
      for (int t = 0; t < tiles; ++t) items.push_back({RI_DEC, gi, t});
    }
    const size_t G = dg.size();
    r->counter_bytes = (1 + 3 * G) * sizeof(unsigned);
    if (cudaMalloc(&r->d_groups, G * sizeof(RaggedGroupDev)) != cudaSuccess ||
        cudaMalloc(&r->d_items, items.size() * sizeof(RaggedItem)) != cudaSuccess ||
        cudaMalloc(&r->d_counters, r->counter_bytes) != cudaSuccess ||
        cudaMemcpy(r->d_groups, dg.data(), G * sizeof(RaggedGroupDev), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(r->d_items, items.data(), items.size() * sizeof(RaggedItem),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(FNT_RS_E_CUDA);
    r->ra.items = r->d_items;
    r->ra.nitems = (int)items.size();
    r->ra.groups = r->d_groups;
    r->ra.next = r->d_counters;
    r->ra.enc_done = r->d_counters + 1;
    r->ra.plan_done = r->d_counters + 1 + G;
    r->ra.spec_done = r->d_counters + 1 + 2 * G;
    r->npersistent = (int)G;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, r->dev);
    r->grid = std::max(1, sms);
    // split-transform scratch: one area per persistent CTA, as large as the
    // largest split item of the batch needs
    size_t cta_words = 0;
    for (int i : pers) cta_words = std::max(cta_words, cta_scratch_words(r->groups[i]));
    if (cta_words) {
      cta_words = (cta_words + 63) / 64 * 64;
      if (cudaMalloc(&r->cta_scratch, (size_t)r->grid * cta_words * 4) != cudaSuccess)
        return fail(FNT_RS_E_CUDA);
    }
    r->ra.cta_scratch = r->cta_scratch;
    r->ra.cta_words = cta_words;
  }
  // schedules of the per-group launches: tune each such plan on its widest group
  {
    const char* e = std::getenv("FNTRS_AUTOTUNE");
    if (!(e && e[0] == '0')) {
      std::map<fnt_rs_plan_s*, std::pair<size_t, bool>> widest;  // W, any decode
      for (auto& rg : r->groups) {
        if (rg.persistent) continue;
        auto& w = widest[rg.plan];
        w.first = std::max(w.first, rg.g.W);
        w.second = w.second || rg.g.positions != nullptr;
      }
      for (auto& kv : widest) {
        fnt_rs_tune_result res[8];
        int rc = fnt_rs_autotune(kv.first, kv.second.first, FNT_RS_OP_ENCODE, res, 8, stream);
        if (rc >= 0 && kv.second.second)
          rc = fnt_rs_autotune(kv.first, kv.second.first, FNT_RS_OP_DECODE, res, 8, stream);
        if (rc < 0) return fail(rc);
        ++r->tuned;
      }
    }
  }
  // the other groups' plan classes -> streams, heaviest first onto the least-loaded stream
  std::map<fnt_rs_plan_s*, double> work;
  for (auto& rg : r->groups) {
    if (rg.persistent) continue;
    const double n = rg.plan->n;
    work[rg.plan] += (double)rg.g.W * n * std::log2(n) * (rg.g.positions ? 4.0 : 1.0);
  }
  std::vector<std::pair<double, fnt_rs_plan_s*>> order;
  for (auto& kv : work) order.push_back({kv.second, kv.first});
  std::sort(order.begin(), order.end(), [](auto& a, auto& b) { return a.first > b.first; });
  const uint32_t S = std::max<uint32_t>(1, std::min<uint32_t>(nstreams, (uint32_t)order.size()));
  std::vector<double> load(S, 0.0);
  std::map<fnt_rs_plan_s*, int> assign;
  for (auto& o : order) {
    const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    assign[o.second] = s;
    load[s] += o.first;
  }
  r->streams.resize(S);
  r->ws.assign(S, nullptr);
  // Workspace per stream: for the per-group launches of the graph, and for
  // fnt_rs_ragged_run_plain, which runs every group (persistent ones too, on
  // stream 0's workspace) one after another through the plain calls.
  std::vector<size_t> wsb(S, 0);
  for (auto& rg : r->groups) {
    rg.stream = rg.persistent ? 0 : assign[rg.plan];
    fnt_rs_plan_s* p = rg.plan;
    // every schedule the plan may run (the tuner may have picked the direct product)
    size_t need = std::max(ws_bytes(p, rg.g.W, enc_nbuf_max(p)), direct_ws_bytes(p, rg.g.W));
    if (rg.g.positions) need = std::max(need, dec_ws_max(p, rg.g.W));
    wsb[rg.stream] = std::max(wsb[rg.stream], need);
  }
  for (uint32_t s = 0; s < S; ++s) {
    if (cudaStreamCreateWithFlags(&r->streams[s], cudaStreamNonBlocking) != cudaSuccess)
      return fail(FNT_RS_E_CUDA);
    if (wsb[s] && cudaMalloc(&r->ws[s], wsb[s]) != cudaSuccess) return fail(FNT_RS_E_CUDA);
  }
  // warm-up run (uncaptured): sets kernel attributes, fills table caches
  {
    int rc = run_persistent(r, st);
    if (rc) return fail(rc);
  }
  for (auto& rg : r->groups) {
    if (rg.persistent) continue;
    const int rc = run_group(rg, r->ws[rg.stream], st);
    if (rc) return fail(rc);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(FNT_RS_E_CUDA);
  // capture the batch
  if (cudaStreamCreateWithFlags(&r->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(FNT_RS_E_CUDA);
  r->joins.resize(S);
  for (uint32_t s = 0; s < S; ++s)
    if (cudaEventCreateWithFlags(&r->joins[s], cudaEventDisableTiming) != cudaSuccess)
      return fail(FNT_RS_E_CUDA);
  if (cudaStreamBeginCapture(r->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(FNT_RS_E_CUDA);
  int rc = FNT_RS_OK;
  cudaEventRecord(r->fork, r->cap);
  for (uint32_t s = 0; s < S; ++s) cudaStreamWaitEvent(r->streams[s], r->fork, 0);
  for (auto& rg : r->groups) {
    if (!rc && !rg.persistent) rc = run_group(rg, r->ws[rg.stream], r->streams[rg.stream]);
  }
  if (!rc) rc = run_persistent(r, r->cap);
  for (uint32_t s = 0; s < S; ++s) {
    cudaEventRecord(r->joins[s], r->streams[s]);
    cudaStreamWaitEvent(r->cap, r->joins[s], 0);
  }
  const cudaError_t ce = cudaStreamEndCapture(r->cap, &r->graph);
  if (rc) return fail(rc);
  if (ce != cudaSuccess || cudaGraphInstantiate(&r->exec, r->graph, 0) != cudaSuccess)
    return fail(FNT_RS_E_CUDA);
  *out = r;
  return FNT_RS_OK;
}

int fnt_rs_ragged_run(fnt_rs_ragged r, void* stream) {
  if (!r) return FNT_RS_E_ARG;
  return cudaGraphLaunch(r->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FNT_RS_OK
             : FNT_RS_E_CUDA;
}

int fnt_rs_ragged_run_plain(fnt_rs_ragged r, void* stream) {
  if (!r) return FNT_RS_E_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (auto& rg : r->groups) {
    const int rc = run_group(rg, r->ws[rg.stream], st);
    if (rc) return rc;
  }
  return FNT_RS_OK;
}

int fnt_rs_ragged_status(fnt_rs_ragged r, void* stream) {
  if (!r) return FNT_RS_E_ARG;
  int worst = FNT_RS_OK;
  for (auto& kv : r->plans) {
    const int s = fnt_rs_status(kv.second, stream);
    if (s == FNT_RS_E_TIMEOUT || (s == FNT_RS_E_RANGE && worst == FNT_RS_OK) ||
        s == FNT_RS_E_CUDA)
      worst = s;
  }
  return worst;
}

int fnt_rs_ragged_info(fnt_rs_ragged r, int* info, int cap) {
  if (!r || !info) return 0;
  int vals[6] = {(int)r->groups.size(), (int)r->plans.size(), (int)r->streams.size(),
                 r->npersistent, r->ra.nitems, r->tuned};
  const int m = std::min(cap, 6);
  for (int i = 0; i < m; ++i) info[i] = vals[i];
  return m;
}

}  // extern "C"
