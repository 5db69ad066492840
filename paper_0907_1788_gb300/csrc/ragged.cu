// Ragged batches: many groups of codewords, each with its own (n, k, W,
// erasure pattern), run by one CUDA graph launch.
//
// Every group is a full round trip: encode its source (Sec. II.B, e = FNT of
// the zero-padded source), build its pattern tables (steps 1-3), decode every
// codeword from the encoded matrix used as the receiver's slot buffer
// (steps 4-6).  Groups sharing (n, k) share one plan and run in order on one
// stream (their pattern builds share the plan's scratch); plan classes are
// spread over several streams by estimated work so that small groups overlap
// large ones.  The streams are captured into a single graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "internal.h"

namespace fntrs {

struct RaggedGroup {
  fnt_rs_group g{};
  fnt_rs_plan_s* plan = nullptr;
  PatternSlot tab;  // decode groups only
  int stream = 0;
};

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

static void free_group(RaggedGroup& rg) { free_pattern_tables(rg.tab); }

}  // namespace fntrs

extern "C" {

void fnt_rs_ragged_destroy(fnt_rs_ragged r) {
  if (!r) return;
  cudaDeviceSynchronize();
  if (r->exec) cudaGraphExecDestroy(r->exec);
  if (r->graph) cudaGraphDestroy(r->graph);
  for (auto& g : r->groups) free_group(g);
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
  // plan classes -> streams, heaviest first onto the least-loaded stream
  std::map<fnt_rs_plan_s*, double> work;
  for (auto& rg : r->groups) {
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
  std::vector<size_t> wsb(S, 0);
  for (auto& rg : r->groups) {
    rg.stream = assign[rg.plan];
    fnt_rs_plan_s* p = rg.plan;
    size_t need = ws_bytes(p, rg.g.W, enc_nbuf(p));
    if (rg.g.positions) need = std::max(need, ws_bytes(p, rg.g.W, dec_nbuf(p)));
    wsb[rg.stream] = std::max(wsb[rg.stream], need);
  }
  for (uint32_t s = 0; s < S; ++s) {
    if (cudaStreamCreateWithFlags(&r->streams[s], cudaStreamNonBlocking) != cudaSuccess)
      return fail(FNT_RS_E_CUDA);
    if (wsb[s] && cudaMalloc(&r->ws[s], wsb[s]) != cudaSuccess) return fail(FNT_RS_E_CUDA);
  }
  // warm-up run (uncaptured): sets kernel attributes, fills table caches
  for (auto& rg : r->groups) {
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
    if (!rc) rc = run_group(rg, r->ws[rg.stream], r->streams[rg.stream]);
  }
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
  int vals[3] = {(int)r->groups.size(), (int)r->plans.size(), (int)r->streams.size()};
  const int m = std::min(cap, 3);
  for (int i = 0; i < m; ++i) info[i] = vals[i];
  return m;
}

}  // extern "C"
