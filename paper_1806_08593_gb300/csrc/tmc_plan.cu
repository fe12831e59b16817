// tmc_plan.cu -- host runtime behind the C ABI of include/tmc.h.
//
// A plan turns the problem description into:
//   * a node table (one entry per latent of every instance) with all buffer offsets,
//   * the elimination schedule of Section 2.2: tree levels processed from the deepest up
//     (forward: messages to parents) and from the root down (adjoint),
//   * tile lists (node, first sample row) for every kernel, and
//   * one device workspace holding samples, means, messages, weights and gradient partials.
// Calls only enqueue kernels on the caller's stream; nothing allocates after creation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/tmc.h"
#include "tmc_internal.cuh"
#include "tmc_tc.cuh"

using namespace tmc;

namespace {

struct ProfileSlot {
  cudaEvent_t start, stop;
  int cls;
};

}  // namespace

struct tmc_plan_s {
  // description
  int B = 0, shared = 0, precision = 0;
  double prior_var = 1.0, obs_var = 1.0;
  int maxK = 0, maxd = 0, maxobs = 0, maxlevel = 0, maxn = 0;
  long long c_total = 0;  // size of dC (per-instance dC partials with shared parameters)
  int coupled = 0;      // coupled (non-factorised) proposal
  bool ragged = false;  // some instance has a different K or d from latent to latent
  long long shared_nW = 0, shared_nb = 0, shared_nC = 0, shared_rootW = 0;  // one instance's parameter sizes
  long long shared_nS = 0;  // one instance's packed dp x dp blocks of the non-root latents
  long long shared_nL2 = 0; // the leaves' dimension squared (the instance sum of the leaf moments)
  int root_fanout = 0;  // most children of any instance's root
  long long tot_nk = 0, tot_nkd = 0, tot_q = 0, tot_W = 0;

  std::vector<NodeInfo> nodes;
  std::vector<InstInfo> insts;
  std::vector<int> children, nonroot;
  std::vector<long long> fac_off;  // unfused baseline: start of each edge's K x K factor block
  std::vector<int4> root_chunks;     // wide roots: chunks of children (instance, begin, end)
  std::vector<int> root_chunk_off;   // [B + 1]
  int4* d_root_chunks = nullptr;
  int* d_root_chunk_off = nullptr;
  long long fac_total = 0;
  long long* d_fac_off = nullptr;

  // tile lists: [begin, end) ranges into one device array
  std::vector<Tile> tiles;
  int t_sample_b = 0, t_sample_e = 0, t_leaf_b = 0, t_leaf_e = 0, t_proj_b = 0, t_proj_e = 0;
  std::vector<int> t_level_b, t_level_e;    // per level: edges whose child is there, parent rows
  std::vector<int> t_clevel_b, t_clevel_e;  // the same edges, child rows (columns adjoint pass)

  // device
  NodeInfo* d_nodes = nullptr;
  InstInfo* d_insts = nullptr;
  int* d_children = nullptr;
  int* d_nonroot = nullptr;
  Tile* d_tiles = nullptr;
  // FP32 path, latents with more than kParamChunk children: their 64-row tiles, the chunk count
  // of the largest, and the size of all their [K][d] children sums
  std::vector<Tile> cs_items;
  Tile* d_cs_items = nullptr;
  int cs_chunks = 0;
  long long cs_total = 0;
  float* cs_part = nullptr;
  int* d_err = nullptr;
  void* ws = nullptr;
  float* dc_part = nullptr;  // FP32 path: per-chunk dC partials of instances with many latents
  size_t ws_bytes = 0;
  Dev dev{};
  tc::TcWork tcw{};

  // fault injection (TMC_FAULT, read at creation) and the dependency-wait budget
  int fault = 0;
  long long wait_limit = kWaitLimitDefault;

  // state
  bool fwd_done = false;
  tmc_inputs last_in{};

  // profiling
  bool prof = false;
  std::vector<ProfileSlot> slots;
  size_t slot_next = 0;
  double prof_ms[TMC_KC_COUNT] = {0};
  long long prof_n[TMC_KC_COUNT] = {0};
};

namespace {

tmc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? TMC_OK : TMC_ERR_CUDA; }

// Host-side fault injection for tests of the error paths (nothing here makes a GPU fault).
enum { kFaultNone = 0, kFaultAlloc = 1, kFaultLaunch = 2, kFaultStall = 3 };
int fault_from_env() {
  const char* f = std::getenv("TMC_FAULT");
  if (!f) return kFaultNone;
  if (!std::strcmp(f, "alloc")) return kFaultAlloc;
  if (!std::strcmp(f, "launch")) return kFaultLaunch;
  if (!std::strcmp(f, "stall")) return kFaultStall;
  return kFaultNone;
}

void drain_profile(tmc_plan p) {
  for (size_t i = 0; i < p->slot_next; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->slots[i].start, p->slots[i].stop) == cudaSuccess) {
      p->prof_ms[p->slots[i].cls] += ms;
      p->prof_n[p->slots[i].cls] += 1;
    }
  }
  p->slot_next = 0;
}

// Launch wrapper: optional event pair around the launch, then the launch error check.
template <class F>
tmc_status timed(tmc_plan p, int cls, cudaStream_t s, F&& launch) {
  ProfileSlot* slot = nullptr;
  if (p->prof) {
    if (p->slot_next == p->slots.size()) {  // pool exhausted: settle and reuse
      cudaStreamSynchronize(s);
      drain_profile(p);
    }
    slot = &p->slots[p->slot_next++];
    slot->cls = cls;
    cudaEventRecord(slot->start, s);
  }
  launch();
  cudaError_t e = cudaGetLastError();
  if (slot) cudaEventRecord(slot->stop, s);
  return cuda_status(e);
}

#define TRY(x)                        \
  do {                                \
    tmc_status _st = (x);             \
    if (_st != TMC_OK) return _st;    \
  } while (0)

template <class T>
tmc_status upload(T** dst, const std::vector<T>& v) {
  if (v.empty()) { *dst = nullptr; return TMC_OK; }
  if (cudaMalloc(dst, sizeof(T) * v.size()) != cudaSuccess) return TMC_ERR_NOMEM;
  return cuda_status(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
}

tmc_status build_plan(const tmc_problem_desc* ds, tmc_plan p) {
  const int B = ds->num_instances;
  if (B < 1 || !ds->n || !ds->parent || !ds->K || !ds->d || !ds->obs_dim) return TMC_ERR_INVALID_ARG;
  if (!(ds->prior_var > 0.0) || !(ds->obs_var > 0.0) || !std::isfinite(ds->prior_var) ||
      !std::isfinite(ds->obs_var))
    return TMC_ERR_INVALID_ARG;
  if (ds->precision != TMC_PREC_FP32 && ds->precision != TMC_PREC_FP16_TC &&
      ds->precision != TMC_PREC_FP32_UNFUSED)
    return TMC_ERR_INVALID_ARG;
  p->B = B;
  p->shared = ds->shared_params ? 1 : 0;
  p->coupled = ds->coupled_proposal ? 1 : 0;
  p->precision = ds->precision;
  p->prior_var = ds->prior_var;
  p->obs_var = ds->obs_var;

  long long poff = 0, off_nk = 0, off_nkd = 0, off_e = 0, off_q = 0, off_W = 0, off_bias = 0,
            off_C = 0, off_x = 0, off_pW = 0, off_pC = 0;
  for (int b = 0; b < B; ++b) {
    const int n = ds->n[b], obs = ds->obs_dim[b];
    if (n < 1 || obs < 1) return TMC_ERR_INVALID_ARG;
    if (obs > kMaxD) return TMC_ERR_UNSUPPORTED;
    const int* par = ds->parent + poff;
    if (par[0] != -1) return TMC_ERR_INVALID_ARG;
    for (int i = 1; i < n; ++i)
      if (par[i] < 0 || par[i] >= i) return TMC_ERR_INVALID_ARG;
    // per-latent sizes: K_node / d_node when given, else the instance's K[b] / d[b]
    std::vector<int> Kv(n), dv(n);
    for (int i = 0; i < n; ++i) {
      Kv[i] = ds->K_node ? ds->K_node[poff + i] : ds->K[b];
      dv[i] = ds->d_node ? ds->d_node[poff + i] : ds->d[b];
      if (Kv[i] < 1 || dv[i] < 1) return TMC_ERR_INVALID_ARG;
      if (Kv[i] > kMaxK || dv[i] > kMaxD) return TMC_ERR_UNSUPPORTED;
      if (Kv[i] != Kv[0] || dv[i] != dv[0]) p->ragged = true;
    }
    const int node0 = (int)p->nodes.size();
    // children lists, levels, and the leaves' common dimension (one C per instance)
    std::vector<std::vector<int>> ch(n);
    std::vector<int> level(n, 0);
    for (int i = 1; i < n; ++i) {
      ch[par[i]].push_back(i);
      level[i] = level[par[i]] + 1;
    }
    int dl = -1, Kmax = 0;
    for (int i = 0; i < n; ++i) {
      Kmax = std::max(Kmax, Kv[i]);
      if (ch[i].empty()) {
        if (dl >= 0 && dl != dv[i]) return TMC_ERR_INVALID_ARG;
        dl = dv[i];
      }
    }
    if (p->coupled)  // sample k of a latent is drawn given its parent's sample k
      for (int i = 1; i < n; ++i)
        if (Kv[i] > Kv[par[i]]) return TMC_ERR_INVALID_ARG;
    if (p->shared && b > 0) {
      if (n != ds->n[0] || obs != ds->obs_dim[0]) return TMC_ERR_INVALID_ARG;
      for (int i = 0; i < n; ++i)
        if (par[i] != ds->parent[i] || dv[i] != p->nodes[i].d) return TMC_ERR_INVALID_ARG;
    }
    // instance-level offsets.  Per-sample workspace blocks hold Kmax rows per latent, so a
    // latent's block also holds the K_parent values indexed by its parent's samples (the
    // message it sends, the parent-sample conditional means).
    const long long iW = p->shared ? 0 : off_W, ib = p->shared ? 0 : off_bias,
                    iC = p->shared ? 0 : off_C;
    int leaves = 0;
    long long e = 0, q = 0, w = 0, kd = 0, sq = 0;
    for (int i = 0; i < n; ++i) {
      NodeInfo nd{};
      nd.b = b;
      nd.i = i;
      nd.parent = i ? node0 + par[i] : -1;
      nd.K = Kv[i];
      nd.log_K = std::log((double)Kv[i]);
      nd.d = dv[i];
      nd.Kp = i ? Kv[par[i]] : 0;
      nd.dp = i ? dv[par[i]] : dv[0];
      nd.obs = obs;
      nd.leaf_slot = ch[i].empty() ? leaves++ : -1;
      nd.child_begin = (int)p->children.size();
      for (int c : ch[i]) p->children.push_back(node0 + c);
      nd.child_end = (int)p->children.size();
      if (i == 0) p->root_fanout = std::max(p->root_fanout, nd.child_end - nd.child_begin);
      nd.level = level[i];
      nd.root = node0;
      nd.off_nk = off_nk + (long long)i * Kmax;
      nd.off_nkd = off_nkd + kd;
      nd.off_e = off_e + e;
      nd.off_q = off_q + q;
      nd.off_W = iW + w;
      nd.off_bias = ib + q;
      nd.off_C = iC;
      nd.off_x = off_x + (long long)(nd.leaf_slot >= 0 ? nd.leaf_slot : 0) * obs;
      nd.off_pW = off_pW + w;
      nd.off_A = off_pW + w;  // the couplings are per instance, laid out like unshared W
      nd.off_S = sq;
      if (i) sq += (long long)nd.dp * nd.dp;
      p->nodes.push_back(nd);
      p->maxlevel = std::max(p->maxlevel, level[i]);
      e += (long long)Kv[i] * dv[i];
      kd += (long long)Kmax * dv[i];
      q += dv[i];
      w += (long long)dv[i] * nd.dp;
      p->maxK = std::max(p->maxK, Kv[i]);
      p->maxd = std::max(p->maxd, dv[i]);
    }
    InstInfo in{};
    in.node0 = node0;
    in.n = n;
    in.K = Kv[0];
    in.d = dl;
    in.obs = obs;
    in.off_C = iC;
    in.off_pC = off_pC;
    p->insts.push_back(in);
    p->maxobs = std::max(p->maxobs, obs);
    p->maxn = std::max(p->maxn, n);
    if (b == 0) {  // sizes of one instance's parameters (the shared reduction)
      p->shared_nW = w;
      p->shared_nb = q;
      p->shared_nC = (long long)obs * dl;
      p->shared_rootW = (long long)dv[0] * dv[0];
      p->shared_nS = sq;
      p->shared_nL2 = (long long)dl * dl;
    }
    poff += n;
    off_nk += (long long)n * Kmax;
    off_nkd += kd;
    off_e += e;
    off_q += q;
    off_x += (long long)leaves * obs;
    off_pW += w;
    off_pC += (long long)obs * dl;
    if (!p->shared) {
      off_W += w;
      off_bias += q;
      off_C += (long long)obs * dl;
    }
  }
  p->tot_nk = off_nk;
  p->tot_nkd = off_nkd;
  p->tot_q = off_q;
  p->c_total = p->shared ? off_pC : off_C;
  // the materialised-factor baseline is built for one K and d per instance and a factorised
  // proposal
  if ((p->ragged || p->coupled) && p->precision == TMC_PREC_FP32_UNFUSED) return TMC_ERR_UNSUPPORTED;

  // tile lists (a tile is a node and 64 of its rows: its own samples, or, for the tiles of an
  // edge p -> i in the projection, forward and rows-adjoint lists, the parent's samples)
  auto add_tiles = [&](int g) {
    for (int r = 0; r < p->nodes[g].K; r += kTile) p->tiles.push_back(Tile{g, r});
  };
  auto add_parent_tiles = [&](int g) {
    for (int r = 0; r < p->nodes[g].Kp; r += kTile) p->tiles.push_back(Tile{g, r});
  };
  const int G = (int)p->nodes.size();
  p->t_sample_b = (int)p->tiles.size();
  for (int g = 0; g < G; ++g) add_tiles(g);
  p->t_sample_e = (int)p->tiles.size();
  p->t_leaf_b = (int)p->tiles.size();
  for (int g = 0; g < G; ++g)
    if (p->nodes[g].leaf_slot >= 0) add_tiles(g);
  p->t_leaf_e = (int)p->tiles.size();
  p->t_proj_b = (int)p->tiles.size();
  for (int g = 0; g < G; ++g)
    if (p->nodes[g].parent >= 0) {
      add_parent_tiles(g);
      p->nonroot.push_back(g);
    }
  p->t_proj_e = (int)p->tiles.size();
  if (p->precision == TMC_PREC_FP32_UNFUSED) {
    p->fac_off.assign(G, 0);
    for (int g = 0; g < G; ++g)
      if (p->nodes[g].parent >= 0) {
        p->fac_off[g] = p->fac_total;
        p->fac_total += (long long)p->nodes[g].Kp * p->nodes[g].K;
      }
  }
  p->t_level_b.assign(p->maxlevel + 1, 0);
  p->t_level_e.assign(p->maxlevel + 1, 0);
  p->t_clevel_b.assign(p->maxlevel + 1, 0);
  p->t_clevel_e.assign(p->maxlevel + 1, 0);
  p->t_clevel_b[0] = (int)p->tiles.size();  // the roots' own rows (coupled proposals' T)
  for (int g = 0; g < G; ++g)
    if (p->nodes[g].level == 0) add_tiles(g);
  p->t_clevel_e[0] = (int)p->tiles.size();
  for (int L = 1; L <= p->maxlevel; ++L) {
    p->t_level_b[L] = (int)p->tiles.size();
    for (int g = 0; g < G; ++g)
      if (p->nodes[g].level == L) add_parent_tiles(g);
    p->t_level_e[L] = (int)p->tiles.size();
    p->t_clevel_b[L] = (int)p->tiles.size();
    for (int g = 0; g < G; ++g)
      if (p->nodes[g].level == L) add_tiles(g);
    p->t_clevel_e[L] = (int)p->tiles.size();
  }
  return TMC_OK;
}

tmc_status alloc_device(tmc_plan p) {
  if (p->fault == kFaultAlloc) return TMC_ERR_NOMEM;  // as if the first cudaMalloc failed
  if (p->root_fanout > kRootChunk) {  // chunks of every root's children (fixed summation order)
    p->root_chunks.clear();
    p->root_chunk_off.assign(p->B + 1, 0);
    for (int b = 0; b < p->B; ++b) {
      p->root_chunk_off[b] = (int)p->root_chunks.size();
      const NodeInfo& r = p->nodes[p->insts[b].node0];
      for (int c = r.child_begin; c < r.child_end; c += kRootChunk)
        p->root_chunks.push_back(int4{b, c, std::min(r.child_end, c + kRootChunk), 0});
    }
    p->root_chunk_off[p->B] = (int)p->root_chunks.size();
    TRY(upload(&p->d_root_chunks, p->root_chunks));
    TRY(upload(&p->d_root_chunk_off, p->root_chunk_off));
  }
  p->cs_items.clear();
  p->cs_chunks = 0;
  p->cs_total = 0;
  for (int g = 0; g < (int)p->nodes.size(); ++g) {
    NodeInfo& nd = p->nodes[g];
    nd.off_cs = -1;
    const int nch = nd.child_end - nd.child_begin;
    if (p->precision == TMC_PREC_FP16_TC || nch <= kParamChunk) continue;
    nd.off_cs = p->cs_total;
    p->cs_total += (long long)nd.K * nd.d;
    p->cs_chunks = std::max(p->cs_chunks, (nch + kParamChunk - 1) / kParamChunk);
    for (int r = 0; r < nd.K; r += kTile) p->cs_items.push_back(Tile{g, r});
  }
  if (!p->cs_items.empty()) TRY(upload(&p->d_cs_items, p->cs_items));
  TRY(upload(&p->d_nodes, p->nodes));
  TRY(upload(&p->d_insts, p->insts));
  TRY(upload(&p->d_children, p->children));
  TRY(upload(&p->d_nonroot, p->nonroot));
  TRY(upload(&p->d_tiles, p->tiles));
  TRY(upload(&p->d_fac_off, p->fac_off));
  if (cudaMalloc(&p->d_err, sizeof(int)) != cudaSuccess) return TMC_ERR_NOMEM;
  if (cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess) return TMC_ERR_CUDA;

  const long long nk = p->tot_nk, nkd = p->tot_nkd, G = (long long)p->nodes.size();
  // per-instance dW partials: the FP32 path with shared parameters (the tensor-core path sums
  // its dW terms per instance group itself)
  const long long nW = (p->shared && p->precision != TMC_PREC_FP16_TC) ? (long long)p->B * p->shared_nW : 0;
  const long long nb = p->shared ? (long long)p->B * p->shared_nb : 0;
  const long long nC = p->shared ? (long long)p->B * p->shared_nC : 0;
  // layout: 256-byte aligned sub-buffers
  struct Sub { void** dst; size_t bytes; };
  float *zt, *mut, *zn, *mun, *u, *beta, *lam, *q, *nodemax, *dmu, *gz, *pW, *pbias, *pC, *fac, *rsum;
  // row-sum scratch: B instances (or fewer instance groups) of one instance's largest block
  const bool tc_plan = p->precision == TMC_PREC_FP16_TC;
  // FP32 path: the dC sum of an instance with more than kParamChunk latents is split into
  // chunks (partials, then rows_sum)
  const long long dc_chunks = tc_plan ? 1 : (p->maxn + kParamChunk - 1) / kParamChunk;
  const long long ndcp = dc_chunks > 1 ? dc_chunks * p->c_total : 0;
  const long long ncsp = p->cs_total ? (long long)p->cs_chunks * p->cs_total : 0;
  const long long nrs = std::max(std::max(
      p->shared ? rows_sum_scratch(p->B, std::max(std::max(std::max(p->shared_nW, p->shared_nS), p->shared_nL2),
                                                  std::max(p->shared_nb, p->shared_nC)))
                : 0ll,
      ndcp ? rows_sum_scratch(dc_chunks, p->c_total) : 0ll),
      ncsp ? rows_sum_scratch(p->cs_chunks, p->cs_total) : 0ll);
  float* csum = nullptr;
  double *nodeconst, *root_part;
  // FP32-path sample vectors (unused on the tc path, except T and G of coupled proposals, kept
  // in mut and gz)
  const long long nkd32 = tc_plan ? 0 : nkd, nkdc = (tc_plan && p->coupled) ? nkd : nkd32;
  const long long nkdt = p->coupled ? nkd : 0;  // T of coupled proposals (its own buffer: mu~
                                                // must survive for a second backward call)
  float* tqb = nullptr;
  std::vector<Sub> subs = {
      {(void**)&zt, sizeof(float) * nkd},      {(void**)&mut, sizeof(float) * nkd32},
      {(void**)&dmu, sizeof(float) * nkd32},   {(void**)&gz, sizeof(float) * nkdc},
      {(void**)&tqb, sizeof(float) * nkdt},
      {(void**)&zn, sizeof(float) * nk},       {(void**)&mun, sizeof(float) * nk},
      {(void**)&u, sizeof(float) * nk},        {(void**)&beta, sizeof(float) * nk},
      {(void**)&lam, sizeof(float) * nk},      {(void**)&q, sizeof(float) * nk},
      {(void**)&nodemax, sizeof(float) * G},   {(void**)&nodeconst, sizeof(double) * G},
      {(void**)&pW, sizeof(float) * nW},       {(void**)&pbias, sizeof(float) * nb},
      {(void**)&pC, sizeof(float) * nC},       {(void**)&rsum, sizeof(float) * nrs},
      {(void**)&p->dc_part, sizeof(float) * ndcp},
      {(void**)&p->cs_part, sizeof(float) * ncsp},
      {(void**)&csum, sizeof(float) * p->cs_total},
      {(void**)&fac, sizeof(float) * p->fac_total},
      {(void**)&root_part, sizeof(double) * p->root_chunks.size() * p->maxK},
  };
  std::vector<tc::TcSub> tsubs;
  p->tcw.t.shared = p->shared;
  p->tcw.precision = p->precision;
  p->tcw.shared_nW = p->shared_nW;
  p->tcw.shared_nS = p->shared_nS;
  p->tcw.shared_nb = p->shared_nb;
  if (tc_plan) tc::workspace_layout(p->tcw, p->nodes, nk, nkd, tsubs);
  size_t total = 0;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  for (auto& s : subs) total += al(s.bytes);
  for (auto& s : tsubs) total += al(s.bytes);
  if (cudaMalloc(&p->ws, total) != cudaSuccess) { p->ws = nullptr; return TMC_ERR_NOMEM; }
  p->ws_bytes = total;
  char* base = (char*)p->ws;
  for (auto& s : subs) { *s.dst = base; base += al(s.bytes); }
  for (auto& s : tsubs) { *s.dst = base; base += al(s.bytes); }

  Dev& D = p->dev;
  D.nodes = p->d_nodes;
  D.insts = p->d_insts;
  D.children = p->d_children;
  D.num_nodes = (int)G;
  D.num_inst = p->B;
  D.inv_var = (float)(1.0 / p->prior_var);
  D.inv_obs_var = (float)(1.0 / p->obs_var);
  D.prior_var = p->prior_var;
  D.obs_var = p->obs_var;
  D.log_prior_var = std::log(p->prior_var);
  D.log_obs_var = std::log(p->obs_var);
  D.shared = p->shared;
  D.zt = zt; D.mut = mut; D.zn = zn; D.mun = mun; D.u = u; D.beta = beta; D.lam = lam; D.q = q;
  D.nodemax = nodemax; D.nodeconst = nodeconst; D.dmu = dmu; D.gz = gz;
  D.pW = nW ? pW : nullptr; D.pbias = nb ? pbias : nullptr; D.pC = nC ? pC : nullptr;
  D.rsum = nrs ? rsum : nullptr;
  D.csum = p->cs_total ? csum : nullptr;
  D.err = p->d_err;
  D.wait_limit = p->wait_limit;
  D.coupled = p->coupled;
  D.tq = p->coupled ? tqb : nullptr;
  D.gsrc = p->coupled ? gz : nullptr;  // G: written by the FP32 node gradients or k_dz_tc
  D.fac = p->fac_total ? fac : nullptr;
  D.fac_off = p->d_fac_off;
  D.root_chunks = p->d_root_chunks;
  D.root_chunk_off = p->d_root_chunk_off;
  D.root_part = p->root_chunks.empty() ? nullptr : root_part;
  D.root_nchunk = (int)p->root_chunks.size();
  D.root_ld = p->maxK;
  if (tc_plan && p->fault == kFaultStall) {
    // the deepest non-root node of instance 0: its forward tiles are left out of the
    // persistent launch, so its parent's tiles wait on a count that never arrives
    for (int i = p->insts[0].n - 1; i >= 1; --i) {
      const int g = p->insts[0].node0 + i;
      if (p->tcw.stall_node < 0 || p->nodes[g].level > p->nodes[p->tcw.stall_node].level) p->tcw.stall_node = g;
    }
  }
  if (tc_plan) TRY(tc::prepare(p->tcw, p->nodes, p->tiles, p->maxK, p->maxd));
  return TMC_OK;
}

void free_plan(tmc_plan p) {
  cudaFree(p->d_nodes);
  cudaFree(p->d_insts);
  cudaFree(p->d_children);
  cudaFree(p->d_nonroot);
  cudaFree(p->d_tiles);
  cudaFree(p->d_cs_items);
  cudaFree(p->d_fac_off);
  cudaFree(p->d_root_chunks);
  cudaFree(p->d_root_chunk_off);
  cudaFree(p->d_err);
  cudaFree(p->ws);
  tc::release(p->tcw);
  for (auto& s : p->slots) {
    cudaEventDestroy(s.start);
    cudaEventDestroy(s.stop);
  }
  delete p;
}

bool inputs_ok(const tmc_inputs* in) {
  return in && in->eps && in->q_mean && in->q_logstd && in->W && in->bias && in->C && in->x;
}

}  // namespace

extern "C" {

const char* tmc_status_string(tmc_status s) {
  switch (s) {
    case TMC_OK: return "TMC_OK";
    case TMC_ERR_INVALID_ARG: return "TMC_ERR_INVALID_ARG";
    case TMC_ERR_UNSUPPORTED: return "TMC_ERR_UNSUPPORTED";
    case TMC_ERR_NOMEM: return "TMC_ERR_NOMEM";
    case TMC_ERR_CUDA: return "TMC_ERR_CUDA";
    case TMC_ERR_NUMERIC: return "TMC_ERR_NUMERIC";
    case TMC_ERR_TIMEOUT: return "TMC_ERR_TIMEOUT";
    case TMC_ERR_STATE: return "TMC_ERR_STATE";
  }
  return "TMC_ERR_UNKNOWN";
}

tmc_status tmc_plan_create(const tmc_problem_desc* desc, tmc_plan* out) {
  if (!desc || !out) return TMC_ERR_INVALID_ARG;
  *out = nullptr;
  tmc_plan p = new (std::nothrow) tmc_plan_s();
  if (!p) return TMC_ERR_NOMEM;
  p->fault = fault_from_env();
  tmc_status st = build_plan(desc, p);
  if (st == TMC_OK && p->precision == TMC_PREC_FP16_TC)
    st = tc::supported(p->nodes, p->precision);
  if (st == TMC_OK) st = alloc_device(p);
  if (st != TMC_OK) {
    free_plan(p);
    return st;
  }
  *out = p;
  return TMC_OK;
}

tmc_status tmc_plan_destroy(tmc_plan p) {
  if (!p) return TMC_OK;
  cudaDeviceSynchronize();
  free_plan(p);
  return TMC_OK;
}

tmc_status tmc_plan_workspace_bytes(tmc_plan p, size_t* bytes) {
  if (!p || !bytes) return TMC_ERR_INVALID_ARG;
  *bytes = p->ws_bytes;
  return TMC_OK;
}

tmc_status tmc_log_marginal(tmc_plan p, const tmc_inputs* in, double* log_phat, void* stream) {
  if (!p || !inputs_ok(in) || !log_phat) return TMC_ERR_INVALID_ARG;
  if (p->coupled && !in->q_A) return TMC_ERR_INVALID_ARG;
  if (p->fault == kFaultLaunch) return TMC_ERR_CUDA;  // as if the first launch failed
  cudaStream_t s = (cudaStream_t)stream;
  Dev D = p->dev;
  D.eps = in->eps; D.q_mean = in->q_mean; D.q_logstd = in->q_logstd;
  D.W = in->W; D.bias = in->bias; D.C = in->C; D.x = in->x;
  D.q_A = p->coupled ? in->q_A : nullptr;
  D.log_phat = log_phat;
  const Tile* T = p->d_tiles;
  const bool tc_path = p->precision == TMC_PREC_FP16_TC;
  // coupled proposals: z~_i += A_i z~_p, level by level from the root (FP32 samples)
  auto couple_samples = [&]() -> tmc_status {
    for (int L = 1; L <= p->maxlevel; ++L) {
      const int b = p->t_clevel_b[L], e = p->t_clevel_e[L];
      TRY(timed(p, TMC_KC_SAMPLE, s, [&] { launch_couple_fwd(D, T + b, e - b, s); }));
    }
    return TMC_OK;
  };
  TRY(timed(p, TMC_KC_SAMPLE, s, [&] { launch_node_const(D, s); }));
  if (tc_path) {
    // split W_i and c_i first: the sampling kernel forms z~ . c_i, the conditional means are
    // formed inside the edge kernels
    TRY(timed(p, TMC_KC_PROJECT, s, [&] { tc::launch_pack(p->tcw, D, s); }));
    if (p->coupled) {  // FP32 samples through the couplings, then split into the tc operands
      TRY(timed(p, TMC_KC_SAMPLE, s, [&] { launch_sample(D, T + p->t_sample_b, p->t_sample_e - p->t_sample_b, s); }));
      TRY(couple_samples());
      TRY(timed(p, TMC_KC_SAMPLE, s, [&] { tc::launch_pack_z(p->tcw, D, s); }));
    } else {
      TRY(timed(p, TMC_KC_SAMPLE, s, [&] { tc::launch_sample(p->tcw, D, s); }));
    }
    TRY(timed(p, TMC_KC_SAMPLE, s, [&] { tc::launch_obs(p->tcw, D, s); }));
  } else {
    TRY(timed(p, TMC_KC_SAMPLE, s, [&] { launch_sample(D, T + p->t_sample_b, p->t_sample_e - p->t_sample_b, s); }));
    if (p->coupled) TRY(couple_samples());
    TRY(timed(p, TMC_KC_SAMPLE, s, [&] { launch_obs_fwd(D, T + p->t_leaf_b, p->t_leaf_e - p->t_leaf_b, s); }));
    TRY(timed(p, TMC_KC_PROJECT, s, [&] { launch_project(D, T + p->t_proj_b, p->t_proj_e - p->t_proj_b, s); }));
  }
  if (tc_path) {
    if (p->maxlevel >= 1) TRY(timed(p, TMC_KC_EDGE_FWD, s, [&] { tc::launch_edge_fwd(p->tcw, D, s); }));
  } else {
    const bool unfused = p->precision == TMC_PREC_FP32_UNFUSED;
    if (unfused)  // every pairwise log-factor of every edge into device memory first
      TRY(timed(p, TMC_KC_EDGE_FWD, s, [&] { launch_factors_f32(D, T + p->t_proj_b, p->t_proj_e - p->t_proj_b, p->maxK, s); }));
    for (int L = p->maxlevel; L >= 1; --L) {
      const int b = p->t_level_b[L], e = p->t_level_e[L];
      if (unfused)
        TRY(timed(p, TMC_KC_EDGE_FWD, s, [&] { launch_lse_rows_f32(D, T + b, e - b, p->maxK, s); }));
      else
        TRY(timed(p, TMC_KC_EDGE_FWD, s, [&] { launch_edge_fwd_f32(D, T + b, e - b, p->maxK, s); }));
    }
  }
  TRY(timed(p, TMC_KC_ROOT, s, [&] { launch_root(D, p->maxK, p->root_fanout, s); }));
  p->fwd_done = true;
  p->last_in = *in;
  return TMC_OK;
}

tmc_status tmc_backward(tmc_plan p, const tmc_inputs* in, const double* grad_out,
                        const tmc_grads* g, void* stream) {
  if (!p || !inputs_ok(in) || !g) return TMC_ERR_INVALID_ARG;
  if (!p->fwd_done || std::memcmp(&p->last_in, in, sizeof(tmc_inputs)) != 0) return TMC_ERR_STATE;
  if (p->fault == kFaultLaunch) return TMC_ERR_CUDA;
  const bool tc_path = p->precision == TMC_PREC_FP16_TC;
  cudaStream_t s = (cudaStream_t)stream;
  Dev D = p->dev;
  D.eps = in->eps; D.q_mean = in->q_mean; D.q_logstd = in->q_logstd;
  D.W = in->W; D.bias = in->bias; D.C = in->C; D.x = in->x;
  D.grad_out = grad_out;
  D.dz = g->dz; D.deps = g->deps; D.dq_mean = g->dq_mean; D.dq_logstd = g->dq_logstd;
  D.dW = g->dW; D.dbias = g->dbias; D.dC = g->dC;
  D.q_A = p->coupled ? in->q_A : nullptr;
  D.dq_A = p->coupled ? g->dq_A : nullptr;
  const Tile* T = p->d_tiles;
  // per-sample path gradients are needed for dz / deps, and, with coupled proposals, for the
  // proposal gradients too (they run through the couplings sample by sample)
  const bool sample_grads = g->dz || g->deps || p->coupled;
  if (tc_path) {
    if (p->maxlevel >= 1) TRY(timed(p, TMC_KC_EDGE_BWD, s, [&] { tc::launch_edge_bwd(p->tcw, D, s); }));
    if (sample_grads && p->maxlevel >= 1)
      TRY(timed(p, TMC_KC_SAMPLE_GRAD, s, [&] { tc::launch_edge_rows(p->tcw, D, s); }));
  } else {
    for (int L = 1; L <= p->maxlevel; ++L) {
      const int b = p->t_level_b[L], e = p->t_level_e[L], cb = p->t_clevel_b[L], ce = p->t_clevel_e[L];
      TRY(timed(p, TMC_KC_EDGE_BWD, s, [&] { launch_edge_bwd_cols_f32(D, T + cb, ce - cb, p->maxK, s); }));
      TRY(timed(p, TMC_KC_EDGE_BWD, s, [&] { launch_edge_bwd_rows_f32(D, T + b, e - b, p->maxK, s); }));
    }
  }
  // coupled proposals: T = G + sum_c A_c^T T_c from the leaves up, then dz, deps, dlogs, dA
  auto couple_grads = [&]() -> tmc_status {
    for (int L = p->maxlevel; L >= 0; --L) {
      const int b = p->t_clevel_b[L], e = p->t_clevel_e[L];
      TRY(timed(p, TMC_KC_SAMPLE_GRAD, s, [&] { launch_couple_T(D, T + b, e - b, s); }));
    }
    return timed(p, TMC_KC_SAMPLE_GRAD, s, [&] {
      launch_couple_out(D, T + p->t_sample_b, p->t_sample_e - p->t_sample_b, p->d_nonroot,
                        (int)p->nonroot.size(), p->maxd, s);
    });
  };
  if (tc_path) {
    TRY(timed(p, TMC_KC_PARAM, s, [&] { tc::launch_unpack_grads(p->tcw, D, s); }));
    if (sample_grads) TRY(timed(p, TMC_KC_SAMPLE_GRAD, s, [&] { tc::launch_dz(p->tcw, D, s); }));
    if (p->coupled) TRY(couple_grads());  // (k_dz_tc wrote the path gradients G)
  } else {
    if (!p->cs_items.empty())
      TRY(timed(p, TMC_KC_PARAM, s, [&] {
        launch_child_sum(D, p->d_cs_items, (int)p->cs_items.size(), p->maxd, p->cs_chunks, p->cs_total,
                         p->cs_part, s);
      }));
    TRY(timed(p, TMC_KC_PARAM, s, [&] { launch_node_grad(D, T + p->t_sample_b, p->t_sample_e - p->t_sample_b, s); }));
    TRY(timed(p, TMC_KC_PARAM, s, [&] { launch_node_reduce(D, s); }));
    if (p->coupled) TRY(couple_grads());
    if (g->dW || g->dbias)
      TRY(timed(p, TMC_KC_PARAM, s, [&] { launch_param_dW(D, p->d_nonroot, (int)p->nonroot.size(), p->maxd, s); }));
    if (g->dC)
      TRY(timed(p, TMC_KC_PARAM, s, [&] {
        launch_param_dC(D, p->maxd, p->maxobs, p->maxn, p->c_total, p->dc_part, s);
      }));
  }
  if (p->shared && (g->dW || g->dbias || g->dC))
    TRY(timed(p, TMC_KC_PARAM, s, [&] {
      launch_shared_reduce(D, p->shared_nW, p->shared_nb, p->shared_nC, p->shared_rootW, tc_path, s);
    }));
  return TMC_OK;
}

tmc_status tmc_plan_sync_status(tmc_plan p, void* stream) {
  if (!p) return TMC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TMC_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TMC_ERR_CUDA;
  if (err && cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess) return TMC_ERR_CUDA;
  if (err & kErrTimeout) return TMC_ERR_TIMEOUT;
  if (err & kErrNumeric) return TMC_ERR_NUMERIC;
  return TMC_OK;
}

tmc_status tmc_plan_set_wait_limit(tmc_plan p, long long cycles) {
  if (!p || cycles < 1) return TMC_ERR_INVALID_ARG;
  p->wait_limit = cycles;
  p->dev.wait_limit = cycles;
  return TMC_OK;
}

tmc_status tmc_plan_set_schedule(tmc_plan p, int schedule) {
  if (!p) return TMC_ERR_INVALID_ARG;
  if (!(p->precision == TMC_PREC_FP16_TC)) return TMC_ERR_UNSUPPORTED;
  return tc::set_schedule(p->tcw, p->nodes, schedule);
}

tmc_status tmc_plan_get_schedule(tmc_plan p, int* schedule) {
  if (!p || !schedule) return TMC_ERR_INVALID_ARG;
  *schedule = p->tcw.schedule;
  return TMC_OK;
}

tmc_status tmc_plan_set_tuning(tmc_plan p, int knob, int value) {
  if (!p) return TMC_ERR_INVALID_ARG;
  if (!(p->precision == TMC_PREC_FP16_TC)) return TMC_ERR_UNSUPPORTED;
  switch (knob) {
    case TMC_TUNE_SCHEDULE: return tc::set_schedule(p->tcw, p->nodes, value);
    case TMC_TUNE_PROLOGUE_LEAD:
      if (value < 1 || value > 3) return TMC_ERR_INVALID_ARG;
      p->tcw.pro_lead = value;
      return TMC_OK;
    case TMC_TUNE_GRID:
      if (value < 0) return TMC_ERR_INVALID_ARG;
      p->tcw.grid_ctas = value;
      return TMC_OK;
    default: return TMC_ERR_INVALID_ARG;
  }
}

tmc_status tmc_plan_get_tuning(tmc_plan p, int knob, int* value) {
  if (!p || !value) return TMC_ERR_INVALID_ARG;
  switch (knob) {
    case TMC_TUNE_SCHEDULE: *value = p->tcw.schedule; return TMC_OK;
    case TMC_TUNE_PROLOGUE_LEAD: *value = p->tcw.pro_lead; return TMC_OK;
    case TMC_TUNE_GRID: *value = p->tcw.grid_ctas; return TMC_OK;
    default: return TMC_ERR_INVALID_ARG;
  }
}

tmc_status tmc_plan_instance_times(tmc_plan p, double* fwd_us, double* bwd_us) {
  if (!p || (!fwd_us && !bwd_us)) return TMC_ERR_INVALID_ARG;
  if (!(p->precision == TMC_PREC_FP16_TC)) return TMC_ERR_UNSUPPORTED;
  return tc::instance_times(p->tcw, p->B, fwd_us, bwd_us);
}

tmc_status tmc_profile_enable(tmc_plan p, int enable) {
  if (!p) return TMC_ERR_INVALID_ARG;
  if (enable && p->slots.empty()) {
    p->slots.resize(8192);
    for (auto& s : p->slots) {
      if (cudaEventCreate(&s.start) != cudaSuccess || cudaEventCreate(&s.stop) != cudaSuccess)
        return TMC_ERR_CUDA;
    }
  }
  p->prof = enable != 0;
  p->slot_next = 0;
  for (int i = 0; i < TMC_KC_COUNT; ++i) { p->prof_ms[i] = 0.0; p->prof_n[i] = 0; }
  return TMC_OK;
}

tmc_status tmc_profile_read(tmc_plan p, int cls, double* total_ms, long long* launches) {
  if (!p || cls < 0 || cls >= TMC_KC_COUNT || !total_ms || !launches) return TMC_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return TMC_ERR_CUDA;
  drain_profile(p);
  *total_ms = p->prof_ms[cls];
  *launches = p->prof_n[cls];
  return TMC_OK;
}

}  // extern "C"
