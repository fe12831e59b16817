// tmc_noalloc.cu -- log P_TMC (FP32 path, forward only) without any allocation.
//
// For callers that must not allocate: code running where cudaMalloc is forbidden or would
// stall (inside a real-time loop, under a memory pool that owns the whole device, or in a
// process whose allocator is not CUDA's).  All scratch lives in one file-scope device array
// of fixed size, and the host-side tables in fixed static host arrays: nothing here calls
// cudaMalloc, cudaFree, malloc or new.
//
// The device array belongs to the loaded library, so every GPU that runs this entry point
// holds kNoAllocScratchBytes until the process exits.  Every call shares it: a call rewrites
// all of it that it reads, and two calls whose work overlaps on the GPU (different streams,
// or different host threads) race on it -- serialise them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/tmc.h"
#include "tmc_internal.cuh"

using namespace tmc;

namespace {

// Size limits of one call (checked before any device work).
constexpr int kNaMaxNodes = 2048;           // latents over all instances
constexpr int kNaMaxInst = 1024;            // instances
constexpr long long kNaMaxNK = 65536;       // sum over latents of K
constexpr long long kNaMaxNKD = 1 << 20;    // sum over latents of K * d
constexpr int kNaMaxTiles = 8192;           // 64-row tiles over all kernels
constexpr int kNaMaxDevices = 64;

// Byte layout of the scratch array (256-byte aligned pieces).
constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffZt = 0;
constexpr size_t kOffMut = kOffZt + al256(sizeof(float) * kNaMaxNKD);
constexpr size_t kOffVec = kOffMut + al256(sizeof(float) * kNaMaxNKD);  // 6 [nk] float arrays
constexpr size_t kOffNodemax = kOffVec + 6 * al256(sizeof(float) * kNaMaxNK);
constexpr size_t kOffNodeconst = kOffNodemax + al256(sizeof(float) * kNaMaxNodes);
constexpr size_t kOffNodes = kOffNodeconst + al256(sizeof(double) * kNaMaxNodes);
constexpr size_t kOffInsts = kOffNodes + al256(sizeof(NodeInfo) * kNaMaxNodes);
constexpr size_t kOffChildren = kOffInsts + al256(sizeof(InstInfo) * kNaMaxInst);
constexpr size_t kOffTiles = kOffChildren + al256(sizeof(int) * kNaMaxNodes);
constexpr size_t kOffErr = kOffTiles + al256(sizeof(Tile) * kNaMaxTiles);
constexpr size_t kNoAllocScratchBytes = kOffErr + 256;

__device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

// Per-device address of g_scratch, looked up once per device with that device current.
std::mutex g_mu;
void* g_addr[kNaMaxDevices] = {nullptr};

// Host tables, filled per call (static storage; the mutex serialises callers).
NodeInfo h_nodes[kNaMaxNodes];
InstInfo h_insts[kNaMaxInst];
int h_children[kNaMaxNodes];
Tile h_tiles[kNaMaxTiles];

struct Layout {
  int G = 0, B = 0, nchild = 0, ntiles = 0, maxK = 0, maxlevel = 0;
  int t_sample_b, t_sample_e, t_leaf_b, t_leaf_e, t_proj_b, t_proj_e;
  int lv_b[kNaMaxNodes + 1], lv_e[kNaMaxNodes + 1];
};
Layout h_lay;

bool add_tile(Layout& L, int g, int row0) {
  if (L.ntiles >= kNaMaxTiles) return false;
  h_tiles[L.ntiles++] = Tile{g, row0};
  return true;
}

// Validates the description and fills the static host tables.
tmc_status build_tables(const tmc_problem_desc* ds, Layout& L) {
  const int B = ds->num_instances;
  if (B < 1 || !ds->n || !ds->parent || !ds->K || !ds->d || !ds->obs_dim) return TMC_ERR_INVALID_ARG;
  if (!(ds->prior_var > 0.0) || !(ds->obs_var > 0.0)) return TMC_ERR_INVALID_ARG;
  if (ds->precision != TMC_PREC_FP32) return TMC_ERR_UNSUPPORTED;
  if (ds->K_node || ds->d_node) return TMC_ERR_UNSUPPORTED;  // one K and d per instance here
  if (ds->coupled_proposal) return TMC_ERR_UNSUPPORTED;      // factorised proposals here
  if (B > kNaMaxInst) return TMC_ERR_UNSUPPORTED;
  L = Layout();
  L.B = B;
  const int shared = ds->shared_params ? 1 : 0;
  long long poff = 0, off_nk = 0, off_nkd = 0, off_q = 0, off_W = 0, off_bias = 0, off_C = 0, off_x = 0;
  int G = 0;
  for (int b = 0; b < B; ++b) {
    const int n = ds->n[b], K = ds->K[b], d = ds->d[b], obs = ds->obs_dim[b];
    if (n < 1 || K < 1 || d < 1 || obs < 1) return TMC_ERR_INVALID_ARG;
    if (K > kMaxK || d > kMaxD || obs > kMaxD) return TMC_ERR_UNSUPPORTED;
    const int* par = ds->parent + poff;
    if (par[0] != -1) return TMC_ERR_INVALID_ARG;
    for (int i = 1; i < n; ++i)
      if (par[i] < 0 || par[i] >= i) return TMC_ERR_INVALID_ARG;
    if (shared && b > 0) {
      if (n != ds->n[0] || d != ds->d[0] || obs != ds->obs_dim[0]) return TMC_ERR_INVALID_ARG;
      for (int i = 0; i < n; ++i)
        if (par[i] != ds->parent[i]) return TMC_ERR_INVALID_ARG;
    }
    if (G + n > kNaMaxNodes || off_nk + (long long)n * K > kNaMaxNK ||
        off_nkd + (long long)n * K * d > kNaMaxNKD)
      return TMC_ERR_UNSUPPORTED;
    const int node0 = G;
    const long long iW = shared ? 0 : off_W, ib = shared ? 0 : off_bias, iC = shared ? 0 : off_C;
    // levels and leaves: a node is a leaf when no later node names it as parent
    int leaves = 0;
    for (int i = 0; i < n; ++i) {
      NodeInfo& nd = h_nodes[node0 + i];
      nd = NodeInfo{};
      nd.off_cs = -1;
      nd.b = b;
      nd.i = i;
      nd.parent = i ? node0 + par[i] : -1;
      nd.K = K;
      nd.log_K = std::log((double)K);
      nd.d = d;
      nd.Kp = i ? K : 0;
      nd.dp = d;
      nd.obs = obs;
      nd.level = i ? h_nodes[node0 + par[i]].level + 1 : 0;
      nd.root = node0;
      nd.off_nk = off_nk + (long long)i * K;
      nd.off_nkd = off_nkd + (long long)i * K * d;
      nd.off_e = nd.off_nkd;
      nd.off_q = off_q + (long long)i * d;
      nd.off_W = iW + (long long)i * d * d;
      nd.off_bias = ib + (long long)i * d;
      nd.off_C = iC;
      L.maxlevel = nd.level > L.maxlevel ? nd.level : L.maxlevel;
    }
    for (int i = 0; i < n; ++i) {
      NodeInfo& nd = h_nodes[node0 + i];
      nd.child_begin = L.nchild;
      for (int c = i + 1; c < n; ++c)
        if (par[c] == i) h_children[L.nchild++] = node0 + c;
      nd.child_end = L.nchild;
      nd.leaf_slot = (nd.child_end == nd.child_begin) ? leaves++ : -1;
      nd.off_x = off_x + (long long)(nd.leaf_slot >= 0 ? nd.leaf_slot : 0) * obs;
    }
    InstInfo& in = h_insts[b];
    in = InstInfo{};
    in.node0 = node0;
    in.n = n;
    in.K = K;
    in.d = d;
    in.obs = obs;
    in.off_C = iC;
    L.maxK = K > L.maxK ? K : L.maxK;
    G += n;
    poff += n;
    off_nk += (long long)n * K;
    off_nkd += (long long)n * K * d;
    off_q += (long long)n * d;
    off_x += (long long)leaves * obs;
    if (!shared) {
      off_W += (long long)n * d * d;
      off_bias += (long long)n * d;
      off_C += (long long)obs * d;
    }
  }
  L.G = G;
  L.t_sample_b = L.ntiles;
  for (int g = 0; g < G; ++g)
    for (int r = 0; r < h_nodes[g].K; r += kTile)
      if (!add_tile(L, g, r)) return TMC_ERR_UNSUPPORTED;
  L.t_sample_e = L.ntiles;
  L.t_leaf_b = L.ntiles;
  for (int g = 0; g < G; ++g)
    if (h_nodes[g].leaf_slot >= 0)
      for (int r = 0; r < h_nodes[g].K; r += kTile)
        if (!add_tile(L, g, r)) return TMC_ERR_UNSUPPORTED;
  L.t_leaf_e = L.ntiles;
  L.t_proj_b = L.ntiles;
  for (int g = 0; g < G; ++g)
    if (h_nodes[g].parent >= 0)
      for (int r = 0; r < h_nodes[g].K; r += kTile)
        if (!add_tile(L, g, r)) return TMC_ERR_UNSUPPORTED;
  L.t_proj_e = L.ntiles;
  for (int lv = 1; lv <= L.maxlevel; ++lv) {
    L.lv_b[lv] = L.ntiles;
    for (int g = 0; g < G; ++g)
      if (h_nodes[g].level == lv)
        for (int r = 0; r < h_nodes[g].K; r += kTile)
          if (!add_tile(L, g, r)) return TMC_ERR_UNSUPPORTED;
    L.lv_e[lv] = L.ntiles;
  }
  return TMC_OK;
}

}  // namespace

extern "C" tmc_status tmc_log_marginal_noalloc(const tmc_problem_desc* desc, const tmc_inputs* in,
                                               double* log_phat, void* stream) {
  if (!desc || !in || !log_phat || !in->eps || !in->q_mean || !in->q_logstd || !in->W || !in->bias ||
      !in->C || !in->x)
    return TMC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // Refused under stream capture: the tables below are uploaded from static host arrays that
  // the next call rewrites, so a captured copy would replay another call's tables under this
  // call's grid sizes.  (The legacy stream reports an implicit capture as an error.)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing(s, &cap);
  if (ce != cudaSuccess) {
    (void)cudaGetLastError();  // not sticky: leave no error behind for the caller
    return ce == cudaErrorStreamCaptureImplicit ? TMC_ERR_UNSUPPORTED : TMC_ERR_CUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) return TMC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  Layout& L = h_lay;
  tmc_status st = build_tables(desc, L);
  if (st != TMC_OK) return st;

  // set-up, once per device: the device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return TMC_ERR_CUDA;
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return TMC_ERR_CUDA;
    g_addr[dev] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(g_addr[dev]);

  // tables -> scratch (copies from static host arrays; no staging allocation by us)
  if (cudaMemcpyAsync(base + kOffNodes, h_nodes, sizeof(NodeInfo) * L.G, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + kOffInsts, h_insts, sizeof(InstInfo) * L.B, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      (L.nchild && cudaMemcpyAsync(base + kOffChildren, h_children, sizeof(int) * L.nchild,
                                   cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      cudaMemcpyAsync(base + kOffTiles, h_tiles, sizeof(Tile) * L.ntiles, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(base + kOffErr, 0, sizeof(int), s) != cudaSuccess)
    return TMC_ERR_CUDA;

  Dev D{};
  D.nodes = reinterpret_cast<const NodeInfo*>(base + kOffNodes);
  D.insts = reinterpret_cast<const InstInfo*>(base + kOffInsts);
  D.children = reinterpret_cast<const int*>(base + kOffChildren);
  D.num_nodes = L.G;
  D.num_inst = L.B;
  D.inv_var = (float)(1.0 / desc->prior_var);
  D.inv_obs_var = (float)(1.0 / desc->obs_var);
  D.prior_var = desc->prior_var;
  D.obs_var = desc->obs_var;
  D.log_prior_var = std::log(desc->prior_var);
  D.log_obs_var = std::log(desc->obs_var);
  D.shared = desc->shared_params ? 1 : 0;
  D.eps = in->eps; D.q_mean = in->q_mean; D.q_logstd = in->q_logstd;
  D.W = in->W; D.bias = in->bias; D.C = in->C; D.x = in->x;
  const size_t vec = al256(sizeof(float) * kNaMaxNK);
  D.zt = reinterpret_cast<float*>(base + kOffZt);
  D.mut = reinterpret_cast<float*>(base + kOffMut);
  D.zn = reinterpret_cast<float*>(base + kOffVec + 0 * vec);
  D.mun = reinterpret_cast<float*>(base + kOffVec + 1 * vec);
  D.u = reinterpret_cast<float*>(base + kOffVec + 2 * vec);
  D.beta = reinterpret_cast<float*>(base + kOffVec + 3 * vec);
  D.lam = reinterpret_cast<float*>(base + kOffVec + 4 * vec);
  D.q = reinterpret_cast<float*>(base + kOffVec + 5 * vec);
  D.nodemax = reinterpret_cast<float*>(base + kOffNodemax);
  D.nodeconst = reinterpret_cast<double*>(base + kOffNodeconst);
  D.err = reinterpret_cast<int*>(base + kOffErr);
  D.wait_limit = kWaitLimitDefault;
  D.log_phat = log_phat;

  const Tile* T = reinterpret_cast<const Tile*>(base + kOffTiles);
  launch_node_const(D, s);
  launch_sample(D, T + L.t_sample_b, L.t_sample_e - L.t_sample_b, s);
  launch_obs_fwd(D, T + L.t_leaf_b, L.t_leaf_e - L.t_leaf_b, s);
  launch_project(D, T + L.t_proj_b, L.t_proj_e - L.t_proj_b, s);
  for (int lv = L.maxlevel; lv >= 1; --lv)
    launch_edge_fwd_f32(D, T + L.lv_b[lv], L.lv_e[lv] - L.lv_b[lv], L.maxK, s);
  launch_root(D, L.maxK, 0, s);
  return cudaGetLastError() == cudaSuccess ? TMC_OK : TMC_ERR_CUDA;
}
