// tmc_internal.cuh -- data structures shared by the host runtime and the kernels.
//
// Every latent of every instance is a "node" with a global id g.  Per-sample scalars
// (node term, messages, weights) live in [g][k] blocks, per-sample vectors (centred samples,
// conditional means, gradients) in [g][k][j] blocks; NodeInfo carries the offsets.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tmc {

constexpr int kTile = 64;       // rows / columns of one FP32 SIMT tile
constexpr int kThreads = 256;   // threads of every FP32 SIMT tile kernel (16 x 16, 4x4 each)
constexpr int kMaxK = 16384;    // samples per latent supported (edge prologue keeps K floats)
constexpr int kMaxD = 1024;     // latent / observation dimension supported

struct NodeInfo {
  int b, i;            // instance, local node index
  int parent;          // global id of the parent node, -1 for the root
  int K, d, obs;       // samples and dimension of this latent, observation dim of the instance
  int Kp, dp;          // the parent's K and d (root: 0 and its own d)
  int leaf_slot;       // >= 0: index of this leaf among the instance's leaves; -1 otherwise
  int child_begin;     // children[child_begin .. child_end) are global ids of the children
  int child_end;
  int level;           // depth below the root
  int root;            // global id of the instance's root
  long long off_nk;    // start of this node's block in per-sample scalar arrays (Kmax entries
                       // of the instance: its own K values, or the Kp values its edge keeps
                       // per parent sample: message, |mu~|^2)
  long long off_nkd;   // start of this node's [Kmax][d] block in per-sample vector arrays
  long long off_e;     // start of this node's [K][d] block in eps / dz / deps (the caller's layout)
  long long off_q;     // start of m_i / logs_i ([d]) in q_mean / q_logstd
  long long off_W;     // start of W_i ([d][dp]) in W
  long long off_bias;  // start of bias_i ([d]) in bias
  long long off_C;     // start of the instance's C ([obs][d])
  long long off_x;     // start of this leaf's observation ([obs]) in x (leaves only)
  long long off_pW;    // start of this node's block in the per-(instance, node) dW partials
  long long off_A;     // start of A_i ([d][dp]) in q_A / dq_A (per instance, like unshared W)
  long long off_S;     // start of this latent's dp x dp block in one instance's packed [dp x dp]
                       // blocks of the non-root latents (the root's block is empty)
  double log_K;        // log K_i (host-computed)
  long long off_cs;    // FP32 path, latents with more than kParamChunk children: start of the
                       // [K][d] sum over children of dmu_c W_c (k_child_sum); -1 otherwise
};

struct InstInfo {
  int node0;           // global id of the root
  int n, K, d, obs;    // K of the root, d of the leaves (the dimension C acts on)
  long long off_C, off_pC;  // instance C offset; per-instance dC partial offset
};

// One unit of work of a tiled kernel: a node and the first sample row of the tile.
struct Tile {
  int node;
  int row0;
};

// Device-side error word bits.
enum : int { kErrNumeric = 1, kErrTimeout = 2 };
// Default budget of a cross-CTA dependency wait: 2^31 cycles, about a second at 2 GHz.
constexpr long long kWaitLimitDefault = 1ll << 31;

// Everything a kernel may touch, passed by value.
struct Dev {
  const NodeInfo* nodes;
  const InstInfo* insts;
  const int* children;
  int num_nodes, num_inst;
  float inv_var, inv_obs_var;   // 1/prior_var, 1/obs_var
  double prior_var, obs_var;
  double log_prior_var, log_obs_var;  // their logarithms (host-computed: FP64 log is slow here)
  int shared;

  // inputs (caller's device memory)
  const float *eps, *q_mean, *q_logstd, *W, *bias, *C, *x;

  // workspace
  float* zt;      // [nkd] centred samples  z~ = exp(logs) * eps
  float* mut;     // [nkd] centred conditional means mu~_i[k] = W_i z_p^k + bias_i - m_i
  float* zn;      // [nk]  ||z~||^2
  float* mun;     // [nk]  ||mu~||^2
  float* u;       // [nk]  per-sample node term (constants removed)
  float* beta;    // [nk]  normalised node log-potential: node term + children messages - max
  float* lam;     // [nk]  message to the parent (constants removed)
  float* q;       // [nk]  marginal weight of each sample
  float* nodemax; // [nodes] max over k of the unnormalised beta
  double* nodeconst; // [nodes] FP64 constants of the node term
  float* dmu;     // [nkd] d logP / d mu_i[k]
  float* gz;      // [nkd] d logP / d z_i[k] without the proposal's own score term
  float* pW;      // per-(instance, node) dW partials  (shared params only)
  float* pbias;   // per-(instance, node) dbias partials (shared params only)
  float* pC;      // per-instance dC partials (shared params only)
  float* rsum;    // scratch of the row sums (rows_sum)
  float* csum;    // FP32 path: children sums of the latents with many children (NodeInfo::off_cs)
  int* err;       // device error word
  long long wait_limit;   // clock cycles a cross-CTA dependency wait polls before giving up
  // coupled proposals (sample k of a latent drawn given its parent's sample k)
  int coupled;
  const float* q_A;       // input: A_i blocks
  float* dq_A;            // output
  float* tq;              // [nkd] total derivative T of every sample (eps held fixed)
  float* gsrc;            // [nkd] path gradient G of every sample (FP32 path: gz)
  float* fac;             // unfused baseline: every edge's K x K log-factors (relative)
  const long long* fac_off;  // per node: start of its edge's block in fac
  // roots with more than kRootChunk children: their messages are summed in chunks of children
  // by k_root_children (one CTA per chunk) into root_part, then in a fixed order by k_root
  const int4* root_chunks;   // per chunk: instance, first and end index into children
  const int* root_chunk_off; // [B + 1] first chunk of each instance
  double* root_part;         // [chunks][root_ld] partial sums over a chunk's children
  int root_nchunk, root_ld;

  // outputs of the current call
  double* log_phat;
  const double* grad_out;
  float *dz, *deps, *dq_mean, *dq_logstd, *dW, *dbias, *dC;
};

// ---- launchers (defined in the .cu files) -------------------------------------------------
// FP32 SIMT path
void launch_node_const(const Dev& D, cudaStream_t s);
void launch_sample(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s);
void launch_obs_fwd(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s);
void launch_project(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s);
void launch_edge_fwd_f32(const Dev& D, const Tile* tiles, int ntiles, int maxK, cudaStream_t s);
void launch_factors_f32(const Dev& D, const Tile* tiles, int ntiles, int maxK, cudaStream_t s);
void launch_lse_rows_f32(const Dev& D, const Tile* tiles, int ntiles, int maxK, cudaStream_t s);
constexpr int kRootChunk = 64;  // children per chunk of a wide root's message sum
// root_fanout: most children of any root (wide roots get a 1024-thread block; with chunks
// prepared in D, the chunk sums run first)
void launch_root(const Dev& D, int maxK, int root_fanout, cudaStream_t s);
void launch_edge_bwd_rows_f32(const Dev& D, const Tile* tiles, int ntiles, int maxK,
                              cudaStream_t s);
void launch_edge_bwd_cols_f32(const Dev& D, const Tile* tiles, int ntiles, int maxK,
                              cudaStream_t s);
void launch_node_grad(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s);
void launch_node_reduce(const Dev& D, cudaStream_t s);
void launch_param_dW(const Dev& D, const int* nonroot, int n_nonroot, int maxd, cudaStream_t s);
// Instances with more than kParamChunk latents split the dC sum over their leaves into chunks:
// part holds chunks x c_total floats (c_total: the size of dC, or of the per-instance dC
// partials with shared parameters) and D.rsum the row-sum scratch of chunks x c_total.
constexpr int kParamChunk = 64;
// Latents with more than kParamChunk children (FP32 path): the sum over children of
// dmu_c W_c is formed in chunks of kParamChunk children, part[chunk][cs_total], then summed
// in order into D.csum.  items: (node, first sample row) of every 64-row tile of those latents.
void launch_child_sum(const Dev& D, const Tile* items, int nitems, int maxd, int chunks, long long cs_total,
                      float* part, cudaStream_t s);
void launch_param_dC(const Dev& D, int maxd, int maxobs, int maxn, long long c_total, float* part,
                     cudaStream_t s);
// out[e] = sum over rows r < R of in[r * stride + e], e < E: rows in order within chunks of
// kRowChunk, chunk sums in order (a tree with a fixed shape: the result does not depend on the
// launch).  scratch: rows_sum_scratch(R, E) floats.
constexpr int kRowChunk = 64;
inline long long rows_sum_scratch(long long R, long long E) {
  return R > kRowChunk ? 2 * ((R + kRowChunk - 1) / kRowChunk) * E : 0;
}
void rows_sum(const float* in, long long R, long long E, long long stride, float* out, float* scratch,
              cudaStream_t s);
// Several row sums at once: each segment with R <= kRowChunk rows is summed exactly as rows_sum
// sums it (one launch for all of them); longer ones go through rows_sum.
struct RowSeg {
  const float* in;
  float* out;
  long long R, E, stride;
};
constexpr int kMaxRowSegs = 6;
void rows_sum_batch(const RowSeg* segs, int n, float* scratch, cudaStream_t s);
// nW, nb, nC: one instance's W, bias, C sizes; rootW: its unused root block of W; tc_done: dW
// past the root block, dbias and dC are already written (the tensor-core path), only the root
// block of dW is zeroed
void launch_shared_reduce(const Dev& D, long long nW, long long nb, long long nC, long long rootW,
                          bool tc_done, cudaStream_t s);
void launch_root_bias(const Dev& D, cudaStream_t s);
// coupled proposals (k_couple.cu)
void launch_couple_fwd(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s);
void launch_couple_T(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s);
void launch_couple_out(const Dev& D, const Tile* tiles, int ntiles, const int* nonroot, int n_nonroot,
                       int maxd, cudaStream_t s);

}  // namespace tmc
