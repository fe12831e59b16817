// tmc_tc.cuh -- tensor-core (tcgen05) path: packed operands, tile lists and launchers.
//
// Operands of the pairwise contraction are carried as split fp16 pairs (x = hi + lo, both
// fp16), and every product that feeds an exponent is formed as hi*hi + lo*hi + hi*lo with
// FP32 accumulation (about 22 significant bits), which keeps |delta log P| far below the
// tolerance of the reduced-precision path at d = 128.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>

#include <vector>

#include "../../include/tmc.h"
#include "tmc_internal.cuh"

namespace tmc {
namespace tc {

constexpr int kRows = 128;      // rows of a tensor-core tile (samples)
constexpr int kLdp = 128;       // row stride (elements) of every packed fp16 operand array
constexpr int kTcMaxD = 128;    // latent dimension covered by the tensor-core kernels
constexpr int kTcMaxK = 4096;   // samples per latent covered by the tensor-core kernels

// A leaf of the tensor-core assembly: node id and the offsets of its proposal mean and
// observation (the leaves of an instance are contiguous, leaf_off[b] .. leaf_off[b + 1]).
// One item of the node-moment launch: up to 1024 consecutive samples of one node.
struct MoItem {
  long long row;  // first sample row of the item in the packed sample tensors
  int node, nrows, d;
  int whole;      // the item covers every sample of its node
};
struct LeafInfo {
  int node;
  int pad;
  long long off_q;
  long long off_x;
};

struct TcSub {
  void** dst;
  size_t bytes;
};

// Device pointers of the tensor-core path (part of the plan's workspace).
struct TcDev {
  __half *ZH, *ZL;             // [rows][128] split centred samples, row = node.off_nk + k
  float* zc;                   // [nk]  z~_i^k . c_i  (row term of the adjoint exponent)
  __half *WH, *WL;             // [slots*128][128] split W_i   ([r][c])
  __half *WTH, *WTL;           // [slots*128][128] split W_i^T ([c][r])
  float* cvec;                 // [nodes][128]  c_i = W_i m_p + bias_i - m_i
  float* G;                    // [nodes][128*128] edge moment sum pi z~_p z~_i^T (child node)
  float* M2;                   // [nodes][128*128] sum_k q_i[k] z~_i^k z~_i^k^T
  float* zbar;                 // [nodes][128]  sum_k q_i[k] z~_i^k
  float* sgC;                  // [nodes][128]  per-edge parts of the node gradient sums
  float* tgC;
  float* sgP;
  float* tgP;
  float* CtC;                  // [1 or B][128*128]  C^T C per observation matrix
  // shared parameters (one W_c per position = local node index): W_c^T W_c ([slot][128*128]);
  // per instance group the partial sums of dW without the W_c M2_p term (Ppart, [group][W
  // layout of one instance]) and of go M2_p / var (Spart, [group][packed dp x dp blocks,
  // NodeInfo::off_S]); P and S2 = their sums over the groups
  float *WtW, *P, *S2, *Ppart, *Spart;
  float* Ssum;                 // shared C: sum_b go_b S_b / obs_var ([d][d], d = the leaves' dimension)
  __half *CH, *CL;             // [c_rows][128] split observation matrices, row = c_row[b] + o
  int* c_row;                  // [1 or B] first row of each observation matrix in CH / CL
  float* xs;                   // centred observations x - C m of the leaves (layout of x)
  const LeafInfo* leaf_info;   // [leaves] in node order
  const int* leaf_off;         // [B + 1] leaves of instance b: leaf_off[b] .. leaf_off[b + 1]
  float* S;                    // [B][128*128] sum over an instance's leaves of M2 + zbar m^T
  // sample gradients (dz, deps): written only when they are requested
  __half *VH, *VL;             // [rows][128] split V / q = E[z~_p | sample] of the adjoint (non-root)
  __half *EH, *EL;             // [rows][128] split R - mu~ per edge, rows = the parent's samples
  __half *CCH, *CCL;           // [num_c*128][128] split -(prior_var / obs_var) C^T C
  int* done;                   // [nodes] tiles finished per node in the running edge launch
  int* claim;                  // [8] next unclaimed item of each persistent edge launch
  unsigned long long* inst_t;  // [2][B] %globaltimer when an instance's last tile finished (fwd, adjoint)
  unsigned long long* t_start; // [2]    %globaltimer at the first tile of each launch
  int shared;
};

struct TcWork {
  int precision = 0;
  int num_nodes = 0, num_slots = 0, maxlevel = 0, num_inst = 0, maxobs = 0;
  long long rows = 0;
  TcDev t{};
  CUtensorMap mZH, mZL, mWH, mWL, mWTH, mWTL;
  CUtensorMap mZH64, mZL64;       // the sample tiles in 64-row boxes (node moments)
  // edge tiles in dependency order: [direction][class] ranges into d_tiles; direction 0 =
  // forward (deepest level first, rows = the parent's samples), 1 = adjoint (level 1 first,
  // rows = the child's samples), 2 = the row-direction pass of the sample gradients (rows = the
  // parent's samples, no dependencies); class 0: every latent of the instance has d <= 64,
  // class 1: d <= 128 (one class per instance, so no dependency crosses launches)
  std::vector<Tile> tiles;
  int it_b[3][2] = {{0, 0}, {0, 0}, {0, 0}}, it_e[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  std::vector<int> inst_dp;       // per instance: widest padded latent dimension (64 or 128)
  int num_sms = 148;
  Tile* d_tiles = nullptr;
  std::vector<int> nonroot;
  int* d_nonroot = nullptr;
  int maxK = 0;
  int schedule = 0;               // work order of the persistent launches (see build_items)
  int pro_lead = 2;               // forward: chunks before an item's end for the next prologue
  int grid_ctas = 0;              // CTAs per persistent edge launch (0: one per SM)
  int stall_node = -1;            // fault injection: node whose forward tiles are left out
  int maxdp = 128;                // widest padded latent dimension (64 or 128)
  int n_pack_w = 0;               // leading non-root nodes whose W is packed
  // shared parameters: one instance's W size, its root block, its packed dp x dp blocks, and
  // the instance groups of the gradient assembly
  long long shared_nW = 0, shared_rootW = 0, shared_nS = 0, shared_nb = 0;
  int asm_groups = 0, leaf_d = 0, obs0 = 0;
  // observation term: split C rows and the 128-sample leaf tiles per d class
  long long c_rows = 0;
  int num_c = 0;                  // distinct observation matrices (1 when shared)
  CUtensorMap mCH, mCL;
  CUtensorMap mG;                 // fp32 [nodes*128][128] view of G for TMA reductions
  CUtensorMap mVH, mVL, mEH, mEL, mCCH, mCCL;  // sample-gradient operands
  std::vector<Tile> dz_tiles;     // 128-row tiles of every node, per d class
  int dz_b[2] = {0, 0}, dz_e[2] = {0, 0};
  Tile* d_dz_tiles = nullptr;
  std::vector<Tile> obs_tiles;
  int ob_b[2] = {0, 0}, ob_e[2] = {0, 0};
  Tile* d_obs_tiles = nullptr;
  std::vector<int> leaves;        // leaf nodes
  int* d_leaves = nullptr;
  LeafInfo* d_leaf_info = nullptr;
  std::vector<MoItem> mo_items;   // node-moment items (every node, up to 1024 samples), per d class
  int mo_b[2] = {0, 0}, mo_e[2] = {0, 0};
  bool mo_split = false;          // some node spans several moment items
  MoItem* d_mo_items = nullptr;
  int* d_leaf_off = nullptr;
  std::vector<Tile> sample_tiles; // sampler tiles (rows per tile grow as d shrinks)
  Tile* d_sample_tiles = nullptr;
};

tmc_status supported(const std::vector<NodeInfo>& nodes, int precision);
void build_items(TcWork& w, const std::vector<NodeInfo>& nodes, int schedule);
tmc_status set_schedule(TcWork& w, const std::vector<NodeInfo>& nodes, int schedule);
tmc_status instance_times(TcWork& w, int B, double* fwd_us, double* bwd_us);
void workspace_layout(TcWork& w, const std::vector<NodeInfo>& nodes, long long nk, long long nkd,
                      std::vector<TcSub>& subs);
tmc_status prepare(TcWork& w, const std::vector<NodeInfo>& nodes, const std::vector<Tile>& tiles,
                   int maxK, int maxd);
void release(TcWork& w);
void launch_sample(TcWork& w, const Dev& D, cudaStream_t s);
void launch_pack(TcWork& w, const Dev& D, cudaStream_t s);
void launch_obs(TcWork& w, const Dev& D, cudaStream_t s);  // leaf observation term
void launch_edge_fwd(TcWork& w, const Dev& D, cudaStream_t s);  // one persistent launch per d class
void launch_edge_bwd(TcWork& w, const Dev& D, cudaStream_t s);
void launch_unpack_grads(TcWork& w, const Dev& D, cudaStream_t s);
// Sample gradients dz / deps (after launch_edge_bwd, which stores V / q when D.dz or D.deps is
// set, and launch_unpack_grads, which forms C^T C): the row-direction edge pass, then the
// assembly (k_dz_tc.cu).
void launch_edge_rows(TcWork& w, const Dev& D, cudaStream_t s);
// Coupled proposals: split the FP32 samples (after the couplings) into the packed operands,
// with z~ . c_i (the other per-sample terms come from the FP32 sampler).
void launch_pack_z(TcWork& w, const Dev& D, cudaStream_t s);
void launch_dz(TcWork& w, const Dev& D, cudaStream_t s);
tmc_status prepare_dz(TcWork& w, const std::vector<NodeInfo>& nodes);
void release_dz(TcWork& w);

}  // namespace tc
}  // namespace tmc
