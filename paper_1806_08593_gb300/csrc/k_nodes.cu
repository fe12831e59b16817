// k_nodes.cu -- per-node kernels of the TMC hot path (both precisions use them):
// proposal samples and node terms, observation residuals, conditional means, the FP64 root
// reduction, and the gradient assembly after the fused edge adjoint.
//
// Notation (Appendix, typical factors): for latent i with parent p,
//   f_i^{(k', k)} = P(z_i^{k'} | z_p^k) / Q_i(z_i^{k'}),  f_root^{k} = P(z_0^k) / Q_0(z_0^k),
//   and every leaf carries P(x_l | z_l^k).
// Everything indexed by one sample k of latent i alone is collected in the node term
//   u_i[k] = -log Q_i(z_i^k) [+ log P(z_0^k) at the root] [+ log P(x_i | z_i^k) at a leaf],
// split into an FP64 constant (nodeconst) and an FP32 per-sample part (u).
// Samples and means are kept centred on the proposal mean m_i: z~ = z - m_i, mu~ = mu - m_i,
// which leaves every pairwise distance unchanged and keeps FP32 magnitudes small.
#include "simt_tile.cuh"

namespace tmc {

namespace {
constexpr double kLog2Pi = 1.8378770664093454835606594728112;

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}
__device__ __forceinline__ double block_max_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = -INFINITY;
  for (int i = 0; i < nw; ++i) t = fmax(t, red[i]);
  return t;
}
__device__ __forceinline__ float block_max_f(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float t = -INFINITY;
  for (int i = 0; i < nw; ++i) t = fmaxf(t, red[i]);
  return t;
}
__device__ __forceinline__ float block_sum_f(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}
}  // namespace

// ---------------------------------------------------------------------------------------
// FP64 node constants: sum_j logs_ij + (d/2) log 2pi  (from -log Q_i)
//   - (d/2) log(2 pi prior_var)  (the prior or transition normaliser)
//   - log K_i for i >= 1  (Eq. (is)'s 1 / K_i; the root's is added by k_root)
//   + leaf: -(obs/2) log(2 pi obs_var)
// ---------------------------------------------------------------------------------------
// One warp per node (8 nodes per CTA): lanes sum logs_i over the dimension in FP64.
constexpr int kConstNodesPerCta = 8;
__global__ void __launch_bounds__(32 * kConstNodesPerCta) k_node_const(Dev D) {
  const int g = blockIdx.x * kConstNodesPerCta + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (g >= D.num_nodes) return;
  const NodeInfo nd = D.nodes[g];
  double s = 0.0;
  for (int j = lane; j < nd.d; j += 32) s += (double)D.q_logstd[nd.off_q + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {  // proposal and prior normalisers, the observation's, and 1 / K_i (Eq. (is))
    double c = s + 0.5 * nd.d * kLog2Pi - 0.5 * nd.d * (kLog2Pi + D.log_prior_var);
    if (nd.parent >= 0) c -= nd.log_K;
    if (nd.leaf_slot >= 0) c += -0.5 * nd.obs * (kLog2Pi + D.log_obs_var);
    D.nodeconst[g] = c;
  }
}

// ---------------------------------------------------------------------------------------
// Samples (Section 2.1: z_i^k ~ Q_i, reparameterised) and the per-sample node term:
//   z~ = exp(logs) * eps,  u = |eps|^2 / 2  [ - |z_0 - bias_0|^2 / (2 prior_var) at the root ]
// One warp per sample row, lanes over the latent dimension.
// ---------------------------------------------------------------------------------------
__global__ void k_sample(Dev D, const Tile* __restrict__ tiles) {
  extern __shared__ float sm[];
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const int d = nd.d;
  float* s_std = sm;         // exp(logs)
  float* s_off = sm + d;     // m_0 - bias_0 (root only)
  const bool root = nd.parent < 0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    s_std[j] = expf(D.q_logstd[nd.off_q + j]);
    s_off[j] = root ? D.q_mean[nd.off_q + j] - D.bias[nd.off_bias + j] : 0.f;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bool bad = false;
  for (int r = w; r < kTile; r += kThreads / 32) {
    const int k = t.row0 + r;
    if (k >= nd.K) break;
    const long long base = nd.off_nkd + (long long)k * d, ebase = nd.off_e + (long long)k * d;
    float se = 0.f, sz = 0.f, sr = 0.f;
    for (int j = lane; j < d; j += 32) {
      const float e = D.eps[ebase + j];
      const float z = s_std[j] * e;
      bad |= !isfinite(z);
      D.zt[base + j] = z;
      se = fmaf(e, e, se);
      sz = fmaf(z, z, sz);
      const float rr = z + s_off[j];
      sr = fmaf(rr, rr, sr);
    }
    for (int o = 16; o > 0; o >>= 1) {
      se += __shfl_xor_sync(0xffffffffu, se, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
    }
    if (lane == 0) {
      float u = 0.5f * se;
      if (root) u -= 0.5f * sr * D.inv_var;
      D.u[nd.off_nk + k] = u;
      D.zn[nd.off_nk + k] = sz;
    }
  }
  if (bad) flag_error(D.err, kErrNumeric);
}

// x~ = x_l - C m_l for the leaf of node nd (into shared memory, obs floats).
__device__ __forceinline__ void centred_obs(const Dev& D, const NodeInfo& nd, float* xs) {
  for (int o = threadIdx.x; o < nd.obs; o += blockDim.x) {
    const float* c = D.C + nd.off_C + (long long)o * nd.d;
    const float* m = D.q_mean + nd.off_q;
    float s = 0.f;
    for (int j = 0; j < nd.d; ++j) s = fmaf(c[j], m[j], s);
    xs[o] = D.x[nd.off_x + o] - s;
  }
}

// ---------------------------------------------------------------------------------------
// Observation term at a leaf: u[k] -= |x - C z^k|^2 / (2 obs_var), residual r = x~ - C z~^k.
// Grid: (leaf node, 64-sample tile); loops over 64-wide observation tiles.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_obs_fwd(Dev D, const Tile* __restrict__ tiles) {
  extern __shared__ float xs[];
  __shared__ TileSmem sm;
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  centred_obs(D, nd, xs);
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int rows = min(kTile, nd.K - t.row0);
  const float* Z = D.zt + nd.off_nkd + (long long)t.row0 * nd.d;
  float rs[4] = {0.f, 0.f, 0.f, 0.f};
  for (int o0 = 0; o0 < nd.obs; o0 += kTile) {
    float acc[4][4];
    zero_acc(acc);
    tile_gemm<true, true>(acc, Z, nd.d, rows, D.C + nd.off_C + (long long)o0 * nd.d, nd.d,
                          min(kTile, nd.obs - o0), nd.d, sm);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int o = o0 + tx * 4 + b;
      if (o < nd.obs) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float r = xs[o] - acc[a][b];
          rs[a] = fmaf(r, r, rs[a]);
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float s = row_group_sum(rs[a]);
    const int k = t.row0 + ty * 4 + a;
    if (tx == 0 && k < nd.K) D.u[nd.off_nk + k] -= 0.5f * s * D.inv_obs_var;
  }
}

// ---------------------------------------------------------------------------------------
// Conditional means (the linear cost of Section 2.4): mu~_i[k] = W_i z_p^k + bias_i - m_i
//   = W_i z~_p^k + c_i,  c_i = W_i m_p + bias_i - m_i;  also |mu~_i[k]|^2.
// Grid: (non-root node i, 64-sample tile of the parent's samples).  W_i is d_i x d_p.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_project(Dev D, const Tile* __restrict__ tiles) {
  extern __shared__ float cs[];
  __shared__ TileSmem sm;
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const NodeInfo pn = D.nodes[nd.parent];
  const int d = nd.d, dp = nd.dp, Kp = nd.Kp;
  const float* Wi = D.W + nd.off_W;
  for (int r = threadIdx.x; r < d; r += blockDim.x) {
    const float* w = Wi + (long long)r * dp;
    const float* mp = D.q_mean + pn.off_q;
    float s = 0.f;
    for (int c = 0; c < dp; ++c) s = fmaf(w[c], mp[c], s);
    cs[r] = s + D.bias[nd.off_bias + r] - D.q_mean[nd.off_q + r];
  }
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int rows = min(kTile, Kp - t.row0);
  const float* Zp = D.zt + pn.off_nkd + (long long)t.row0 * dp;
  float rs[4] = {0.f, 0.f, 0.f, 0.f};
  for (int r0 = 0; r0 < d; r0 += kTile) {
    float acc[4][4];
    zero_acc(acc);
    tile_gemm<true, true>(acc, Zp, dp, rows, Wi + (long long)r0 * dp, dp, min(kTile, d - r0), dp, sm);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int k = t.row0 + ty * 4 + a;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int r = r0 + tx * 4 + b;
        if (k < Kp && r < d) {
          const float v = acc[a][b] + cs[r];
          D.mut[nd.off_nkd + (long long)k * d + r] = v;
          rs[a] = fmaf(v, v, rs[a]);
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float s = row_group_sum(rs[a]);
    const int k = t.row0 + ty * 4 + a;
    if (tx == 0 && k < Kp) D.mun[nd.off_nk + k] = s;
  }
}

constexpr int kRootThreads = 1024;
// ---------------------------------------------------------------------------------------
// Root: closes the sum of Eq. (is) in FP64.
//   beta'_0 = u_0 + sum_children lam_c (FP64: a root may have thousands of children),
//   M_0 = max beta'_0,  beta_0 = beta'_0 - M_0,
//   log P = sum_nodes (nodeconst + M) + log sum_k exp(beta_0[k]) - log K_0,
// and the root's sample weights q_0[k] = exp(beta_0[k] - logsumexp(beta_0)).
// ---------------------------------------------------------------------------------------
// A chunk of a wide root's children: their messages summed per sample, in child order.
__global__ void __launch_bounds__(256) k_root_children(Dev D) {
  const int4 ch = D.root_chunks[blockIdx.x];
  const int K = D.nodes[D.insts[ch.x].node0].K;
  double* out = D.root_part + (long long)blockIdx.x * D.root_ld;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double v = 0.0;
#pragma unroll 4
    for (int c = ch.y; c < ch.z; ++c) v += D.lam[D.nodes[D.children[c]].off_nk + k];
    out[k] = v;
  }
}

// The children's messages come from the chunk sums of k_root_children when the plan made
// them (summed in chunk order); otherwise they are summed here by G = blockDim / K groups of
// threads when K < blockDim
// (group g takes children g, g + G, ...; a root may have thousands), the group partials then
// in a fixed order, so the result does not depend on timing.
__global__ void k_root(Dev D) {
  extern __shared__ double sbd[];  // [K] beta'_0, then [G][Kb] group partials
  __shared__ double redd[32];
  __shared__ float redf[32];
  const InstInfo in = D.insts[blockIdx.x];
  const NodeInfo nd = D.nodes[in.node0];
  const int K = nd.K;
  const int Kb = K < (int)blockDim.x ? K : (int)blockDim.x;
  const int G = (int)blockDim.x / Kb, grp = (int)threadIdx.x / Kb, kt = (int)threadIdx.x % Kb;
  double* part = sbd + K;
  const bool chunked = D.root_part != nullptr;
  if (!chunked && grp < G)
    for (int k = kt; k < K; k += Kb) {
      double v = 0.0;
#pragma unroll 4
      for (int c = nd.child_begin + grp; c < nd.child_end; c += G)
        v += D.lam[D.nodes[D.children[c]].off_nk + k];
      if (G == 1) sbd[k] = v;
      else part[grp * Kb + kt] = v;  // K == Kb here
    }
  __syncthreads();
  double mxd = -INFINITY;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double v = D.u[nd.off_nk + k];
    if (chunked) {
      const int c0 = D.root_chunk_off[blockIdx.x], c1 = D.root_chunk_off[blockIdx.x + 1];
#pragma unroll 8
      for (int ci = c0; ci < c1; ++ci) v += D.root_part[(long long)ci * D.root_ld + k];
    }
    else if (G == 1) v += sbd[k];
    else
      for (int g = 0; g < G; ++g) v += part[g * Kb + k];
    sbd[k] = v;
    mxd = fmax(mxd, v);
  }
  mxd = block_max_d(mxd, redd);
  const float mx = (float)mxd;
  float s = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const float b = (float)(sbd[k] - mxd);
    D.beta[nd.off_nk + k] = b;
    s += expf(b);
  }
  s = block_sum_f(s, redf);
  const float lse = logf(s);
  for (int k = threadIdx.x; k < K; k += blockDim.x) D.q[nd.off_nk + k] = expf((float)(sbd[k] - mxd) - lse);
  double acc = 0.0;
  for (int g = in.node0 + threadIdx.x; g < in.node0 + in.n; g += blockDim.x)
    acc += D.nodeconst[g] + ((g == in.node0) ? mxd : (double)D.nodemax[g]);
  acc = block_sum_d(acc, redd);
  if (threadIdx.x == 0) {
    D.nodemax[in.node0] = mx;
    const double lp = acc + (double)lse - nd.log_K;
    D.log_phat[blockIdx.x] = lp;
    if (!isfinite(lp)) flag_error(D.err, kErrNumeric);
  }
}

// ---------------------------------------------------------------------------------------
// Sample gradients without the proposal's own score (the "path" part):
//   gz_i[k] = [edge part, written by the edge adjoint, if i is not the root]
//           + sum_{children c} W_c^T dmu_c[k]                      (mu_c = W_c z_i + bias_c)
//           - q_0[k] (z_0^k - bias_0) / prior_var                   (root prior)
//           + q_i[k] C^T (x_i - C z_i^k) / obs_var                  (leaf observation)
// and the requested sample gradients dz = grad_out * (gz + q z~ / exp(2 logs)),
// deps = exp(logs) * dz.
// Grid: (node, 64-sample tile); loops over 64-wide latent-dimension tiles.
// ---------------------------------------------------------------------------------------
// Sum over one chunk of a wide latent's children of dmu_c W_c for 64 sample rows and 64 columns.
// Grid: (item = node and first row, chunk of kParamChunk children, 64-column tile).  Chunks past
// the latent's children write zeros (every chunk row of part is summed).
__global__ void __launch_bounds__(kThreads) k_child_sum(Dev D, const Tile* __restrict__ items, float* __restrict__ part,
                                                         long long cs_total) {
  __shared__ TileSmem sm;
  const Tile t = items[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const int d = nd.d, K = nd.K;
  const int c0 = blockIdx.z * kTile;
  if (c0 >= d) return;
  const int rows = min(kTile, K - t.row0), ncol = min(kTile, d - c0);
  const int cb = nd.child_begin + blockIdx.y * kParamChunk, ce = min(nd.child_end, cb + kParamChunk);
  float acc[4][4];
  zero_acc(acc);
  for (int ci = cb; ci < ce; ++ci) {
    const NodeInfo ch = D.nodes[D.children[ci]];
    tile_gemm<true, false>(acc, D.dmu + ch.off_nkd + (long long)t.row0 * ch.d, ch.d, rows,
                           D.W + ch.off_W + c0, d, ncol, ch.d, sm);
  }
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float* out = part + (long long)blockIdx.y * cs_total + nd.off_cs;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int k = t.row0 + ty * 4 + a;
    if (k >= K) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c < d) out[(long long)k * d + c] = acc[a][b];
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_node_grad(Dev D, const Tile* __restrict__ tiles) {
  extern __shared__ float xs[];  // centred observation (leaves)
  __shared__ TileSmem sm;
  __shared__ float rsm[kTile * kLd];  // residual tile, [o][k]
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const int d = nd.d, K = nd.K;
  const bool root = nd.parent < 0, leaf = nd.leaf_slot >= 0;
  if (leaf) centred_obs(D, nd, xs);
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int rows = min(kTile, K - t.row0);
  const float* Z = D.zt + nd.off_nkd + (long long)t.row0 * d;
  const float go = D.grad_out ? (float)D.grad_out[nd.b] : 1.f;
  float qk[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int k = t.row0 + ty * 4 + a;
    qk[a] = (k < K) ? D.q[nd.off_nk + k] : 0.f;
  }
  for (int c0 = 0; c0 < d; c0 += kTile) {
    const int ncol = min(kTile, d - c0);
    float acc[4][4];
    zero_acc(acc);
    // children: out[k][c] += sum_r dmu_c[k][r] W_c[r][c]   (W_c is d_c x d); a latent with
    // many children reads the sum formed beforehand by k_child_sum
    if (nd.off_cs >= 0) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int k = t.row0 + ty * 4 + a, c = c0 + tx * 4 + b;
          acc[a][b] = (k < K && c < d) ? D.csum[nd.off_cs + (long long)k * d + c] : 0.f;
        }
    } else {
      for (int ci = nd.child_begin; ci < nd.child_end; ++ci) {
        const NodeInfo ch = D.nodes[D.children[ci]];
        tile_gemm<true, false>(acc, D.dmu + ch.off_nkd + (long long)t.row0 * ch.d, ch.d, rows,
                               D.W + ch.off_W + c0, d, ncol, ch.d, sm);
      }
    }
    if (leaf) {
      // out[k][c] += q[k] / obs_var * sum_o r[k][o] C[o][c],  r = x~ - C z~
      float acc2[4][4];
      zero_acc(acc2);
      for (int o0 = 0; o0 < nd.obs; o0 += kTile) {
        const int nob = min(kTile, nd.obs - o0);
        float racc[4][4];
        zero_acc(racc);
        tile_gemm<true, true>(racc, Z, d, rows, D.C + nd.off_C + (long long)o0 * d, d, nob, d, sm);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int o = o0 + tx * 4 + b;
            rsm[(tx * 4 + b) * kLd + ty * 4 + a] = (o < nd.obs) ? xs[o] - racc[a][b] : 0.f;
          }
        __syncthreads();
        for (int l0 = 0; l0 < nob; l0 += kSlice) {
          load_slice<false>(sm.b, D.C + nd.off_C + (long long)o0 * d + c0, d, ncol, l0, nob);
          __syncthreads();
          slice_fma(acc2, rsm + l0 * kLd, sm.b);
          __syncthreads();
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(qk[a] * D.inv_obs_var, acc2[a][b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int k = t.row0 + ty * 4 + a;
      if (k >= K) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + tx * 4 + b;
        if (c >= d) continue;
        const long long idx = nd.off_nkd + (long long)k * d + c;
        float g = acc[a][b];
        const float zt = D.zt[idx];
        if (root) {
          const float off = D.q_mean[nd.off_q + c] - D.bias[nd.off_bias + c];
          g -= qk[a] * (zt + off) * D.inv_var;
        } else {
          g += D.gz[idx];
        }
        D.gz[idx] = g;
        if ((D.dz || D.deps) && !D.coupled) {  // coupled proposals: k_couple_out
          const long long eidx = nd.off_e + (long long)k * d + c;
          const float ls = D.q_logstd[nd.off_q + c];
          const float dzv = go * (g + qk[a] * zt * expf(-2.f * ls));
          if (D.dz) D.dz[eidx] = dzv;
          if (D.deps) D.deps[eidx] = dzv * expf(ls);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Per-latent reductions over samples (reparameterisation z = m + exp(logs) eps):
//   dm_i    = grad_out * sum_k gz_i[k]
//   dlogs_i = grad_out * (sum_k q_i[k] + sum_k gz_i[k] * z~_i[k])
// Root also: dbias_0 = grad_out * sum_k q_0[k] (z_0^k - bias_0) / prior_var.
// Non-shared parameters: writes the instance's dW_0 = 0 (the root has no W).
// ---------------------------------------------------------------------------------------
__global__ void k_node_reduce(Dev D) {
  __shared__ float red[3][8][33];
  const NodeInfo nd = D.nodes[blockIdx.x];
  const int d = nd.d, K = nd.K;
  const bool root = nd.parent < 0;
  const float go = D.grad_out ? (float)D.grad_out[nd.b] : 1.f;
  const int grp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float qs = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) qs += D.q[nd.off_nk + k];
  for (int o = 16; o > 0; o >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, o);
  __shared__ float qred[8];
  if (lane == 0) qred[grp] = qs;
  __syncthreads();
  float qtot = 0.f;
  for (int i = 0; i < 8; ++i) qtot += qred[i];
  for (int j0 = 0; j0 < d; j0 += 32) {
    const int j = j0 + lane;
    float sm_ = 0.f, sl = 0.f, sb = 0.f;
    if (j < d) {
      const float off = root ? D.q_mean[nd.off_q + j] - D.bias[nd.off_bias + j] : 0.f;
      for (int k = grp; k < K; k += 8) {
        const long long idx = nd.off_nkd + (long long)k * d + j;
        const float g = D.gz[idx], zt = D.zt[idx];
        sm_ += g;
        sl = fmaf(g, zt, sl);
        if (root) sb = fmaf(D.q[nd.off_nk + k], zt + off, sb);
      }
    }
    red[0][grp][lane] = sm_;
    red[1][grp][lane] = sl;
    red[2][grp][lane] = sb;
    __syncthreads();
    if (grp == 0 && j < d) {
      float a = 0.f, b = 0.f, c = 0.f;
      for (int i = 0; i < 8; ++i) { a += red[0][i][lane]; b += red[1][i][lane]; c += red[2][i][lane]; }
      if (D.dq_mean) D.dq_mean[nd.off_q + j] = go * a;
      if (D.dq_logstd) D.dq_logstd[nd.off_q + j] = go * (qtot + b);
      if (root) {
        const float db = go * c * D.inv_var;
        if (D.shared) { if (D.pbias) D.pbias[nd.off_q + j] = db; }
        else if (D.dbias) D.dbias[nd.off_bias + j] = db;
      }
    }
    __syncthreads();
  }
  if (root && !D.shared && D.dW)
    for (long long e = threadIdx.x; e < (long long)d * d; e += blockDim.x) D.dW[nd.off_W + e] = 0.f;
}

// ---------------------------------------------------------------------------------------
// dW_i = grad_out * sum_k dmu_i[k] z_p^k^T,  dbias_i = grad_out * sum_k dmu_i[k]
// (z_p = m_p + z~_p).  Grid: (non-root node, 64-row tile of W, 64-col tile of W).
// Shared parameters go to per-(instance, node) partials, summed later in a fixed order.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_param_dW(Dev D, const int* __restrict__ nonroot) {
  __shared__ TileSmem sm;
  __shared__ float colsum[kTile];
  const int g = nonroot[blockIdx.x];
  const NodeInfo nd = D.nodes[g];
  const NodeInfo pn = D.nodes[nd.parent];
  const int d = nd.d, dp = nd.dp, K = nd.Kp;  // dmu_i[k] for the parent's samples k
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.z * kTile;
  if (r0 >= d || c0 >= dp) return;
  const float go = D.grad_out ? (float)D.grad_out[nd.b] : 1.f;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  if (threadIdx.x < kTile) {
    const int r = r0 + threadIdx.x;
    float s = 0.f;
    if (r < d)
      for (int k = 0; k < K; ++k) s += D.dmu[nd.off_nkd + (long long)k * d + r];
    colsum[threadIdx.x] = s;
  }
  float acc[4][4];
  zero_acc(acc);
  // opA(m = r, l = k) = dmu[k][r0 + m];  opB(n = c, l = k) = z~_p[k][c0 + n]
  tile_gemm<false, false>(acc, D.dmu + nd.off_nkd + r0, d, min(kTile, d - r0),
                          D.zt + pn.off_nkd + c0, dp, min(kTile, dp - c0), K, sm);
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = r0 + ty * 4 + a;
    if (r >= d) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c >= dp) continue;
      const float v = go * (acc[a][b] + colsum[ty * 4 + a] * D.q_mean[pn.off_q + c]);
      if (D.shared) D.pW[nd.off_pW + (long long)r * dp + c] = v;
      else if (D.dW) D.dW[nd.off_W + (long long)r * dp + c] = v;
    }
  }
  if (c0 == 0 && threadIdx.x < kTile && r0 + threadIdx.x < d) {
    const float v = go * colsum[threadIdx.x];
    if (D.shared) D.pbias[nd.off_q + r0 + threadIdx.x] = v;
    else if (D.dbias) D.dbias[nd.off_bias + r0 + threadIdx.x] = v;
  }
}

// ---------------------------------------------------------------------------------------
// dC = grad_out * sum_{leaves l} sum_k q_l[k] (x_l - C z_l^k) z_l^k^T / obs_var.
// Grid: (instance, 64 x 64 tile of C (observation tile * ctiles + latent tile), chunk of
// kParamChunk nodes).  With one chunk the CTA writes dC (or the shared-parameter partial);
// with several it writes its chunk's partial, part[chunk][same layout], summed afterwards.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_param_dC(Dev D, int ctiles, float* __restrict__ part, long long part_ld) {
  extern __shared__ float xs[];
  __shared__ TileSmem sm;
  __shared__ float rsm[kTile * kLd];  // q-weighted residuals, [k][o]
  __shared__ float rsum[kTile];
  const InstInfo in = D.insts[blockIdx.x];
  const int d = in.d, obs = in.obs;  // d of the leaves
  const int o0 = (blockIdx.y / ctiles) * kTile, c0 = (blockIdx.y % ctiles) * kTile;
  if (o0 >= obs || c0 >= d) return;
  const int g_begin = in.node0 + min(in.n, (int)blockIdx.z * kParamChunk);
  const int g_end = in.node0 + min(in.n, ((int)blockIdx.z + 1) * kParamChunk);
  const int nob = min(kTile, obs - o0), ncol = min(kTile, d - c0);
  const float go = D.grad_out ? (float)D.grad_out[blockIdx.x] : 1.f;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float acc[4][4];
  zero_acc(acc);
  float macc[4][4];                          // sum_k r[k][o] * m[c]: folded at the end per leaf
  zero_acc(macc);
  for (int g = g_begin; g < g_end; ++g) {
    const NodeInfo nd = D.nodes[g];
    if (nd.leaf_slot < 0) continue;
    __syncthreads();
    centred_obs(D, nd, xs);
    __syncthreads();
    const int K = nd.K;
    float leaf_rsum[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += kTile) {
      const int rows = min(kTile, K - k0);
      float racc[4][4];
      zero_acc(racc);
      tile_gemm<true, true>(racc, D.zt + nd.off_nkd + (long long)k0 * d, d, rows,
                            D.C + nd.off_C + (long long)o0 * d, d, nob, d, sm);
      // racc[a][b]: k = k0 + ty*4 + a, o = o0 + tx*4 + b; store rsm[k][o] as [l = k][m = o]
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int k = k0 + ty * 4 + a;
        const float qv = (k < K) ? D.q[nd.off_nk + k] * D.inv_obs_var : 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int o = o0 + tx * 4 + b;
          rsm[(ty * 4 + a) * kLd + tx * 4 + b] = (o < obs && k < K) ? qv * (xs[o] - racc[a][b]) : 0.f;
        }
      }
      __syncthreads();
      // acc[o][c] += sum_k rsm[k][o] * z~[k][c]
      for (int l0 = 0; l0 < rows; l0 += kSlice) {
        load_slice<false>(sm.b, D.zt + nd.off_nkd + (long long)k0 * d + c0, d, ncol, l0, rows);
        __syncthreads();
        slice_fma(acc, rsm + l0 * kLd, sm.b);
        __syncthreads();
      }
      // row sums of the weighted residual for the m_l term
      if (threadIdx.x < kTile) {
        float s = 0.f;
        for (int k = 0; k < rows; ++k) s += rsm[k * kLd + threadIdx.x];
        rsum[threadIdx.x] = s;
      }
      __syncthreads();
#pragma unroll
      for (int a = 0; a < 4; ++a) leaf_rsum[a] += rsum[ty * 4 + a];
      __syncthreads();
    }
    // + (sum_k r[k][o]) * m_l[c]
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + tx * 4 + b;
        const float m = (c < d) ? D.q_mean[nd.off_q + c] : 0.f;
        macc[a][b] = fmaf(leaf_rsum[a], m, macc[a][b]);
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int o = o0 + ty * 4 + a;
    if (o >= obs) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c >= d) continue;
      const float v = go * (acc[a][b] + macc[a][b]);
      const long long e = (D.shared ? in.off_pC : in.off_C) + (long long)o * d + c;
      if (part) part[(long long)blockIdx.z * part_ld + e] = v;
      else if (D.shared) D.pC[e] = v;
      else D.dC[e] = v;
    }
  }
}

// One level of rows_sum: out[g * E + e] = sum of rows g * kRowChunk .. +kRowChunk - 1 (in order).
// 32 rows' loads are issued before they are added.
__global__ void __launch_bounds__(256) k_rows_sum(const float* __restrict__ in, long long R, long long E,
                                                  long long stride, float* __restrict__ out) {
  const long long e = blockIdx.x * 256ll + threadIdx.x;
  if (e >= E) return;
  const long long r0 = (long long)blockIdx.y * kRowChunk, r1 = min(R, r0 + kRowChunk);
  float s = 0.f;
  for (long long r = r0; r < r1; r += 32) {
    float v[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) v[u] = r + u < r1 ? __ldg(in + (r + u) * stride + e) : 0.f;
#pragma unroll
    for (int u = 0; u < 32; ++u) s += v[u];
  }
  out[(long long)blockIdx.y * E + e] = s;
}

// ---- launchers ----------------------------------------------------------------------------
void launch_node_const(const Dev& D, cudaStream_t s) {
  k_node_const<<<(D.num_nodes + kConstNodesPerCta - 1) / kConstNodesPerCta, 32 * kConstNodesPerCta, 0, s>>>(D);
}
void launch_sample(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s) {
  k_sample<<<ntiles, kThreads, 2 * kMaxD * sizeof(float), s>>>(D, tiles);
}
void launch_obs_fwd(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s) {
  if (ntiles) k_obs_fwd<<<ntiles, kThreads, kMaxD * sizeof(float), s>>>(D, tiles);
}
void launch_project(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s) {
  if (ntiles) k_project<<<ntiles, kThreads, kMaxD * sizeof(float), s>>>(D, tiles);
}
void launch_root(const Dev& D, int maxK, int root_fanout, cudaStream_t s) {
  static bool once = (cudaFuncSetAttribute(k_root, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (kMaxK + kRootThreads) * (int)sizeof(double)), true);
  (void)once;
  if (D.root_part) k_root_children<<<D.root_nchunk, 256, 0, s>>>(D);
  // wide roots summed in the kernel take kRootThreads; otherwise 256, or one or a few warps
  // when every root has few samples (many small instances)
  const int threads = (root_fanout > 32 && !D.root_part) ? kRootThreads
                      : maxK <= 128                      ? std::max(32, (maxK + 31) / 32 * 32)
                                                         : 256;
  k_root<<<D.num_inst, threads, (maxK + threads) * sizeof(double), s>>>(D);
}
void launch_node_grad(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s) {
  k_node_grad<<<ntiles, kThreads, kMaxD * sizeof(float), s>>>(D, tiles);
}
void launch_child_sum(const Dev& D, const Tile* items, int nitems, int maxd, int chunks, long long cs_total,
                      float* part, cudaStream_t s) {
  if (!nitems) return;
  k_child_sum<<<dim3(nitems, chunks, (maxd + kTile - 1) / kTile), kThreads, 0, s>>>(D, items, part, cs_total);
  rows_sum(part, chunks, cs_total, cs_total, D.csum, D.rsum, s);
}
void launch_node_reduce(const Dev& D, cudaStream_t s) { k_node_reduce<<<D.num_nodes, 256, 0, s>>>(D); }
void launch_param_dW(const Dev& D, const int* nonroot, int n_nonroot, int maxd, cudaStream_t s) {
  if (!n_nonroot) return;
  const int t = (maxd + kTile - 1) / kTile;
  k_param_dW<<<dim3(n_nonroot, t, t), kThreads, 0, s>>>(D, nonroot);
}
void launch_param_dC(const Dev& D, int maxd, int maxobs, int maxn, long long c_total, float* part,
                     cudaStream_t s) {
  const int ctiles = (maxd + kTile - 1) / kTile, chunks = (maxn + kParamChunk - 1) / kParamChunk;
  float* out = D.shared ? D.pC : D.dC;
  k_param_dC<<<dim3(D.num_inst, ((maxobs + kTile - 1) / kTile) * ctiles, chunks), kThreads,
               kMaxD * sizeof(float), s>>>(D, ctiles, chunks > 1 ? part : nullptr, c_total);
  if (chunks > 1 && out) rows_sum(part, chunks, c_total, c_total, out, D.rsum, s);
}
struct RowSegs {
  RowSeg s[kMaxRowSegs];
  int blk0[kMaxRowSegs + 1];  // first block of each segment
  int n;
};
// Single-level sums of several segments (R <= kRowChunk each): block b belongs to the last
// segment whose first block is <= b; the sum is the one k_rows_sum forms (rows in order, 32
// loads in flight).
__global__ void __launch_bounds__(256) k_rows_sum_multi(RowSegs S) {
  int si = 0;
  while (si + 1 < S.n && (int)blockIdx.x >= S.blk0[si + 1]) ++si;
  const RowSeg g = S.s[si];
  const long long e = (long long)(blockIdx.x - S.blk0[si]) * 256 + threadIdx.x;
  if (e >= g.E) return;
  float s = 0.f;
  for (long long r = 0; r < g.R; r += 32) {
    float v[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) v[u] = r + u < g.R ? __ldg(g.in + (r + u) * g.stride + e) : 0.f;
#pragma unroll
    for (int u = 0; u < 32; ++u) s += v[u];
  }
  g.out[e] = s;
}

void rows_sum_batch(const RowSeg* segs, int n, float* scratch, cudaStream_t s) {
  RowSegs S{};
  int blocks = 0;
  for (int i = 0; i < n; ++i) {
    if (segs[i].E <= 0) continue;
    if (segs[i].R > kRowChunk) {
      rows_sum(segs[i].in, segs[i].R, segs[i].E, segs[i].stride, segs[i].out, scratch, s);
      continue;
    }
    S.s[S.n] = segs[i];
    S.blk0[S.n] = blocks;
    blocks += (int)((segs[i].E + 255) / 256);
    ++S.n;
  }
  S.blk0[S.n] = blocks;
  if (S.n) k_rows_sum_multi<<<blocks, 256, 0, s>>>(S);
}

void rows_sum(const float* in, long long R, long long E, long long stride, float* out, float* scratch,
              cudaStream_t s) {
  if (E <= 0) return;
  const unsigned ex = (unsigned)((E + 255) / 256);
  const long long half = (R + kRowChunk - 1) / kRowChunk * E;
  const float* src = in;
  long long rows = R, ld = stride;
  int ping = 0;
  while (rows > kRowChunk) {  // one level: chunks of kRowChunk rows -> one row each
    const long long g = (rows + kRowChunk - 1) / kRowChunk;
    float* dst = scratch + ping * half;
    k_rows_sum<<<dim3(ex, (unsigned)g), 256, 0, s>>>(src, rows, E, ld, dst);
    src = dst;
    rows = g;
    ld = E;
    ping ^= 1;
  }
  k_rows_sum<<<dim3(ex, 1), 256, 0, s>>>(src, rows, E, ld, out);
}

// Shared parameters: dW, dbias, dC = sum over instances of the per-instance partials (rows_sum,
// fixed order); the root's block of W (the first rootW entries) is zero.  tc_done: dW past the
// root block and dC were written by the tensor-core path's own kernels.
void launch_shared_reduce(const Dev& D, long long nW, long long nb, long long nC, long long rootW,
                          bool tc_done, cudaStream_t s) {
  const long long B = D.num_inst;
  if (D.dW && rootW) cudaMemsetAsync(D.dW, 0, sizeof(float) * rootW, s);
  if (tc_done) return;
  RowSeg segs[3];
  int n = 0;
  if (D.dW && nW > rootW) segs[n++] = RowSeg{D.pW + rootW, D.dW + rootW, B, nW - rootW, nW};
  if (D.dbias && nb) segs[n++] = RowSeg{D.pbias, D.dbias, B, nb, nb};
  if (D.dC && nC) segs[n++] = RowSeg{D.pC, D.dC, B, nC, nC};
  rows_sum_batch(segs, n, D.rsum, s);
}
void launch_root_bias(const Dev&, cudaStream_t) {}

}  // namespace tmc
