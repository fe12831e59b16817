// k_couple.cu -- coupled (non-factorised) proposals (Section 2.3 "Non-factorised proposals";
// appendix: the proposal of a latent may depend on the samples of other latents, and the
// estimator keeps the form of Eq. (is) because each proposal factor is indexed by k_i alone).
//
// Here sample k of latent i is drawn given its parent's sample k:
//   z_i^k = m_i + A_i (z_p^k - m_p) + s_i eps_i^k,   i.e.  z~_i^k = A_i z~_p^k + s_i eps_i^k,
//   Q_i(z_i^k | parent samples) = N(m_i + A_i z~_p^k, diag(s_i^2)),  s_i = exp(logs_i).
// In terms of eps, -log Q_i = sum_j (eps_j^2/2 + logs_j) + const -- the node term is the
// factorised one -- so only the samples change in the forward pass.  Gradients with eps held
// fixed see every descendant's sample k move with z_i^k:
//   T_i^k = G_i^k + sum_{children c} A_c^T T_c^k     (G: the path gradient of log P(x, z))
//   dz_i^k = grad_out (T_i^k + q_i[k] eps_i^k / s_i)  (= (d/d eps) / s; the factorised dz
//                                                       when A = 0),  deps = s dz,
//   dm_i = grad_out sum_k G_i^k,  dlogs_i = grad_out (sum_k q_i[k] + sum_k T_i^k s_i eps_i^k),
//   dA_i = grad_out sum_k T_i^k z~_p^k^T.
// FP32 tile GEMMs, one launch per tree level (parents before children forward, children
// before parents for T).
#include "simt_tile.cuh"

namespace tmc {

// z~_i += z~_p A_i^T (sample k of the parent for sample k of the child), then |z~_i|^2.
// Grid: (coupled node, 64-sample tile of its own samples).
__global__ void __launch_bounds__(kThreads) k_couple_fwd(Dev D, const Tile* __restrict__ tiles) {
  __shared__ TileSmem sm;
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const NodeInfo pn = D.nodes[nd.parent];
  const int d = nd.d, dp = nd.dp, K = nd.K;
  const float* A = D.q_A + nd.off_A;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int rows = min(kTile, K - t.row0);
  const float* Zp = D.zt + pn.off_nkd + (long long)t.row0 * dp;
  float* Z = D.zt + nd.off_nkd + (long long)t.row0 * d;
  float rs[4] = {0.f, 0.f, 0.f, 0.f};
  for (int r0 = 0; r0 < d; r0 += kTile) {
    float acc[4][4];
    zero_acc(acc);
    tile_gemm<true, true>(acc, Zp, dp, rows, A + (long long)r0 * dp, dp, min(kTile, d - r0), dp, sm);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = ty * 4 + a;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = r0 + tx * 4 + b;
        if (r < rows && c < d) {
          const float v = Z[(long long)r * d + c] + acc[a][b];
          Z[(long long)r * d + c] = v;
          rs[a] = fmaf(v, v, rs[a]);
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float s = row_group_sum(rs[a]);
    const int k = t.row0 + ty * 4 + a;
    if (tx == 0 && k < K) D.zn[nd.off_nk + k] = s;
  }
}

// T_i = G_i + sum_children T_c A_c (rows: this node's samples).  Grid: (node, 64-sample tile);
// loops over 64-wide latent tiles.
__global__ void __launch_bounds__(kThreads) k_couple_T(Dev D, const Tile* __restrict__ tiles) {
  __shared__ TileSmem sm;
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const int d = nd.d, K = nd.K;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int rows = min(kTile, K - t.row0);
  for (int c0 = 0; c0 < d; c0 += kTile) {
    const int ncol = min(kTile, d - c0);
    float acc[4][4];
    zero_acc(acc);
    for (int ci = nd.child_begin; ci < nd.child_end; ++ci) {
      const NodeInfo ch = D.nodes[D.children[ci]];
      // acc[k][c] += sum_r T_c[k][r] A_c[r][c]   (A_c is d_c x d); only the child's samples
      // k < K_c were drawn given this node's sample k (K_c <= K)
      const int crows = min(rows, ch.K - t.row0);
      if (crows <= 0) continue;  // uniform over the CTA: tile_gemm's barriers stay matched
      tile_gemm<true, false>(acc, D.tq + ch.off_nkd + (long long)t.row0 * ch.d, ch.d, crows,
                             D.q_A + ch.off_A + c0, d, ncol, ch.d, sm);
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
        D.tq[idx] = D.gsrc[idx] + acc[a][b];
      }
    }
  }
}

// dz = grad_out (T + q eps / s), deps = s dz.  Grid: (node, 64-sample tile).
__global__ void __launch_bounds__(kThreads) k_couple_out(Dev D, const Tile* __restrict__ tiles) {
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const int d = nd.d;
  const float go = D.grad_out ? (float)D.grad_out[nd.b] : 1.f;
  const int rows = min(kTile, nd.K - t.row0);
  for (int e = threadIdx.x; e < rows * d; e += blockDim.x) {
    const int r = e / d, j = e % d, k = t.row0 + r;
    const float s = expf(D.q_logstd[nd.off_q + j]);
    const long long ei = nd.off_e + (long long)k * d + j;
    const float v = go * (D.tq[nd.off_nkd + (long long)k * d + j] + D.q[nd.off_nk + k] * D.eps[ei] / s);
    if (D.dz) D.dz[ei] = v;
    if (D.deps) D.deps[ei] = v * s;
  }
}

// dlogs_i = grad_out (sum_k q_i[k] + sum_k T_i^k s_i eps_i^k).  One CTA of 256 threads per node.
__global__ void __launch_bounds__(256) k_couple_logs(Dev D) {
  __shared__ float red[8][33];
  __shared__ float qred[8];
  const NodeInfo nd = D.nodes[blockIdx.x];
  const int d = nd.d, K = nd.K;
  const float go = D.grad_out ? (float)D.grad_out[nd.b] : 1.f;
  const int grp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float qs = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) qs += D.q[nd.off_nk + k];
  for (int o = 16; o > 0; o >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, o);
  if (lane == 0) qred[grp] = qs;
  __syncthreads();
  float qtot = 0.f;
  for (int i = 0; i < 8; ++i) qtot += qred[i];
  for (int j0 = 0; j0 < d; j0 += 32) {
    const int j = j0 + lane;
    float sl = 0.f;
    if (j < d) {
      const float s = expf(D.q_logstd[nd.off_q + j]);
      for (int k = grp; k < K; k += 8)
        sl = fmaf(D.tq[nd.off_nkd + (long long)k * d + j], s * D.eps[nd.off_e + (long long)k * d + j], sl);
    }
    red[grp][lane] = sl;
    __syncthreads();
    if (grp == 0 && j < d) {
      float b = 0.f;
      for (int i = 0; i < 8; ++i) b += red[i][lane];
      if (D.dq_logstd) D.dq_logstd[nd.off_q + j] = go * (qtot + b);
    }
    __syncthreads();
  }
}

// dA_i = grad_out sum_k T_i^k z~_p^k^T.  Grid: (non-root node, 64-row tile, 64-col tile).
__global__ void __launch_bounds__(kThreads) k_couple_dA(Dev D, const int* __restrict__ nonroot) {
  __shared__ TileSmem sm;
  const int g = nonroot[blockIdx.x];
  const NodeInfo nd = D.nodes[g];
  const NodeInfo pn = D.nodes[nd.parent];
  const int d = nd.d, dp = nd.dp, K = nd.K;
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.z * kTile;
  if (r0 >= d || c0 >= dp) return;
  const float go = D.grad_out ? (float)D.grad_out[nd.b] : 1.f;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float acc[4][4];
  zero_acc(acc);
  // opA(m = r, l = k) = T[k][r0 + m];  opB(n = c, l = k) = z~_p[k][c0 + n]
  tile_gemm<false, false>(acc, D.tq + nd.off_nkd + r0, d, min(kTile, d - r0),
                          D.zt + pn.off_nkd + c0, dp, min(kTile, dp - c0), K, sm);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = r0 + ty * 4 + a;
    if (r >= d) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c < dp) D.dq_A[nd.off_A + (long long)r * dp + c] = go * acc[a][b];
    }
  }
}

// The root's block of dq_A is zero (it has no parent to couple to).
__global__ void k_couple_dA_root(Dev D) {
  const NodeInfo nd = D.nodes[D.insts[blockIdx.x].node0];
  for (int e = threadIdx.x; e < nd.d * nd.d; e += blockDim.x) D.dq_A[nd.off_A + e] = 0.f;
}

void launch_couple_fwd(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s) {
  if (ntiles) k_couple_fwd<<<ntiles, kThreads, 0, s>>>(D, tiles);
}
void launch_couple_T(const Dev& D, const Tile* tiles, int ntiles, cudaStream_t s) {
  if (ntiles) k_couple_T<<<ntiles, kThreads, 0, s>>>(D, tiles);
}
void launch_couple_out(const Dev& D, const Tile* tiles, int ntiles, const int* nonroot, int n_nonroot,
                       int maxd, cudaStream_t s) {
  if (D.dz || D.deps) k_couple_out<<<ntiles, kThreads, 0, s>>>(D, tiles);
  if (D.dq_logstd) k_couple_logs<<<D.num_nodes, 256, 0, s>>>(D);
  if (D.dq_A) {
    k_couple_dA_root<<<D.num_inst, 256, 0, s>>>(D);
    if (n_nonroot) {
      const int tt = (maxd + kTile - 1) / kTile;
      k_couple_dA<<<dim3(n_nonroot, tt, tt), kThreads, 0, s>>>(D, nonroot);
    }
  }
}

}  // namespace tmc
