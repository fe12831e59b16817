// k_unfused.cu -- the materialised baseline of the forward messages (FP32).
//
// The fused kernels never store the K x K block of pairwise log-factors of an edge.  This
// baseline does what a plain tensor-op implementation of Section 2.2 does: it first writes
// every factor of every edge to device memory,
//   F[k][k'] = (mu~^k . z~^{k'} - |z~^{k'}|^2 / 2 - |mu~^k|^2 / 2) / var   (constants removed),
// and then, level by level, reduces each row with a log-sum-exp against beta_i,
//   lam_i[k] = log sum_k' exp(F[k][k'] + beta_i[k']).
// Results equal the fused FP32 kernels up to rounding; the cost is 4 bytes written and read
// per factor entry.
#include "simt_tile.cuh"

namespace tmc {

// Grid: (edge tile of 64 parent samples, 64-wide tile of child samples).
__global__ void __launch_bounds__(kThreads) k_factors_f32(Dev D, const Tile* __restrict__ tiles) {
  __shared__ TileSmem sm;
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const int K = nd.K, d = nd.d;
  const int c0 = blockIdx.y * kTile;
  if (c0 >= K) return;
  const int rows = min(kTile, K - t.row0), cols = min(kTile, K - c0);
  float acc[4][4];
  zero_acc(acc);
  tile_gemm<true, true>(acc, D.mut + nd.off_nkd + (long long)t.row0 * d, d, rows,
                        D.zt + nd.off_nkd + (long long)c0 * d, d, cols, d, sm);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float* F = D.fac + D.fac_off[t.node];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int k = t.row0 + ty * 4 + a;
    if (k >= K) continue;
    const float hm = 0.5f * D.mun[nd.off_nk + k];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int kk = c0 + tx * 4 + b;
      if (kk < K) F[(long long)k * K + kk] = (acc[a][b] - 0.5f * D.zn[nd.off_nk + kk] - hm) * D.inv_var;
    }
  }
}

// Grid: edge tile of 64 parent samples; one warp per row, lanes over the child samples.
__global__ void __launch_bounds__(kThreads) k_lse_rows_f32(Dev D, const Tile* __restrict__ tiles) {
  extern __shared__ float sb[];  // [K]: normalised beta_i
  __shared__ float red[kThreads / 32];
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const int K = nd.K;
  float mx = -INFINITY;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    float v = D.u[nd.off_nk + k];
    for (int c = nd.child_begin; c < nd.child_end; ++c) v += D.lam[D.nodes[D.children[c]].off_nk + k];
    sb[k] = v;
    mx = fmaxf(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = -INFINITY;
  for (int i = 0; i < kThreads / 32; ++i) mx = fmaxf(mx, red[i]);
  const bool store = (t.row0 == 0);
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const float b = sb[k] - mx;
    sb[k] = b;
    if (store) D.beta[nd.off_nk + k] = b;
  }
  if (store && threadIdx.x == 0) D.nodemax[t.node] = mx;
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* F = D.fac + D.fac_off[t.node];
  for (int r = w; r < kTile; r += kThreads / 32) {
    const int k = t.row0 + r;
    if (k >= K) break;
    const float* row = F + (long long)k * K;
    float m = -INFINITY;
    for (int kk = lane; kk < K; kk += 32) m = fmaxf(m, row[kk] + sb[kk]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    float s = 0.f;
    for (int kk = lane; kk < K; kk += 32) s += __expf(row[kk] + sb[kk] - m);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) D.lam[nd.off_nk + k] = m + logf(s);
  }
}

void launch_factors_f32(const Dev& D, const Tile* tiles, int ntiles, int maxK, cudaStream_t s) {
  if (ntiles) k_factors_f32<<<dim3(ntiles, (maxK + kTile - 1) / kTile), kThreads, 0, s>>>(D, tiles);
}
void launch_lse_rows_f32(const Dev& D, const Tile* tiles, int ntiles, int maxK, cudaStream_t s) {
  static bool once = (cudaFuncSetAttribute(k_lse_rows_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           kMaxK * (int)sizeof(float)),
                      true);
  (void)once;
  if (ntiles) k_lse_rows_f32<<<ntiles, kThreads, maxK * sizeof(float), s>>>(D, tiles);
}

}  // namespace tmc
