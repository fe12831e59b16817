// k_edge_f32.cu -- fused pairwise factor + log-sum-exp kernels on FP32 CUDA cores.
//
// For an edge p -> i (Section 2.2, summing out k_i; Appendix factors) the log-factor of
// parent sample k and child sample k' is, with centred samples / means,
//   log P(z_i^{k'} | z_p^k) = -|z~_i^{k'} - mu~_i^k|^2 / (2 var) - (d/2) log(2 pi var)
//                           = (mu~^k . z~^{k'} - |z~^{k'}|^2/2 - |mu~^k|^2/2) / var + const.
// The K x K block of these values is formed tile by tile in registers and never stored:
//   forward : lam_i[k] = log sum_k' exp(F[k,k'] + beta_i[k'])        (online max / sum)
//   adjoint : pi[k,k'] = q_p[k] exp(F[k,k'] + beta_i[k'] - lam_i[k]) (no max needed: each row
//             of pi sums to q_p[k] <= 1 and each column to q_i[k'] <= 1)
//     rows pass  (CTA owns 64 parent samples): dmu_i[k]  = (sum_k' pi z~^{k'} - q_p[k] mu~^k) / var
//     cols pass  (CTA owns 64 child samples) : q_i[k']   = sum_k pi,
//                                              gz_i[k']  = (sum_k pi mu~^k - q_i[k'] z~^{k'}) / var
// The FP64 constants (-(d/2) log(2 pi var) - log K and the max of beta) are added at the
// root in FP64, so lam and beta stay O(100) in FP32.
#include "simt_tile.cuh"

namespace tmc {

// Exponent given to padding columns.  Finite so that the online update never forms
// (-inf) - (-inf); any real column has a far larger exponent, and a row always has one.
constexpr float kInvalid = -1.0e30f;

// ---------------------------------------------------------------------------------------
// Forward message of one edge, 64 parent samples per CTA.
// ---------------------------------------------------------------------------------------
// Latents with d <= kResD keep the CTA's 64 x d block of mu~ in shared memory for the whole
// sweep over the child's samples (only the z~ tiles stream, in 64-deep slices); wider latents
// stream both operands in 16-deep slices.
constexpr int kResD = 128;
__host__ __device__ constexpr int res_smem_floats(int maxK) {
  return ((maxK + 3) & ~3) + (kResD + 2 * kDeep) * kLd;
}

__global__ void __launch_bounds__(kThreads) k_edge_fwd_f32(Dev D, const Tile* __restrict__ tiles) {
  extern __shared__ __align__(16) float cb[];  // [K]: beta - |z~|^2 / (2 var); then sa, sb
  __shared__ TileSmem sm;
  __shared__ float red[32];
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const int K = nd.K, Kp = nd.Kp, d = nd.d;  // child samples (columns), parent samples (rows)
  const float iv = D.inv_var;
  // beta_i and its max
  float mx = -INFINITY;
  for (int k = threadIdx.x; k < K; k += kThreads) {
    float v = D.u[nd.off_nk + k];
    for (int c = nd.child_begin; c < nd.child_end; ++c) v += D.lam[D.nodes[D.children[c]].off_nk + k];
    cb[k] = v;
    mx = fmaxf(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = -INFINITY;
#pragma unroll
  for (int i = 0; i < kThreads / 32; ++i) mx = fmaxf(mx, red[i]);
  const bool store = (t.row0 == 0);
  for (int k = threadIdx.x; k < K; k += kThreads) {
    const float b = cb[k] - mx;
    if (store) D.beta[nd.off_nk + k] = b;
    cb[k] = b - 0.5f * D.zn[nd.off_nk + k] * iv;
  }
  if (store && threadIdx.x == 0) D.nodemax[t.node] = mx;
  __syncthreads();

  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int rows = min(kTile, Kp - t.row0);
  const float* M = D.mut + nd.off_nkd + (long long)t.row0 * d;
  const float* Z = D.zt + nd.off_nkd;
  const bool res = d <= kResD;
  float* sa = cb + ((K + 3) & ~3);  // [kResD][kLd], then sb [kDeep][kLd]
  float* sb = sa + kResD * kLd;
  if (res) load_resident<true>(sa, M, d, rows, d);
  float rm[4], rs[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) { rm[a] = -INFINITY; rs[a] = 0.f; }
  for (int c0 = 0; c0 < K; c0 += kTile) {
    float acc[4][4];
    zero_acc(acc);
    if (res) tile_gemm_resA<true>(acc, sa, Z + (long long)c0 * d, d, min(kTile, K - c0), d, sb);
    else tile_gemm<true, true>(acc, M, d, rows, Z + (long long)c0 * d, d, min(kTile, K - c0), d, sm);
    float cv[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      cv[b] = (c < K) ? cb[c] : kInvalid;  // finite sentinel: exp(sentinel - max) = 0 later
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float e[4], tmax = -INFINITY;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        e[b] = fmaf(acc[a][b], iv, cv[b]);
        tmax = fmaxf(tmax, e[b]);
      }
      if (tmax > rm[a]) {
        rs[a] *= __expf(rm[a] - tmax);
        rm[a] = tmax;
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) rs[a] += __expf(e[b] - rm[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float gm = row_group_max(rm[a]);
    const float s = row_group_sum(rs[a] * __expf(rm[a] - gm));
    const int k = t.row0 + ty * 4 + a;
    if (tx == 0 && k < Kp) D.lam[nd.off_nk + k] = gm + logf(s) - 0.5f * D.mun[nd.off_nk + k] * iv;
  }
}

// Row bias of the adjoint: log q_p[k] - lam_i[k] - |mu~^k|^2 / (2 var)
__device__ __forceinline__ float adj_row_bias(const Dev& D, const NodeInfo& nd, const NodeInfo& pn,
                                              int k) {
  return logf(D.q[pn.off_nk + k]) - D.lam[nd.off_nk + k] - 0.5f * D.mun[nd.off_nk + k] * D.inv_var;
}

// ---------------------------------------------------------------------------------------
// Adjoint, rows pass: CTA owns 64 parent samples k; writes dmu_i[k] (all d columns).
// The d columns are covered 128 at a time (two 64-wide accumulators); wider d repeats
// the sweep over k' per 128-column chunk.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 2) k_edge_bwd_rows_f32(Dev D, const Tile* __restrict__ tiles) {
  extern __shared__ __align__(16) float cb[];  // [K]: beta - |z~|^2 / (2 var); then sa, sb, sb2
  __shared__ TileSmem sm;
  __shared__ float ps[kTile * kLd];  // pi tile stored [k'][k]
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const NodeInfo pn = D.nodes[nd.parent];
  const int K = nd.K, Kp = nd.Kp, d = nd.d;  // child samples (columns), parent samples (rows)
  const float iv = D.inv_var;
  for (int k = threadIdx.x; k < K; k += kThreads)
    cb[k] = D.beta[nd.off_nk + k] - 0.5f * D.zn[nd.off_nk + k] * iv;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int rows = min(kTile, Kp - t.row0);
  float ra[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int k = t.row0 + ty * 4 + a;
    ra[a] = (k < Kp) ? adj_row_bias(D, nd, pn, k) : -INFINITY;
  }
  __syncthreads();
  const float* M = D.mut + nd.off_nkd + (long long)t.row0 * d;
  const float* Z = D.zt + nd.off_nkd;
  const bool res = d <= kResD;
  float* sa = cb + ((K + 3) & ~3);  // [kResD][kLd]: mu~ of the CTA's rows, resident
  float* sb = sa + kResD * kLd;     // [kDeep][kLd] x 2: streamed z~ slices
  float* sb2 = sb + kDeep * kLd;
  if (res) load_resident<true>(sa, M, d, rows, d);
  for (int j0 = 0; j0 < d; j0 += 2 * kTile) {
    float o0[4][4], o1[4][4], rsum[4] = {0.f, 0.f, 0.f, 0.f};
    zero_acc(o0);
    zero_acc(o1);
    for (int c0 = 0; c0 < K; c0 += kTile) {
      const int cols = min(kTile, K - c0);
      float acc[4][4];
      zero_acc(acc);
      if (res) tile_gemm_resA<true>(acc, sa, Z + (long long)c0 * d, d, cols, d, sb);
      else tile_gemm<true, true>(acc, M, d, rows, Z + (long long)c0 * d, d, cols, d, sm);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + tx * 4 + b;
        const float cv = (c < K) ? cb[c] : -INFINITY;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float p = __expf(fmaf(acc[a][b], iv, ra[a] + cv));
          rsum[a] += p;
          ps[(tx * 4 + b) * kLd + ty * 4 + a] = p;
        }
      }
      // o[k][j] += sum_k' pi[k][k'] z~[k'][j]
      const float* Zc = Z + (long long)c0 * d + j0;
      if (res) {  // the tile's 64 rows of z~ in one round of loads
        float rv[kDeepVals];
        fetch_deep<false>(rv, Zc, d, min(kTile, d - j0), 0, cols);
        __syncthreads();  // the pi tile is written; the readers of sb are done
        store_deep<false>(sb, rv);
        if (j0 + kTile < d) {
          fetch_deep<false>(rv, Zc + kTile, d, min(kTile, d - j0 - kTile), 0, cols);
          store_deep<false>(sb2, rv);
        }
        __syncthreads();
        const int nq = (cols + kSlice - 1) / kSlice;
        for (int q = 0; q < nq; ++q) {
          slice_fma(o0, ps + q * kSlice * kLd, sb + q * kSlice * kLd);
          if (j0 + kTile < d) slice_fma(o1, ps + q * kSlice * kLd, sb2 + q * kSlice * kLd);
        }
        __syncthreads();  // ps and sb are rewritten by the next tile
      } else {
        __syncthreads();
        for (int l0 = 0; l0 < cols; l0 += kSlice) {
          load_slice<false>(sm.a, Zc, d, min(kTile, d - j0), l0, cols);
          if (j0 + kTile < d) load_slice<false>(sm.b, Zc + kTile, d, min(kTile, d - j0 - kTile), l0, cols);
          __syncthreads();
          slice_fma(o0, ps + l0 * kLd, sm.a);
          if (j0 + kTile < d) slice_fma(o1, ps + l0 * kLd, sm.b);
          __syncthreads();
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float rq = row_group_sum(rsum[a]);
      const int k = t.row0 + ty * 4 + a;
      if (k >= Kp) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int j = j0 + tx * 4 + b;
        const long long base = nd.off_nkd + (long long)k * d;
        if (j < d) D.dmu[base + j] = (o0[a][b] - rq * D.mut[base + j]) * iv;
        j += kTile;
        if (j < d) D.dmu[base + j] = (o1[a][b] - rq * D.mut[base + j]) * iv;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Adjoint, columns pass: CTA owns 64 child samples k'; writes q_i[k'] and the edge part of
// gz_i[k'] (all d columns).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 2) k_edge_bwd_cols_f32(Dev D, const Tile* __restrict__ tiles) {
  extern __shared__ __align__(16) float rb[];  // [Kp]: row bias per parent sample k; then sa, sb, sb2
  __shared__ TileSmem sm;
  __shared__ float ps[kTile * kLd];  // pi^T tile stored [k][k']
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const NodeInfo pn = D.nodes[nd.parent];
  const int K = nd.K, Kp = nd.Kp, d = nd.d;  // child samples (owned rows), parent samples
  const float iv = D.inv_var;
  for (int k = threadIdx.x; k < Kp; k += kThreads) rb[k] = adj_row_bias(D, nd, pn, k);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int cols = min(kTile, K - t.row0);  // child samples owned
  float cva[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int c = t.row0 + ty * 4 + a;
    cva[a] = (c < K) ? D.beta[nd.off_nk + c] - 0.5f * D.zn[nd.off_nk + c] * iv : -INFINITY;
  }
  __syncthreads();
  const float* Zo = D.zt + nd.off_nkd + (long long)t.row0 * d;
  const float* M = D.mut + nd.off_nkd;
  const bool res = d <= kResD;
  float* sa = rb + ((Kp + 3) & ~3);  // [kResD][kLd]: z~ of the CTA's child samples, resident
  float* sb = sa + kResD * kLd;      // [kDeep][kLd] x 2: streamed mu~ slices
  float* sb2 = sb + kDeep * kLd;
  if (res) load_resident<true>(sa, Zo, d, cols, d);
  for (int j0 = 0; j0 < d; j0 += 2 * kTile) {
    float o0[4][4], o1[4][4], qsum[4] = {0.f, 0.f, 0.f, 0.f};
    zero_acc(o0);
    zero_acc(o1);
    for (int r0 = 0; r0 < Kp; r0 += kTile) {
      const int rws = min(kTile, Kp - r0);
      float acc[4][4];  // acc[a][b]: child k' = row0 + ty*4 + a, parent k = r0 + tx*4 + b
      zero_acc(acc);
      if (res) tile_gemm_resA<true>(acc, sa, M + (long long)r0 * d, d, rws, d, sb);
      else tile_gemm<true, true>(acc, Zo, d, cols, M + (long long)r0 * d, d, rws, d, sm);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int k = r0 + tx * 4 + b;
        const float rv = (k < Kp) ? rb[k] : -INFINITY;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float p = __expf(fmaf(acc[a][b], iv, cva[a] + rv));
          qsum[a] += p;
          ps[(tx * 4 + b) * kLd + ty * 4 + a] = p;
        }
      }
      const float* Mr = M + (long long)r0 * d + j0;
      if (res) {  // the tile's 64 rows of mu~ in one round of loads
        float rv[kDeepVals];
        fetch_deep<false>(rv, Mr, d, min(kTile, d - j0), 0, rws);
        __syncthreads();  // the pi tile is written; the readers of sb are done
        store_deep<false>(sb, rv);
        if (j0 + kTile < d) {
          fetch_deep<false>(rv, Mr + kTile, d, min(kTile, d - j0 - kTile), 0, rws);
          store_deep<false>(sb2, rv);
        }
        __syncthreads();
        const int nq = (rws + kSlice - 1) / kSlice;
        for (int q = 0; q < nq; ++q) {
          slice_fma(o0, ps + q * kSlice * kLd, sb + q * kSlice * kLd);
          if (j0 + kTile < d) slice_fma(o1, ps + q * kSlice * kLd, sb2 + q * kSlice * kLd);
        }
        __syncthreads();  // ps and sb are rewritten by the next tile
      } else {
        __syncthreads();
        for (int l0 = 0; l0 < rws; l0 += kSlice) {
          load_slice<false>(sm.a, Mr, d, min(kTile, d - j0), l0, rws);
          if (j0 + kTile < d) load_slice<false>(sm.b, Mr + kTile, d, min(kTile, d - j0 - kTile), l0, rws);
          __syncthreads();
          slice_fma(o0, ps + l0 * kLd, sm.a);
          if (j0 + kTile < d) slice_fma(o1, ps + l0 * kLd, sm.b);
          __syncthreads();
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float qs = row_group_sum(qsum[a]);
      const int c = t.row0 + ty * 4 + a;
      if (c >= K) continue;
      if (tx == 0 && j0 == 0) D.q[nd.off_nk + c] = qs;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int j = j0 + tx * 4 + b;
        const long long base = nd.off_nkd + (long long)c * d;
        if (j < d) D.gz[base + j] = (o0[a][b] - qs * D.zt[base + j]) * iv;
        j += kTile;
        if (j < d) D.gz[base + j] = (o1[a][b] - qs * D.zt[base + j]) * iv;
      }
    }
  }
}

// The K-float prologue array lives in dynamic shared memory; K up to kMaxK needs the opt-in.
template <class Kern>
static void allow_dynamic_smem(Kern k) {
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxK * (int)sizeof(float));
}

void launch_edge_fwd_f32(const Dev& D, const Tile* tiles, int ntiles, int maxK, cudaStream_t s) {
  static bool once = (cudaFuncSetAttribute(k_edge_fwd_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           res_smem_floats(kMaxK) * (int)sizeof(float)),
                      true);
  (void)once;
  if (ntiles) k_edge_fwd_f32<<<ntiles, kThreads, res_smem_floats(maxK) * sizeof(float), s>>>(D, tiles);
}
void launch_edge_bwd_rows_f32(const Dev& D, const Tile* tiles, int ntiles, int maxK, cudaStream_t s) {
  static bool once = (cudaFuncSetAttribute(k_edge_bwd_rows_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           res_smem_floats(kMaxK) * (int)sizeof(float)),
                      true);
  (void)once;
  if (ntiles) k_edge_bwd_rows_f32<<<ntiles, kThreads, res_smem_floats(maxK) * sizeof(float), s>>>(D, tiles);
}
void launch_edge_bwd_cols_f32(const Dev& D, const Tile* tiles, int ntiles, int maxK, cudaStream_t s) {
  static bool once = (cudaFuncSetAttribute(k_edge_bwd_cols_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           res_smem_floats(kMaxK) * (int)sizeof(float)),
                      true);
  (void)once;
  if (ntiles) k_edge_bwd_cols_f32<<<ntiles, kThreads, res_smem_floats(maxK) * sizeof(float), s>>>(D, tiles);
}

}  // namespace tmc
