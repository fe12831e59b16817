// k_loopy.cu -- TMC on the loopy graph of Fig. 1 with matrix messages (Section 2.2, Fig. 1 C/D;
// the log-domain matrix product of the Appendix, "Numerically stable matrix (tensor) products").
//
// Model per instance (all latents of dimension d, K samples each, sigma^2 = prior_var):
//   z1 ~ N(b_0, s2),  z2 | z1 ~ N(W_1 z1 + b_1, s2),  z3 | z1 ~ N(W_2 z1 + b_2, s2),
//   z4 | z2, z3 ~ N(W_3 z2 + W_4 z3 + b_3, s2),  x | z4 ~ N(C z4, obs_var).
// With centred samples z~_i = z_i - m_i:  mu2~^{k1} = W_1 z~1 + c2, mu3~^{k1} = W_2 z~1 + c3,
// a^{k2} = W_3 z~2 + c4, c^{k3} = W_4 z~3  (c2 = W_1 m1 + b_1 - m2, c3 = W_2 m1 + b_2 - m3,
// c4 = W_3 m2 + W_4 m3 + b_3 - m4), and per-sample node terms u_i (-log Q_i, the root prior,
// the observation).  Summing out k4 and k1 leaves two matrix messages over (k2, k3):
//   L4[k2][k3] = log sum_k4 exp(X4[k2][k4] + Y4[k3][k4]),
//       X4 = a.z~4 / s2 + beta4[k4],  Y4 = c.z~4 / s2,  beta4 = u4 - |z~4|^2 / (2 s2)
//   L1[k2][k3] = log sum_k1 exp(X1[k2][k1] + Y1[k3][k1]),
//       X1 = z~2.mu2~ / s2 + beta1[k1],  Y1 = z~3.mu3~ / s2,
//       beta1 = u1 - (|mu2~|^2 + |mu3~|^2) / (2 s2)
//   log P = const - 4 log K + log sum_{k2,k3} exp(P23 + L4 + L1),
//       P23 = -a.c / s2 + u2 - (|a|^2 + |z~2|^2) / (2 s2) + u3 - (|c|^2 + |z~3|^2) / (2 s2).
// The five K x K factor matrices are d-long contractions; the two messages are K-long
// contractions of exponentials: C = exp(X - x) exp(Y - y)^T with the row maxima x, y
// subtracted (the Appendix's logmmexp), then L = log C + x + y.  Both run on one tcgen05 GEMM
// kernel with split operands (v = hi + lo; hi*hi + lo*hi + hi*lo, FP32 accumulation): fp16
// pairs for the factors (about 22 bits), bf16 pairs (or single bf16) for the exponentials
// (about 16 bits, with the exponent range of FP32).  The maxima are lowered by a fixed shift
// so that exponentials up to e^38 are kept: an entry of C underflows only where every term
// lies below e^-163 relative to the row maxima, and such an entry is recomputed exactly in
// the final pass with the combined maximum.  The
// final (k2, k3) sum is a bandwidth-bound pass over P23, L4 and L1.
#include <algorithm>
#include <cstdio>
#include <vector>

#include <cuda.h>

#include "../../include/tmc.h"
#include <cuda_bf16.h>

#include "simt_tile.cuh"
#include "tc_ptx.cuh"
#include "tmc_tc.cuh"

using namespace tmc;
using namespace tmc::tc;

namespace {
constexpr int kLBox = 16384;             // one [128 rows x 64] 16-bit box, 128-byte swizzle
constexpr int kLNS = 3;                  // ring stages
constexpr int kLStage = 4 * kLBox;       // A hi, A lo, B hi, B lo of one 64-wide K slice
constexpr double kLog2Pi = 1.8378770664093454835606594728112;

enum { kProjMu2 = 0, kProjMu3 = 1, kProjA = 2, kProjC = 3 };

// Everything the loopy kernels touch (device pointers), passed by value.
struct LDev {
  int B, K, d, obs, dp, Kp, shared;
  int msplit;      // message operands: 1 split bf16 pairs, 0 single bf16
  float iv, iov;  // 1 / prior_var, 1 / obs_var
  // inputs
  const float *eps, *q_mean, *q_logstd, *W, *bias, *C, *x;
  // workspace
  float* zt;       // [B][4][K][d] centred samples
  float* pr;       // [B][4][K][d] mu2~, mu3~, a, c
  float* cv;       // [B][3][d]   c2, c3, c4
  float* xo;       // [B][obs]    x - C m4
  float* u;        // [B][4][K]   per-sample node terms
  float* zn;       // [B][4][K]   |z~|^2
  float* pn;       // [B][4][K]   |mu2~|^2, |mu3~|^2, |a|^2, |c|^2
  float* rowt;     // [B][5][K]   beta4, beta1, row2, col3, (unused)
  __half *oh, *ol; // [B][7][K][dp] split fp16 operands: z~2, z~3, z~4, mu2~, mu3~, a, c
  float* fac;      // [B][5][K][Kp] X4, Y4, X1, Y1, P23 (rows padded to Kp)
  __nv_bfloat16 *eh, *el;  // [B][4][K][Kp] split bf16 exp(X4 - x4), exp(Y4 - y4), exp(X1 - x1), exp(Y1 - y1)
  float* rmax;     // [B][4][K]   row maxima of X4, Y4, X1, Y1
  float* msg;      // [B][2][K][Kp] L4, L1 (rows padded to Kp)
  float2* part;    // [B][chunks] (max, sum) of the final sum, per chunk of kFinalRows rows
  double* cst;     // [B] FP64 constants
  double* log_phat;
  int* nfix;       // entries recomputed by the exact pass (diagnostic)
};

__device__ __forceinline__ const float* Wof(const LDev& L, int b, int w) {
  return L.W + ((L.shared ? 0 : (long long)b) * 5 + w) * L.d * L.d;
}
__device__ __forceinline__ const float* biasof(const LDev& L, int b, int i) {
  return L.bias + ((L.shared ? 0 : (long long)b) * 4 + i) * L.d;
}
__device__ __forceinline__ const float* Cof(const LDev& L, int b) {
  return L.C + (L.shared ? 0 : (long long)b) * L.obs * L.d;
}

// ---------------------------------------------------------------------------------------
// Samples, node terms and FP64 constants.  Grid: (instance, node, 64-sample tile); one warp
// per sample row.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dia_samples(LDev L) {
  const int b = blockIdx.x, i = blockIdx.y, d = L.d, K = L.K;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* ls = L.q_logstd + ((long long)b * 4 + i) * d;
  const float* m = L.q_mean + ((long long)b * 4 + i) * d;
  for (int r = w; r < kTile; r += 8) {
    const int k = blockIdx.z * kTile + r;
    if (k >= K) break;
    const long long row = (((long long)b * 4 + i) * K + k) * d;
    float se = 0.f, sz = 0.f, sr = 0.f;
    for (int j = lane; j < d; j += 32) {
      const float e = L.eps[row + j];
      const float z = expf(ls[j]) * e;
      L.zt[row + j] = z;
      se = fmaf(e, e, se);
      sz = fmaf(z, z, sz);
      if (i == 0) {
        const float rr = z + m[j] - biasof(L, b, 0)[j];
        sr = fmaf(rr, rr, sr);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      se += __shfl_xor_sync(0xffffffffu, se, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
    }
    if (lane == 0) {
      L.u[((long long)b * 4 + i) * K + k] = 0.5f * se - 0.5f * sr * L.iv;
      L.zn[((long long)b * 4 + i) * K + k] = sz;
    }
  }
  if (blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x < 32) {
    // sum_i (sum_j logs_ij + (d/2) log 2pi) - 4 (d/2) log(2 pi s2) - (obs/2) log(2 pi obs_var)
    double s = 0.0;
    for (int j = lane; j < 4 * d; j += 32) s += (double)L.q_logstd[(long long)b * 4 * d + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0)
      L.cst[b] = s + 4.0 * 0.5 * d * kLog2Pi - 4.0 * 0.5 * d * (kLog2Pi - log((double)L.iv)) -
                 0.5 * L.obs * (kLog2Pi - log((double)L.iov));
  }
}

// c2, c3, c4 and x~ = x - C m4 per instance (one CTA of 128 threads).
__global__ void __launch_bounds__(128) k_dia_consts(LDev L) {
  const int b = blockIdx.x, d = L.d;
  const float* m1 = L.q_mean + ((long long)b * 4 + 0) * d;
  const float* m2 = L.q_mean + ((long long)b * 4 + 1) * d;
  const float* m3 = L.q_mean + ((long long)b * 4 + 2) * d;
  const float* m4 = L.q_mean + ((long long)b * 4 + 3) * d;
  for (int r = threadIdx.x; r < d; r += blockDim.x) {
    float s2 = 0.f, s3 = 0.f, s4 = 0.f;
    for (int c = 0; c < d; ++c) {
      s2 = fmaf(Wof(L, b, 1)[r * d + c], m1[c], s2);
      s3 = fmaf(Wof(L, b, 2)[r * d + c], m1[c], s3);
      s4 = fmaf(Wof(L, b, 3)[r * d + c], m2[c], s4);
      s4 = fmaf(Wof(L, b, 4)[r * d + c], m3[c], s4);
    }
    L.cv[((long long)b * 3 + 0) * d + r] = s2 + biasof(L, b, 1)[r] - m2[r];
    L.cv[((long long)b * 3 + 1) * d + r] = s3 + biasof(L, b, 2)[r] - m3[r];
    L.cv[((long long)b * 3 + 2) * d + r] = s4 + biasof(L, b, 3)[r] - m4[r];
  }
  for (int o = threadIdx.x; o < L.obs; o += blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < d; ++c) s = fmaf(Cof(L, b)[(long long)o * d + c], m4[c], s);
    L.xo[(long long)b * L.obs + o] = L.x[(long long)b * L.obs + o] - s;
  }
}

// Projections: out[k] = z~_src[k] W_w^T + cvec, and |out|^2.  Grid: (instance, which, 64-row
// tile); which: mu2~ (z~1, W_1, c2), mu3~ (z~1, W_2, c3), a (z~2, W_3, c4), c (z~3, W_4, 0).
__global__ void __launch_bounds__(kThreads) k_dia_proj(LDev L) {
  __shared__ TileSmem sm;
  const int b = blockIdx.x, which = blockIdx.y, d = L.d, K = L.K;
  const int src = which <= kProjMu3 ? 0 : which == kProjA ? 1 : 2;
  const int wi = which + 1;  // W_1 .. W_4
  const float* cvec = which == kProjC ? nullptr : L.cv + ((long long)b * 3 + which) * d;
  const int row0 = blockIdx.z * kTile, rows = min(kTile, K - row0);
  const float* Z = L.zt + (((long long)b * 4 + src) * K + row0) * d;
  float* out = L.pr + (((long long)b * 4 + which) * K + row0) * d;
  const float* Wm = Wof(L, b, wi);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float rs[4] = {0.f, 0.f, 0.f, 0.f};
  for (int r0 = 0; r0 < d; r0 += kTile) {
    float acc[4][4];
    zero_acc(acc);
    tile_gemm<true, true>(acc, Z, d, rows, Wm + (long long)r0 * d, d, min(kTile, d - r0), d, sm);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int k = ty * 4 + a;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int r = r0 + tx * 4 + c;
        if (k < rows && r < d) {
          const float v = acc[a][c] + (cvec ? cvec[r] : 0.f);
          out[(long long)k * d + r] = v;
          rs[a] = fmaf(v, v, rs[a]);
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float s = row_group_sum(rs[a]);
    const int k = row0 + ty * 4 + a;
    if (tx == 0 && k < K) L.pn[((long long)b * 4 + which) * K + k] = s;
  }
}

// Observation: u4[k] -= |x~ - C z~4^k|^2 / (2 obs_var).  Grid: (instance, 64-row tile).
__global__ void __launch_bounds__(kThreads) k_dia_obs(LDev L) {
  __shared__ TileSmem sm;
  const int b = blockIdx.x, d = L.d, K = L.K, obs = L.obs;
  const int row0 = blockIdx.y * kTile, rows = min(kTile, K - row0);
  const float* Z = L.zt + (((long long)b * 4 + 3) * K + row0) * d;
  const float* xs = L.xo + (long long)b * obs;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float rs[4] = {0.f, 0.f, 0.f, 0.f};
  for (int o0 = 0; o0 < obs; o0 += kTile) {
    float acc[4][4];
    zero_acc(acc);
    tile_gemm<true, true>(acc, Z, d, rows, Cof(L, b) + (long long)o0 * d, d, min(kTile, obs - o0), d, sm);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int o = o0 + tx * 4 + c;
        if (o < obs) {
          const float r = xs[o] - acc[a][c];
          rs[a] = fmaf(r, r, rs[a]);
        }
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float s = row_group_sum(rs[a]);
    const int k = row0 + ty * 4 + a;
    if (tx == 0 && k < K) L.u[((long long)b * 4 + 3) * K + k] -= 0.5f * s * L.iov;
  }
}

// Per-sample vectors of the factor matrices: beta4, beta1, row2 (k2), col3 (k3).
__global__ void k_dia_terms(LDev L) {
  const int b = blockIdx.x, K = L.K;
  const float h = 0.5f * L.iv;
  const float* u = L.u + (long long)b * 4 * K;
  const float* zn = L.zn + (long long)b * 4 * K;
  const float* pn = L.pn + (long long)b * 4 * K;
  float* rt = L.rowt + (long long)b * 5 * K;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    rt[0 * K + k] = u[3 * K + k] - h * zn[3 * K + k];                      // beta4
    rt[1 * K + k] = u[0 * K + k] - h * (pn[0 * K + k] + pn[1 * K + k]);   // beta1
    rt[2 * K + k] = u[1 * K + k] - h * (pn[2 * K + k] + zn[1 * K + k]);   // row2
    rt[3 * K + k] = u[2 * K + k] - h * (pn[3 * K + k] + zn[2 * K + k]);   // col3
  }
}

// Split fp16 operand rows (hi, lo) of the seven [K][d] vectors, zero padded to dp columns.
// Grid: (instance, operand, 64-row tile); one warp per row.
__global__ void __launch_bounds__(256) k_dia_split16(LDev L) {
  const int b = blockIdx.x, op = blockIdx.y, d = L.d, K = L.K, dp = L.dp;
  const float* src = op < 3 ? L.zt + (((long long)b * 4 + 1 + op) * K) * d
                            : L.pr + (((long long)b * 4 + (op - 3)) * K) * d;
  __half* oh = L.oh + (((long long)b * 7 + op) * K) * dp;
  __half* ol = L.ol + (((long long)b * 7 + op) * K) * dp;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = w; r < kTile; r += 8) {
    const int k = blockIdx.z * kTile + r;
    if (k >= K) break;
    for (int j = lane; j < dp; j += 32) {
      const float v = j < d ? src[(long long)k * d + j] : 0.f;
      float hi, lo;
      split_half(v, hi, lo);
      oh[(long long)k * dp + j] = __float2half_rn(hi);
      ol[(long long)k * dp + j] = __float2half_rn(lo);
    }
  }
}

// exp(row - r) of the four message operands as split bf16 rows (zero padded to Kp), with
// r = max(row) - kExpShift: every exponential is at most e^kExpShift, so a product of two is at
// most e^(2 kExpShift) and a sum of K <= 16384 of them stays below the FP32 maximum, while
// a product now underflows only where the two exponents sum below -(87 + 2 kExpShift).
// Grid: (instance, matrix, 8-row group); one warp per row.
constexpr float kExpShift = 38.f;
__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__global__ void __launch_bounds__(256) k_dia_expsplit(LDev L) {
  const int b = blockIdx.x, mi = blockIdx.y, K = L.K, Kp = L.Kp;
  const int fi = mi;  // X4, Y4, X1, Y1 are factor matrices 0..3
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.z * 8 + w;
  if (k >= K) return;
  // rows are Kp floats (a multiple of 64): 8-column chunks are 32-byte aligned; columns >= K
  // of the factor rows are padding (read but masked)
  const float* row = L.fac + (((long long)b * 5 + fi) * K + k) * Kp;
  float mx = -INFINITY;
  for (int j = lane * 8; j < K; j += 256) {
    const float4 u0 = *reinterpret_cast<const float4*>(row + j);
    const float4 u1 = *reinterpret_cast<const float4*>(row + j + 4);
    const float e[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
    for (int x = 0; x < 8; ++x)
      if (j + x < K) mx = fmaxf(mx, e[x]);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float r = mx - kExpShift;
  __nv_bfloat16* eh = L.eh + (((long long)b * 4 + mi) * K + k) * Kp;
  __nv_bfloat16* el = L.el + (((long long)b * 4 + mi) * K + k) * Kp;
  for (int j = lane * 8; j < Kp; j += 256) {
    const float4 u0 = *reinterpret_cast<const float4*>(row + j);
    const float4 u1 = *reinterpret_cast<const float4*>(row + j + 4);
    const float e[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    float v[8], lo[8];
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      v[x] = j + x < K ? __expf(e[x] - r) : 0.f;
      lo[x] = v[x] - __bfloat162float(__float2bfloat16_rn(v[x]));
    }
    *reinterpret_cast<uint4*>(eh + j) =
        make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]), pack_bf2(v[6], v[7]));
    if (L.msplit)
      *reinterpret_cast<uint4*>(el + j) =
          make_uint4(pack_bf2(lo[0], lo[1]), pack_bf2(lo[2], lo[3]), pack_bf2(lo[4], lo[5]), pack_bf2(lo[6], lo[7]));
  }
  if (lane == 0) L.rmax[((long long)b * 4 + mi) * K + k] = r;
}

// ---------------------------------------------------------------------------------------
// Split-operand tcgen05 GEMM over a batch of (item, matrix) pairs: for output tile (ti, tk) of
// matrix m of item z,
//   acc[i][k] = sum_j (Ah + Al)[i][j] (Bh + Bl)[k][j]     (without Al * Bl; hi only if !split)
// with A rows z * a_step + a_off[m] + i and B rows z * b_step + b_off[m] + k of their tensor
// maps (K-major, 64-column boxes), nsl slices of 64 along j.  Epilogues:
//   MODE 0 (factor)   out[i][k] = alpha[m] acc + rt[i] + ct[k]
//   MODE 1 (message)  out[i][k] = log acc + rt[i] + ct[k]   (-inf where the sum underflowed:
//                     the final pass recomputes those entries exactly)
// rt / ct: terms + z * t_step + rt_off[m] / ct_off[m] (offset -1: none).  The output tile
// (columns, rows, item z * out_zmul + out_off[m]) leaves through a TMA store.
// Persistent and warp-specialised: one CTA per SM walks the tiles (ti fastest); warp 0 streams
// the slices through the shared-memory ring (3 stages of four boxes, or 6 of two when !split),
// warp 1 issues the MMAs into one of two TMEM accumulators, warps 2-9 drain the other: warp w
// reads TMEM lane quarter w % 4 (its 32 rows) and column half (w - 2) / 4, writes each 32 x 32
// block into a 128-byte-swizzled shared-memory buffer and stores it with one TMA copy, while
// the next tile is multiplied.
// ---------------------------------------------------------------------------------------
constexpr int kMaxMat = 5;
struct GemmArgs {
  int M, N, nsl, items, nmat;      // rows, columns of each output; 64-wide K slices; items; matrices
  long long a_step, b_step;        // operand rows per item
  int a_off[kMaxMat], b_off[kMaxMat];  // operand first rows of matrix m within an item
  const float* terms;              // row / column terms
  long long t_step;                // term elements per item
  int rt_off[kMaxMat], ct_off[kMaxMat];
  float alpha[kMaxMat];
  int out_zmul, out_off[kMaxMat];  // output item coordinate z * out_zmul + out_off[m]
  int bf16;                        // operands are bf16 (else fp16)
  int split;                       // 1: hi*hi + lo*hi + hi*lo; 0: hi*hi only (the lo maps unused)
};

constexpr int kGemmThreads = 320;                          // TMA warp, MMA warp, 8 epilogue warps
constexpr int kEpiWarps = 8;
constexpr int kStgBytes = 32 * 32 * 4;                     // one 32 x 32 fp32 block
// Shared memory per mode: the factor GEMM (2 slices per tile, epilogue-bound) keeps a 2-stage
// ring and two staging blocks per epilogue warp, so one block's TMA store overlaps the next
// block's math; the message GEMM keeps a 192 KB ring and one staging block per warp.
__host__ __device__ constexpr size_t ring_bytes(int mode) { return mode == 0 ? 2 * (size_t)kLStage : (size_t)kLNS * kLStage; }
__host__ __device__ constexpr int stg_bufs(int mode) { return mode == 0 ? 2 : 1; }
__host__ __device__ constexpr size_t gemm_smem(int mode) {
  return 1024 + ring_bytes(mode) + (size_t)kEpiWarps * stg_bufs(mode) * kStgBytes;
}
constexpr float kLn2 = 0.693147180559945309f;

__device__ __forceinline__ void tile_of(const GemmArgs& g, int bn, int t, int& z, int& m, int& ti, int& tk) {
  const int nti = (g.M + 127) >> 7, ntk = (g.N + bn - 1) / bn;
  const int zz = t / (nti * ntk);
  const int r = t - zz * nti * ntk;
  z = zz / g.nmat;
  m = zz - z * g.nmat;
  ti = r % nti;
  tk = r / nti;
}

__device__ __forceinline__ void tma_store_3d(const void* tmap, const void* src, int x, int y, int zc) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(tmap)),
               "r"(smem_u32(src)), "r"(x), "r"(y), "r"(zc)
               : "memory");
}

template <int MODE, int BN>
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm_split(GemmArgs g, int* err,
                                                                const __grid_constant__ CUtensorMap mAh,
                                                                const __grid_constant__ CUtensorMap mAl,
                                                                const __grid_constant__ CUtensorMap mBh,
                                                                const __grid_constant__ CUtensorMap mBl,
                                                                const __grid_constant__ CUtensorMap mOut) {
  extern __shared__ unsigned char smraw[];
  unsigned char* ring = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[2 * kLNS], empty[2 * kLNS], tfull[2], tempty[2];
  __shared__ uint32_t tbase;
  __shared__ volatile int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // stage: A hi [128 x 64], B hi [BN x 64] (, A lo, B lo)
  constexpr int kBBox = kLBox * BN / 128;
  const int shalf = kLBox + kBBox;
  const int sstride = g.split ? 2 * shalf : shalf;
  constexpr size_t kRing = ring_bytes(MODE);
  const int nst = (int)(kRing / sstride);  // messages: 3 or 6 stages (BN = 128), 2 or 4 (BN = 256)
  const int nti = (g.M + 127) >> 7, ntk = (g.N + BN - 1) / BN;
  const int total = nti * ntk * g.items * g.nmat;
  if (warp == 1) tmem_alloc(&tbase, 2 * BN);
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
    }
    fence_barrier_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  auto give_up = [&]() {
    s_abort = 1;
    atomicOr(err, kErrTimeout);
  };
  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int t = blockIdx.x; t < total && !s_abort; t += gridDim.x) {
        int z, m, ti, tk;
        tile_of(g, BN, t, z, m, ti, tk);
        const int arow = (int)((long long)z * g.a_step + g.a_off[m] + (long long)ti * 128);
        const int brow = (int)((long long)z * g.b_step + g.b_off[m] + (long long)tk * BN);
        bool ok = true;
        for (int s = 0; s < g.nsl; ++s, ++it) {
          const int st = it % nst, fill = it / nst;
          if (fill >= 1 && !mbar_wait(&empty[st], (uint32_t)((fill - 1) & 1))) { ok = false; break; }
          unsigned char* sp = ring + st * sstride;
          mbar_arrive_expect_tx(&full[st], (uint32_t)sstride);
          tma_load_2d(sp, &mAh, &full[st], s * 64, arow);
          tma_load_2d(sp + kLBox, &mBh, &full[st], s * 64, brow);
          if (g.split) {
            tma_load_2d(sp + shalf, &mAl, &full[st], s * 64, arow);
            tma_load_2d(sp + shalf + kLBox, &mBl, &full[st], s * 64, brow);
          }
        }
        if (!ok) { give_up(); break; }
      }
      // every issued copy has landed before the CTA may exit (bounded; normally immediate)
      for (int q = 0; q < nst && q < it; ++q) {
        const int f = it - 1 - q;
        mbar_wait(&full[f % nst], (uint32_t)((f / nst) & 1));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id = idesc_f16(128, BN, g.bf16 != 0, false, false);
      int it = 0, tl = 0;
      for (int t = blockIdx.x; t < total && !s_abort; t += gridDim.x, ++tl) {
        const int buf = tl & 1, use = tl >> 1;
        if (use >= 1 && !mbar_wait(&tempty[buf], (uint32_t)((use - 1) & 1))) { give_up(); break; }
        tc_fence_after();
        const uint32_t acc = tmem + buf * BN;
        bool ok = true;
        for (int s = 0; s < g.nsl; ++s, ++it) {
          const int st = it % nst;
          if (!mbar_wait(&full[st], (uint32_t)((it / nst) & 1))) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(ring + st * sstride);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            // 16-wide K step inside the 128-byte swizzled rows: start address + 32 bytes
            const uint64_t dah = smem_desc_sw128(sa + kk * 32, 16, 1024),
                           dbh = smem_desc_sw128(sa + kLBox + kk * 32, 16, 1024);
            mma_ss(acc, dah, dbh, id, (s > 0 || kk > 0) ? 1u : 0u);
            if (g.split) {
              const uint64_t dal = smem_desc_sw128(sa + shalf + kk * 32, 16, 1024),
                             dbl = smem_desc_sw128(sa + shalf + kLBox + kk * 32, 16, 1024);
              mma_ss(acc, dal, dbh, id, 1u);
              mma_ss(acc, dah, dbl, id, 1u);
            }
          }
          mma_commit(&empty[st]);
        }
        mma_commit(&tfull[buf]);
        if (!ok) { give_up(); break; }
      }
    }
  } else {
    const int e = warp - 2, q = warp & 3, h = e >> 2;  // lane quarter q, column half h
    constexpr int kBufs = stg_bufs(MODE);
    unsigned char* stg_base = ring + kRing + e * kBufs * kStgBytes;  // 1024-byte aligned
    int nstore = 0;  // TMA stores issued by this warp
    int tl = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++tl) {
      const int buf = tl & 1, use = tl >> 1;
      const bool ok = !s_abort && mbar_wait(&tfull[buf], (uint32_t)(use & 1));
      if (!ok) {
        if (lane == 0) give_up();
        break;
      }
      tc_fence_after();
      int z, m, ti, tk;
      tile_of(g, BN, t, z, m, ti, tk);
      const int i = ti * 128 + q * 32 + lane;  // accumulator row of this lane
      const float* tz = g.terms + (long long)z * g.t_step;
      const float rti = (g.rt_off[m] >= 0 && i < g.M) ? tz[g.rt_off[m] + i] : 0.f;
      const bool has_ct = g.ct_off[m] >= 0;
      const float alpha = g.alpha[m];
#pragma unroll 1
      for (int gg = 0; gg < BN / 64; ++gg) {
        const int grp = (BN / 64) * h + gg;  // 32-column group of this warp's half
        const int k0 = tk * BN + grp * 32;
        uint32_t v[32];
        tmem_ld32(tmem + buf * BN + ((uint32_t)(q * 32) << 16) + grp * 32, v);
        const float ctl = (has_ct && k0 + lane < g.N) ? tz[g.ct_off[m] + k0 + lane] : 0.f;
        tmem_wait_ld();
        unsigned char* stg = stg_base + (nstore % kBufs) * kStgBytes;
        if (nstore >= kBufs) {
          // the TMA store that last used this buffer has read it
          if (lane == 0) {
            if (kBufs == 2) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            else asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          }
          __syncwarp();
        }
#pragma unroll
        for (int c4 = 0; c4 < 8; ++c4) {
          float o[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int x = c4 * 4 + u;
            const float a = __uint_as_float(v[x]);
            const float ck = has_ct ? __shfl_sync(0xffffffffu, ctl, x) : 0.f;
            // MODE 1: lg2(0) = -inf marks an underflowed sum
            o[u] = MODE == 0 ? fmaf(a, alpha, rti) + ck : fmaf(__log2f(a), kLn2, rti) + ck;
          }
          // row = lane (128 bytes), 16-byte chunk c4 stored at chunk c4 ^ (row % 8)
          *reinterpret_cast<float4*>(stg + lane * 128 + ((c4 ^ (lane & 7)) << 4)) = make_float4(o[0], o[1], o[2], o[3]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_store_3d(&mOut, stg, k0, ti * 128 + q * 32, z * g.out_zmul + g.out_off[m]);
          bulk_commit_group();
        }
        ++nstore;
      }
      // the accumulator buffer is drained: the MMA warp may reuse it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
    if (lane == 0) bulk_wait_group0();  // every store has completed before the kernel ends
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * BN);
  }
}

// log sum_j exp(X[j] + Y[j]) over n terms, with the maximum of the whole exponent subtracted.
__device__ __noinline__ float exact_lse(const float* __restrict__ X, const float* __restrict__ Y, int n) {
  float mx = -INFINITY;
  for (int j = 0; j < n; ++j) mx = fmaxf(mx, X[j] + Y[j]);
  float s = 0.f;
  for (int j = 0; j < n; ++j) s += __expf(X[j] + Y[j] - mx);
  return mx + __logf(s);
}

// The final sum over (k2, k3) of exp(P23 + L4 + L1), by chunks of kFinalRows rows: each block
// writes the (max, sum exp(v - max)) of its chunk.  Message entries whose tensor-core sum
// underflowed (-inf) are recomputed here from the factor rows (rare).  Grid: (chunk, instance).
constexpr int kFinalRows = 8;
__device__ __forceinline__ void lse_add(float& m, float& s, float v) {
  if (v > m) {
    s = s * __expf(m - v) + 1.f;
    m = v;
  } else {
    s += __expf(v - m);
  }
}
__global__ void __launch_bounds__(256) k_dia_final(LDev L) {
  __shared__ float sm_m[8], sm_s[8];
  const int b = blockIdx.y, K = L.K, Kp = L.Kp;
  const long long mat = (long long)K * Kp;
  const float* P = L.fac + ((long long)b * 5 + 4) * mat;
  const float* L4 = L.msg + ((long long)b * 2 + 0) * mat;
  const float* L1 = L.msg + ((long long)b * 2 + 1) * mat;
  float m = -INFINITY, s = 0.f;
  const int r0 = blockIdx.x * kFinalRows, r1 = min(K, r0 + kFinalRows);
  // rows are Kp floats (a multiple of 64): 4-column chunks are 16-byte aligned
#pragma unroll 2
  for (int r = r0; r < r1; ++r) {
    for (int c = threadIdx.x * 4; c < K; c += blockDim.x * 4) {
      const long long e = (long long)r * Kp + c;
      const float4 p = *reinterpret_cast<const float4*>(P + e);
      const float4 a = *reinterpret_cast<const float4*>(L4 + e);
      const float4 q = *reinterpret_cast<const float4*>(L1 + e);
      float v[4] = {p.x + a.x + q.x, p.y + a.y + q.y, p.z + a.z + q.z, p.w + a.w + q.w};
      const float l4[4] = {a.x, a.y, a.z, a.w}, l1[4] = {q.x, q.y, q.z, q.w}, pp[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        if (c + x >= K) continue;
        if (!(v[x] > -INFINITY)) {
          // a message entry underflowed (or, defensively, is not a number): recompute it
          float f4 = l4[x], f1 = l1[x];
          if (!(f4 > -INFINITY)) {
            f4 = exact_lse(L.fac + (((long long)b * 5 + 0) * K + r) * Kp,
                           L.fac + (((long long)b * 5 + 1) * K + c + x) * Kp, K);
            atomicAdd(L.nfix, 1);
          }
          if (!(f1 > -INFINITY)) {
            f1 = exact_lse(L.fac + (((long long)b * 5 + 2) * K + r) * Kp,
                           L.fac + (((long long)b * 5 + 3) * K + c + x) * Kp, K);
            atomicAdd(L.nfix, 1);
          }
          v[x] = pp[x] + f4 + f1;
        }
        lse_add(m, s, v[x]);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float m2 = __shfl_xor_sync(0xffffffffu, m, o), s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float nm = fmaxf(m, m2);
    if (nm > -INFINITY) {
      s = s * __expf(m - nm) + s2 * __expf(m2 - nm);
      m = nm;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    sm_m[threadIdx.x >> 5] = m;
    sm_s[threadIdx.x >> 5] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = -INFINITY, ss = 0.f;
    for (int w = 0; w < 8; ++w) {
      const float nm = fmaxf(mm, sm_m[w]);
      if (nm > -INFINITY) {
        ss = ss * __expf(mm - nm) + sm_s[w] * __expf(sm_m[w] - nm);
        mm = nm;
      }
    }
    L.part[(long long)b * gridDim.x + blockIdx.x] = make_float2(mm, ss);
  }
}

// log P = const - 4 log K + log sum_{k2,k3} exp(P23 + L4 + L1), per instance, from the chunk
// (max, sum) pairs (FP64).
__global__ void __launch_bounds__(256) k_dia_combine(LDev L, int nchunks) {
  __shared__ double sm_m[8], sm_s[8];
  const int b = blockIdx.x;
  const float2* pp = L.part + (long long)b * nchunks;
  double m = -INFINITY;
  for (int t = threadIdx.x; t < nchunks; t += blockDim.x) m = fmax(m, (double)pp[t].x);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm_m[threadIdx.x >> 5] = m;
  __syncthreads();
  m = -INFINITY;
  for (int w = 0; w < 8; ++w) m = fmax(m, sm_m[w]);
  double s = 0.0;
  for (int t = threadIdx.x; t < nchunks; t += blockDim.x)
    if (pp[t].x > -INFINITY) s += (double)pp[t].y * exp((double)pp[t].x - m);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm_s[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sm_s[w];
    L.log_phat[b] = L.cst[b] - 4.0 * log((double)L.K) + m + log(t);
  }
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn loopy_encode() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
  }
  return fn;
}
// [rows][ld] 16-bit array, box 64 columns x box_rows rows, 128-byte swizzle (rows past the end
// read 0)
bool map16(CUtensorMap* m, void* ptr, long long rows, long long ld, bool bf16, int box_rows = 128) {
  EncodeFn enc = loopy_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ptr, dims, strides,
             box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
// [items][rows][ld] fp32 output (columns >= ld and rows >= rows are clipped), box 32 x 32 x 1,
// 128-byte swizzle
bool map_out(CUtensorMap* m, float* ptr, long long items, long long rows, long long ld) {
  EncodeFn enc = loopy_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)rows, (cuuint64_t)items};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)(ld * rows * 4)};
  cuuint32_t box[3] = {32, 32, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}
}  // namespace

struct tmc_loopy_plan_s {
  LDev L{};
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int* d_nfix = nullptr;
  int* d_err = nullptr;
  CUtensorMap mOh, mOl, mEh, mEl, mEh256, mEl256, mFac, mMsg;
  bool prof = false;
  cudaEvent_t ev[TMC_LOOPY_STAGE_COUNT + 1] = {};
  double stage_ms[TMC_LOOPY_STAGE_COUNT] = {};
  int num_sms = 148;
  int n_tile = 0;  // message GEMM N tile: 0 automatic, 128 or 256
  long long calls = 0;
};

extern "C" {

tmc_status tmc_loopy_plan_create(const tmc_loopy_desc* ds, tmc_loopy_plan* out) {
  if (!ds || !out) return TMC_ERR_INVALID_ARG;
  *out = nullptr;
  if (ds->num_instances < 1 || ds->K < 1 || ds->d < 1 || ds->obs_dim < 1 || !(ds->prior_var > 0.0) ||
      !(ds->obs_var > 0.0) || (ds->message_precision != 0 && ds->message_precision != 1))
    return TMC_ERR_INVALID_ARG;
  if (ds->d > kTcMaxD || ds->obs_dim > kMaxD || ds->K > kMaxK) return TMC_ERR_UNSUPPORTED;
  // tile row coordinates of the operand maps are 32-bit
  if ((long long)ds->num_instances * 7 * ds->K > (1ll << 30)) return TMC_ERR_UNSUPPORTED;
  tmc_loopy_plan p = new (std::nothrow) tmc_loopy_plan_s();
  if (!p) return TMC_ERR_NOMEM;
  LDev& L = p->L;
  L.B = ds->num_instances;
  L.K = ds->K;
  L.d = ds->d;
  L.obs = ds->obs_dim;
  L.shared = ds->shared_params ? 1 : 0;
  L.msplit = ds->message_precision == 0 ? 1 : 0;
  L.dp = (ds->d + 63) / 64 * 64;
  L.Kp = (ds->K + 63) / 64 * 64;
  L.iv = (float)(1.0 / ds->prior_var);
  L.iov = (float)(1.0 / ds->obs_var);
  const long long B = L.B, K = L.K, d = L.d, Kp = L.Kp;
  struct Sub { void** dst; size_t bytes; };
  const size_t kkp = (size_t)K * Kp;
  std::vector<Sub> subs = {
      {(void**)&L.zt, sizeof(float) * B * 4 * K * d}, {(void**)&L.pr, sizeof(float) * B * 4 * K * d},
      {(void**)&L.cv, sizeof(float) * B * 3 * d},     {(void**)&L.xo, sizeof(float) * B * L.obs},
      {(void**)&L.u, sizeof(float) * B * 4 * K},      {(void**)&L.zn, sizeof(float) * B * 4 * K},
      {(void**)&L.pn, sizeof(float) * B * 4 * K},     {(void**)&L.rowt, sizeof(float) * B * 5 * K},
      {(void**)&L.oh, sizeof(__half) * B * 7 * K * L.dp}, {(void**)&L.ol, sizeof(__half) * B * 7 * K * L.dp},
      {(void**)&L.fac, sizeof(float) * B * 5 * kkp}, {(void**)&L.eh, sizeof(__nv_bfloat16) * B * 4 * kkp},
      {(void**)&L.el, sizeof(__nv_bfloat16) * B * 4 * kkp}, {(void**)&L.rmax, sizeof(float) * B * 4 * K},
      {(void**)&L.msg, sizeof(float) * B * 2 * kkp}, {(void**)&L.cst, sizeof(double) * B},
      {(void**)&L.part, sizeof(float2) * B * ((K + kFinalRows - 1) / kFinalRows)},
  };
  size_t total = 0;
  auto al = [](size_t x) { return (x + 1023) & ~size_t(1023); };
  for (auto& s : subs) total += al(s.bytes);
  if (cudaMalloc(&p->ws, total) != cudaSuccess || cudaMalloc(&p->d_nfix, 2 * sizeof(int)) != cudaSuccess) {
    cudaFree(p->ws);
    delete p;
    return TMC_ERR_NOMEM;
  }
  p->d_err = p->d_nfix + 1;
  cudaMemset(p->d_nfix, 0, 2 * sizeof(int));
  p->ws_bytes = total;
  char* base = (char*)p->ws;
  for (auto& s : subs) { *s.dst = base; base += al(s.bytes); }
  L.nfix = p->d_nfix;
  if (!map16(&p->mOh, L.oh, B * 7 * K, L.dp, false) || !map16(&p->mOl, L.ol, B * 7 * K, L.dp, false) ||
      !map16(&p->mEh, L.eh, B * 4 * K, Kp, true) || !map16(&p->mEl, L.el, B * 4 * K, Kp, true) ||
      !map16(&p->mEh256, L.eh, B * 4 * K, Kp, true, 256) || !map16(&p->mEl256, L.el, B * 4 * K, Kp, true, 256) ||
      !map_out(&p->mFac, L.fac, B * 5, K, Kp) || !map_out(&p->mMsg, L.msg, B * 2, K, Kp)) {
    cudaFree(p->ws);
    cudaFree(p->d_nfix);
    delete p;
    return TMC_ERR_CUDA;
  }
  cudaFuncSetAttribute(k_gemm_split<0, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem(0));
  cudaFuncSetAttribute(k_gemm_split<1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem(1));
  cudaFuncSetAttribute(k_gemm_split<1, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem(1));
  for (auto& e : p->ev) cudaEventCreate(&e);
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  *out = p;
  return cudaGetLastError() == cudaSuccess ? TMC_OK : TMC_ERR_CUDA;
}

tmc_status tmc_loopy_log_marginal(tmc_loopy_plan p, const tmc_inputs* in, double* log_phat, void* stream) {
  if (!p || !in || !in->eps || !in->q_mean || !in->q_logstd || !in->W || !in->bias || !in->C || !in->x || !log_phat)
    return TMC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  LDev L = p->L;
  L.eps = in->eps; L.q_mean = in->q_mean; L.q_logstd = in->q_logstd;
  L.W = in->W; L.bias = in->bias; L.C = in->C; L.x = in->x;
  L.log_phat = log_phat;
  const int B = L.B, K = L.K, tiles64 = (K + kTile - 1) / kTile;
  if (p->prof) cudaEventRecord(p->ev[0], s);
  k_dia_samples<<<dim3(B, 4, tiles64), 256, 0, s>>>(L);
  k_dia_consts<<<B, 128, 0, s>>>(L);
  k_dia_proj<<<dim3(B, 4, tiles64), kThreads, 0, s>>>(L);
  k_dia_obs<<<dim3(B, tiles64), kThreads, 0, s>>>(L);
  k_dia_terms<<<B, 256, 0, s>>>(L);
  k_dia_split16<<<dim3(B, 7, tiles64), 256, 0, s>>>(L);
  if (p->prof) cudaEventRecord(p->ev[1], s);
  const int nt = (K + 127) / 128;
  // the five factor matrices in one launch.  Operands (rows of [B][7][K]): 0 z~2, 1 z~3,
  // 2 z~4, 3 mu2~, 4 mu3~, 5 a, 6 c; terms [B][5][K]: beta4, beta1, row2, col3.
  {
    GemmArgs g{};
    g.M = K; g.N = K; g.nsl = L.dp / 64; g.items = B; g.nmat = 5;
    g.a_step = 7ll * K; g.b_step = 7ll * K;
    g.terms = L.rowt; g.t_step = 5ll * K;
    g.out_zmul = 5;
    g.bf16 = 0;
    g.split = 1;
    struct F { int a, b, rt, ct; float alpha; };
    const F f[5] = {
        {5, 2, -1, 0, L.iv},   // X4[k2][k4] = a . z~4 / s2 + beta4[k4]
        {6, 2, -1, -1, L.iv},  // Y4[k3][k4] = c . z~4 / s2
        {0, 3, -1, 1, L.iv},   // X1[k2][k1] = z~2 . mu2~ / s2 + beta1[k1]
        {1, 4, -1, -1, L.iv},  // Y1[k3][k1] = z~3 . mu3~ / s2
        {5, 6, 2, 3, -L.iv},   // P23[k2][k3] = -a . c / s2 + row2[k2] + col3[k3]
    };
    for (int m = 0; m < 5; ++m) {
      g.a_off[m] = f[m].a * K;
      g.b_off[m] = f[m].b * K;
      g.rt_off[m] = f[m].rt < 0 ? -1 : f[m].rt * K;
      g.ct_off[m] = f[m].ct < 0 ? -1 : f[m].ct * K;
      g.alpha[m] = f[m].alpha;
      g.out_off[m] = m;
    }
    const int grid = std::min(nt * nt * B * 5, p->num_sms);
    k_gemm_split<0, 128><<<grid, kGemmThreads, gemm_smem(0), s>>>(g, p->d_err, p->mOh, p->mOl, p->mOh, p->mOl, p->mFac);
  }
  if (p->prof) cudaEventRecord(p->ev[2], s);
  k_dia_expsplit<<<dim3(B, 4, (K + 7) / 8), 256, 0, s>>>(L);
  if (p->prof) cudaEventRecord(p->ev[3], s);
  // the two messages in one launch: L[i][k] = log sum_j exp(X[i][j] + Y[k][j]) for (X4, Y4) and
  // (X1, Y1); terms [B][4][K]: the lowered row maxima of X4, Y4, X1, Y1
  {
    GemmArgs g{};
    g.M = K; g.N = K; g.nsl = L.Kp / 64; g.items = B; g.nmat = 2;
    g.a_step = 4ll * K; g.b_step = 4ll * K;
    g.terms = L.rmax; g.t_step = 4ll * K;
    g.out_zmul = 2;
    g.bf16 = 1;
    g.split = L.msplit;
    for (int m = 0; m < 2; ++m) {
      g.a_off[m] = 2 * m * K;
      g.b_off[m] = (2 * m + 1) * K;
      g.rt_off[m] = 2 * m * K;
      g.ct_off[m] = (2 * m + 1) * K;
      g.alpha[m] = 1.f;
      g.out_off[m] = m;
    }
    const bool wide = p->n_tile == 256 || (p->n_tile == 0 && K > 128);
    if (wide) {  // 128 x 256 tiles: a third fewer operand bytes per flop
      const int grid = std::min(nt * ((K + 255) / 256) * B * 2, p->num_sms);
      k_gemm_split<1, 256><<<grid, kGemmThreads, gemm_smem(1), s>>>(g, p->d_err, p->mEh, p->mEl, p->mEh256, p->mEl256,
                                                              p->mMsg);
    } else {
      const int grid = std::min(nt * nt * B * 2, p->num_sms);
      k_gemm_split<1, 128><<<grid, kGemmThreads, gemm_smem(1), s>>>(g, p->d_err, p->mEh, p->mEl, p->mEh, p->mEl, p->mMsg);
    }
  }
  if (p->prof) cudaEventRecord(p->ev[4], s);
  const int nchunks = (K + kFinalRows - 1) / kFinalRows;
  k_dia_final<<<dim3(nchunks, B), 256, 0, s>>>(L);
  k_dia_combine<<<B, 256, 0, s>>>(L, nchunks);
  if (p->prof) cudaEventRecord(p->ev[5], s);
  if (cudaGetLastError() != cudaSuccess) return TMC_ERR_CUDA;
  if (p->prof) {
    if (cudaEventSynchronize(p->ev[TMC_LOOPY_STAGE_COUNT]) != cudaSuccess) return TMC_ERR_CUDA;
    for (int st = 0; st < TMC_LOOPY_STAGE_COUNT; ++st) {
      float a = 0.f;
      cudaEventElapsedTime(&a, p->ev[st], p->ev[st + 1]);
      p->stage_ms[st] += a;
    }
    ++p->calls;
  }
  return TMC_OK;
}

tmc_status tmc_loopy_profile(tmc_loopy_plan p, int enable, double* stage_ms, long long* calls,
                             int* exact_entries) {
  if (!p) return TMC_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return TMC_ERR_CUDA;
  if (stage_ms)
    for (int st = 0; st < TMC_LOOPY_STAGE_COUNT; ++st) stage_ms[st] = p->stage_ms[st];
  if (calls) *calls = p->calls;
  if (exact_entries && cudaMemcpy(exact_entries, p->d_nfix, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return TMC_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TMC_ERR_CUDA;
  p->prof = enable != 0;
  for (double& v : p->stage_ms) v = 0.0;
  p->calls = 0;
  if (cudaMemset(p->d_nfix, 0, 2 * sizeof(int)) != cudaSuccess) return TMC_ERR_CUDA;
  return (err & kErrTimeout) ? TMC_ERR_TIMEOUT : TMC_OK;
}

tmc_status tmc_loopy_plan_set_tile(tmc_loopy_plan p, int n_tile) {
  if (!p || (n_tile != 0 && n_tile != 128 && n_tile != 256)) return TMC_ERR_INVALID_ARG;
  p->n_tile = n_tile;
  return TMC_OK;
}

tmc_status tmc_loopy_plan_destroy(tmc_loopy_plan p) {
  if (!p) return TMC_OK;
  cudaDeviceSynchronize();
  cudaFree(p->ws);
  cudaFree(p->d_nfix);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  delete p;
  return TMC_OK;
}

}  // extern "C"
