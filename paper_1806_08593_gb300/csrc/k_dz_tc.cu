// k_dz_tc.cu -- per-sample gradients (dz, deps) on the tensor-core path.
//
// d log P / d z_i^k collects, for sample k of latent i (Section 2.2: gradient of log P_TMC;
// weights pi of the adjoint, q_i[k] = sum over the other index of pi), with everything centred
// (z~ = z - m_i, mu~_c^k = W_c z~_i^k + c_c, c_c = W_c m_i + bias_c - m_c):
//   through the edge pa(i) -> i:   (sum_k' pi_i[k',k] mu~_i^{k'} - q_i[k] z~_i^k) / var
//                                 = q_i[k] (Vt_i[k] W_i^T + c_i - z~_i^k) / var,
//        Vt_i[k] = sum_k' pi_i[k',k] z~_p^{k'} / q_i[k]         (k_edge_bwd_tc stores it)
//   through each edge i -> c:      q_i[k] W_c^T (R_c[k] - mu~_c^k) / var,
//        R_c[k] = sum_k' softmax_k'(F_c[k,.] + beta_c)[k'] z~_c^{k'}   (the row pass stores
//        E_c[k] = R_c[k] - mu~_c^k)
//   the root prior:                -q_0[k] (z~_0^k + m_0 - bias_0) / var
//   a leaf's observation:          q_i[k] C^T (x~ - C z~_i^k) / obs_var,   x~ = x - C m_i
//   the proposal (density at z):   q_i[k] z~_i^k / s_i^2
// so that, as rows, with a = var / obs_var,
//   var dz_i[k] = q_i[k] ( Vt_i[k] W_i^T + sum_c E_c[k] W_c - a z~_i^k C^T C
//                          + vec_i + z~_i^k (var / s_i^2 - 1) ),
//   vec_i = c_i (non-root) or bias_0 - m_0 (root), + a C^T x~ (leaf).
// The three products are one accumulator on the tensor core: each term is an A tile of 128
// sample rows (split fp16: Vt, E or z~) against a d x d B matrix (split W_i, W_c^T, or
// -a C^T C), as hi*hi + lo*hi + hi*lo with FP32 accumulation; the epilogue adds the element-
// wise terms, scales by q_i[k] grad_out_b / var and writes dz and deps = s_i dz.
#include <algorithm>

#include "tc_ptx.cuh"
#include "tmc_tc.cuh"

namespace tmc {
namespace tc {

namespace {
constexpr int kBoxDz = 16384;  // one [128 x 64] fp16 box, 128-byte swizzle
constexpr int kDzThreads = 128;
constexpr size_t kDzSmem = 1024 + 4 * kBoxDz;  // A hi, A lo, B hi, B lo of one 64-wide K slice

__device__ __forceinline__ uint64_t box_desc(const unsigned char* base) {
  return smem_desc_sw128(smem_u32(base), 16, 1024);
}
// K-step kk (16 fp16) inside a 64-column box: 32 bytes along the swizzled row.
__device__ __forceinline__ uint64_t box_step(uint64_t d0, int kk) { return d0 + (uint64_t)((kk * 32) >> 4); }

// -(prior_var / obs_var) C^T C, split, per observation matrix (C^T C from k_ctc; its padding
// beyond d is zero).
__global__ void __launch_bounds__(256) k_pack_cc(Dev D, TcDev T) {
  const float a = (float)(D.prior_var / D.obs_var);
  const long long o = (long long)blockIdx.x * kLdp * kLdp;
  for (int e = threadIdx.x; e < kLdp * kLdp; e += blockDim.x) {
    float hi, lo;
    split_half(-a * T.CtC[o + e], hi, lo);
    T.CCH[o + e] = __float2half_rn(hi);
    T.CCL[o + e] = __float2half_rn(lo);
  }
}

// One CTA per 128-sample tile of one node.  Thread 0 streams the terms' K slices through one
// shared-memory stage (TMA) and issues their MMAs into a DP-column accumulator; every thread
// then owns one sample row (TMEM lane) for the epilogue.  Several CTAs share an SM (64 KB of
// shared memory, DP TMEM columns each), so one CTA's loads overlap another's MMAs and stores.
// gmode (coupled proposals): the path gradient G = dz without the proposal's own term and
// without grad_out, from the FP32 samples, into D.gsrc (layout of the FP32 sample vectors).
template <int DP>
__global__ void __launch_bounds__(kDzThreads) k_dz_tc(
    Dev D, TcDev T, const Tile* __restrict__ tiles, int gmode, const __grid_constant__ CUtensorMap mVH,
    const __grid_constant__ CUtensorMap mVL, const __grid_constant__ CUtensorMap mEH,
    const __grid_constant__ CUtensorMap mEL, const __grid_constant__ CUtensorMap mZH,
    const __grid_constant__ CUtensorMap mZL, const __grid_constant__ CUtensorMap mWH,
    const __grid_constant__ CUtensorMap mWL, const __grid_constant__ CUtensorMap mWTH,
    const __grid_constant__ CUtensorMap mWTL, const __grid_constant__ CUtensorMap mCCH,
    const __grid_constant__ CUtensorMap mCCL) {
  constexpr int SLICES = DP / 64;
  extern __shared__ unsigned char smraw[];
  unsigned char* st = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full, mdone;
  __shared__ uint32_t tbase;
  __shared__ int s_ok;
  __shared__ float vec[kTcMaxD], diag[kTcMaxD], sd[kTcMaxD];
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = nd.d;
  if (warp == 1) tmem_alloc(&tbase, DP);
  if (threadIdx.x == 0) {
    mbar_init(&full, 1);
    mbar_init(&mdone, 1);
    fence_barrier_init();
    s_ok = 1;
  }
  {  // per-node vectors, thread j = latent dimension j
    const int j = threadIdx.x;
    if (j < d) {
      const float ls = D.q_logstd[nd.off_q + j];
      sd[j] = expf(ls);
      diag[j] = gmode ? -1.f : (float)D.prior_var * expf(-2.f * ls) - 1.f;
      float v = nd.parent >= 0 ? T.cvec[(long long)t.node * kLdp + j]
                               : D.bias[nd.off_bias + j] - D.q_mean[nd.off_q + j];
      if (nd.leaf_slot >= 0) {
        const float* C = D.C + nd.off_C;
        const float* xt = T.xs + nd.off_x;
        float a0 = 0.f, a1 = 0.f;
        int o = 0;
        for (; o + 1 < nd.obs; o += 2) {
          a0 = fmaf(__ldg(C + (long long)o * d + j), __ldg(xt + o), a0);
          a1 = fmaf(__ldg(C + (long long)(o + 1) * d + j), __ldg(xt + o + 1), a1);
        }
        if (o < nd.obs) a0 = fmaf(__ldg(C + (long long)o * d + j), __ldg(xt + o), a0);
        v += (float)(D.prior_var / D.obs_var) * (a0 + a1);
      }
      vec[j] = v;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t acc = tbase;

  if (threadIdx.x == 0) {
    const uint32_t id = idesc_f16(kRows, DP, false, false, false);
    int u = 0;
    bool ok = true;
    // one term: A rows arow of (ah, al) against B rows brow of (bh, bl), K slice by K slice
    auto term = [&](const CUtensorMap* ah, const CUtensorMap* al, int arow, const CUtensorMap* bh,
                    const CUtensorMap* bl, int brow) {
      for (int sl = 0; sl < SLICES && ok; ++sl, ++u) {
        if (u > 0 && !mbar_wait(&mdone, (uint32_t)((u - 1) & 1))) { ok = false; break; }  // stage free
        mbar_arrive_expect_tx(&full, 4 * kBoxDz);
        tma_load_2d(st, ah, &full, sl * 64, arow);
        tma_load_2d(st + kBoxDz, al, &full, sl * 64, arow);
        tma_load_2d(st + 2 * kBoxDz, bh, &full, sl * 64, brow);
        tma_load_2d(st + 3 * kBoxDz, bl, &full, sl * 64, brow);
        if (!mbar_wait(&full, (uint32_t)(u & 1))) { ok = false; break; }
        tc_fence_after();
        const uint64_t dah = box_desc(st), dal = box_desc(st + kBoxDz), dbh = box_desc(st + 2 * kBoxDz),
                       dbl = box_desc(st + 3 * kBoxDz);
        for (int kk = 0; kk < 4; ++kk) mma_ss(acc, box_step(dah, kk), box_step(dbh, kk), id, (u > 0 || kk > 0) ? 1u : 0u);
        for (int kk = 0; kk < 4; ++kk) mma_ss(acc, box_step(dal, kk), box_step(dbh, kk), id, 1u);
        for (int kk = 0; kk < 4; ++kk) mma_ss(acc, box_step(dah, kk), box_step(dbl, kk), id, 1u);
        mma_commit(&mdone);
      }
    };
    const int arow = (int)(nd.off_nk + t.row0);
    if (nd.parent >= 0) term(&mVH, &mVL, arow, &mWH, &mWL, (D.shared ? nd.i : t.node) * kLdp);
    for (int c = nd.child_begin; c < nd.child_end && ok; ++c) {
      const int cg = D.children[c];
      const NodeInfo cn = D.nodes[cg];
      term(&mEH, &mEL, (int)(cn.off_nk + t.row0), &mWTH, &mWTL, (D.shared ? cn.i : cg) * kLdp);
    }
    if (nd.leaf_slot >= 0) term(&mZH, &mZL, arow, &mCCH, &mCCL, (D.shared ? 0 : nd.b) * kLdp);
    if (ok && u > 0) ok = mbar_wait(&mdone, (uint32_t)((u - 1) & 1));
    if (!ok) {
      atomicOr(D.err, kErrTimeout);
      s_ok = 0;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  // epilogue: thread r owns sample t.row0 + r (TMEM lane r)
  const int k = t.row0 + (int)threadIdx.x;
  const bool valid = s_ok && k < nd.K;
  const float gb = (D.grad_out && !gmode) ? (float)D.grad_out[nd.b] : 1.f;
  const float w = valid ? D.q[nd.off_nk + k] * gb * D.inv_var : 0.f;
  const uint32_t lane_acc = acc + ((uint32_t)(32 * warp) << 16);
  const long long row = nd.off_e + (long long)k * d;  // eps / dz / deps: the caller's layout
  const bool vec4 = ((nd.off_e | (long long)d) & 3) == 0;
  if (gmode) {  // G from the FP32 samples (z~ is no longer s eps with couplings)
    const long long zrow = nd.off_nkd + (long long)k * d;
#pragma unroll 1
    for (int g = 0; g < DP / 32 && g * 32 < d; ++g) {  // warp-uniform
      uint32_t v[32];
      tmem_ld32(lane_acc + g * 32, v);
      tmem_wait_ld();
      if (!valid) continue;
#pragma unroll
      for (int x = 0; x < 32; ++x) {
        const int c = g * 32 + x;
        if (c < d) D.gsrc[zrow + c] = w * (__uint_as_float(v[x]) + vec[c] + D.zt[zrow + c] * diag[c]);
      }
    }
  } else
#pragma unroll 1
  for (int g = 0; g < DP / 32 && g * 32 < d; ++g) {  // warp-uniform
    uint32_t v[32];
    tmem_ld32(lane_acc + g * 32, v);
    tmem_wait_ld();
    if (!valid) continue;
    const int c0 = g * 32;
    if (vec4 && c0 + 32 <= d) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c0 + 4 * q;
        const float4 e = __ldg(reinterpret_cast<const float4*>(D.eps + row + c));
        const float ev[4] = {e.x, e.y, e.z, e.w};
        float o[4], oe[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const float zt = sd[c + x] * ev[x];
          o[x] = w * (__uint_as_float(v[4 * q + x]) + vec[c + x] + zt * diag[c + x]);
          oe[x] = o[x] * sd[c + x];
        }
        if (D.dz) *reinterpret_cast<float4*>(D.dz + row + c) = make_float4(o[0], o[1], o[2], o[3]);
        if (D.deps) *reinterpret_cast<float4*>(D.deps + row + c) = make_float4(oe[0], oe[1], oe[2], oe[3]);
      }
    } else {
#pragma unroll
      for (int x = 0; x < 32; ++x) {
        const int c = c0 + x;
        if (c < d) {
          const float zt = sd[c] * __ldg(D.eps + row + c);
          const float o = w * (__uint_as_float(v[x]) + vec[c] + zt * diag[c]);
          if (D.dz) D.dz[row + c] = o;
          if (D.deps) D.deps[row + c] = o * sd[c];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(acc, DP);
  }
}
}  // namespace

tmc_status prepare_dz(TcWork& w, const std::vector<NodeInfo>& nodes) {
  w.dz_tiles.clear();
  for (int c = 0; c < 2; ++c) {
    w.dz_b[c] = (int)w.dz_tiles.size();
    for (int g = 0; g < (int)nodes.size(); ++g)  // the instance's class: its terms' K-dims vary
      if ((w.inst_dp[nodes[g].b] > 64 ? 1 : 0) == c)
        for (int r = 0; r < nodes[g].K; r += kRows) w.dz_tiles.push_back(Tile{g, r});
    w.dz_e[c] = (int)w.dz_tiles.size();
  }
  if (!w.dz_tiles.empty()) {
    if (cudaMalloc(&w.d_dz_tiles, sizeof(Tile) * w.dz_tiles.size()) != cudaSuccess) return TMC_ERR_NOMEM;
    if (cudaMemcpy(w.d_dz_tiles, w.dz_tiles.data(), sizeof(Tile) * w.dz_tiles.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return TMC_ERR_CUDA;
  }
  // the split V / E rows are read whole by the MMAs: padding columns and spare rows must be
  // finite (zero); the kernels that write them fill only valid rows and columns < DP
  for (__half* a : {w.t.VH, w.t.VL, w.t.EH, w.t.EL})
    if (cudaMemset(a, 0, (size_t)w.rows * kLdp * sizeof(__half)) != cudaSuccess) return TMC_ERR_CUDA;
  cudaFuncSetAttribute(k_dz_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDzSmem);
  cudaFuncSetAttribute(k_dz_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDzSmem);
  return cudaGetLastError() == cudaSuccess ? TMC_OK : TMC_ERR_CUDA;
}

void release_dz(TcWork& w) {
  cudaFree(w.d_dz_tiles);
  w.d_dz_tiles = nullptr;
}

void launch_dz(TcWork& w, const Dev& D, cudaStream_t s) {
  k_pack_cc<<<w.num_c, 256, 0, s>>>(D, w.t);
  const int gmode = D.coupled ? 1 : 0;
  for (int c = 0; c < 2; ++c) {
    const int b = w.dz_b[c], n = w.dz_e[c] - b;
    if (!n) continue;
    if (c == 0)
      k_dz_tc<64><<<n, kDzThreads, kDzSmem, s>>>(D, w.t, w.d_dz_tiles + b, gmode, w.mVH, w.mVL, w.mEH, w.mEL, w.mZH,
                                                 w.mZL, w.mWH, w.mWL, w.mWTH, w.mWTL, w.mCCH, w.mCCL);
    else
      k_dz_tc<128><<<n, kDzThreads, kDzSmem, s>>>(D, w.t, w.d_dz_tiles + b, gmode, w.mVH, w.mVL, w.mEH, w.mEL,
                                                  w.mZH, w.mZL, w.mWH, w.mWL, w.mWTH, w.mWTL, w.mCCH, w.mCCL);
  }
}

// Coupled proposals: rows of the FP32 samples -> split fp16 operand rows, and z~ . c_i.
// One warp per sample row (lanes over the latent dimension); grid: 128-row tiles of every node.
__global__ void __launch_bounds__(256) k_pack_z(Dev D, TcDev T, const Tile* __restrict__ tiles) {
  const Tile t = tiles[blockIdx.x];
  const NodeInfo nd = D.nodes[t.node];
  const int d = nd.d, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool root = nd.parent < 0;
  for (int r = w; r < kRows; r += 8) {
    const int k = t.row0 + r;
    if (k >= nd.K) break;
    const float* z = D.zt + nd.off_nkd + (long long)k * d;
    __half* zh = T.ZH + (nd.off_nk + k) * kLdp;
    __half* zl = T.ZL + (nd.off_nk + k) * kLdp;
    float zc = 0.f;
    for (int j = lane; j < d; j += 32) {
      const float v = z[j];
      float hi, lo;
      split_half(v, hi, lo);
      zh[j] = __float2half_rn(hi);
      zl[j] = __float2half_rn(lo);
      if (!root) zc = fmaf(v, T.cvec[(long long)t.node * kLdp + j], zc);
    }
    for (int o = 16; o > 0; o >>= 1) zc += __shfl_xor_sync(0xffffffffu, zc, o);
    if (lane == 0) T.zc[nd.off_nk + k] = zc;
  }
}

void launch_pack_z(TcWork& w, const Dev& D, cudaStream_t s) {
  const int n = (int)w.dz_tiles.size();
  if (n) k_pack_z<<<n, 256, 0, s>>>(D, w.t, w.d_dz_tiles);
}

}  // namespace tc
}  // namespace tmc
