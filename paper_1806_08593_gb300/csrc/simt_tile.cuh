// simt_tile.cuh -- FP32 CUDA-core 64x64 tile products used by the FP32 path.
//
// A CTA of 256 threads owns a 64x64 output tile; thread (ty, tx) = (tid / 16, tid % 16)
// holds rows ty*4 .. ty*4+3 and columns tx*4 .. tx*4+3 in acc[4][4].  Operands are staged
// through shared memory in 16-deep slices laid out [l][m] (contraction index major), so the
// inner loop reads one float4 of each operand per step.
#pragma once
#include "tmc_internal.cuh"

namespace tmc {

constexpr int kSlice = 16;
constexpr int kLd = kTile + 4;  // padded shared-memory row (floats)

struct TileSmem {
  float a[kSlice * kLd];
  float b[kSlice * kLd];
};

// A 16 x 64 slice s[l][m] is fetched into registers (4 values per thread) and then stored to
// shared memory, so the next slice's loads can be in flight while the current one is used.
//   TRANS = true : element (m, l) of a row-major matrix src[m * ld + l] ("row m, depth l")
//   TRANS = false: element (l, m) of a row-major matrix src[l * ld + m]
// Out-of-range entries (m >= mlim or l0 + l >= llim) are zero.
constexpr int kSliceVals = kSlice * kTile / kThreads;
template <bool TRANS>
__device__ __forceinline__ void fetch_slice(float (&r)[kSliceVals], const float* __restrict__ src, long long ld,
                                            int mlim, int l0, int llim) {
#pragma unroll
  for (int x = 0; x < kSliceVals; ++x) {
    const int e = threadIdx.x + x * kThreads;
    int l, m;
    if (TRANS) { m = e >> 4; l = e & 15; }
    else       { l = e >> 6; m = e & 63; }
    const int gl = l0 + l;
    r[x] = (m < mlim && gl < llim) ? (TRANS ? src[(long long)m * ld + gl] : src[(long long)gl * ld + m]) : 0.f;
  }
}
template <bool TRANS>
__device__ __forceinline__ void store_slice(float* s, const float (&r)[kSliceVals]) {
#pragma unroll
  for (int x = 0; x < kSliceVals; ++x) {
    const int e = threadIdx.x + x * kThreads;
    int l, m;
    if (TRANS) { m = e >> 4; l = e & 15; }
    else       { l = e >> 6; m = e & 63; }
    s[l * kLd + m] = r[x];
  }
}
template <bool TRANS>
__device__ __forceinline__ void load_slice(float* s, const float* __restrict__ src, long long ld,
                                           int mlim, int l0, int llim) {
  float r[kSliceVals];
  fetch_slice<TRANS>(r, src, ld, mlim, l0, llim);
  store_slice<TRANS>(s, r);
}

__device__ __forceinline__ void slice_fma(float acc[4][4], const float* sa, const float* sb) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int l = 0; l < kSlice; ++l) {
    const float4 a = *reinterpret_cast<const float4*>(sa + l * kLd + ty * 4);
    const float4 b = *reinterpret_cast<const float4*>(sb + l * kLd + tx * 4);
    const float av[4] = {a.x, a.y, a.z, a.w};
    const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
}

// acc += opA * opB over contraction length L, where
//   opA(m, l) = A_TRANS ? A[m*lda + l] : A[l*lda + m]     (m < ma)
//   opB(n, l) = B_TRANS ? B[n*ldb + l] : B[l*ldb + n]     (n < nb)
// and the product is sum_l opA(m, l) * opB(n, l).
// The loads of slice l0 + 16 are issued before slice l0 is multiplied (register double
// buffering), so the global-memory latency of a slice overlaps the previous slice's FMAs.
template <bool A_TRANS, bool B_TRANS>
__device__ __forceinline__ void tile_gemm(float acc[4][4], const float* __restrict__ A,
                                          long long lda, int ma, const float* __restrict__ B,
                                          long long ldb, int nb, int L, TileSmem& sm) {
  float ra[kSliceVals], rb[kSliceVals];
  if (L > 0) {
    fetch_slice<A_TRANS>(ra, A, lda, ma, 0, L);
    fetch_slice<B_TRANS>(rb, B, ldb, nb, 0, L);
  }
  for (int l0 = 0; l0 < L; l0 += kSlice) {
    store_slice<A_TRANS>(sm.a, ra);
    store_slice<B_TRANS>(sm.b, rb);
    __syncthreads();
    if (l0 + kSlice < L) {
      fetch_slice<A_TRANS>(ra, A, lda, ma, l0 + kSlice, L);
      fetch_slice<B_TRANS>(rb, B, ldb, nb, l0 + kSlice, L);
    }
    slice_fma(acc, sm.a, sm.b);
    __syncthreads();
  }
}

// The same product in 64-deep slices (short contractions, L <= a few hundred): each slice is
// one round of loads (16 values per operand and thread), the next slice's loads are issued
// before the current one is multiplied, so a 128-deep product waits on global memory twice
// instead of eight times.
constexpr int kDeep = 64;
constexpr int kDeepVals = kDeep * kTile / kThreads;
struct TileSmemDeep {
  float a[kDeep * kLd];
  float b[kDeep * kLd];
};
template <bool TRANS>
__device__ __forceinline__ void fetch_deep(float (&r)[kDeepVals], const float* __restrict__ src, long long ld,
                                           int mlim, int l0, int llim) {
#pragma unroll
  for (int x = 0; x < kDeepVals; ++x) {
    const int e = threadIdx.x + x * kThreads;
    int l, m;
    if (TRANS) { m = e >> 6; l = e & 63; }
    else       { l = e >> 6; m = e & 63; }
    const int gl = l0 + l;
    r[x] = (m < mlim && gl < llim) ? (TRANS ? src[(long long)m * ld + gl] : src[(long long)gl * ld + m]) : 0.f;
  }
}
template <bool TRANS>
__device__ __forceinline__ void store_deep(float* s, const float (&r)[kDeepVals]) {
#pragma unroll
  for (int x = 0; x < kDeepVals; ++x) {
    const int e = threadIdx.x + x * kThreads;
    int l, m;
    if (TRANS) { m = e >> 6; l = e & 63; }
    else       { l = e >> 6; m = e & 63; }
    s[l * kLd + m] = r[x];
  }
}
template <bool A_TRANS, bool B_TRANS>
__device__ __forceinline__ void tile_gemm_deep(float acc[4][4], const float* __restrict__ A,
                                               long long lda, int ma, const float* __restrict__ B,
                                               long long ldb, int nb, int L, TileSmemDeep& sm) {
  float ra[kDeepVals], rb[kDeepVals];
  if (L > 0) {
    fetch_deep<A_TRANS>(ra, A, lda, ma, 0, L);
    fetch_deep<B_TRANS>(rb, B, ldb, nb, 0, L);
  }
  for (int l0 = 0; l0 < L; l0 += kDeep) {
    store_deep<A_TRANS>(sm.a, ra);
    store_deep<B_TRANS>(sm.b, rb);
    __syncthreads();
    if (l0 + kDeep < L) {
      fetch_deep<A_TRANS>(ra, A, lda, ma, l0 + kDeep, L);
      fetch_deep<B_TRANS>(rb, B, ldb, nb, l0 + kDeep, L);
    }
#pragma unroll
    for (int q = 0; q < kDeep / kSlice; ++q) slice_fma(acc, sm.a + q * kSlice * kLd, sm.b + q * kSlice * kLd);
    __syncthreads();
  }
}

// acc += opA * opB with opA resident in shared memory, sa[l * kLd + m] for every l < L rounded
// up to kDeep (rows past L zero), and opB streamed through sb ([kDeep * kLd]) in 64-deep
// slices (register prefetch of the next slice).  The first barrier also orders the caller's
// stores of sa.
template <bool B_TRANS>
__device__ __forceinline__ void tile_gemm_resA(float acc[4][4], const float* sa, const float* __restrict__ B,
                                               long long ldb, int nb, int L, float* sb) {
  float rb[kDeepVals];
  fetch_deep<B_TRANS>(rb, B, ldb, nb, 0, L);
  for (int l0 = 0; l0 < L; l0 += kDeep) {
    __syncthreads();  // the previous readers of sb are done
    store_deep<B_TRANS>(sb, rb);
    __syncthreads();
    if (l0 + kDeep < L) fetch_deep<B_TRANS>(rb, B, ldb, nb, l0 + kDeep, L);
    const int nq = (min(kDeep, L - l0) + kSlice - 1) / kSlice;
    for (int q = 0; q < nq; ++q) slice_fma(acc, sa + (l0 + q * kSlice) * kLd, sb + q * kSlice * kLd);
  }
}
// Stores opA (A_TRANS layout as in tile_gemm) of an ma x L tile into sa[l * kLd + m], in
// 64-deep slices (zeros past L up to the next multiple of kDeep).
template <bool A_TRANS>
__device__ __forceinline__ void load_resident(float* sa, const float* __restrict__ A, long long lda, int ma, int L) {
  for (int l0 = 0; l0 < L; l0 += kDeep) {
    float r[kDeepVals];
    fetch_deep<A_TRANS>(r, A, lda, ma, l0, L);
    store_deep<A_TRANS>(sa + l0 * kLd, r);
  }
}

__device__ __forceinline__ void zero_acc(float acc[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
}

// Sum over the 16 threads that share a row group (tx = 0..15 live in one half-warp).
__device__ __forceinline__ float row_group_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  return v;
}
__device__ __forceinline__ float row_group_max(float v) {
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 1));
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 2));
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 4));
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 8));
  return v;
}

__device__ __forceinline__ void flag_error(int* err, int bit) { atomicOr(err, bit); }

}  // namespace tmc
