// k_edge_tc.cu -- tcgen05 tensor-core path of the TMC hot path (sm_103a).
//
// Edge p -> i of the elimination (Section 2.2; factors of the Appendix), centred samples
// z~ = z - m_i and conditional means mu~^k = W_i z~_p^k + c_i (c_i = W_i m_p + bias_i - m_i):
//   log P(z_i^{k'} | z_p^k) = (mu~^k . z~^{k'} - |z~^{k'}|^2/2 - |mu~^k|^2/2) / var + const.
//
// Forward (k_edge_fwd_tc): an item is 128 parent samples k of one edge.  Prologue: mu~ tile =
//   Z~_p W_i^T on the tensor core (split operands), + c_i, |mu~|^2 in FP32, split again into
//   the A operand.  Main loop over 128-sample chunks of the child: S = mu~ z~^T (3 split MMAs
//   into TMEM, double-buffered), then the math warps run an online log-sum-exp over k' (base
//   2) giving lam_i[k] = log sum_k' exp(F[k,k'] + beta_i[k']).
//
// Adjoint (k_edge_bwd_tc): an item is 128 child samples k'.  With the weight of an entry
//   pi[k,k'] = q_p[k] exp(F[k,k'] + beta_i[k'] - lam_i[k])  (Section 2.2, d log P / d log f),
//   S^T[k',k] = (Z~_i W_i)[k'] . z~_p^k is formed from A' = Z~_i W_i (prologue) against chunks
//   of the parent's samples; the CTA accumulates
//     q_i[k']  = sum_k pi                    (row sums, in registers)
//     V[k']    = sum_k pi z~_p^k             (tensor core, P from TMEM)
//   and its epilogue adds the edge moment  G_i = sum_k' V[k'] z~_i^{k'T}  into a global
//   accumulator (TMA reductions).  The node moments M2_i = sum_k' q_i[k'] z~_i^{k'} z~_i^{k'T}
//   and zbar_i = sum q z~ come from k_moments_tc; every parameter and proposal gradient
//   follows from these d x d moments (k_asm_*), so no K x d gradient tensor is formed.
//
// Both edge kernels are persistent (one CTA per SM, 384 threads): warp 0 issues TMA, warp 1
// issues MMAs, warp 2 owns the TMEM allocation, warp 3 prepares per-item vectors (forward:
// messages of the next item; adjoint: the next item's records), warps 4..11 (two groups of 128
// threads, one sample row each) run the exponentials on alternate chunks.
// Every mbarrier wait is bounded; on a timeout the kernel records kErrTimeout and winds down.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "simt_tile.cuh"
#include "tc_ptx.cuh"
#include "tmc_tc.cuh"

namespace tmc {
namespace tc {

namespace {
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr int kThreadsTc = 384;  // 4 control warps + 8 math warps
constexpr int kMath = 256;       // math threads
constexpr int kJt = kTcMaxK / kMath;  // per-thread share of a K-long prologue vector
constexpr int kBox = 16384;  // bytes of one 128-row x 128-byte swizzled box

__device__ __forceinline__ int slot_of(const Dev& D, const NodeInfo& nd, int g) {
  return D.shared ? nd.i : g;
}

// Named barrier among the 256 math threads (warps 4..11).
__device__ __forceinline__ void sync_math() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// The same barrier, returning the OR of `v` over the 256 math threads (the same value in each).
__device__ __forceinline__ bool sync_math_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 256, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// Writes 8 consecutive values of row r (columns 8*chunk .. 8*chunk+7) of a [128 x DP]
// 128-byte-swizzled fp16 tile as hi / lo splits.
__device__ __forceinline__ void store_split8(unsigned char* th, unsigned char* tl, int r, int chunk,
                                             const float* v) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float h0, l0, h1, l1;
    split_half(v[2 * q], h0, l0);
    split_half(v[2 * q + 1], h1, l1);
    h[q] = pack_half2(h0, h1);
    l[q] = pack_half2(l0, l1);
  }
  const uint32_t off = (uint32_t)(chunk >> 3) * kBox + sw128_offset(r, chunk & 7);
  *reinterpret_cast<uint4*>(th + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(tl + off) = make_uint4(l[0], l[1], l[2], l[3]);
}
__device__ __forceinline__ void store_half8(unsigned char* t, int r, int chunk, const float* v) {
  uint32_t h[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) h[q] = pack_half2(v[2 * q], v[2 * q + 1]);
  const uint32_t off = (uint32_t)(chunk >> 3) * kBox + sw128_offset(r, chunk & 7);
  *reinterpret_cast<uint4*>(t + off) = make_uint4(h[0], h[1], h[2], h[3]);
}
__device__ __forceinline__ void load_half8(const unsigned char* t, int r, int chunk, float* v) {
  const uint32_t off = (uint32_t)(chunk >> 3) * kBox + sw128_offset(r, chunk & 7);
  const uint4 u = *reinterpret_cast<const uint4*>(t + off);
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __half2 hh = *reinterpret_cast<const __half2*>(&w[q]);
    float2 f = __half22float2(hh);
    v[2 * q] = f.x;
    v[2 * q + 1] = f.y;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%"
      "15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// 32 FP32 values -> split fp16 pairs packed two per 32-bit word (hi[16], lo[16]).
__device__ __forceinline__ void split_pack32(const float* f, uint32_t* hi, uint32_t* lo) {
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    float h0, l0, h1, l1;
    split_half(f[2 * q], h0, l0);
    split_half(f[2 * q + 1], h1, l1);
    hi[q] = pack_half2(h0, h1);
    lo[q] = pack_half2(l0, l1);
  }
}

// K-major descriptor of K-step kk (16 fp16) of a [rows x DP] swizzled tile.
__device__ __forceinline__ uint64_t kdesc(const unsigned char* base, int kk) {
  return smem_desc_sw128(smem_u32(base) + (kk >> 2) * kBox + (kk & 3) * 32, 16, 1024);
}
// MN-major descriptor of K-step kk (16 rows) of a [128 rows (K) x N] swizzled tile.
__device__ __forceinline__ uint64_t mndesc(const unsigned char* base, int kk) {
  return smem_desc_sw128(smem_u32(base) + kk * 2048, kBox, 1024);
}
// The same descriptors from the K-step-0 descriptor of the tile: the start-address field holds
// the byte address >> 4 and every tile lies below 256 KB, so adding the step offset cannot
// carry out of the field.  One 64-bit add per MMA instead of a descriptor build.
__device__ __forceinline__ uint64_t kstep(uint64_t d0, int kk) {
  return d0 + (uint64_t)((((kk >> 2) * kBox) + (kk & 3) * 32) >> 4);
}
__device__ __forceinline__ uint64_t mnstep(uint64_t d0, int kk) { return d0 + (uint64_t)((kk * 2048) >> 4); }

__device__ __forceinline__ void set_timeout(const Dev& D) { atomicOr(D.err, kErrTimeout); }

// Cross-CTA completion counters of the persistent edge kernels (per node, per launch).
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Bounded wait until *p >= need (`limit` cycles of polling, the plan's wait limit); false on
// timeout.
__device__ __forceinline__ bool wait_count(const int* p, int need, long long limit) {
  if (ld_acquire(p) >= need) return true;
  const long long t0 = clock64();
  while (ld_acquire(p) < need) {
    if (clock64() - t0 > limit) return false;
    __nanosleep(64);
  }
  return true;
}
__host__ __device__ constexpr int tiles_of(int K) { return (K + kRows - 1) / kRows; }
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Per-instance completion stamps of a persistent edge launch (direction dir).
__device__ __forceinline__ void stamp_item_start(TcDev& T, int dir, bool first) {
  if (first) atomicMin(T.t_start + dir, global_ns());
}
// An instance's end time is the latest end time of its tiles (a fire-and-forget max).
__device__ __forceinline__ void stamp_item_end(const Dev& D, TcDev& T, int dir, int b) {
  atomicMax(T.inst_t + (long long)dir * D.num_inst + b, global_ns());
}

// Stages of the adjoint kernel's ring of (hi, lo) parent sample chunks (192 KB either way).
__host__ __device__ constexpr int bwd_stages(int DP) { return DP == 64 ? 6 : 3; }
// Use index of chunk c's stage within an item (stages 0 and 1 start with the prologue).
__host__ __device__ constexpr int bwd_use(int c, int NS) { return (c + 2) / NS - ((c + 2) % NS < 2 ? 1 : 0); }
// Bytes of that ring: the stages, and at least the prologue operands (Z~ hi / lo, W^T hi / lo)
// and the epilogue's (Z~ hi, Z~ lo, V tile of two atoms).
__host__ __device__ constexpr int ring_bytes(int DP) {
  return bwd_stages(DP) * 2 * kRows * DP * 2 > 4 * kRows * DP * 2 ? bwd_stages(DP) * 2 * kRows * DP * 2
                                                                   : 4 * kRows * DP * 2;
}
static_assert(ring_bytes(64) >= 2 * kRows * 64 * 2 + 2 * kBox && ring_bytes(128) >= 2 * kRows * 128 * 2 + 2 * kBox,
              "adjoint epilogue fits in the ring");
// the G boxes (DP / 32 of them) fill stage 2, beyond the epilogue operands
static_assert(4 * kRows * 64 * 2 >= 2 * kRows * 64 * 2 + 2 * kBox && 4 * kRows * 64 * 2 + 2 * kBox <= ring_bytes(64) &&
                  4 * kRows * 128 * 2 >= 2 * kRows * 128 * 2 + 2 * kBox && 4 * kRows * 128 * 2 + 4 * kBox <= ring_bytes(128),
              "adjoint G boxes fit in stage 2");
}  // namespace

// =======================================================================================
// Samples for the tensor-core path: z~ = exp(logs) eps split into fp16 hi / lo rows of the
// packed operand array, |z~|^2, z~ . c_i and the per-sample node term (as in the FP32 path);
// FP32 samples are kept for the root (its moments are formed from them).
// =======================================================================================
// Persistent, warp-specialised sampler.  A tile is a node and up to sample_rows(d) of its
// rows (32 KB of eps whatever d is).  Warp 0 is the producer: for each tile of the CTA it
// reads the tile's node record, forms the per-dimension vectors (exp(logs), m - bias at the
// root, c_i), and bulk-copies the tile's eps rows into a ring stage; warps 1..8 consume the
// stages: split z~ = exp(logs) eps into fp16 hi / lo rows and form the row sums.  Tiles whose
// eps rows are not 16-byte aligned (d not a multiple of 4) are read from global memory by the
// consumers instead.
// Consumer lane mapping: 2^LG lanes per sample row (4 at d <= 16, else 8); lane `sub` owns the
// float4 groups at columns 4 sub + 4 L q (q < Q), so a row sum needs LG shuffle steps per
// 32 / L rows.
__host__ __device__ constexpr int sample_rows(int d) { return d > 64 ? 64 : d > 32 ? 128 : d > 16 ? 256 : 512; }
// Above this many nodes the per-node set-up kernels take several nodes per CTA.
constexpr int kManyNodes = 8192;
constexpr int kSampleStage = 64 * kTcMaxD * 4;  // bytes of one eps stage (= rows x d x 4 at most)
constexpr int kSampleNS = 3;                    // ring stages
constexpr int kSampleConsumers = 8;             // consumer warps (64 rows at d = 128: two full passes)

struct __align__(16) SampleStage {  // 16-byte aligned: the vectors are read as float4
  float std_[kTcMaxD], off[kTcMaxD], c[kTcMaxD];
  long long off_nk, off_nkd, off_e;
  int d, row0, rows, root, bulk;
};
constexpr size_t kSampleSmem = kSampleNS * (kSampleStage + sizeof(SampleStage)) + 64;
static_assert(sizeof(SampleStage) % 16 == 0 && kSampleStage % 64 == 0, "sampler stage alignment");

__device__ __forceinline__ bool sample_bulk_ok(const Dev& D, const NodeInfo& nd) {
  return (nd.d & 3) == 0 && (nd.off_e & 3) == 0 && ((uintptr_t)D.eps & 15) == 0;
}

// Rows of one stage; element (r, col) of the tile is src[r * d + col].
template <int LG, int Q>
__device__ __forceinline__ bool sample_stage(const Dev& D, const TcDev& T, const SampleStage& st, const float* src) {
  constexpr int L = 1 << LG, RPW = 32 >> LG, PASS = kSampleConsumers * RPW;
  const int w = (threadIdx.x >> 5) - 1, lane = threadIdx.x & 31;
  const int sub = lane & (L - 1), rl = w * RPW + (lane >> LG);
  const int d = st.d, rows = st.rows;
  const bool root = st.root != 0;
  const bool vec = (d & 3) == 0 && ((uintptr_t)src & 15) == 0;
  bool bad = false;
  for (int base = 0; base < rows; base += PASS) {
    const int r = base + rl;
    const long long k = st.row0 + r;
    const bool live = r < rows;
    float se = 0.f, sz = 0.f, sr = 0.f, szc = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int col = 4 * sub + 4 * L * q;
      float e[4] = {0.f, 0.f, 0.f, 0.f};
      if (live && col < d) {
        if (vec) {
          const float4 x = *reinterpret_cast<const float4*>(src + (long long)r * d + col);
          e[0] = x.x; e[1] = x.y; e[2] = x.z; e[3] = x.w;
        } else {
#pragma unroll
          for (int x = 0; x < 4; ++x)
            if (col + x < d) e[x] = src[(long long)r * d + col + x];
        }
      }
      const float4 sd = *reinterpret_cast<const float4*>(st.std_ + col);
      const float4 sc = *reinterpret_cast<const float4*>(st.c + col);
      const float z[4] = {sd.x * e[0], sd.y * e[1], sd.z * e[2], sd.w * e[3]};
      const float cv[4] = {sc.x, sc.y, sc.z, sc.w};
      float hi[4], lo[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        se = fmaf(e[x], e[x], se);
        sz = fmaf(z[x], z[x], sz);
        szc = fmaf(z[x], cv[x], szc);
        split_half(z[x], hi[x], lo[x]);
      }
      if (root) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const float rr = (col + x < d) ? z[x] + st.off[col + x] : 0.f;
          sr = fmaf(rr, rr, sr);
        }
      }
      if (live && col < d) {  // padding columns stay zero from plan creation
        if (root)
          for (int x = 0; x < 4; ++x)
            if (col + x < d) D.zt[st.off_nkd + k * d + col + x] = z[x];
        const long long prow = (st.off_nk + k) * kLdp + col;
        *reinterpret_cast<uint2*>(T.ZH + prow) = make_uint2(pack_half2(hi[0], hi[1]), pack_half2(hi[2], hi[3]));
        *reinterpret_cast<uint2*>(T.ZL + prow) = make_uint2(pack_half2(lo[0], lo[1]), pack_half2(lo[2], lo[3]));
      }
    }
#pragma unroll
    for (int o = L >> 1; o > 0; o >>= 1) {
      se += __shfl_xor_sync(0xffffffffu, se, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
      szc += __shfl_xor_sync(0xffffffffu, szc, o);
      if (root) sr += __shfl_xor_sync(0xffffffffu, sr, o);
    }
    if (live && sub == 0) {
      bad |= !isfinite(sz) || !isfinite(se);
      float uu = 0.5f * se;
      if (root) uu -= 0.5f * sr * D.inv_var;
      D.u[st.off_nk + k] = uu;
      D.zn[st.off_nk + k] = sz;
      T.zc[st.off_nk + k] = szc;
    }
  }
  return bad;
}

constexpr int kSampleThreads = 32 * (1 + kSampleConsumers);
__global__ void __launch_bounds__(kSampleThreads, 2) k_sample_tc(Dev D, TcDev T, const Tile* __restrict__ tiles, int ntiles) {
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 63) & ~(uintptr_t)63);
  float* buf = reinterpret_cast<float*>(sm);                                        // [NS][stage]
  SampleStage* st = reinterpret_cast<SampleStage*>(sm + kSampleNS * kSampleStage);  // [NS]
  __shared__ uint64_t full[kSampleNS], empty[kSampleNS];
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSampleNS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kSampleConsumers);
    }
    fence_barrier_init();
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    // ------------------------------------------------------------------ producer
    // tiles blockIdx.x, + gridDim.x, ...; the next tile's record, node and proposal vectors
    // are loaded right after the current tile's copy is issued, so their latency overlaps the
    // wait for the next free stage
    int n = 0;
    bool ok = true;
    Tile t{};
    NodeInfo nd{};
    float lsv[4], ofv[4], ccv[4];
    auto fetch = [&](int item) {
      t = tiles[item];
      nd = D.nodes[t.node];
      const bool rt = nd.parent < 0;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int j = lane + 32 * x;
        lsv[x] = j < nd.d ? __ldg(D.q_logstd + nd.off_q + j) : 0.f;
        ofv[x] = (rt && j < nd.d) ? __ldg(D.q_mean + nd.off_q + j) - __ldg(D.bias + nd.off_bias + j) : 0.f;
        ccv[x] = (rt || j >= nd.d) ? 0.f : __ldg(T.cvec + (long long)t.node * kLdp + j);
      }
    };
    if (blockIdx.x < ntiles) fetch(blockIdx.x);
    for (int item = blockIdx.x; item < ntiles; item += gridDim.x, ++n) {
      const int s = n % kSampleNS, fill = n / kSampleNS;
      if (fill >= 1 && !mbar_wait(&empty[s], (fill - 1) & 1)) { ok = false; break; }
      const bool root = nd.parent < 0;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int j = lane + 32 * x;
        st[s].std_[j] = j < nd.d ? expf(lsv[x]) : 0.f;
        st[s].off[j] = ofv[x];
        st[s].c[j] = ccv[x];
      }
      const bool bulk = sample_bulk_ok(D, nd);
      const int rows = min(sample_rows(nd.d), nd.K - t.row0);
      if (lane == 0) {
        st[s].off_nk = nd.off_nk;
        st[s].off_nkd = nd.off_nkd;
        st[s].off_e = nd.off_e;
        st[s].d = nd.d;
        st[s].row0 = t.row0;
        st[s].rows = rows;
        st[s].root = root ? 1 : 0;
        st[s].bulk = bulk ? 1 : 0;
      }
      __syncwarp();
      if (lane == 0) {
        if (bulk) {
          const uint32_t bytes = (uint32_t)rows * nd.d * 4;
          mbar_arrive_expect_tx(&full[s], bytes);
          bulk_load(buf + (size_t)s * (kSampleStage / 4), D.eps + nd.off_e + (long long)t.row0 * nd.d, bytes,
                    &full[s]);
        } else {
          mbar_arrive(&full[s]);  // release of the stage record; the rows are read from global
        }
      }
      __syncwarp();  // every lane has read this tile's record before it is replaced
      if (item + (int)gridDim.x < ntiles) fetch(item + gridDim.x);
    }
    if (!ok && lane == 0) set_timeout(D);
    // the last fills still in flight land before the CTA exits
    if (lane == 0)
      for (int m = (n > kSampleNS ? n - kSampleNS : 0); m < n; ++m)
        mbar_wait(&full[m % kSampleNS], (m / kSampleNS) & 1);
  } else {
    // ------------------------------------------------------------------ consumers
    int n = 0;
    bool bad = false, ok = true;
    for (int item = blockIdx.x; item < ntiles; item += gridDim.x, ++n) {
      const int s = n % kSampleNS;
      if (!mbar_wait(&full[s], (n / kSampleNS) & 1)) { ok = false; break; }
      const SampleStage& stg = st[s];
      const float* src = stg.bulk ? buf + (size_t)s * (kSampleStage / 4) : D.eps + stg.off_e + (long long)stg.row0 * stg.d;
      const int d = stg.d;
      if (d > 64) bad |= sample_stage<3, 4>(D, T, stg, src);
      else if (d > 32) bad |= sample_stage<3, 2>(D, T, stg, src);
      else if (d > 16) bad |= sample_stage<3, 1>(D, T, stg, src);
      else bad |= sample_stage<2, 1>(D, T, stg, src);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (!ok && lane == 0) set_timeout(D);
    if (bad) atomicOr(D.err, kErrNumeric);
  }
}

// Split W_i (and its transpose) into fp16 hi / lo blocks, one 128-row slot per W_i; only the
// d_pad x d_pad corner is read by the kernels (the rest of a slot stays zero from creation).
// Grid: (non-root node, 32-row tile, 32-column tile) of that corner; the transpose goes
// through shared memory so both writes are coalesced.
__global__ void k_pack_w(Dev D, TcDev T, const int* __restrict__ nonroot) {
  __shared__ float tile[32][33];
  const int g = nonroot[blockIdx.x];
  const NodeInfo nd = D.nodes[g];
  if (D.shared && nd.b != 0) return;  // shared parameters: pack once (instance 0's nodes)
  const int d = nd.d, dq = nd.dp;  // W_i is d x dq (dq: the parent's dimension)
  const int r0 = blockIdx.y * 32, c0 = blockIdx.z * 32;
  if (r0 >= d || c0 >= dq) return;  // tiles beyond d x dq stay zero from plan creation
  const int slot = slot_of(D, nd, g);
  const long long o = (long long)slot * kLdp * kLdp;
  const float* Wi = D.W + nd.off_W;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  float v[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {  // every load before the first store
    const int r = r0 + ty + 8 * x, c = c0 + tx;
    v[x] = (r < d && c < dq) ? __ldg(Wi + (long long)r * dq + c) : 0.f;
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int i = ty + 8 * x, r = r0 + i, c = c0 + tx;
    tile[i][tx] = v[x];
    float hi, lo;
    split_half(v[x], hi, lo);
    T.WH[o + (long long)r * kLdp + c] = __float2half_rn(hi);
    T.WL[o + (long long)r * kLdp + c] = __float2half_rn(lo);
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {  // WT[c][r] = W[r][c]
    const float v = tile[tx][i];
    float hi, lo;
    split_half(v, hi, lo);
    const int c = c0 + i, r = r0 + tx;
    T.WTH[o + (long long)c * kLdp + r] = __float2half_rn(hi);
    T.WTL[o + (long long)c * kLdp + r] = __float2half_rn(lo);
  }
}

// c_i = W_i m_p + bias_i - m_i per non-root node (zero in the padding up to d_pad).  One
// thread per row of W_i, each streaming its own row (independent loads).
// NPB nodes per CTA (128 / NPB threads each): several nodes per CTA when there are many small
// latents (one CTA per latent spends its time on launch and latency).
template <int NPB>
__global__ void __launch_bounds__(128) k_pack_c(Dev D, TcDev T, const int* __restrict__ nonroot, int n) {
  constexpr int TPN = 128 / NPB;
  __shared__ __align__(16) float mp_all[NPB][kTcMaxD];
  const int slot = threadIdx.x / TPN, tid = threadIdx.x % TPN;
  const int idx = blockIdx.x * NPB + slot;
  const bool live = idx < n;
  const int g = live ? nonroot[idx] : 0;
  const NodeInfo nd = D.nodes[live ? g : nonroot[0]];
  const NodeInfo pn = D.nodes[nd.parent];
  const int d = nd.d, dq = nd.dp, dp = kTcMaxD;  // W_i is d x dq; c_i padded to 128 with zeros
  float* mp = mp_all[slot];
  for (int j = tid; j < kTcMaxD; j += TPN) mp[j] = j < dq ? D.q_mean[pn.off_q + j] : 0.f;
  __syncthreads();
  if (!live) return;
  const bool vec = (dq & 3) == 0 && (nd.off_W & 3) == 0;
  for (int r = tid; r < dp; r += TPN) {
    float s = 0.f;
    if (r < d) {
      const float* wr = D.W + nd.off_W + (long long)r * dq;
      float s0 = 0.f, s1 = 0.f;
      if (vec) {
        for (int c = 0; c < dq; c += 8) {
          const float4 a = *reinterpret_cast<const float4*>(wr + c);
          s0 = fmaf(a.x, mp[c], s0); s0 = fmaf(a.y, mp[c + 1], s0);
          s0 = fmaf(a.z, mp[c + 2], s0); s0 = fmaf(a.w, mp[c + 3], s0);
          if (c + 4 < dq) {
            const float4 b = *reinterpret_cast<const float4*>(wr + c + 4);
            s1 = fmaf(b.x, mp[c + 4], s1); s1 = fmaf(b.y, mp[c + 5], s1);
            s1 = fmaf(b.z, mp[c + 6], s1); s1 = fmaf(b.w, mp[c + 7], s1);
          }
        }
      } else {
        for (int c = 0; c < dq; ++c) s0 = fmaf(wr[c], mp[c], s0);
      }
      s = (s0 + s1) + D.bias[nd.off_bias + r] - D.q_mean[nd.off_q + r];
    }
    T.cvec[(long long)g * kLdp + r] = s;
  }
}

// Centred observations of the leaves, x~_l = x_l - C m_l, kept for the observation kernel
// and the gradient assembly.  Grid: one CTA per leaf; thread per observation row, each thread
// streaming its own row of C (independent loads, no per-row reduction chain).
template <int NPB>
__global__ void __launch_bounds__(128) k_obs_center(Dev D, TcDev T, const int* __restrict__ leaves, int n) {
  constexpr int TPN = 128 / NPB;
  __shared__ __align__(16) float m_all[NPB][kTcMaxD];
  const int slot = threadIdx.x / TPN, tid = threadIdx.x % TPN;
  const int idx = blockIdx.x * NPB + slot;
  const bool live = idx < n;
  const NodeInfo nd = D.nodes[leaves[live ? idx : 0]];
  const int d = nd.d;
  float* m = m_all[slot];
  for (int j = tid; j < kTcMaxD; j += TPN) m[j] = j < d ? D.q_mean[nd.off_q + j] : 0.f;
  __syncthreads();
  if (!live) return;
  const bool vec = (d & 3) == 0 && (nd.off_C & 3) == 0;
  for (int o = tid; o < nd.obs; o += TPN) {
    const float* c = D.C + nd.off_C + (long long)o * d;
    float s0 = 0.f, s1 = 0.f;
    if (vec) {
      for (int i = 0; i < d; i += 8) {
        const float4 a = *reinterpret_cast<const float4*>(c + i);
        s0 = fmaf(a.x, m[i], s0); s0 = fmaf(a.y, m[i + 1], s0);
        s0 = fmaf(a.z, m[i + 2], s0); s0 = fmaf(a.w, m[i + 3], s0);
        if (i + 4 < d) {
          const float4 b = *reinterpret_cast<const float4*>(c + i + 4);
          s1 = fmaf(b.x, m[i + 4], s1); s1 = fmaf(b.y, m[i + 5], s1);
          s1 = fmaf(b.z, m[i + 6], s1); s1 = fmaf(b.w, m[i + 7], s1);
        }
      }
    } else {
      for (int i = 0; i < d; ++i) s0 = fmaf(c[i], m[i], s0);
    }
    T.xs[nd.off_x + o] = D.x[nd.off_x + o] - (s0 + s1);
  }
}

// Split observation matrices: CH / CL row c_row[b] + o = C_b[o][0..d) as fp16 hi / lo, zero
// beyond d.  Grid: (distinct matrix, 8 rows); thread = (row parity, column), 4 rows each.
__global__ void __launch_bounds__(256) k_pack_cobs(Dev D, TcDev T) {
  const InstInfo in = D.insts[blockIdx.x];
  const int j = threadIdx.x & 127;
  const long long r0 = T.c_row[blockIdx.x];
  float v[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {  // rows 8 y + 2 x + (thread >> 7); every load before the first store
    const int o = blockIdx.y * 8 + 2 * x + (threadIdx.x >> 7);
    v[x] = (o < in.obs && j < in.d) ? __ldg(D.C + in.off_C + (long long)o * in.d + j) : 0.f;
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int o = blockIdx.y * 8 + 2 * x + (threadIdx.x >> 7);
    if (o >= in.obs) break;
    float hi, lo;
    split_half(v[x], hi, lo);
    T.CH[(r0 + o) * kLdp + j] = __float2half_rn(hi);
    T.CL[(r0 + o) * kLdp + j] = __float2half_rn(lo);
  }
}

// =======================================================================================
// Observation term of the leaves on the tensor cores:
//   u_l[k] -= |x~ - C z~^k|^2 / (2 obs_var),   x~ = x - C m_l   (z = m_l + z~),
// with C z~^k formed as split-fp16 products (hi*hi + lo*hi + hi*lo, FP32 accumulation) in
// 128-observation chunks.  Grid: one CTA per 128-sample tile of a leaf; 128 threads: thread 0
// issues the TMA loads and the MMAs, all four warps form x~ and reduce the accumulator rows
// (thread t owns sample row t = TMEM lane t).
// =======================================================================================
template <int DP>
__global__ void __launch_bounds__(128) k_obs_tc(Dev D, TcDev T, const Tile* __restrict__ tiles, int ntiles,
                                                 const __grid_constant__ CUtensorMap mZH,
                                                 const __grid_constant__ CUtensorMap mZL,
                                                 const __grid_constant__ CUtensorMap mCH,
                                                 const __grid_constant__ CUtensorMap mCL) {
  constexpr int TB = kRows * DP * 2;
  constexpr int NB = DP / 64;
  constexpr int KS = DP / 16;
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  unsigned char *ah = sm, *al = sm + TB, *bh = sm + 2 * TB, *bl = sm + 3 * TB;
  float* xs = reinterpret_cast<float*>(sm + 4 * TB);  // centred observation (obs floats)
  __shared__ uint64_t bar_ld, bar_mma;
  __shared__ uint32_t tbase;
  __shared__ int s_ok;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) tmem_alloc(&tbase, 128);
  if (threadIdx.x == 0) {
    mbar_init(&bar_ld, 1);
    mbar_init(&bar_mma, 1);
    fence_barrier_init();
    s_ok = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = tbase;
  const uint32_t idesc = idesc_f16(kRows, kRows, false, false, false);
  uint32_t nld = 0, nmma = 0;  // completed phases of the two barriers (same in every thread)
  bool run = true;
  // persistent loop over the leaf tiles
  for (int item = blockIdx.x; run && item < ntiles; item += gridDim.x) {
    const Tile t = tiles[item];
    const NodeInfo nd = D.nodes[t.node];
    const int obs = nd.obs;
    const int nchunk = (obs + kRows - 1) / kRows;
    const int crow = T.c_row[D.shared ? 0 : nd.b];
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(&bar_ld, 4 * TB);
      const int arow = (int)(nd.off_nk + t.row0);
      for (int b = 0; b < NB; ++b) {
        tma_load_2d(ah + b * kBox, &mZH, &bar_ld, b * 64, arow);
        tma_load_2d(al + b * kBox, &mZL, &bar_ld, b * 64, arow);
        tma_load_2d(bh + b * kBox, &mCH, &bar_ld, b * 64, crow);
        tma_load_2d(bl + b * kBox, &mCL, &bar_ld, b * 64, crow);
      }
    }
    for (int o = threadIdx.x; o < obs; o += blockDim.x) xs[o] = __ldg(T.xs + nd.off_x + o);  // x~ = x - C m
    __syncthreads();
    float rs = 0.f;
    for (int c = 0; c < nchunk; ++c) {
      if (threadIdx.x == 0) {
        if (c > 0) {
          mbar_arrive_expect_tx(&bar_ld, 2 * TB);
          for (int b = 0; b < NB; ++b) {
            tma_load_2d(bh + b * kBox, &mCH, &bar_ld, b * 64, crow + c * kRows);
            tma_load_2d(bl + b * kBox, &mCL, &bar_ld, b * 64, crow + c * kRows);
          }
        }
        if (mbar_wait(&bar_ld, nld & 1)) {
          tc_fence_after();
          for (int kk = 0; kk < KS; ++kk) mma_ss(tb, kdesc(ah, kk), kdesc(bh, kk), idesc, kk > 0);
          for (int kk = 0; kk < KS; ++kk) mma_ss(tb, kdesc(al, kk), kdesc(bh, kk), idesc, 1);
          for (int kk = 0; kk < KS; ++kk) mma_ss(tb, kdesc(ah, kk), kdesc(bl, kk), idesc, 1);
          mma_commit(&bar_mma);
        } else {
          set_timeout(D);
          mbar_wait(&bar_ld, nld & 1);  // once more (bounded) for the copies still in flight
          s_ok = 0;
        }
      }
      ++nld;
      __syncthreads();
      if (!s_ok) { run = false; break; }
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar_mma, nmma & 1));
      tc_fence_after();
      if (ok) {
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
          const int o0 = c * kRows + q * 32;
          if (o0 >= obs) break;
          uint32_t v[32];
          tmem_ld32(tb + ((uint32_t)(warp * 32) << 16) + q * 32, v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float r = (o0 + j < obs) ? xs[o0 + j] - __uint_as_float(v[j]) : 0.f;
            rs = fmaf(r, r, rs);
          }
        }
      } else {
        if (lane == 0) set_timeout(D);
        mbar_wait(&bar_mma, nmma & 1);  // once more (bounded) before the accumulator is reused
      }
      ++nmma;
      tc_fence_before();
      if (!__syncthreads_and(ok)) { run = false; break; }  // block-uniform
    }
    const int k = t.row0 + threadIdx.x;
    if (run && k < nd.K) D.u[nd.off_nk + k] -= 0.5f * rs * D.inv_obs_var;
    __syncthreads();  // xs and the operand tiles are free for the next item
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tb, 128);
  }
}

// =======================================================================================
// Forward edge kernel, pipelined across the CTA's items.
// Roles: warp 0 lane 0 issues TMA; warp 1 lane 0 issues MMAs; warp 2 owns the TMEM
// allocation; warp 3 prepares the next item's message vector (dependency
// wait, beta_i, its maximum); warps 4..11 run the exponentials in two groups: group h =
// (w-4)/4 takes the chunks in S buffer h (warp w serves TMEM lanes 32*(w%4)..) and half h of
// the latent dimension in the prologue split.
// The A operand is double-buffered in TMEM: item j's mu~ accumulates (FP32) into region
// j & 1 and is split there in place (each 32-column group becomes 16 columns of hi pairs and
// 16 of lo pairs), so item j + 1's split never waits for item j's last S MMA, and it reads
// c_i from global memory, so it never waits for item j + 1's message vector either.
// The barriers are initialised once; every role walks the same item sequence and derives the
// phase of each barrier from running counters:
//   ring uses   : per item [Z~_p tile, W_i, chunk 0 .. chunk nch-1], stage = use % NS
//   S buffers   : running chunk count, buffer = chunk & 1
//   per item    : mu_full (mu~ in TMEM region j & 1), a_full (A operand written), phase = j & 1
//   beta buffers: NCB (1 or 2) SMEM copies of cb / c_i, written by warp 3, freed by the math warps
// so the TMA and MMA warps run into item j + 1 (its operands, mu~ = Z~_p W^T into TMEM) while
// the math warps still finish item j, and warp 3 has item j + 1's message vector ready.
// =======================================================================================
template <int DP>
struct FwdCfg {
  static constexpr int TB = kRows * DP * 2;  // bytes of one [128 x DP] fp16 tile
  static constexpr int NB = DP / 64;         // 64-column boxes per tile
  static constexpr int KS = DP / 16;         // K-steps over the latent dimension
  static constexpr int GH = DP / 64;         // 32-column groups of the latent dimension per half
  static constexpr int NS = DP == 64 ? 6 : 3;  // ring stages of (hi, lo) tiles
};

// Chunk of an item before which the next item's prologue operands and mu~ MMAs are placed
// in the ring / MMA order: two chunks before the end, so they overlap this item's tail.
__host__ __device__ constexpr int pro_slot(int nch, int lead) { return nch >= lead ? nch - lead : 0; }
// Items of a persistent edge launch are claimed from a counter in list order, which is
// dependency order: every item an item depends on was claimed earlier by a running CTA, so the
// launch progresses however many of its CTAs are resident.  -1 once the list is exhausted.
__device__ __forceinline__ int claim_item(int* counter, int ntiles) {
  const int v = atomicAdd(counter, 1);
  return v < ntiles ? v : -1;
}
constexpr int kSeq = 4;                     // forward item-sequence ring
constexpr int kSeqReaders = 2 + kMath / 32; // MMA issuer, warp 3, one arrival per math warp
// TMEM column (within an A region) of the hi pairs of K-step kk after the in-place split
__device__ __forceinline__ uint32_t a_col(int kk) { return (uint32_t)(32 * (kk >> 1) + 8 * (kk & 1)); }

// Bounded wait that also gives up as soon as another role of the CTA has given up.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_test_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort || clock64() - t0 > (1ll << 31)) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

template <int DP>
__global__ void __launch_bounds__(kThreadsTc, 1)
    k_edge_fwd_tc(Dev D, TcDev T, const Tile* __restrict__ tiles, int ntiles, int* __restrict__ done,
                  int* __restrict__ claim, int lead, int ncb, int cbk,
                  const __grid_constant__ CUtensorMap mZH, const __grid_constant__ CUtensorMap mZL,
                  const __grid_constant__ CUtensorMap mWH, const __grid_constant__ CUtensorMap mWL) {
  using C = FwdCfg<DP>;
  constexpr int TB = C::TB, NB = C::NB, KS = C::KS, GH = C::GH, NS = C::NS;
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  unsigned char* ring = sm;  // NS stages x (hi, lo)
  float* cbuf = reinterpret_cast<float*>(ring + NS * 2 * TB);  // [ncb][cbk], cbk = max K rounded up to 128
  __shared__ uint64_t full[NS], empty[NS], sfull[2], sfree[2], mu_full, a_full, cb_full[2], cb_empty[2],
      bar_done;
  __shared__ uint32_t tbase;
  __shared__ int s_abort;
  __shared__ __align__(16) float cvn[2][kTcMaxD];  // c_i of item j in cvn[j & 1], for its split
  // The CTA's item sequence: the producer claims items from the launch's counter in list
  // (dependency) order, one ahead of the item it loads, into a ring of kSeq slots; the MMA
  // issuer, warp 3 and the math warps read it (an entry < 0 ends the sequence).
  __shared__ int s_seq[kSeq];
  __shared__ uint64_t q_full[kSeq], q_empty[kSeq];
  __shared__ float nrm_h[2][2][kRows], m_h[2][kRows], s_h[2][kRows];
  volatile int* abort = &s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float iv = D.inv_var;
  if (warp == 2) tmem_alloc(&tbase, 512);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sfull[i], 1);
      mbar_init(&sfree[i], kMath / 2);  // the warp group of buffer i
      mbar_init(&cb_full[i], 1);
      mbar_init(&cb_empty[i], kMath);
    }
    mbar_init(&mu_full, 1);
    mbar_init(&a_full, kMath);
    mbar_init(&bar_done, 1);
    for (int i = 0; i < kSeq; ++i) {
      mbar_init(&q_full[i], 1);
      mbar_init(&q_empty[i], kSeqReaders);
    }
    fence_barrier_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = tbase;
  // TMEM: S double buffer [0,256); A regions [256,384) and [384,512): item j's mu~ (FP32), then
  // its A operand (split in place) in region j & 1
  const uint32_t tS[2] = {tb, tb + 128}, tR[2] = {tb + 256, tb + 384};
  // entry j of the item sequence (every reader waits; one arrival per reading unit on release)
  auto seq_get = [&](int j, int& v) -> bool {
    if (!mbar_wait_ab(&q_full[j % kSeq], (uint32_t)((j / kSeq) & 1), abort)) return false;
    v = s_seq[j % kSeq];
    return true;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------------- TMA producer
      prefetch_tmap(&mZH);
      prefetch_tmap(&mZL);
      prefetch_tmap(&mWH);
      prefetch_tmap(&mWL);
      long long gu = 0;  // ring uses issued
      bool ok = true;
      // one ring use: wait for the stage, then load a (hi, lo) pair of [128 x DP] tiles
      auto load_use = [&](const CUtensorMap* mh, const CUtensorMap* ml, int row) -> bool {
        const int s = (int)(gu % NS);
        const long long fill = gu / NS;
        if (fill >= 1 && !mbar_wait_ab(&empty[s], (uint32_t)((fill - 1) & 1), abort)) return false;
        unsigned char* st = ring + s * 2 * TB;
        mbar_arrive_expect_tx(&full[s], 2 * TB);
        for (int b = 0; b < NB; ++b) {
          tma_load_2d(st + b * kBox, mh, &full[s], b * 64, row);
          tma_load_2d(st + TB + b * kBox, ml, &full[s], b * 64, row);
        }
        ++gu;
        return true;
      };
      // an item's prologue operands: its Z~_p tile and W_i
      auto load_pro = [&](int item) -> bool {
        const Tile t = tiles[item];
        const NodeInfo nd = D.nodes[t.node];
        return load_use(&mZH, &mZL, (int)(D.nodes[nd.parent].off_nk + t.row0)) &&
               load_use(&mWH, &mWL, slot_of(D, nd, t.node) * kLdp);
      };
      // publish entry j of the sequence: a claimed item, or -1 once the list is exhausted
      auto publish = [&](int j) -> int {
        if (j >= kSeq && !mbar_wait_ab(&q_empty[j % kSeq], (uint32_t)(((j / kSeq) - 1) & 1), abort)) return -2;
        const int v = claim_item(claim, ntiles);
        s_seq[j % kSeq] = v;
        mbar_arrive(&q_full[j % kSeq]);  // (release)
        return v;
      };
      int cur = publish(0), nxt = cur >= 0 ? publish(1) : -1;
      if (cur == -2 || nxt == -2) ok = false;
      if (ok && cur >= 0) ok = load_pro(cur);
      for (int j = 0; ok && cur >= 0; ++j) {
        const int item = cur;
        const Tile t = tiles[item];
        const NodeInfo nd = D.nodes[t.node];
        const int nch = tiles_of(nd.K);
        stamp_item_start(T, 0, j == 0);
        // the 8 row tiles of an edge walk the child's chunks in the same order; each pulls
        // "its" chunk (index = its row tile) into L2 up front
        for (int b = 0; b < NB; ++b) {
          tma_prefetch_l2_2d(&mZH, b * 64, (int)(nd.off_nk + t.row0));
          tma_prefetch_l2_2d(&mZL, b * 64, (int)(nd.off_nk + t.row0));
        }
        for (int c = 0; ok && c < nch; ++c) {
          if (c == pro_slot(nch, lead) && nxt >= 0) ok = load_pro(nxt);
          ok = ok && load_use(&mZH, &mZL, (int)(nd.off_nk + c * kRows));
        }
        // the next item becomes current; claim the one after it
        cur = nxt;
        if (ok && cur >= 0) {
          nxt = publish(j + 2);
          if (nxt == -2) ok = false;
        }
      }
      if (!ok) set_timeout(D);
      // the last fills still in flight land before the CTA exits
      for (long long g = (gu > NS ? gu - NS : 0); g < gu; ++g)
        mbar_wait(&full[(int)(g % NS)], (uint32_t)((g / NS) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------------------------- MMA issuer
      const uint32_t id_mu = idesc_f16(kRows, DP, false, false, false);
      const uint32_t id_s = idesc_f16(kRows, kRows, false, false, false);
      long long gu = 0, gc = 0;
      int it = 0;
      bool ok = true;
      // mu~ = Z~_p W_i^T (split products) of item `itm` from the next two ring uses into
      // region itm & 1 (its previous A, read by MMAs issued before these)
      auto mu_mmas = [&](int itm) -> bool {
        const uint32_t tMU = tR[itm & 1];
        const int sz = (int)(gu % NS), sw = (int)((gu + 1) % NS);
        if (!mbar_wait_ab(&full[sz], (uint32_t)((gu / NS) & 1), abort) ||
            !mbar_wait_ab(&full[sw], (uint32_t)(((gu + 1) / NS) & 1), abort))
          return false;
        tc_fence_after();
        unsigned char *zh = ring + sz * 2 * TB, *wh = ring + sw * 2 * TB;
        const uint64_t dzh = kdesc(zh, 0), dzl = kdesc(zh + TB, 0), dwh = kdesc(wh, 0), dwl = kdesc(wh + TB, 0);
        for (int kk = 0; kk < KS; ++kk) mma_ss(tMU, kstep(dzh, kk), kstep(dwh, kk), id_mu, kk > 0);
        for (int kk = 0; kk < KS; ++kk) mma_ss(tMU, kstep(dzl, kk), kstep(dwh, kk), id_mu, 1);
        for (int kk = 0; kk < KS; ++kk) mma_ss(tMU, kstep(dzh, kk), kstep(dwl, kk), id_mu, 1);
        mma_commit(&mu_full);
        mma_commit(&empty[sz]);
        mma_commit(&empty[sw]);
        gu += 2;
        return true;
      };
      int cur = -1, nxt = -1;
      ok = seq_get(0, cur);
      if (ok && cur >= 0) ok = mu_mmas(0);
      for (; ok && cur >= 0; ++it) {
        const int item = cur;
        if (!seq_get(it + 1, nxt)) { ok = false; break; }
        mbar_arrive(&q_empty[it % kSeq]);
        const NodeInfo nd = D.nodes[tiles[item].node];
        const int nch = tiles_of(nd.K);
        const bool has_next = nxt >= 0;
        // A of this item written by the math warps (they have also read MU, so the next
        // item's mu~ may go there)
        if (!mbar_wait_ab(&a_full, (uint32_t)(it & 1), abort)) { ok = false; break; }
        for (int c = 0; c < nch; ++c, ++gu, ++gc) {
          // the next item's mu~ between this item's chunks, where the tensor pipe has room
          if (c == pro_slot(nch, lead) && has_next && !mu_mmas(it + 1)) { ok = false; break; }
          const int s = (int)(gu % NS), b = (int)(gc & 1);
          if (!mbar_wait_ab(&full[s], (uint32_t)((gu / NS) & 1), abort)) { ok = false; break; }
          if (gc >= 2 && !mbar_wait_ab(&sfree[b], (uint32_t)(((gc >> 1) + 1) & 1), abort)) { ok = false; break; }
          tc_fence_after();
          const uint64_t dbh = kdesc(ring + s * 2 * TB, 0), dbl = kdesc(ring + s * 2 * TB + TB, 0);
          // S = (A_hi + A_lo)(B_hi + B_lo)^T without lo*lo; A from tensor memory (2 fp16 / column):
          // K-step kk's 16 elements are hi pairs at columns 32 (kk / 2) + 8 (kk % 2), lo 16 further
          const uint32_t tA = tR[it & 1];
          for (int kk = 0; kk < KS; ++kk) mma_ts(tS[b], tA + a_col(kk), kstep(dbh, kk), id_s, kk > 0);
          for (int kk = 0; kk < KS; ++kk) mma_ts(tS[b], tA + a_col(kk) + 16, kstep(dbh, kk), id_s, 1);
          for (int kk = 0; kk < KS; ++kk) mma_ts(tS[b], tA + a_col(kk), kstep(dbl, kk), id_s, 1);
          mma_commit(&sfull[b]);
          mma_commit(&empty[s]);
        }
        cur = nxt;
      }
      if (!ok) set_timeout(D);
      mma_commit(&bar_done);
      mbar_wait(&bar_done, 0);
    }
  } else if (warp == 3) {
    // ------------------------------------------------------------------ message vectors
    // cb[k'] = (beta_i[k'] - max beta_i - |z~_i^{k'}|^2 / (2 var)) log2(e), -inf past K; c_i.
    int it = 0;
    bool ok = true;
    for (;; ++it) {
      int item = -1;
      if (lane == 0) ok = seq_get(it, item);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      item = __shfl_sync(0xffffffffu, item, 0);
      if (lane == 0) mbar_arrive(&q_empty[it % kSeq]);
      if (!ok || item < 0) break;
      const Tile t = tiles[item];
      const NodeInfo nd = D.nodes[t.node];
      const int K = nd.K, nch = tiles_of(K);
      const int ib = it % ncb;
      if (it >= ncb && !mbar_wait_ab(&cb_empty[ib], (uint32_t)(((it / ncb) - 1) & 1), abort)) { ok = false; break; }
      // every child of the edge's child node must have sent its message (all its tiles)
      bool dep_ok = true;
      if (lane == 0)
        for (int c = nd.child_begin; c < nd.child_end; ++c) {
          const int cg = D.children[c];
          dep_ok = wait_count(done + cg, tiles_of(D.nodes[cg].Kp), D.wait_limit) && dep_ok;
        }
      dep_ok = __shfl_sync(0xffffffffu, dep_ok, 0);
      __syncwarp();  // lane 0's acquire of the counters orders the other lanes' reads below
      if (!dep_ok) { *abort = 1; ok = false; break; }
      float* cb = cbuf + (size_t)ib * cbk;
      // pass 1: beta = u + sum of the children's messages (into cb), and its maximum; 32
      // values per lane per batch, every load of a batch issued before the first use
      constexpr int kB = 32;
      float mx = -INFINITY;
      for (int j0 = 0; j0 < K; j0 += 32 * kB) {
        float bv[kB];
#pragma unroll
        for (int x = 0; x < kB; ++x) {
          const int j = j0 + x * 32 + lane;
          bv[x] = j < K ? __ldg(D.u + nd.off_nk + j) : 0.f;
        }
        for (int c = nd.child_begin; c < nd.child_end; ++c) {
          const long long co = D.nodes[D.children[c]].off_nk;
          float lv[kB];
#pragma unroll
          for (int x = 0; x < kB; ++x) {
            const int j = j0 + x * 32 + lane;
            lv[x] = j < K ? __ldcg(D.lam + co + j) : 0.f;  // written by other CTAs of this launch
          }
#pragma unroll
          for (int x = 0; x < kB; ++x) bv[x] += lv[x];
        }
#pragma unroll
        for (int x = 0; x < kB; ++x) {
          const int j = j0 + x * 32 + lane;
          if (j < K) {
            cb[j] = bv[x];
            mx = fmaxf(mx, bv[x]);
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      // pass 2: normalise, fold in the row term, pad to whole chunks
      const bool store = (t.row0 == 0);
      for (int j0 = 0; j0 < nch * kRows; j0 += 32 * kB) {
        float zv[kB];
#pragma unroll
        for (int x = 0; x < kB; ++x) {
          const int j = j0 + x * 32 + lane;
          zv[x] = j < K ? __ldg(D.zn + nd.off_nk + j) : 0.f;
        }
#pragma unroll
        for (int x = 0; x < kB; ++x) {
          const int j = j0 + x * 32 + lane;
          if (j < K) {
            const float bb = cb[j] - mx;
            if (store) D.beta[nd.off_nk + j] = bb;
            cb[j] = (bb - 0.5f * zv[x] * iv) * kLog2e;
          } else if (j < nch * kRows) {
            cb[j] = -INFINITY;
          }
        }
      }
      if (store && lane == 0) D.nodemax[t.node] = mx;
      __syncwarp();
      if (lane == 0) mbar_arrive(&cb_full[ib]);  // release: cb visible to the math warps
    }
    if (!ok) set_timeout(D);
  } else if (warp >= 4) {
    // ------------------------------------------------------------------ exponentials
    const int mt = threadIdx.x - 128;
    const int qd = warp & 3, h = (warp - 4) >> 2;
    const int r = 32 * qd + lane;  // tile row = TMEM lane
    const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
    const float sc = iv * kLog2e;
    // A failed wait leaves `ok` false for this thread: it skips its remaining work of the
    // item but still reaches every named barrier; after the item's last barrier all math
    // threads read the shared abort flag and stop together.
    // Per item: the chunk loop (the group without the item's last chunk splits the next
    // item's mu~ after its own last chunk), then this item's messages are combined and
    // published.
    bool ok = true;
    // mu~ of item `it_s` (+ c_i) -> A operand, in place in region it_s & 1; its squared norm
    // into nrm_h[it_s & 1].  Each group splits its half of the columns, or (all) one group
    // splits every column and arrives on a_full for the other group's threads too.
    auto split = [&](int it_s, bool all) {
      ok = ok && mbar_wait_ab(&mu_full, (uint32_t)(it_s & 1), abort);
      tc_fence_after();
      const uint32_t tMU = tR[it_s & 1];
      const float* cvg = cvn[it_s & 1];
      // the two column halves keep separate norm partials, so the norm is the same sum
      // whichever way the split ran (the results do not depend on the work order)
      float nrm_lo = 0.f, nrm_hi = 0.f;  // columns [0, DP/2) and [DP/2, DP)
      if (ok) {
        const int g0 = all ? 0 : h * GH, g1 = all ? 2 * GH : (h + 1) * GH;
#pragma unroll 1
        for (int g = g0; g < g1; ++g) {
          uint32_t v[32];
          tmem_ld32(tMU + lane_off + g * 32, v);
          tmem_wait_ld();
          float f[32], nrm = g >= GH ? nrm_hi : nrm_lo;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            f[j] = __uint_as_float(v[j]) + cvg[g * 32 + j];
            nrm = fmaf(f[j], f[j], nrm);
          }
          if (g >= GH) nrm_hi = nrm;
          else nrm_lo = nrm;
          uint32_t hi[16], lo[16];
          split_pack32(f, hi, lo);
          // in place: this thread has read its row's 32 columns of the group
          tmem_st16(tMU + lane_off + g * 32, hi);
          tmem_st16(tMU + lane_off + g * 32 + 16, lo);
        }
        tmem_wait_st();
      }
      tc_fence_before();
      if (all) {
        nrm_h[it_s & 1][0][r] = nrm_lo;
        nrm_h[it_s & 1][1][r] = nrm_hi;
      } else {
        nrm_h[it_s & 1][h][r] = h ? nrm_hi : nrm_lo;
      }
      mbar_arrive(&a_full);
      if (all) mbar_arrive(&a_full);
    };
    long long gc = 0;
    int it = 0;
    int cur = -1, nxt = -1;
    ok = seq_get(0, cur);
    if (__any_sync(0xffffffffu, !ok)) cur = -1;  // (a failed read ends every thread's loop below)
    cur = sync_math_or(cur < 0) ? -1 : cur;
    if (cur >= 0) {
      if (mt < kTcMaxD) cvn[0][mt] = __ldg(T.cvec + (long long)tiles[cur].node * kLdp + mt);
      sync_math();
      split(0, false);
    }
    for (; cur >= 0; ++it) {
      const int item = cur;
      ok = ok && seq_get(it + 1, nxt);
      __syncwarp();
      if (lane == 0) mbar_arrive(&q_empty[it % kSeq]);
      const Tile t = tiles[item];
      const NodeInfo nd = D.nodes[t.node];
      const int K = nd.Kp, nch = tiles_of(nd.K);  // rows: parent samples; chunks: child samples
      const int k = t.row0 + r;
      const int ib = it % ncb;
      const float* cb = cbuf + (size_t)ib * cbk;
      // this item's message vector (warp 3, after the item's dependencies) before any chunk
      ok = ok && mbar_wait_ab(&cb_full[ib], (uint32_t)((it / ncb) & 1), abort);
      sync_math();  // both half norms of this item are complete
      const float nrm_all = nrm_h[it & 1][0][r] + nrm_h[it & 1][1][r];
      if (ok && h == 0 && k < K) D.mun[nd.off_nk + k] = nrm_all;
      float m = -INFINITY, ssum = 0.f;
      // The group that does not hold the item's last chunk splits the next item's mu~ (every
      // column) into the other A region as soon as it is done with its own chunks, while the
      // other group still works on the last chunk; its threads fetch that item's c_i now, so
      // the loads complete under the chunks.
      const bool has_next = ok && nxt >= 0;
      const int blast = (int)((gc + nch - 1) & 1);
      if (h != blast && has_next) {
        const int ml = mt - h * (kMath / 2);
        if (ml < kTcMaxD) cvn[(it + 1) & 1][ml] = __ldg(T.cvec + (long long)tiles[nxt].node * kLdp + ml);
      }
      // the two warp groups take alternate chunks (group h: the chunks in S buffer h), each
      // thread a whole 128-column row of its chunks, so one group's TMEM loads and
      // exponentials overlap the other's
      for (int c = 0; ok && c < nch; ++c) {
        const long long gcc = gc + c;
        const int b = (int)(gcc & 1);
        if (b != h) continue;
        if (!mbar_wait_ab(&sfull[b], (uint32_t)((gcc >> 1) & 1), abort)) { ok = false; break; }
        tc_fence_after();
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t v[2][32];
          tmem_ld32(tS[b] + lane_off + 64 * hh, v[0]);
          tmem_ld32(tS[b] + lane_off + 64 * hh + 32, v[1]);
          tmem_wait_ld();
          if (hh == 1) {
            tc_fence_before();
            mbar_arrive(&sfree[b]);  // the MMA may overwrite this S buffer now
          }
          const float* cbc = cb + c * kRows + 64 * hh;
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            float e[32], gm = -INFINITY;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              const float4 c4 = *reinterpret_cast<const float4*>(cbc + g * 32 + j);
              e[j] = fmaf(__uint_as_float(v[g][j]), sc, c4.x);
              e[j + 1] = fmaf(__uint_as_float(v[g][j + 1]), sc, c4.y);
              e[j + 2] = fmaf(__uint_as_float(v[g][j + 2]), sc, c4.z);
              e[j + 3] = fmaf(__uint_as_float(v[g][j + 3]), sc, c4.w);
              gm = fmaxf(gm, fmaxf(fmaxf(e[j], e[j + 1]), fmaxf(e[j + 2], e[j + 3])));
            }
            if (gm == -INFINITY) continue;  // every column of the group lies past K
            if (gm > m) {
              ssum *= ex2_ftz(m - gm);
              m = gm;
            }
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
              s0 += ex2_ftz(e[j] - m);
              s1 += ex2_ftz(e[j + 1] - m);
            }
            ssum += s0 + s1;
          }
        }
      }
      if (h != blast && has_next) {
        asm volatile("bar.sync 3, 128;" ::: "memory");  // this group's c_i loads are in cvn
        split(it + 1, true);
      }
      gc += nch;
      mbar_arrive(&cb_empty[ib]);  // cb of this item is no longer read
      m_h[h][r] = m;
      s_h[h][r] = ssum;
      sync_math();  // m_h / s_h complete
      if (ok && h == 0 && k < K) {
        const float m0 = m_h[0][r], m1 = m_h[1][r];
        const float M = fmaxf(m0, m1);
        const float S = s_h[0][r] * ex2_ftz(m0 - M) + (m1 == -INFINITY ? 0.f : s_h[1][r] * ex2_ftz(m1 - M));
        D.lam[nd.off_nk + k] = (M + log2f(S)) * kLn2 - 0.5f * nrm_all * iv;
      }
      // Every row's message is written; m_h / s_h are free for the next item.  Whether to stop
      // is an OR over the math threads taken inside the barrier, so all of them take the same
      // branch even when another role raises the abort flag meanwhile.
      const bool stop = sync_math_or(!ok || *abort != 0);
      if (stop) *abort = 1;
      if (mt == 0 && !stop) {
        __threadfence();  // the CTA's messages visible device-wide before the count moves
        red_release_add(done + t.node, 1);
        stamp_item_end(D, T, 0, nd.b);
      }
      if (stop) {
        if (mt == 0) set_timeout(D);
        break;
      }
      cur = nxt;  // the same value in every math thread (every read succeeded)
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tb, 512);
  }
}

// =======================================================================================
// Adjoint edge kernel (ROWS = false) and its row-direction twin (ROWS = true).
// TMEM: S double buffer [0,256), V [256, 256+DP), P double buffer [384, 512) (fp16 pairs).
//
// ROWS: the parent-side part of the sample gradient.  An item is 128 PARENT samples k of edge
// p -> i (tile.node = i, tile.row0 = first parent row); the prologue forms mu~ = Z~_p W_i^T + c_i
// (the forward's A operand), the chunks run over the child's samples k', and with the weights
// normalised per parent sample (P[k,k'] = exp(F[k,k'] + beta_i[k'] - lam_i[k]), known from the
// forward) the same TS MMA accumulates R[k] = sum_k' P[k,k'] z~_i^{k'}.  The epilogue stores
// E[k] = R[k] - mu~^k (split fp16) for the sample-gradient assembly (k_dz_tc), which forms
// q_p[k] E[k] W_i (d log P / d z_p^k through this edge).  The weights of this direction need
// nothing of the adjoint, so the items carry no dependencies.
// In ROWS mode the mWTH / mWTL arguments carry W itself (B operand of Z~_p W_i^T) and mG is
// unused.
// =======================================================================================
template <int DP, bool ROWS>
__global__ void __launch_bounds__(kThreadsTc, 1)
    k_edge_bwd_tc(Dev D, TcDev T, const Tile* __restrict__ tiles, int ntiles, int* __restrict__ done,
                  int* __restrict__ claim,
                  const __grid_constant__ CUtensorMap mZH, const __grid_constant__ CUtensorMap mZL,
                  const __grid_constant__ CUtensorMap mWTH, const __grid_constant__ CUtensorMap mWTL,
                  const __grid_constant__ CUtensorMap mG) {
  constexpr int TB = kRows * DP * 2;
  constexpr int NB = DP / 64;
  constexpr int KS = DP / 16;
  constexpr int GH = DP / 64;
  constexpr int NS = bwd_stages(DP);
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  // NS stages x (hi, lo) of parent sample chunks.  Chunk c of an item goes to stage
  // (c + 2) % NS: stages 0 and 1 hold the prologue operands until its MMAs complete, so the
  // first NS - 2 chunks stream in beside them.
  unsigned char* ring = sm;
  float* ak = reinterpret_cast<float*>(ring + ring_bytes(DP));
  unsigned char* eG = ring + 4 * TB;   // G boxes: DP / 32 x [128 x 32] fp32 in stage 2
  __shared__ uint64_t bar_pro, bar_mu, bar_A, full[NS], empty[NS], sfull[2], pready[2];
  __shared__ uint64_t bar_v, bar_etma, bar_eready, bar_gm, bar_gst;
  __shared__ uint32_t tbase;
  __shared__ float q_h[2][kRows];
  // the records of this item and the next (slot = item iteration & 1), loaded by warp 3 while
  // the item before runs, and whether the next item's dependency was already seen satisfied
  __shared__ Tile s_tile[2];
  __shared__ NodeInfo s_nd[2], s_pn[2];
  __shared__ int s_dep[2];
  // the items of this CTA, claimed from the launch's counter in list (dependency) order: thread
  // 0 claims item iter + 1 at the start of item iter (slot iter & 1 holds item iter)
  __shared__ int s_claim[2];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float iv = D.inv_var;
  if (warp == 2) tmem_alloc(&tbase, 512);
  if (threadIdx.x == 0) {
    const int first = claim_item(claim, ntiles);
    s_claim[0] = first;
    if (first >= 0) {
      s_tile[0] = tiles[first];
      s_nd[0] = D.nodes[s_tile[0].node];
      s_pn[0] = D.nodes[s_nd[0].parent];
      s_dep[0] = 0;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = tbase;
  // TMEM: S double buffer [0,256), V [256,384), A'_hi [384,448), A'_lo [448,512).  The two math
  // warp groups take alternate chunks (group h: the chunks in S buffer h), one thread per row.
  // P of a chunk (fp16 pairs) overwrites the S row it came from: the thread reads S columns
  // [0,64) and writes P pairs to [0,32), then reads [64,128) and writes [32,64); the MMA warp
  // issues V(c) before S(c+2) into the same buffer, and tcgen05 MMAs of one thread run in
  // issue order.
  const uint32_t tS[2] = {tb, tb + 128}, tV = tb + 256, tAH = tb + 384, tAL = tb + 448;
  const uint32_t tG = tb;

  // persistent loop over the edge tiles of every level, root side first
  for (int iter = 0;; ++iter) {
  const int sl = iter & 1;
  const int item = s_claim[sl];  // written before the last CTA-wide barrier
  if (item < 0) break;
  const Tile t = s_tile[sl];
  const NodeInfo nd = s_nd[sl];
  const NodeInfo pn = s_pn[sl];
  // the node whose samples fill the chunks, and the node whose 128 rows the item owns
  const NodeInfo& chn = ROWS ? nd : pn;
  const long long own_off = ROWS ? pn.off_nk : nd.off_nk;
  const int Kch = chn.K, Krow = ROWS ? nd.Kp : nd.K;  // chunk samples, row samples
  const int nch = (Kch + kRows - 1) / kRows;
  // Epilogue operands in the ring.  With 3 or more chunks this CTA's own Z~ tile is loaded
  // into the stage of chunk nch - 3 as soon as its V MMAs are done (no later chunk uses that
  // stage), under the last two chunks, and the V tile goes to the last chunk's stage; with
  // fewer chunks both sit at the ring start, loaded after every V MMA.
  const bool early_ez = nch >= 3;
  unsigned char* eZH = early_ez ? ring + ((nch - 1) % NS) * 2 * TB : ring;  // Z~_i hi (N atoms)
  unsigned char* eZL = eZH + TB;                                            // Z~_i lo
  unsigned char* eSV = early_ez ? ring + ((nch + 1) % NS) * 2 * TB : ring + 2 * TB;  // V tile
  if (threadIdx.x == 0) {
    s_claim[sl ^ 1] = claim_item(claim, ntiles);  // the next item (its records: warp 3)
    // the parent's sample weights must be final (the root's come from an earlier launch)
    if (!ROWS) {
      if (pn.parent >= 0 && !s_dep[sl] && !wait_count(done + nd.parent, tiles_of(pn.K), D.wait_limit))
        set_timeout(D);
      stamp_item_start(T, 1, iter == 0);
    }
    mbar_init(&bar_pro, 1);
    mbar_init(&bar_mu, 1);
    mbar_init(&bar_A, kMath);
    mbar_init(&bar_v, 1);
    mbar_init(&bar_etma, 1);
    mbar_init(&bar_eready, kMath);
    mbar_init(&bar_gm, 1);
    mbar_init(&bar_gst, kMath);
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) mbar_init(&sfull[i], 1);
    mbar_init(&pready[0], kMath / 2);
    mbar_init(&pready[1], kMath / 2);
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------------ TMA producer
    prefetch_tmap(&mZH);
    prefetch_tmap(&mZL);
    // pull the chunk with this CTA's tile index into L2 (see the forward kernel)
    for (int b = 0; b < NB; ++b) {
      tma_prefetch_l2_2d(&mZH, b * 64, (int)(chn.off_nk + t.row0));
      tma_prefetch_l2_2d(&mZL, b * 64, (int)(chn.off_nk + t.row0));
    }
    const int slot = slot_of(D, nd, t.node);
    const int own = (int)(own_off + t.row0);
    mbar_arrive_expect_tx(&bar_pro, 4 * TB);
    for (int b = 0; b < NB; ++b) {
      tma_load_2d(ring + b * kBox, &mZH, &bar_pro, b * 64, own);
      tma_load_2d(ring + TB + b * kBox, &mZL, &bar_pro, b * 64, own);
      tma_load_2d(ring + 2 * TB + b * kBox, &mWTH, &bar_pro, b * 64, slot * kLdp);
      tma_load_2d(ring + 3 * TB + b * kBox, &mWTL, &bar_pro, b * 64, slot * kLdp);
    }
    if (s_claim[sl ^ 1] >= 0) {  // next item's own tile into L2 while this one runs
      const Tile tn = tiles[s_claim[sl ^ 1]];
      const NodeInfo& nn = D.nodes[tn.node];
      const int row_n = (int)((ROWS ? D.nodes[nn.parent].off_nk : nn.off_nk) + tn.row0);
      for (int b = 0; b < NB; ++b) {
        tma_prefetch_l2_2d(&mZH, b * 64, row_n);
        tma_prefetch_l2_2d(&mZL, b * 64, row_n);
      }
    }
    bool ok = true, mu_seen = false;
    int issued = 0;
    for (int c = 0; ok && c < nch; ++c) {
      const int s = (c + 2) % NS, ui = bwd_use(c, NS);
      if (ui >= 1) {
        if (!mbar_wait(&empty[s], (ui - 1) & 1)) { ok = false; break; }
      } else if (s < 2 && !mu_seen) {  // first use of a prologue stage
        if (!mbar_wait(&bar_mu, 0)) { ok = false; break; }
        mu_seen = true;
      }
      unsigned char* st = ring + s * 2 * TB;
      if (!ROWS && c == 0) bulk_wait_group_read0();  // stage 2 held the last item's G boxes
      mbar_arrive_expect_tx(&full[s], 2 * TB);
      const int row = (int)(chn.off_nk + c * kRows);
      for (int b = 0; b < NB; ++b) {
        tma_load_2d(st + b * kBox, &mZH, &full[s], b * 64, row);
        tma_load_2d(st + TB + b * kBox, &mZL, &full[s], b * 64, row);
      }
      issued = c + 1;
    }
    if constexpr (ROWS) {
      // the last fills land before the item ends; the epilogue needs no operands
      for (int c = (issued > NS ? issued - NS : 0); c < issued; ++c)
        mbar_wait(&full[(c + 2) % NS], bwd_use(c, NS) & 1);
      if (!ok) set_timeout(D);
    } else {
    // epilogue operands: this CTA's own Z~ tile again (early: once V(nch - 3) is done)
    auto load_ez = [&]() {
      mbar_arrive_expect_tx(&bar_etma, 2 * TB);
      for (int b = 0; b < NB; ++b) {
        tma_load_2d(eZH + b * kBox, &mZH, &bar_etma, b * 64, own);
        tma_load_2d(eZL + b * kBox, &mZL, &bar_etma, b * 64, own);
      }
    };
    bool ez_issued = false;
    if (ok && early_ez) {
      ok = mbar_wait(&empty[(nch - 1) % NS], bwd_use(nch - 3, NS) & 1);
      if (ok) {
        load_ez();
        ez_issued = true;
      }
    }
    for (int c = (issued > NS ? issued - NS : 0); c < issued; ++c)
      mbar_wait(&full[(c + 2) % NS], bwd_use(c, NS) & 1);
    if (ok) ok = mbar_wait(&bar_v, 0);
    if (ok && !ez_issued) {
      load_ez();
      ez_issued = true;
    }
    if (ez_issued) ok = mbar_wait(&bar_etma, 0) && ok;
    // this tile's G partial, staged by the math warps, goes out as TMA reductions; their
    // reads of stage 2 are waited for before the next item's first chunk lands there
    if (ok) ok = mbar_wait(&bar_gst, 0);
    if (ok) {
      const int y = t.node * kLdp;
      for (int g = 0; g < DP / 32; ++g) tma_reduce_add_2d(&mG, eG + g * kBox, g * 32, y);
      bulk_commit_group();
    }
    if (!ok) set_timeout(D);
    }  // !ROWS
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------------ MMA issuer
    bool ok = mbar_wait(&bar_pro, 0);
    if (ok) {
      tc_fence_after();
      const uint32_t id_a = idesc_f16(kRows, DP, false, false, false);
      const uint64_t dzh = kdesc(ring, 0), dzl = kdesc(ring + TB, 0), dwh = kdesc(ring + 2 * TB, 0),
                     dwl = kdesc(ring + 3 * TB, 0);
      for (int kk = 0; kk < KS; ++kk) mma_ss(tS[0], kstep(dzh, kk), kstep(dwh, kk), id_a, kk > 0);
      for (int kk = 0; kk < KS; ++kk) mma_ss(tS[0], kstep(dzl, kk), kstep(dwh, kk), id_a, 1);
      for (int kk = 0; kk < KS; ++kk) mma_ss(tS[0], kstep(dzh, kk), kstep(dwl, kk), id_a, 1);
      mma_commit(&bar_mu);
      ok = mbar_wait(&bar_A, 0);
    }
    const uint32_t id_s = idesc_f16(kRows, kRows, false, false, false);
    const uint32_t id_v = idesc_f16(kRows, DP, false, false, true);
    for (int c = 0; ok && c <= nch; ++c) {
      if (c < nch) {
        const int s = (c + 2) % NS, b = c & 1;
        if (!mbar_wait(&full[s], bwd_use(c, NS) & 1)) { ok = false; break; }
        tc_fence_after();
        const uint64_t dbh = kdesc(ring + s * 2 * TB, 0), dbl = kdesc(ring + s * 2 * TB + TB, 0);
        for (int kk = 0; kk < KS; ++kk) mma_ts(tS[b], tAH + kk * 8, kstep(dbh, kk), id_s, kk > 0);
        for (int kk = 0; kk < KS; ++kk) mma_ts(tS[b], tAL + kk * 8, kstep(dbh, kk), id_s, 1);
        for (int kk = 0; kk < KS; ++kk) mma_ts(tS[b], tAH + kk * 8, kstep(dbl, kk), id_s, 1);
        mma_commit(&sfull[b]);
      }
      if (c >= 1) {
        const int cp = c - 1, s = (cp + 2) % NS;
        if (!mbar_wait(&pready[cp & 1], (cp >> 1) & 1)) { ok = false; break; }
        tc_fence_after();
        const uint64_t dv = mndesc(ring + s * 2 * TB, 0);
        // V[k'][:] += sum_k P[k'][k] z~_p^k   (P: fp16 pairs in columns [0,64) of S buffer cp & 1)
        for (int kk = 0; kk < kRows / 16; ++kk)
          mma_ts(tV, tS[cp & 1] + kk * 8, mnstep(dv, kk), id_v, (cp > 0 || kk > 0) ? 1u : 0u);
        mma_commit(&empty[s]);
      }
    }
    mma_commit(&bar_v);
    if constexpr (ROWS) {
      if (ok) ok = mbar_wait(&bar_v, 0);
      if (!ok) set_timeout(D);
    } else {
    if (ok) ok = mbar_wait(&bar_v, 0);
    if (ok) ok = mbar_wait(&bar_etma, 0) && mbar_wait(&bar_eready, 0);
    if (ok) {
      tc_fence_after();
      // G[a][b] = sum_k' V[k'][a] z~[k'][b]   (the node moments M2, zbar: k_moments_tc)
      const uint32_t id_g = idesc_f16(kRows, DP, false, true, true);
      for (int kk = 0; kk < kRows / 16; ++kk) mma_ss(tG, mndesc(eSV, kk), mndesc(eZH, kk), id_g, kk > 0);
      for (int kk = 0; kk < kRows / 16; ++kk) mma_ss(tG, mndesc(eSV, kk), mndesc(eZL, kk), id_g, 1);
      mma_commit(&bar_gm);
      mbar_wait(&bar_gm, 0);
    } else {
      set_timeout(D);
      mma_commit(&bar_gm);
      mbar_wait(&bar_gm, 0);
    }
    }  // !ROWS
  } else if (warp == 3 && lane == 0) {
    // ------------------------------------------------------------------ next item's records
    // (three dependent loads) and one look at its dependency, while this item runs; if the
    // dependency is not met yet (it may be this very item), thread 0 waits for it at the
    // next item's start.
    const int nx = s_claim[sl ^ 1];
    if (nx >= 0) {
      const Tile tn = tiles[nx];
      const NodeInfo ndn = D.nodes[tn.node];
      const NodeInfo pnn = D.nodes[ndn.parent];
      s_tile[sl ^ 1] = tn;
      s_nd[sl ^ 1] = ndn;
      s_pn[sl ^ 1] = pnn;
      s_dep[sl ^ 1] = ROWS || pnn.parent < 0 || ld_acquire(done + ndn.parent) >= tiles_of(pnn.K);
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------------ exponentials
    const int mt = threadIdx.x - 128;
    const int qd = warp & 3, h = (warp - 4) >> 2;
    const int r = 32 * qd + lane;
    const uint32_t lane_off = (uint32_t)(32 * qd) << 16;
    const int kq = t.row0 + r;  // sample owned by this thread's row (ROWS: a parent sample)
    const bool valid = kq < Krow;
    if constexpr (ROWS) {
      // column (child sample) terms: (beta_i - |z~_i|^2 / (2 var)) log2 e, as in the forward
      float bv[kJt], zv[kJt];
#pragma unroll
      for (int i = 0; i < kJt; ++i) {
        const int j = mt + i * kMath;
        const bool in = j < Kch;
        bv[i] = in ? D.beta[nd.off_nk + j] : 0.f;
        zv[i] = in ? D.zn[nd.off_nk + j] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < kJt; ++i) {
        const int j = mt + i * kMath;
        if (j >= nch * kRows) break;
        ak[j] = (j < Kch) ? (bv[i] - 0.5f * zv[i] * iv) * kLog2e : -INFINITY;
      }
    } else {
      // column (parent sample) terms: (log q_p - lam_i - |mu~|^2 / (2 var)) log2 e; all loads first
      float qv[kJt], lv[kJt], mv[kJt];
#pragma unroll
      for (int i = 0; i < kJt; ++i) {
        const int j = mt + i * kMath;
        const bool in = j < Kch;
        qv[i] = in ? __ldcg(D.q + pn.off_nk + j) : 0.f;  // may come from this launch
        lv[i] = in ? D.lam[nd.off_nk + j] : 0.f;
        mv[i] = in ? D.mun[nd.off_nk + j] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < kJt; ++i) {
        const int j = mt + i * kMath;
        if (j >= nch * kRows) break;
        ak[j] = (j < Kch) ? (logf(qv[i]) - lv[i] - 0.5f * mv[i] * iv) * kLog2e : -INFINITY;
      }
    }
    // row term: adjoint (beta_i - |z~|^2 / (2 var) + z~ . c_i / var) log2 e; ROWS the row
    // normaliser -(lam_i[k] + |mu~^k|^2 / (2 var)) log2 e of the forward's log-sum-exp
    const float crow = !valid ? -INFINITY
                       : ROWS ? -(D.lam[nd.off_nk + kq] + 0.5f * D.mun[nd.off_nk + kq] * iv) * kLog2e
                              : (D.beta[nd.off_nk + kq] - 0.5f * D.zn[nd.off_nk + kq] * iv +
                                 T.zc[nd.off_nk + kq] * iv) * kLog2e;
    // prologue result A' = Z~_i W_i -> this half of the split A operand
    bool ok = mbar_wait(&bar_mu, 0);
    if (ok) {
      tc_fence_after();
#pragma unroll 1
      for (int gg = 0; gg < GH; ++gg) {
        const int g = h * GH + gg;
        uint32_t v[32];
        tmem_ld32(tS[0] + lane_off + g * 32, v);
        tmem_wait_ld();
        float f[32];
        const float* cv = T.cvec + (long long)t.node * kLdp + g * 32;  // ROWS: mu~ = Z~_p W^T + c_i
#pragma unroll
        for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]) + (ROWS ? __ldg(cv + j) : 0.f);
        uint32_t hi[16], lo[16];
        split_pack32(f, hi, lo);
        tmem_st16(tAH + lane_off + g * 16, hi);
        tmem_st16(tAL + lane_off + g * 16, lo);
      }
      tmem_wait_st();
      tc_fence_before();
    }
    mbar_arrive(&bar_A);
    sync_math();  // ak complete
    const float sc = iv * kLog2e;
    float qacc = 0.f;
    for (int c = h; ok && c < nch; c += 2) {  // this group's chunks: S buffer h
      const int b = c & 1;
      if (!mbar_wait(&sfull[b], (c >> 1) & 1)) { ok = false; break; }
      tc_fence_after();
#pragma unroll 1
      for (int hh = 0; hh < 2; ++hh) {
        uint32_t v[2][32];
        tmem_ld32(tS[b] + lane_off + 64 * hh, v[0]);
        tmem_ld32(tS[b] + lane_off + 64 * hh + 32, v[1]);
        tmem_wait_ld();
        const float* akc = ak + c * kRows + 64 * hh;
        uint32_t pk[32];
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            const float4 a4 = *reinterpret_cast<const float4*>(akc + g * 32 + j);
            const float p0 = ex2_ftz(fmaf(__uint_as_float(v[g][j]), sc, crow + a4.x));
            const float p1 = ex2_ftz(fmaf(__uint_as_float(v[g][j + 1]), sc, crow + a4.y));
            const float p2 = ex2_ftz(fmaf(__uint_as_float(v[g][j + 2]), sc, crow + a4.z));
            const float p3 = ex2_ftz(fmaf(__uint_as_float(v[g][j + 3]), sc, crow + a4.w));
            s0 += p0 + p1;
            s1 += p2 + p3;
            pk[g * 16 + j / 2] = pack_half2(p0, p1);
            pk[g * 16 + j / 2 + 1] = pack_half2(p2, p3);
          }
        }
        qacc += s0 + s1;
        tmem_st32(tS[b] + lane_off + 32 * hh, pk);  // P over S columns this thread has read
      }
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&pready[b]);
    }
    if constexpr (ROWS) {
      // E[k] = R[k] - mu~^k (R in V's columns, mu~ = A hi + lo), split, to the E rows
      (void)qacc;
      if (ok) ok = mbar_wait(&bar_v, 0);
      if (ok) {
        tc_fence_after();
        __half* eh = T.EH + (nd.off_nk + kq) * kLdp;
        __half* el = T.EL + (nd.off_nk + kq) * kLdp;
#pragma unroll 1
        for (int gg = 0; gg < GH; ++gg) {
          const int g = h * GH + gg;
          uint32_t v[32], ah[16], al[16];
          tmem_ld32(tV + lane_off + g * 32, v);
          tmem_ld16(tAH + lane_off + g * 16, ah);
          tmem_ld16(tAL + lane_off + g * 16, al);
          tmem_wait_ld();
          float e[32];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float2 fh = __half22float2(*reinterpret_cast<const __half2*>(&ah[q]));
            const float2 fl = __half22float2(*reinterpret_cast<const __half2*>(&al[q]));
            e[2 * q] = __uint_as_float(v[2 * q]) - (fh.x + fl.x);
            e[2 * q + 1] = __uint_as_float(v[2 * q + 1]) - (fh.y + fl.y);
          }
          uint32_t hi[16], lo[16];
          split_pack32(e, hi, lo);
          if (valid)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              reinterpret_cast<uint4*>(eh + g * 32)[q] = make_uint4(hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
              reinterpret_cast<uint4*>(el + g * 32)[q] = make_uint4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
            }
        }
      }
      tc_fence_before();
      if (!ok) set_timeout(D);
    } else {
    q_h[h][r] = qacc;
    sync_math();
    const float qtot = q_h[0][r] + q_h[1][r];
    if (ok && valid && h == 0) D.q[nd.off_nk + kq] = qtot;
    __threadfence();  // weights visible device-wide before the completion count moves
    // sample gradients requested: V / q (the conditional mean of the parent's samples given
    // this child sample) to the V rows, split, for the sample-gradient assembly
    const bool want_v = D.dz != nullptr || D.deps != nullptr || D.coupled;
    const float rq = qtot > 0.f ? 1.f / qtot : 0.f;
    // epilogue: V row -> fp16 A tile of G
    if (ok) ok = mbar_wait(&bar_v, 0);
    if (ok) {
      tc_fence_after();
#pragma unroll 1
      for (int gg = 0; gg < 2; ++gg) {
        const int g = 2 * h + gg;  // 32-column group of the 128-wide tile
        float f[32];
        if (g < DP / 32) {
          uint32_t v[32];
          tmem_ld32(tV + lane_off + g * 32, v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) f[j] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) store_half8(eSV, r, g * 4 + q, f + 8 * q);
        if (want_v && valid && g < DP / 32) {
          float fv[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) fv[j] = f[j] * rq;
          uint32_t hi[16], lo[16];
          split_pack32(fv, hi, lo);
          uint4* vh = reinterpret_cast<uint4*>(T.VH + (nd.off_nk + kq) * kLdp + g * 32);
          uint4* vl = reinterpret_cast<uint4*>(T.VL + (nd.off_nk + kq) * kLdp + g * 32);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            vh[q] = make_uint4(hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
            vl[q] = make_uint4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
          }
        }
      }
      ok = mbar_wait(&bar_etma, 0);
    }
    if (ok) {
      fence_proxy_async_smem();
      tc_fence_before();
    }
    mbar_arrive(&bar_eready);
    if (ok) ok = mbar_wait(&bar_gm, 0);
    // The tile's G partial goes to global memory as TMA reductions (the L2 adds whole
    // lines): TMEM -> 128B-swizzled [128 x 32] fp32 boxes in ring stage 2 (free once the V
    // MMAs are done) -> one cp.reduce.async.bulk.tensor per box, issued by the producer.
    // Rows / columns past d are zero (padding of z~).
    if (ok) {
      tc_fence_after();
      const int a = r;  // TMEM lane = output row a
#pragma unroll 1
      for (int gg = 0; gg < GH; ++gg) {
        const int g = h * GH + gg;  // 32-column box
        uint32_t v[32];
        tmem_ld32(tG + lane_off + g * 32, v);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<uint4*>(eG + g * kBox + sw128_offset(a, q)) =
              make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      fence_proxy_async_smem();
    }
    tc_fence_before();
    mbar_arrive(&bar_gst);  // (release) this thread's rows of the boxes are written
    if (!ok) set_timeout(D);
    }  // !ROWS
  }
  // item end: every role is done with this item's barriers, tensor memory and ring
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (!ROWS && warp == 3 && lane == 0) {  // thread 0 goes straight on to the next item's setup
    red_release_add(done + t.node, 1);
    stamp_item_end(D, T, 1, nd.b);
  }
  }  // items
  if (!ROWS && warp == 0 && lane == 0) bulk_wait_group0();  // the last G reductions are done
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tb, 512);
  }
}

// =======================================================================================
// Node moments on the tensor core, for every node:
//   M2_g = sum_k q_g[k] z~_g^k z~_g^k^T,   zbar_g = sum_k q_g[k] z~_g^k.
// With the samples as the contraction index, A = (q Z~)^T and B = Z~ are MN-major views of
// [samples x DP] fp16 tiles; zbar is the same A against a B whose first column is 1.  q z~ and
// z~ are both split (hi + lo), which keeps about 22 bits.
// Work moves in units of 64 samples: the producer warp streams each unit's Z~ hi / lo (TMA)
// and its weights into an NS-stage ring, the math warps form the unit's q Z~ into one of NQ
// buffers, the MMA warp issues its products.  An item (up to kMoSlabs x 128 samples of one
// node) accumulates in one of two TMEM accumulators; four epilogue warps store its M2 and zbar
// (rows a < d, columns < d) while the next item's units run.
// Both MMA operands come from shared memory (about twice the cycles of a TMEM-operand MMA),
// and those MMAs bound the kernel, so every MMA reads its A once against as wide a B as fits: each ring stage holds
// a constant ones atom next to the Z~ atoms, and B = [Z~ hi | Z~ lo | 1] (DP = 64, N = 144)
// or [Z~ hi | 1] (DP = 128, N = 144) plus Z~ lo (N = 128).
// DP = 64: hi and lo of q Z~ are stacked along M (A rows 0-63 hi, 64-127 lo): one MMA per
// K-step gives qz_hi z~_hi, qz_hi z~_lo, qz_lo z~_hi, qz_lo z~_lo and both zbar halves; the
// epilogue adds the column blocks and the two TMEM halves.  DP = 128: A rows are the 128
// entries of q z~, hi and lo in separate tiles, three MMAs per K-step.
// =======================================================================================
constexpr int kMoSlabs = 8;
constexpr int kMoMath = 256;                 // math warps 0-7
constexpr int kMoProd = kMoMath / 32;        // producer warp; the MMA warp follows, then 4 epilogue warps
constexpr int kMoThreads = kMoMath + 6 * 32;
constexpr int kMoPrefetch = 4;               // units prefetched into L2 ahead of the ring loads
constexpr int kMoUnit = 64;                  // samples per unit
constexpr int kMoAtom = kMoUnit * 128;       // one 64-row, 128-byte-swizzled atom
constexpr int kMoXLd = 68;                   // row stride (floats) of the epilogue scratch
constexpr int kMoXBytes = (64 * kMoXLd + 64) * 4;  // one scratch: 64 x 64 block + 64 zbar
template <int DP>
struct MoCfg {
  static constexpr bool STK = DP == 64;        // q Z~ hi / lo stacked along M
  static constexpr int UT = kMoUnit * DP * 2;  // one [64 x DP] fp16 tile (DP / 64 atoms)
  // ring stage: STK [Z~ hi | Z~ lo | ones], else [Z~ hi (2 atoms) | ones | Z~ lo (2 atoms)]
  static constexpr int ZL_OFF = STK ? kMoAtom : 3 * kMoAtom;
  static constexpr int ONES_OFF = STK ? 2 * kMoAtom : 2 * kMoAtom;
  static constexpr int SB = 2 * UT + kMoAtom;
  static constexpr int QB = STK ? 2 * kMoAtom : 4 * kMoAtom;  // q Z~ buffer
  static constexpr int NQ = STK ? 4 : 2;
  static constexpr int XB = STK ? 2 * kMoXBytes : 0;  // epilogue scratch (two buffers)
  // the opt-in maximum (227 KB) less the alignment pad and 2 KB of static shared memory
  static constexpr int NS0 = (232448 - 1024 - 2048 - NQ * QB - XB) / SB;
  static constexpr int NS = NS0 > 6 ? 6 : NS0;
  static constexpr size_t smem = 1024 + (size_t)NS * SB + (size_t)NQ * QB + XB;
  static constexpr int CPT = DP / 32;          // 16-byte chunks of a q Z~ row per math thread
  static_assert(NS >= 2, "moments ring");
};

__device__ __forceinline__ uint32_t mo_off(int rr, int chunk) {
  return (uint32_t)(chunk >> 3) * kMoAtom + sw128_offset(rr, chunk & 7);
}
__device__ __forceinline__ uint64_t mo_desc(const unsigned char* p) {
  return smem_desc_sw128(smem_u32(p), kMoAtom, 1024);
}

template <int DP>
__global__ void __launch_bounds__(kMoThreads, 1)
    k_moments_tc(Dev D, TcDev T, const MoItem* __restrict__ items, int nitems,
                 const __grid_constant__ CUtensorMap mZH, const __grid_constant__ CUtensorMap mZL) {
  using C = MoCfg<DP>;
  constexpr int SB = C::SB, QB = C::QB, NQ = C::NQ, NS = C::NS, NB = DP / 64, CPT = C::CPT;
  constexpr int ZL_OFF = C::ZL_OFF, ONES_OFF = C::ONES_OFF;
  constexpr bool STK = C::STK;
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  unsigned char* ring = sm;                   // NS x (Z~ hi, Z~ lo, ones) of a unit
  unsigned char* qz = ring + NS * SB;         // NQ x q Z~
  float* xs = reinterpret_cast<float*>(qz + NQ * QB);  // DP = 64: lo-half partials, 2 buffers
  __shared__ uint64_t full[NS], empty[NS], qready[NQ], qfree[NQ], accdone[2], accfree[2], fin;
  __shared__ float qs[NS][kMoUnit];             // the unit's sample weights, beside its ring stage
  __shared__ uint32_t tbase;
  __shared__ int abort_;
  volatile int* abort = &abort_;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == kMoProd + 1) tmem_alloc(&tbase, 512);
  // the ones atom of every stage: row k = (1, 0, ..., 0)
  for (int i = threadIdx.x; i < NS * kMoUnit * 8; i += blockDim.x) {
    const int r = i % kMoUnit, ch = (i / kMoUnit) % 8, st = i / (kMoUnit * 8);
    const uint32_t one = ch == 0 ? 0x3C00u : 0u;  // fp16 1.0 in the low half
    *reinterpret_cast<uint4*>(ring + st * SB + ONES_OFF + mo_off(r, ch)) = make_uint4(one, 0u, 0u, 0u);
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < NQ; ++i) {
      mbar_init(&qready[i], kMoMath / 32);  // one arrival per math warp
      mbar_init(&qfree[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accdone[i], 1);
      mbar_init(&accfree[i], 4);  // one arrival per epilogue warp
    }
    mbar_init(&fin, 1);
    fence_barrier_init();
    abort_ = 0;
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = tbase;

  if (warp == kMoProd) {
    // ---------------- producer: 64-sample units of Z~ hi / lo into the ring (TMA, lane 0) and
    // their sample weights into qs (the whole warp, loaded ahead of the wait for the stage).
    // The warp loads the records of its next 32 items at once (lane i: item i).
    if (lane == 0) {
      prefetch_tmap(&mZH);
      prefetch_tmap(&mZL);
    }
    int gu = 0;
    bool ok = true;
    for (int base = blockIdx.x; base < nitems && ok; base += 32 * gridDim.x) {
      const int mine = base + lane * gridDim.x;
      const MoItem rec = mine < nitems ? items[mine] : MoItem{};
      const int nb = min(32, (nitems - base + (int)gridDim.x - 1) / (int)gridDim.x);
      // L2 prefetch cursor kMoPrefetch units ahead of the loads (within the batch): the ring
      // holds too few bytes to cover the DRAM latency on its own
      int pj = 0, pu = 0;
      auto pf_step = [&]() {
        if (pj >= nb) return;
        const long long prow = __shfl_sync(0xffffffffu, rec.row, pj);
        const int pnr = __shfl_sync(0xffffffffu, rec.nrows, pj);
        if (lane == 0) {
          for (int b = 0; b < NB; ++b) {
            tma_prefetch_l2_2d(&mZH, b * 64, (int)(prow + pu * kMoUnit));
            tma_prefetch_l2_2d(&mZL, b * 64, (int)(prow + pu * kMoUnit));
          }
          // the unit's sample weights (two 128-byte lines), read by the weight loads below
          const float* qp = D.q + prow + pu * kMoUnit;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(qp) : "memory");
          if (pu * kMoUnit + 32 < pnr) asm volatile("prefetch.global.L2 [%0];" ::"l"(qp + 32) : "memory");
        }
        if (++pu * kMoUnit >= pnr) {
          pu = 0;
          ++pj;
        }
      };
      for (int i = 0; i < kMoPrefetch; ++i) pf_step();
      // the sample weights of a unit are loaded one unit ahead of its stage
      auto q_load = [&](int jj, int uu, float& x0, float& x1) {
        const long long r = __shfl_sync(0xffffffffu, rec.row, jj);
        const int nr = __shfl_sync(0xffffffffu, rec.nrows, jj);
        const int k0 = uu * kMoUnit + lane;
        x0 = k0 < nr ? __ldg(D.q + r + k0) : 0.f;
        x1 = k0 + 32 < nr ? __ldg(D.q + r + k0 + 32) : 0.f;
      };
      float q0 = 0.f, q1 = 0.f;
      if (nb > 0) q_load(0, 0, q0, q1);
      for (int j = 0, u = 0; j < nb && ok;) {
        const long long row = __shfl_sync(0xffffffffu, rec.row, j);
        const int nrows = __shfl_sync(0xffffffffu, rec.nrows, j);
        const int nu = (nrows + kMoUnit - 1) / kMoUnit;
        int j2 = j, u2 = u + 1;  // the next unit
        if (u2 >= nu) {
          j2 = j + 1;
          u2 = 0;
        }
        float n0 = 0.f, n1 = 0.f;
        if (j2 < nb) q_load(j2, u2, n0, n1);
        pf_step();
        const int st = gu % NS, use = gu / NS;
        bool w = true;
        if (lane == 0) w = use < 1 || mbar_wait_ab(&empty[st], (uint32_t)((use - 1) & 1), abort);
        if (!__shfl_sync(0xffffffffu, w, 0)) {
          ok = false;
          break;
        }
        qs[st][lane] = q0;
        qs[st][lane + 32] = q1;
        __syncwarp();  // orders the weights before lane 0's arrival (release) on full
        if (lane == 0) {
          mbar_arrive_expect_tx(&full[st], 2 * C::UT);
          for (int b = 0; b < NB; ++b) {
            tma_load_2d(ring + st * SB + b * kMoAtom, &mZH, &full[st], b * 64, (int)(row + u * kMoUnit));
            tma_load_2d(ring + st * SB + ZL_OFF + b * kMoAtom, &mZL, &full[st], b * 64, (int)(row + u * kMoUnit));
          }
        }
        ++gu;
        q0 = n0;
        q1 = n1;
        j = j2;
        u = u2;
      }
    }
    // the copies still in flight land before the CTA leaves (bounded)
    if (lane == 0)
      for (int i = gu - 1; i >= 0 && i >= gu - NS; --i) mbar_wait(&full[i % NS], (uint32_t)((i / NS) & 1));
  } else if (warp == kMoProd + 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t id_w = idesc_f16(kRows, 144, false, true, true);  // [hi | lo | 1] or [hi | 1]
      const uint32_t id_l = idesc_f16(kRows, DP, false, true, true);    // DP = 128: Z~ lo
      int gu = 0, it = 0;
      bool issued = false;
      MoItem mn = blockIdx.x < nitems ? items[blockIdx.x] : MoItem{};
      for (int item = blockIdx.x; item < nitems && !*abort; item += gridDim.x, ++it) {
        const MoItem m = mn;
        if (item + gridDim.x < nitems) mn = items[item + gridDim.x];
        const int nu = (m.nrows + kMoUnit - 1) / kMoUnit;
        const int ab = it & 1;
        const uint32_t acc = tb + ab * 256;
        if (it >= 2 && !mbar_wait_ab(&accfree[ab], (uint32_t)(((it >> 1) - 1) & 1), abort)) break;
        bool ok = true;
        for (int u = 0; u < nu; ++u, ++gu) {
          const int st = gu % NS, qb = gu % NQ;
          if (!mbar_wait_ab(&full[st], (uint32_t)((gu / NS) & 1), abort) ||
              !mbar_wait_ab(&qready[qb], (uint32_t)((gu / NQ) & 1), abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t dbw = mo_desc(ring + st * SB), dzl = mo_desc(ring + st * SB + ZL_OFF);
          const uint64_t dqh = mo_desc(qz + qb * QB), dql = mo_desc(qz + qb * QB + 2 * kMoAtom);
          for (int kk = 0; kk < kMoUnit / 16; ++kk) {
            const uint32_t first = (u == 0 && kk == 0) ? 0u : 1u;
            mma_ss(acc, mnstep(dqh, kk), mnstep(dbw, kk), id_w, first);
            if (!STK) {
              mma_ss(acc, mnstep(dql, kk), mnstep(dbw, kk), id_w, 1u);
              mma_ss(acc, mnstep(dqh, kk), mnstep(dzl, kk), id_l, 1u);
            }
          }
          issued = true;
          mma_commit(&empty[st]);
          mma_commit(&qfree[qb]);
        }
        if (!ok) break;
        mma_commit(&accdone[ab]);
      }
      if (issued) {  // every MMA issued has completed before TMEM is released
        mma_commit(&fin);
        mbar_wait(&fin, 0);
      }
    }
  } else if (warp < kMoProd) {
    // ---------------- math warps: q Z~ units (thread: sample rr of the unit, chunk group cq).
    const int rr = threadIdx.x & (kMoUnit - 1), cq = threadIdx.x / kMoUnit;
    bool ok = true;
    int gu = 0, it = 0;
    // item records are loaded one item ahead; the sample weights come with the ring stage
    MoItem m = blockIdx.x < nitems ? items[blockIdx.x] : MoItem{};
    MoItem mn = blockIdx.x + gridDim.x < nitems ? items[blockIdx.x + gridDim.x] : MoItem{};
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
      const int nu = (m.nrows + kMoUnit - 1) / kMoUnit;
      for (int u = 0; u < nu; ++u, ++gu) {
        const int st = gu % NS, qb = gu % NQ;
        const int k = u * kMoUnit + rr;  // sample within the item
        ok = ok && mbar_wait_ab(&full[st], (uint32_t)((gu / NS) & 1), abort);
        ok = ok && (gu < NQ || mbar_wait_ab(&qfree[qb], (uint32_t)(((gu / NQ) - 1) & 1), abort));
        ok = __all_sync(0xffffffffu, ok);  // one arrival per warp below
        if (ok) {
          const float q = k < m.nrows ? qs[st][rr] : 0.f;
          const unsigned char* zt = ring + st * SB;
          unsigned char* qh = qz + qb * QB;
          unsigned char* ql = qh + (STK ? kMoAtom : 2 * kMoAtom);
#pragma unroll
          for (int i = 0; i < CPT; ++i) {
            const int ch = cq * CPT + i;
            const uint32_t off = mo_off(rr, ch);
            const uint4 uh = *reinterpret_cast<const uint4*>(zt + off);
            const uint4 ul = *reinterpret_cast<const uint4*>(zt + ZL_OFF + off);
            const uint32_t wh[4] = {uh.x, uh.y, uh.z, uh.w}, wl[4] = {ul.x, ul.y, ul.z, ul.w};
            uint32_t hh[4], ll[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float2 fh = __half22float2(*reinterpret_cast<const __half2*>(&wh[e]));
              const float2 fl = __half22float2(*reinterpret_cast<const __half2*>(&wl[e]));
              split_pack2(q * (fh.x + fl.x), q * (fh.y + fl.y), hh[e], ll[e]);
            }
            *reinterpret_cast<uint4*>(qh + off) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
            *reinterpret_cast<uint4*>(ql + off) = make_uint4(ll[0], ll[1], ll[2], ll[3]);
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&qready[qb]);
        }
      }
      m = mn;
      if (item + 2 * gridDim.x < nitems) mn = items[item + 2 * gridDim.x];
    }
    if (!ok) set_timeout(D);
  } else {
    // ---------------- epilogue warps: every item, in item order, as soon as its accumulator
    // is complete (TMEM lane quarter = warp % 4; the four warps cover the four quarters).
    bool ok = true;
    // Epilogue of an item: TMEM lane a holds row a of M2 in columns [0, DP) (DP = 64: the sum
    // of column blocks [0, 64) and [64, 128), and lanes 64-127 the lo-half partial of row
    // a - 64) and entry a of zbar in column 128.  An item that covers its node stores M2 and
    // zbar (the lo-half partials pass through shared memory to the hi-half warps); a node split
    // over several items accumulates with atomics into the zeroed M2 / zbar.  Only rows and
    // columns < d are written: no reader looks past them.
    auto ld_m2 = [&](uint32_t acc, int g, float (&f)[32]) {  // 32 columns of M2, warp-collective
      uint32_t v[32];
      tmem_ld32(acc + g * 32, v);
      tmem_wait_ld();
#pragma unroll
      for (int c = 0; c < 32; ++c) f[c] = __uint_as_float(v[c]);
      if (STK) {
        tmem_ld32(acc + 64 + g * 32, v);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 32; ++c) f[c] += __uint_as_float(v[c]);
      }
    };
    auto ld_zbar = [&](uint32_t acc) {  // warp-collective
      uint32_t v[32];
      tmem_ld32(acc + 128, v);
      tmem_wait_ld();
      return __uint_as_float(v[0]);
    };
    auto epilogue = [&](const MoItem& m, int pit) {
      const int ab = pit & 1;
      ok = ok && mbar_wait_ab(&accdone[ab], (uint32_t)((pit >> 1) & 1), abort);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      const int quarter = warp & 3;
      const int abase = STK ? (quarter & 1) * 32 : quarter * 32;
      const int a = abase + lane;
      const bool lo_half = STK && quarter >= 2;
      const uint32_t acc = tb + ab * 256 + ((uint32_t)(quarter * 32) << 16);
      float* M2row = T.M2 + ((long long)m.node * kLdp + a) * kLdp;
      float* zb = T.zbar + (long long)m.node * kLdp;
      float* x = xs + ab * (kMoXBytes / 4);
      const bool combine = STK && m.whole;
      if (ok) tc_fence_after();
      if (combine) {
        if (ok && lo_half && abase < m.d) {
          for (int part = 0; part < DP / 32 && part * 32 < m.d; ++part) {
            float f[32];
            ld_m2(acc, part, f);
#pragma unroll
            for (int c4 = 0; c4 < 8; ++c4)
              *reinterpret_cast<float4*>(x + a * kMoXLd + part * 32 + c4 * 4) =
                  make_float4(f[4 * c4], f[4 * c4 + 1], f[4 * c4 + 2], f[4 * c4 + 3]);
          }
          x[64 * kMoXLd + a] = ld_zbar(acc);
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");  // every epilogue warp, whatever ok says
        if (ok && !lo_half && abase < m.d) {
          for (int part = 0; part < DP / 32 && part * 32 < m.d; ++part) {
            float f[32];
            ld_m2(acc, part, f);
            if (a < m.d)
#pragma unroll
              for (int c4 = 0; c4 < 8; ++c4)
                if (part * 32 + c4 * 4 < m.d) {
                  const float4 o = *reinterpret_cast<const float4*>(x + a * kMoXLd + part * 32 + c4 * 4);
                  *reinterpret_cast<float4*>(M2row + part * 32 + c4 * 4) =
                      make_float4(f[4 * c4] + o.x, f[4 * c4 + 1] + o.y, f[4 * c4 + 2] + o.z, f[4 * c4 + 3] + o.w);
                }
          }
          const float z = ld_zbar(acc);
          if (a < m.d) zb[a] = z + x[64 * kMoXLd + a];
        }
      } else {
        // (DP = 64: the scratch buffers are reused two items on, with this barrier between)
        if (STK) asm volatile("bar.sync 2, 128;" ::: "memory");
      }
      if (!combine && ok && abase < m.d) {  // warp-uniform
        for (int g = 0; g < DP / 32; ++g) {
          if (g * 32 >= m.d) break;
          float f[32];
          ld_m2(acc, g, f);
          if (a < m.d)
#pragma unroll
            for (int c4 = 0; c4 < 8; ++c4)
              if (g * 32 + c4 * 4 < m.d) {
                const float4 v4 = make_float4(f[4 * c4], f[4 * c4 + 1], f[4 * c4 + 2], f[4 * c4 + 3]);
                if (m.whole) *reinterpret_cast<float4*>(M2row + g * 32 + c4 * 4) = v4;
                else atomicAdd(reinterpret_cast<float4*>(M2row + g * 32 + c4 * 4), v4);
              }
        }
        const float z = ld_zbar(acc);
        if (a < m.d) {
          if (m.whole) zb[a] = z;
          else atomicAdd(zb + a, z);
        }
      }
      if (ok) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accfree[ab]);
      }
    };
    int it = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) epilogue(items[item], it);
    if (!ok) set_timeout(D);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMoProd + 1) {
    tc_fence_after();
    tmem_dealloc(tb, 512);
  }
}

// Zeroes the dp x d block of every node in a [node][128][128] array (the part the readers use:
// G_i = sum pi z~_p z~_i^T is d_parent x d_i; the adjoint launch adds its tile partials into it).
// Rows are zeroed in whole float4s (up to three entries past d, inside the 128-float row);
// NPB nodes per CTA.
template <int NPB>
__global__ void __launch_bounds__(256) k_zero_dd(Dev D, float* __restrict__ base) {
  constexpr int TPN = 256 / NPB;
  const int g = blockIdx.x * NPB + threadIdx.x / TPN, tid = threadIdx.x % TPN;
  if (g >= D.num_nodes) return;
  const int d4 = (D.nodes[g].d + 3) >> 2, dq = D.nodes[g].dp;
  float4* blk = reinterpret_cast<float4*>(base + (long long)g * kLdp * kLdp);
  for (int i = tid; i < dq * d4; i += TPN)
    blk[(i / d4) * (kLdp / 4) + i % d4] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// =======================================================================================
// Gradient assembly from the moments.  For the edge c (parent p):
//   db'_c = (zbar_c - W_c zbar_p - c_c) / var                      (= sum_k dmu_c[k])
//   D_c   = (G_c^T - W_c M2_p - c_c zbar_p^T) / var                (= sum_k dmu_c[k] z~_p^k^T)
//   dW_c  = grad_out (D_c + db'_c m_p^T),  dbias_c = grad_out db'_c
// and the edge's parts of the proposal-gradient sums of its two nodes:
//   child c  : sum_k' g = -db'_c,  sum_k' g z~ = (diag(W_c G_c) + c_c zbar_c - diag(M2_c)) / var
//   parent p : sum_k g = W_c^T db'_c,  sum_k g z~ = diag(W_c^T D_c)
// k_asm_edge_vec: one CTA (128 threads) per edge -- the vector quantities (db', child-side
// sums, parent-side sum_k g, dbias).  k_asm_edge_mat: (edge, 64x64 tile of D_c) -- the d x d
// part on the tiled FP32 GEMM (D_c needs W_c M2_p), dW and the parent-side diag(W_c^T D_c).
// =======================================================================================
__global__ void __launch_bounds__(128) k_asm_edge_vec(Dev D, TcDev T, const int* __restrict__ nonroot) {
  __shared__ float zp[kTcMaxD], dbs[kTcMaxD];
  const int g = nonroot[blockIdx.x];
  const NodeInfo nd = D.nodes[g];
  const int d = nd.d, dq = nd.dp;  // W_c is d x dq
  const float iv = D.inv_var;
  const float go = D.grad_out ? (float)D.grad_out[nd.b] : 1.f;
  const float* W = D.W + nd.off_W;
  const float* zbc = T.zbar + (long long)g * kLdp;
  const float* cc = T.cvec + (long long)g * kLdp;
  const int j = threadIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (j < dq) zp[j] = __ldg(T.zbar + (long long)nd.parent * kLdp + j);
  __syncthreads();
  // (W_c zbar_p)[r]: one warp per row, lanes along the row (coalesced)
  for (int r = w; r < d; r += 4) {
    float s = 0.f;
    for (int c = lane; c < dq; c += 32) s = fmaf(__ldg(W + (long long)r * dq + c), zp[c], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dbs[r] = (__ldg(zbc + r) - s - __ldg(cc + r)) * iv;
  }
  __syncthreads();
  if (j < d) {
    const float db = dbs[j];
    T.sgC[(long long)g * kLdp + j] = -db;
    if (D.shared) { if (D.pbias) D.pbias[nd.off_q + j] = go * db; }
    else if (D.dbias) D.dbias[nd.off_bias + j] = go * db;
  }
  // (W^T db')[j] = sum_a W[a][j] db'[a] (coalesced over j, j < dq).  The child-side sum of
  // g z~ is diag(W_c G_c) / var (k_asm_edge_mat, which holds both tiles, into the zeroed tgC)
  // plus (c_c zbar_c - diag M2_c) / var (added by k_asm_node)
  if (j >= dq) return;
  float sg = 0.f;
  for (int a = 0; a < d; ++a) sg = fmaf(__ldg(W + (long long)a * dq + j), dbs[a], sg);
  T.sgP[(long long)g * kLdp + j] = sg;
}

// Grid: (edge, 64x64 tile of D_c (2 x 2)).  The W_c and G_c^T tiles are staged through
// shared memory (coalesced reads of both); row sums of W_c o G_c^T give diag(W_c G_c), column
// sums of W_c o D_c give diag(W_c^T D_c).
__global__ void __launch_bounds__(kThreads) k_asm_edge_mat(Dev D, TcDev T, const int* __restrict__ nonroot) {
  __shared__ TileSmem sm;
  __shared__ float sW[kTile][kTile + 1], sG[kTile][kTile + 1];
  __shared__ float colpart[16][kTile + 1];
  const int g = nonroot[blockIdx.x];
  const NodeInfo nd = D.nodes[g];
  const NodeInfo pn = D.nodes[nd.parent];
  const int d = nd.d, dq = nd.dp;  // D_c and W_c are d x dq, G_c is dq x d
  const int a0 = (blockIdx.y >> 1) * kTile, b0 = (blockIdx.y & 1) * kTile;
  if (a0 >= d || b0 >= dq) return;
  const float iv = D.inv_var;
  const float go = D.grad_out ? (float)D.grad_out[nd.b] : 1.f;
  const float* W = D.W + nd.off_W;
  const float* Gc = T.G + (long long)g * kLdp * kLdp;
  const float* M2p = T.M2 + (long long)nd.parent * kLdp * kLdp;
  const float* zbp = T.zbar + (long long)nd.parent * kLdp;
  const float* cc = T.cvec + (long long)g * kLdp;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  // sW[r][c] = W[a0 + r][b0 + c],  sG[r][c] = G[b0 + r][a0 + c]  (so G^T[a][b] = sG[b][a]);
  // every load of the stage is issued before the first shared-memory store
  {
    constexpr int NV = kTile * kTile / kThreads;
    float wv[NV], gv[NV];
#pragma unroll
    for (int x = 0; x < NV; ++x) {
      const int e = threadIdx.x + x * kThreads, r = e >> 6, c = e & 63;
      wv[x] = (a0 + r < d && b0 + c < dq) ? __ldg(W + (long long)(a0 + r) * dq + b0 + c) : 0.f;
      gv[x] = (b0 + r < dq && a0 + c < d) ? __ldg(Gc + (long long)(b0 + r) * kLdp + a0 + c) : 0.f;
    }
#pragma unroll
    for (int x = 0; x < NV; ++x) {
      const int e = threadIdx.x + x * kThreads, r = e >> 6, c = e & 63;
      sW[r][c] = wv[x];
      sG[r][c] = gv[x];
    }
  }
  float acc[4][4];
  zero_acc(acc);
  // acc[a][b] = sum_j W[a][j] M2_p[j][b]   (tile_gemm synchronises before its first read)
  tile_gemm<true, false>(acc, W + (long long)a0 * dq, dq, min(kTile, d - a0), M2p + b0, kLdp,
                         min(kTile, dq - b0), dq, sm);
  float tcol[4] = {0.f, 0.f, 0.f, 0.f};
  float wrow[4] = {0.f, 0.f, 0.f, 0.f};
  // every vector operand of the epilogue in registers before the first store
  float dbv[4], cav[4], zpv[4], mpv[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i, bb = b0 + tx * 4 + i;
    dbv[i] = a < d ? -__ldg(T.sgC + (long long)g * kLdp + a) : 0.f;  // db'[a], from k_asm_edge_vec
    cav[i] = a < d ? __ldg(cc + a) : 0.f;
    zpv[i] = bb < dq ? __ldg(zbp + bb) : 0.f;
    mpv[i] = bb < dq ? __ldg(D.q_mean + pn.off_q + bb) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int al = ty * 4 + i, a = a0 + al;
    const float db = dbv[i], ca = cav[i];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int bl = tx * 4 + jj, bb = b0 + bl;
      if (a >= d || bb >= dq) continue;
      const float wab = sW[al][bl], gt = sG[bl][al];
      const float Dab = (gt - acc[i][jj] - ca * zpv[jj]) * iv;
      tcol[jj] = fmaf(wab, Dab, tcol[jj]);
      wrow[i] = fmaf(wab, gt, wrow[i]);
      const float v = go * (Dab + db * mpv[jj]);
      if (D.shared) { if (D.pW) D.pW[nd.off_pW + (long long)a * dq + bb] = v; }
      else if (D.dW) D.dW[nd.off_W + (long long)a * dq + bb] = v;
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {  // the 16 threads of one ty sit in one half-warp
    float v = wrow[i];
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int a = a0 + ty * 4 + i;
    // two column tiles per row into a zeroed entry: the two additions commute exactly
    if (tx == 0 && a < d) atomicAdd(T.tgC + (long long)g * kLdp + a, v * iv);
  }
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) colpart[ty][tx * 4 + jj] = tcol[jj];
  __syncthreads();
  if (threadIdx.x < kTile && b0 + threadIdx.x < dq) {
    float s = 0.f;
    for (int i = 0; i < 16; ++i) s += colpart[i][threadIdx.x];
    atomicAdd(T.tgP + (long long)g * kLdp + b0 + threadIdx.x, s);
  }
}

// ---- shared parameters: every instance uses the same W_c ---------------------------------
// The W_c M2_p term of dW_c is linear in M2_p, so it is applied once to the instance sum:
//   dW_c = sum_b go_b [(G_c,b^T - c_c,b zbar_p,b^T) / var + db'_c,b m_p,b^T]
//          - W_c (sum_b go_b M2_p,b) / var
// and the parent-side sum of each instance needs only O(d^2) work given W_c^T W_c (symmetric,
// as is M2_p):
//   diag(W_c^T D_c,b)[j] = (sum_a W[a][j] (G^T[a][j] - c_a zbar_p[j]) - sum_l (W^T W)[l][j] M2_p[l][j]) / var
// so no d x d x d product is formed per instance.  Positions are the local indices 1 .. n-1
// of the instances' common graph (local index = global id in instance 0).
constexpr int kAsmInst = 8;  // instances per group of k_asm_shared (group sums in a fixed order)

// W_c^T W_c per position.  Grid: (position, 64 x 64 tile (2 x 2)).
__global__ void __launch_bounds__(kThreads) k_wtw(Dev D, TcDev T) {
  __shared__ TileSmemDeep sm;
  const int i = blockIdx.x + 1;
  const NodeInfo nd = D.nodes[i];
  const int d = nd.d, dq = nd.dp;  // W_c is d x dq
  const int l0 = (blockIdx.y >> 1) * kTile, j0 = (blockIdx.y & 1) * kTile;
  if (l0 >= dq || j0 >= dq) return;
  const float* W = D.W + nd.off_W;
  float acc[4][4];
  zero_acc(acc);
  // acc[l][j] = sum_a W[a][l] W[a][j]
  tile_gemm_deep<false, false>(acc, W + l0, dq, min(kTile, dq - l0), W + j0, dq, min(kTile, dq - j0), d, sm);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float* out = T.WtW + (long long)i * kLdp * kLdp;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int l = l0 + ty * 4 + a, j = j0 + tx * 4 + b;
      if (l < dq && j < dq) out[(long long)l * kLdp + j] = acc[a][b];
    }
}

// Grid: (position, 64 x 64 tile (2 x 2), instance group of kAsmInst).  Per instance of the
// group: the child- and parent-side sums of the edge (tgC, tgP) and, summed over the group's
// instances in order, the dW terms without W_c M2_p (into Ppart) and go M2_p / var (into
// Spart).  Thread (ty, tx) holds rows a0 + 4 ty .. +3 (child index a of W_c and G_c^T, and
// parent index l of M2_p) and columns b0 + 4 tx .. +3 (parent index j).  The instances'
// offsets are read once into shared memory, only the edge's own rows and columns are loaded,
// and the column sums of every instance are formed after one barrier at the end.
__global__ void __launch_bounds__(kThreads, 2) k_asm_shared(Dev D, TcDev T, long long nW, long long nS) {
  __shared__ float colpart[kAsmInst][16][kTile + 1];
  __shared__ int s_n0[kAsmInst];
  __shared__ long long s_offq[kAsmInst];
  __shared__ float s_go[kAsmInst];
  const int i = blockIdx.x + 1;
  const NodeInfo nd = D.nodes[i];
  const int d = nd.d, dq = nd.dp, pi = nd.parent;  // local index of the parent = its id in instance 0
  const int a0 = (blockIdx.y >> 1) * kTile, b0 = (blockIdx.y & 1) * kTile;
  if (b0 >= dq || a0 >= max(d, dq)) return;
  const int bb = blockIdx.z * kAsmInst, nb = min(D.num_inst - bb, kAsmInst);
  if (threadIdx.x < nb) {
    const int b = bb + threadIdx.x, n0 = D.insts[b].node0;
    s_n0[threadIdx.x] = n0;
    s_offq[threadIdx.x] = D.nodes[n0 + pi].off_q;
    s_go[threadIdx.x] = D.grad_out ? (float)D.grad_out[b] : 1.f;
  }
  const float iv = D.inv_var;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int ar = a0 + ty * 4, jc = b0 + tx * 4;  // first row / column of the thread
  const float* W = D.W + nd.off_W;
  const float* WtW = T.WtW + (long long)i * kLdp * kLdp;
  float wv[4][4], ww[4][4], pw[4][4], s2[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int a = ar + r, j = jc + c;
      wv[r][c] = (a < d && j < dq) ? __ldg(W + (long long)a * dq + j) : 0.f;
      ww[r][c] = (a < dq && j < dq) ? __ldg(WtW + (long long)a * kLdp + j) : 0.f;
      pw[r][c] = 0.f;
      s2[r][c] = 0.f;
    }
  // loads stay inside the nodes' 128 x 128 blocks; entries outside the edge's sizes are
  // not used (the workspace there is not initialised)
  const bool g_rows = ar < d, m_cols = jc < dq;
  __syncthreads();
  for (int u = 0; u < nb; ++u) {
    const int gc = s_n0[u] + i, gp = s_n0[u] + pi;
    const float go = s_go[u];
    const float* Gc = T.G + (long long)gc * kLdp * kLdp;
    const float* M2p = T.M2 + (long long)gp * kLdp * kLdp;
    // G^T[a][j] = G[j][a]: four consecutive a per column j; M2_p[l][j]: four consecutive j per row l
    float4 gq[4], mq[4];
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      gq[c] = (g_rows && jc + c < dq) ? __ldg(reinterpret_cast<const float4*>(Gc + (long long)(jc + c) * kLdp + ar)) : z4;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      mq[r] = (m_cols && ar + r < dq) ? __ldg(reinterpret_cast<const float4*>(M2p + (long long)(ar + r) * kLdp + jc)) : z4;
    const float4 ca4 = g_rows ? __ldg(reinterpret_cast<const float4*>(T.cvec + (long long)gc * kLdp + ar)) : z4;
    const float4 db4 = g_rows ? __ldg(reinterpret_cast<const float4*>(T.sgC + (long long)gc * kLdp + ar)) : z4;
    const float4 zp4 = m_cols ? __ldg(reinterpret_cast<const float4*>(T.zbar + (long long)gp * kLdp + jc)) : z4;
    float mpv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) mpv[k] = jc + k < dq ? __ldg(D.q_mean + s_offq[u] + jc + k) : 0.f;
    const float cav[4] = {ca4.x, ca4.y, ca4.z, ca4.w};
    const float dbv[4] = {-db4.x, -db4.y, -db4.z, -db4.w};  // db'[a] = -sgC, from k_asm_edge_vec
    const float zpv[4] = {zp4.x, zp4.y, zp4.z, zp4.w};
    const float giv = go * iv;
    float wrow[4] = {0.f, 0.f, 0.f, 0.f}, tcol[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int a = ar + r, j = jc + c;
        const float gt = (a < d && j < dq) ? (&gq[c].x)[r] : 0.f;
        const float m2 = (a < dq && j < dq) ? (&mq[r].x)[c] : 0.f;
        const float ca = a < d ? cav[r] : 0.f, db = a < d ? dbv[r] : 0.f;
        const float zp = j < dq ? zpv[c] : 0.f;
        const float dp = (gt - ca * zp) * iv;
        pw[r][c] = fmaf(go, fmaf(db, mpv[c], dp), pw[r][c]);
        s2[r][c] = fmaf(giv, m2, s2[r][c]);
        wrow[r] = fmaf(wv[r][c], gt, wrow[r]);
        tcol[c] = fmaf(wv[r][c], dp, fmaf(-ww[r][c] * iv, m2, tcol[c]));
      }
#pragma unroll
    for (int r = 0; r < 4; ++r) {  // the 16 threads of one ty sit in one half-warp
      float v = wrow[r];
      for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      // two column tiles per row into a zeroed entry: the two additions commute exactly
      if (tx == 0 && ar + r < d) atomicAdd(T.tgC + (long long)gc * kLdp + ar + r, v * iv);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) colpart[u][ty][tx * 4 + c] = tcol[c];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < nb * kTile; x += kThreads) {
    const int u = x / kTile, col = x % kTile;
    if (b0 + col >= dq) continue;
    float v = 0.f;
    for (int r = 0; r < 16; ++r) v += colpart[u][r][col];
    atomicAdd(T.tgP + (long long)(s_n0[u] + i) * kLdp + b0 + col, v);  // two row tiles, as above
  }
  float* pp = T.Ppart + (long long)blockIdx.z * nW + nd.off_W;
  float* sp = T.Spart + (long long)blockIdx.z * nS + nd.off_S;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int a = ar + r, j = jc + c;
      if (j >= dq) continue;
      if (a < d) pp[(long long)a * dq + j] = pw[r][c];
      if (a < dq) sp[(long long)a * dq + j] = s2[r][c];
    }
}

// dW_c = P_c - W_c S2_c.  Grid: (position, 64 x 64 tile (2 x 2)).
__global__ void __launch_bounds__(kThreads) k_shared_dw(Dev D, TcDev T) {
  __shared__ TileSmemDeep sm;
  const int i = blockIdx.x + 1;
  const NodeInfo nd = D.nodes[i];
  const int d = nd.d, dq = nd.dp;
  const int a0 = (blockIdx.y >> 1) * kTile, b0 = (blockIdx.y & 1) * kTile;
  if (a0 >= d || b0 >= dq) return;
  const float* W = D.W + nd.off_W;
  const float* S2 = T.S2 + nd.off_S;
  float acc[4][4];
  zero_acc(acc);
  // acc[a][j] = sum_l W[a][l] S2[l][j]
  tile_gemm_deep<true, false>(acc, W + (long long)a0 * dq, dq, min(kTile, d - a0), S2 + b0, dq,
                         min(kTile, dq - b0), dq, sm);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int a = a0 + ty * 4 + r, j = b0 + tx * 4 + c;
      if (a >= d || j >= dq) continue;
      const long long e = nd.off_W + (long long)a * dq + j;
      D.dW[e] = T.P[e] - acc[r][c];
    }
}

// C^T C per distinct observation matrix (one for shared parameters, else one per instance).
// Grid: (matrix, 64x64 tile (2 x 2), 64-row slab of C); slabs add into the zeroed C^T C.
__global__ void __launch_bounds__(kThreads) k_ctc(Dev D, TcDev T) {
  __shared__ TileSmemDeep sm;
  const InstInfo in = D.insts[blockIdx.x];
  const int d = in.d, obs = in.obs;
  const int a0 = (blockIdx.y >> 1) * kTile, b0 = (blockIdx.y & 1) * kTile, o0 = blockIdx.z * kTile;
  if (a0 >= d || b0 >= d || o0 >= obs) return;
  const float* C = D.C + in.off_C + (long long)o0 * d;
  float acc[4][4];
  zero_acc(acc);
  tile_gemm_deep<false, false>(acc, C + a0, d, min(kTile, d - a0), C + b0, d, min(kTile, d - b0),
                          min(kTile, obs - o0), sm);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float* out = T.CtC + (long long)blockIdx.x * kLdp * kLdp;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = a0 + ty * 4 + i, b = b0 + tx * 4 + j;
      if (a < d && b < d) atomicAdd(out + (long long)a * kLdp + b, acc[i][j]);
    }
}

// Node sums and outputs: dm_i = grad_out * Sg,  dlogs_i = grad_out * (sum_k q_i + Tg), with
//   Sg, Tg = [edge as child] + sum over child edges + [root prior] + [leaf observation]
//   root : Sg -= (zbar + m_0 - bias_0)/var,  Tg -= (diag M2 + (m_0 - bias_0) zbar)/var,
//          dbias_0 = grad_out (zbar + m_0 - bias_0)/var
//   leaf : Sg += C^T (x~ - C zbar)/obs_var,  Tg += ((C^T x~) zbar - diag(C^T C M2))/obs_var
// One CTA of P x 128 threads per node: thread (part, j) owns latent entry j; with P > 1 the
// leaf sums over the observation rows and over C^T C's rows are split P ways and reduced in
// shared memory, so wide leaves do not run long serial loops.
template <int P>
__global__ void __launch_bounds__(P * kTcMaxD) k_asm_node(Dev D, TcDev T) {
  __shared__ float xs[kMaxD];
  __shared__ float zb[kTcMaxD], ctx[kTcMaxD];
  __shared__ float qred[P * kTcMaxD / 32];
  __shared__ float part_a[P][kTcMaxD], part_b[P][kTcMaxD];
  const int g = blockIdx.x;
  const NodeInfo nd = D.nodes[g];
  const int d = nd.d, K = nd.K;
  const float go = D.grad_out ? (float)D.grad_out[nd.b] : 1.f;
  const float* M2 = T.M2 + (long long)g * kLdp * kLdp;
  const int tid = threadIdx.x, j = tid % kTcMaxD, part = tid / kTcMaxD;
  float qs = 0.f;
#pragma unroll 4
  for (int k = tid; k < K; k += P * kTcMaxD) qs += __ldg(D.q + nd.off_nk + k);
  for (int o = 16; o > 0; o >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, o);
  if ((tid & 31) == 0) qred[tid >> 5] = qs;
  if (part == 0 && j < d) zb[j] = __ldg(T.zbar + (long long)g * kLdp + j);
  const bool leaf = nd.leaf_slot >= 0, root = nd.parent < 0;
  if (leaf)  // x~ = x - C m, formed in the forward pass
    for (int o = tid; o < nd.obs; o += P * kTcMaxD) xs[o] = __ldg(T.xs + nd.off_x + o);
  __syncthreads();
  float qtot = 0.f;
#pragma unroll
  for (int w = 0; w < P * kTcMaxD / 32; ++w) qtot += qred[w];
  float czb = 0.f, dg = 0.f;
  if (leaf) {
    // (C^T x~)[j] over this part's observation rows
    float s0 = 0.f, s1 = 0.f;
    if (j < d) {
      const int ob = (nd.obs * part) / P, oe = (nd.obs * (part + 1)) / P;
      const float* c = D.C + nd.off_C + j;
      int o = ob;
#pragma unroll 4
      for (; o + 1 < oe; o += 2) {
        s0 = fmaf(__ldg(c + (long long)o * d), xs[o], s0);
        s1 = fmaf(__ldg(c + (long long)(o + 1) * d), xs[o + 1], s1);
      }
      if (o < oe) s0 = fmaf(__ldg(c + (long long)o * d), xs[o], s0);
      // (C^T C zbar)[j] and (C^T C M2)[j][j] over this part's rows of C^T C (symmetric: row
      // j read as column j, coalesced over threads)
      const float* ctc = T.CtC + (long long)(D.shared ? 0 : nd.b) * kLdp * kLdp;
      const int ab = (d * part) / P, ae = (d * (part + 1)) / P;
#pragma unroll 4
      for (int a = ab; a < ae; ++a) {
        const float v = __ldg(ctc + (long long)a * kLdp + j);
        czb = fmaf(v, zb[a], czb);
        dg = fmaf(v, __ldg(M2 + (long long)a * kLdp + j), dg);
      }
    }
    if (P == 1) {
      ctx[j] = s0 + s1;
    } else {
      part_a[part][j] = s0 + s1;
      part_b[part][j] = czb;
      __syncthreads();
      if (part == 0) {
        float c = 0.f, z = 0.f;
#pragma unroll
        for (int q = 0; q < P; ++q) {
          c += part_a[q][j];
          z += part_b[q][j];
        }
        ctx[j] = c;
        czb = z;
      }
      __syncthreads();  // part_a reused for dg
      part_a[part][j] = dg;
      __syncthreads();
      if (part == 0) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < P; ++q) t += part_a[q][j];
        dg = t;
      }
    }
  }
  // the children's edge sums (a node may have thousands of children): thread t takes entry
  // t % d of children t / d, t / d + G, ... (G = blockDim / d); the partials are then summed in
  // a fixed order (a node with children is no leaf, so part_a / part_b are free)
  float csg = 0.f, ctg = 0.f;
  if (nd.child_end > nd.child_begin) {
    const int G = (P * kTcMaxD) / d, jj = tid % d, grp = tid / d;
    float* pa = &part_a[0][0];
    float* pb = &part_b[0][0];
    float a = 0.f, b = 0.f;
    if (grp < G)
#pragma unroll 4
      for (int ci = nd.child_begin + grp; ci < nd.child_end; ci += G) {
        const int c = D.children[ci];
        a += T.sgP[(long long)c * kLdp + jj];
        b += T.tgP[(long long)c * kLdp + jj];
      }
    if (grp < G) {
      pa[grp * d + jj] = a;
      pb[grp * d + jj] = b;
    }
    __syncthreads();
    if (part == 0 && j < d)
      for (int g2 = 0; g2 < G; ++g2) {
        csg += pa[g2 * d + j];
        ctg += pb[g2 * d + j];
      }
  }
  if (part != 0 || j >= d) return;
  float Sg = csg, Tg = ctg;
  if (!root) {
    Sg += T.sgC[(long long)g * kLdp + j];
    Tg += T.tgC[(long long)g * kLdp + j] +
          (T.cvec[(long long)g * kLdp + j] * zb[j] - M2[(long long)j * kLdp + j]) * D.inv_var;
  }
  if (root) {
    const float off = D.q_mean[nd.off_q + j] - D.bias[nd.off_bias + j];
    const float t = zb[j] + off;
    Sg -= t * D.inv_var;
    Tg -= (M2[(long long)j * kLdp + j] + off * zb[j]) * D.inv_var;
    const float db = go * t * D.inv_var;
    if (D.shared) { if (D.pbias) D.pbias[nd.off_q + j] = db; }
    else if (D.dbias) D.dbias[nd.off_bias + j] = db;
    if (!D.shared && D.dW)  // the root has no incoming edge: its W slot gets zero
      for (int e = j; e < d * d; e += d) D.dW[nd.off_W + e] = 0.f;
  }
  if (leaf) {
    Sg += (ctx[j] - czb) * D.inv_obs_var;
    Tg += (ctx[j] * zb[j] - dg) * D.inv_obs_var;
  }
  if (D.dq_mean) D.dq_mean[nd.off_q + j] = go * Sg;
  if (D.dq_logstd) D.dq_logstd[nd.off_q + j] = go * (qtot + Tg);
}

// dC = grad_out / obs_var * sum_leaves [ x~ (zbar + m)^T - C (M2 + zbar m^T) ]
//    = grad_out / obs_var * ( X - C S ),   X = sum_l x~_l (zbar_l + m_l)^T,
//                                          S = sum_l (M2_l + zbar_l m_l^T)   (d x d)
// k_leaf_S: grid (instance, 64x64 tile of S (2 x 2)).
// A tile with fewer entries than threads (small d) splits the leaves instead: thread t takes
// entry t % np of leaves t / np, t / np + G, ... (G = threads / np), and the group partials are
// summed in a fixed order -- an instance may have thousands of leaves.
__device__ __forceinline__ float leaf_S_entry(const Dev& D, const TcDev& T, const LeafInfo& li, int a, int c) {
  return __ldg(T.M2 + ((long long)li.node * kLdp + a) * kLdp + c) +
         __ldg(T.zbar + (long long)li.node * kLdp + a) * __ldg(D.q_mean + li.off_q + c);
}
__global__ void __launch_bounds__(kThreads) k_leaf_S(Dev D, TcDev T) {
  __shared__ float part[kThreads];
  const InstInfo in = D.insts[blockIdx.x];
  const int d = in.d;
  const int a0 = (blockIdx.y >> 1) * kTile, b0 = (blockIdx.y & 1) * kTile;
  if (a0 >= d || b0 >= d) return;
  const int rt = min(kTile, d - a0), ct = min(kTile, d - b0), np = rt * ct;
  // shared C: go_b S_b / obs_var, packed d x d (its instance sum multiplies C once); else S_b
  const bool sh = D.shared != 0;
  const long long ld = sh ? d : kLdp;
  const float sc = sh ? (D.grad_out ? (float)D.grad_out[blockIdx.x] : 1.f) * D.inv_obs_var : 1.f;
  float* S = T.S + (long long)blockIdx.x * (sh ? (long long)d * d : (long long)kLdp * kLdp);
  if (np < kThreads) {
    const int G = kThreads / np, e = threadIdx.x % np, grp = threadIdx.x / np;
    const int a = a0 + e / ct, cc = b0 + e % ct;
    float acc = 0.f;
    if (grp < G)
#pragma unroll 4
      for (int l = T.leaf_off[blockIdx.x] + grp; l < T.leaf_off[blockIdx.x + 1]; l += G)
        acc += leaf_S_entry(D, T, T.leaf_info[l], a, cc);
    if (grp < G) part[grp * np + e] = acc;
    __syncthreads();
    if (threadIdx.x < np) {
      float v = 0.f;
      for (int g = 0; g < G; ++g) v += part[g * np + threadIdx.x];
      S[(long long)a * ld + cc] = sh ? v * sc : v;
    }
    return;
  }
  const int c = threadIdx.x & 63, r0 = threadIdx.x >> 6;  // 4 rows per pass, column c
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
#pragma unroll 2
  for (int l = T.leaf_off[blockIdx.x]; l < T.leaf_off[blockIdx.x + 1]; ++l) {
    const LeafInfo li = T.leaf_info[l];
    const int gi = li.node;
    const float* M2 = T.M2 + (long long)gi * kLdp * kLdp;
    const float* zb = T.zbar + (long long)gi * kLdp;
    const float mb = b0 + c < d ? __ldg(D.q_mean + li.off_q + b0 + c) : 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int a = a0 + r0 + 4 * i;
      if (a < d && b0 + c < d) acc[i] += __ldg(M2 + (long long)a * kLdp + b0 + c) + __ldg(zb + a) * mb;
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int a = a0 + r0 + 4 * i;
    if (a < d && b0 + c < d) S[(long long)a * ld + b0 + c] = sh ? acc[i] * sc : acc[i];
  }
}

// Grid: (instance, 64-row tile of observation dims, 64-col tile of latent dims).
// X = sum_leaves x~ (zbar + m)^T is split over the leaves like k_leaf_S when the tile has
// fewer entries than threads.
__global__ void __launch_bounds__(kThreads) k_asm_dC(Dev D, TcDev T) {
  __shared__ TileSmem sm;
  __shared__ float part[kThreads];
  const InstInfo in = D.insts[blockIdx.x];
  const int d = in.d, obs = in.obs;
  const int o0 = blockIdx.y * kTile, c0 = blockIdx.z * kTile;
  if (o0 >= obs || c0 >= d) return;
  const int rows = min(kTile, obs - o0), cols = min(kTile, d - c0);
  const float go = D.grad_out ? (float)D.grad_out[blockIdx.x] : 1.f;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const float* C = D.C + in.off_C;
  float acc[4][4];
  zero_acc(acc);
  // acc = C[o0.., :] S[:, c0..]; a shared C multiplies the instance sum of S once (k_shared_dC)
  if (!D.shared)
    tile_gemm<true, false>(acc, C + (long long)o0 * d, d, rows, T.S + (long long)blockIdx.x * kLdp * kLdp + c0,
                           kLdp, cols, d, sm);
  float X[4][4];
  zero_acc(X);
  const int np = rows * cols;
  if (np < kThreads) {
    const int G = kThreads / np, e = threadIdx.x % np, grp = threadIdx.x / np;
    const int o = o0 + e / cols, c = c0 + e % cols;
    float x = 0.f;
    if (grp < G)
#pragma unroll 4
      for (int l = T.leaf_off[blockIdx.x] + grp; l < T.leaf_off[blockIdx.x + 1]; l += G) {
        const LeafInfo li = T.leaf_info[l];
        x += __ldg(T.xs + li.off_x + o) *
             (__ldg(T.zbar + (long long)li.node * kLdp + c) + __ldg(D.q_mean + li.off_q + c));
      }
    if (grp < G) part[grp * np + e] = x;
    __syncthreads();
    if (threadIdx.x < np) {
      float v = 0.f;
      for (int g = 0; g < G; ++g) v += part[g * np + threadIdx.x];
      part[threadIdx.x] = v;  // each thread rewrites only its own group-0 entry after reading
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int oo = ty * 4 + i, cc = tx * 4 + j;
        if (oo < rows && cc < cols) X[i][j] = part[oo * cols + cc];
      }
  } else
#pragma unroll 2
  for (int l = T.leaf_off[blockIdx.x]; l < T.leaf_off[blockIdx.x + 1]; ++l) {
    const LeafInfo li = T.leaf_info[l];
    const int gi = li.node;
    float xo[4], zm[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int o = o0 + ty * 4 + i;
      xo[i] = o < obs ? __ldg(T.xs + li.off_x + o) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      zm[j] = c < d ? __ldg(T.zbar + (long long)gi * kLdp + c) + __ldg(D.q_mean + li.off_q + c) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) X[i][j] = fmaf(xo[i], zm[j], X[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = o0 + ty * 4 + i, c = c0 + tx * 4 + j;
      if (o >= obs || c >= d) continue;
      const float v = go * (X[i][j] - acc[i][j]) * D.inv_obs_var;
      if (D.shared) { if (D.pC) D.pC[in.off_pC + (long long)o * d + c] = v; }
      else if (D.dC) D.dC[in.off_C + (long long)o * d + c] = v;
    }
}

// Shared C: dC = sum_b go_b X_b / obs_var (already in dC) - C Ssum, Ssum = sum_b go_b S_b / obs_var.
// Grid: (64-row tile of observation dims, 64-col tile of latent dims).
__global__ void __launch_bounds__(kThreads) k_shared_dC(Dev D, TcDev T) {
  __shared__ TileSmemDeep sm;
  const InstInfo in = D.insts[0];
  const int d = in.d, obs = in.obs;
  const int o0 = blockIdx.x * kTile, c0 = blockIdx.y * kTile;
  if (o0 >= obs || c0 >= d) return;
  const int rows = min(kTile, obs - o0), cols = min(kTile, d - c0);
  float acc[4][4];
  zero_acc(acc);
  tile_gemm_deep<true, false>(acc, D.C + (long long)o0 * d, d, rows, T.Ssum + c0, d, cols, d, sm);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = o0 + ty * 4 + i, c = c0 + tx * 4 + j;
      if (o < obs && c < d) D.dC[(long long)o * d + c] -= acc[i][j];
    }
}

// =======================================================================================
// host side
// =======================================================================================
namespace {
typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
  }
  return fn;
}

// [rows][128] fp16 array, box 64 columns x 128 rows, 128-byte swizzle.
// [rows][128] fp32 array, box 32 columns x 128 rows, 128-byte swizzle (the G / M2 reductions).
bool make_map_f32(CUtensorMap* m, void* ptr, long long rows) {
  EncodeFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kLdp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kLdp * 4};
  cuuint32_t box[2] = {32, (cuuint32_t)kRows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_map(CUtensorMap* m, void* ptr, long long rows, int box_rows = kRows) {
  EncodeFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kLdp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kLdp * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ptr, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Dynamic shared memory, at least half of the SM's: one CTA per SM, so the 512-column TMEM
// allocation never waits on a co-resident CTA.
// Dynamic shared memory of the forward kernel: the ring, then one or two cb buffers of the
// longest K (two when they fit beside the ring: warp 3 then prepares item j + 1's vector
// while the math warps use item j's).  At least half of the SM's, so one CTA per SM holds
// the 512-column TMEM allocation.
template <int DP>
size_t fwd_smem(int maxK, int* ncb_out = nullptr, int* cbk_out = nullptr) {
  const int cbk = tiles_of(maxK) * kRows;
  const size_t ring = (size_t)FwdCfg<DP>::NS * 2 * FwdCfg<DP>::TB;
  const size_t limit = 232448 - 8 * 1024;  // opt-in maximum less a margin for static shared memory
  const int ncb = (1024 + ring + 2 * (size_t)cbk * 4 <= limit) ? 2 : 1;
  if (ncb_out) *ncb_out = ncb;
  if (cbk_out) *cbk_out = cbk;
  const size_t need = 1024 + ring + (size_t)ncb * cbk * 4;
  return need > 120 * 1024 ? need : 120 * 1024;
}
template <int DP>
size_t obs_smem() {
  return 1024 + 4 * (size_t)(kRows * DP * 2) + sizeof(float) * kMaxD;
}
template <int DP>
size_t bwd_smem(int maxK) {
  const size_t need = 1024 + ring_bytes(DP) +
                      4 * (size_t)(((maxK + kRows - 1) / kRows) * kRows);
  return need > 120 * 1024 ? need : 120 * 1024;
}
}  // namespace

// Edge tiles of both persistent launches in dependency order (every tile's dependencies sit
// at an earlier level, hence earlier in the list).  Within a level:
//   schedule 0: instance by instance (the tiles of one edge are adjacent)
//   schedule 1: tile index major (tile r of every edge, then tile r+1, ...)
//   schedule 2: instances with more edge work first
void build_items(TcWork& w, const std::vector<NodeInfo>& nodes, int schedule) {
  w.tiles.clear();
  w.schedule = schedule;
  std::vector<double> work(w.num_inst, 0.0);
  for (const NodeInfo& nd : nodes)
    if (nd.parent >= 0) work[nd.b] += (double)nd.Kp * nd.K * nd.d;
  // rows of an edge's tiles: the parent's samples (forward, row pass) or the child's (adjoint)
  auto rows_of = [&](int dir, int g) { return dir == 1 ? nodes[g].K : nodes[g].Kp; };
  for (int dir = 0; dir < 3; ++dir)
    for (int c = 0; c < 2; ++c) {
      w.it_b[dir][c] = (int)w.tiles.size();
      for (int step = 0; step < w.maxlevel; ++step) {
        const int L = dir == 0 ? w.maxlevel - step : 1 + step;
        std::vector<int> lv;
        for (int g = 0; g < (int)nodes.size(); ++g)
          if (nodes[g].level == L && (w.inst_dp[nodes[g].b] > 64 ? 1 : 0) == c) lv.push_back(g);
        if (schedule == 2)
          std::stable_sort(lv.begin(), lv.end(), [&](int x, int y) { return work[nodes[x].b] > work[nodes[y].b]; });
        if (schedule == 1) {
          for (int r = 0;; r += kRows) {
            bool any = false;
            for (int g : lv)
              if (r < rows_of(dir, g) && !(dir == 0 && g == w.stall_node)) {
                w.tiles.push_back(Tile{g, r});
                any = true;
              }
            if (!any) break;
          }
        } else {
          for (int g : lv)
            if (!(dir == 0 && g == w.stall_node))  // (the stall fault drops one node's tiles)
              for (int r = 0; r < rows_of(dir, g); r += kRows) w.tiles.push_back(Tile{g, r});
        }
      }
      w.it_e[dir][c] = (int)w.tiles.size();
    }
}

tmc_status set_schedule(TcWork& w, const std::vector<NodeInfo>& nodes, int schedule) {
  if (schedule < 0 || schedule > 2) return TMC_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return TMC_ERR_CUDA;
  build_items(w, nodes, schedule);
  if (!w.tiles.empty() &&
      cudaMemcpy(w.d_tiles, w.tiles.data(), sizeof(Tile) * w.tiles.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return TMC_ERR_CUDA;
  return TMC_OK;
}

tmc_status supported(const std::vector<NodeInfo>& nodes, int precision) {
  if (precision != TMC_PREC_FP16_TC) return TMC_ERR_UNSUPPORTED;  // split-fp16 kernels only
  for (const NodeInfo& nd : nodes)
    if (nd.d > kTcMaxD || nd.K > kTcMaxK) return TMC_ERR_UNSUPPORTED;
  return TMC_OK;
}

void workspace_layout(TcWork& w, const std::vector<NodeInfo>& nodes, long long nk, long long,
                      std::vector<TcSub>& subs) {
  w.num_nodes = (int)nodes.size();
  w.num_inst = nodes.empty() ? 0 : nodes.back().b + 1;
  int slots = 0;
  for (const NodeInfo& nd : nodes) slots = std::max(slots, (w.t.shared ? nd.i : (int)(&nd - nodes.data())) + 1);
  w.num_slots = slots;
  w.rows = nk + kRows;  // one spare tile of rows so a ragged last tile stays inside the map
  const size_t pk = (size_t)w.rows * kLdp * sizeof(__half);
  const size_t pw = (size_t)slots * kLdp * kLdp * sizeof(__half);
  const size_t nv = (size_t)w.num_nodes * kLdp * sizeof(float);
  const size_t nm = (size_t)w.num_nodes * kLdp * kLdp * sizeof(float);
  subs.push_back({(void**)&w.t.ZH, pk});
  subs.push_back({(void**)&w.t.ZL, pk});
  subs.push_back({(void**)&w.t.zc, (size_t)nk * sizeof(float)});
  subs.push_back({(void**)&w.t.done, (size_t)w.num_nodes * sizeof(int)});
  subs.push_back({(void**)&w.t.claim, 8 * sizeof(int)});  // item counters: fwd, adjoint, rows x 2 classes
  subs.push_back({(void**)&w.t.inst_t, (size_t)2 * w.num_inst * sizeof(unsigned long long)});
  subs.push_back({(void**)&w.t.t_start, 2 * sizeof(unsigned long long)});
  subs.push_back({(void**)&w.t.WH, pw});
  subs.push_back({(void**)&w.t.WL, pw});
  subs.push_back({(void**)&w.t.WTH, pw});
  subs.push_back({(void**)&w.t.WTL, pw});
  subs.push_back({(void**)&w.t.cvec, nv});
  subs.push_back({(void**)&w.t.G, nm});
  subs.push_back({(void**)&w.t.M2, nm});
  subs.push_back({(void**)&w.t.zbar, nv});
  subs.push_back({(void**)&w.t.sgC, nv});
  subs.push_back({(void**)&w.t.tgC, nv});
  subs.push_back({(void**)&w.t.sgP, nv});
  subs.push_back({(void**)&w.t.tgP, nv});
  subs.push_back({(void**)&w.t.CtC, (size_t)(w.t.shared ? 1 : w.num_inst) * kLdp * kLdp * sizeof(float)});
  if (w.t.shared) {  // shared parameters: W^T W per position, the instance-group partials and sums
    w.asm_groups = (w.num_inst + kAsmInst - 1) / kAsmInst;
    w.shared_rootW = (long long)nodes[0].d * nodes[0].d;
    const size_t nw = (size_t)w.shared_nW * sizeof(float), ns = (size_t)w.shared_nS * sizeof(float);
    subs.push_back({(void**)&w.t.WtW, (size_t)slots * kLdp * kLdp * sizeof(float)});
    subs.push_back({(void**)&w.t.P, nw});
    subs.push_back({(void**)&w.t.S2, ns});
    subs.push_back({(void**)&w.t.Ppart, nw * w.asm_groups});
    subs.push_back({(void**)&w.t.Spart, ns * w.asm_groups});
    for (const NodeInfo& nd : nodes)  // the leaves' common dimension and the observation size
      if (nd.b == 0 && nd.leaf_slot >= 0) w.leaf_d = nd.d;
    w.obs0 = nodes[0].obs;
    subs.push_back({(void**)&w.t.Ssum, (size_t)w.leaf_d * w.leaf_d * sizeof(float)});
  }
  w.num_c = w.t.shared ? 1 : w.num_inst;
  long long cr = 0;
  for (const NodeInfo& nd : nodes)
    if (nd.parent < 0 && (!w.t.shared || nd.b == 0)) cr += nd.obs;
  w.c_rows = cr + kRows;  // one spare tile of rows: chunk tails stay inside the map
  subs.push_back({(void**)&w.t.CH, (size_t)w.c_rows * kLdp * sizeof(__half)});
  subs.push_back({(void**)&w.t.CL, (size_t)w.c_rows * kLdp * sizeof(__half)});
  subs.push_back({(void**)&w.t.c_row, (size_t)w.num_c * sizeof(int)});
  long long nx = 0;
  for (const NodeInfo& nd : nodes)
    if (nd.leaf_slot >= 0) nx = std::max(nx, nd.off_x + nd.obs);
  subs.push_back({(void**)&w.t.xs, (size_t)std::max(nx, 1ll) * sizeof(float)});
  // per instance: the leaves' M2 + zbar m^T sum ([128][128]; shared C: packed d x d)
  subs.push_back({(void**)&w.t.S, (size_t)w.num_inst * (w.t.shared ? (size_t)w.leaf_d * w.leaf_d
                                                                    : (size_t)kLdp * kLdp) * sizeof(float)});
  subs.push_back({(void**)&w.t.VH, pk});
  subs.push_back({(void**)&w.t.VL, pk});
  subs.push_back({(void**)&w.t.EH, pk});
  subs.push_back({(void**)&w.t.EL, pk});
  subs.push_back({(void**)&w.t.CCH, (size_t)w.num_c * kLdp * kLdp * sizeof(__half)});
  subs.push_back({(void**)&w.t.CCL, (size_t)w.num_c * kLdp * kLdp * sizeof(__half)});
}

tmc_status prepare(TcWork& w, const std::vector<NodeInfo>& nodes, const std::vector<Tile>&, int maxK,
                   int maxd) {
  w.maxK = maxK;
  w.maxdp = maxd > 64 ? 128 : 64;
  for (const NodeInfo& nd : nodes) w.maxobs = std::max(w.maxobs, nd.obs);
  if (!make_map(&w.mZH, w.t.ZH, w.rows) || !make_map(&w.mZL, w.t.ZL, w.rows) ||
      !make_map(&w.mWH, w.t.WH, (long long)w.num_slots * kLdp) ||
      !make_map(&w.mWL, w.t.WL, (long long)w.num_slots * kLdp) ||
      !make_map(&w.mWTH, w.t.WTH, (long long)w.num_slots * kLdp) ||
      !make_map(&w.mWTL, w.t.WTL, (long long)w.num_slots * kLdp) ||
      !make_map(&w.mCH, w.t.CH, w.c_rows) || !make_map(&w.mCL, w.t.CL, w.c_rows) ||
      !make_map(&w.mZH64, w.t.ZH, w.rows, kMoUnit) || !make_map(&w.mZL64, w.t.ZL, w.rows, kMoUnit) ||
      !make_map_f32(&w.mG, w.t.G, (long long)w.num_nodes * kLdp) ||
      !make_map(&w.mVH, w.t.VH, w.rows) || !make_map(&w.mVL, w.t.VL, w.rows) ||
      !make_map(&w.mEH, w.t.EH, w.rows) || !make_map(&w.mEL, w.t.EL, w.rows) ||
      !make_map(&w.mCCH, w.t.CCH, (long long)w.num_c * kLdp) ||
      !make_map(&w.mCCL, w.t.CCL, (long long)w.num_c * kLdp))
    return TMC_ERR_CUDA;
  {  // observation matrices' first rows, and the leaf tiles of the observation kernel
    std::vector<int> crow(w.num_c, 0);
    int next = 0;
    for (const NodeInfo& nd : nodes)
      if (nd.parent < 0 && nd.b < w.num_c) {
        crow[nd.b] = next;
        next += nd.obs;
      }
    cudaMemcpy(w.t.c_row, crow.data(), sizeof(int) * crow.size(), cudaMemcpyHostToDevice);
    w.obs_tiles.clear();
    for (int c = 0; c < 2; ++c) {
      w.ob_b[c] = (int)w.obs_tiles.size();
      for (int g = 0; g < (int)nodes.size(); ++g)
        if (nodes[g].leaf_slot >= 0 && nodes[g].obs > 0 && ((nodes[g].d > 64) ? 1 : 0) == c)
          for (int r = 0; r < nodes[g].K; r += kRows) w.obs_tiles.push_back(Tile{g, r});
      w.ob_e[c] = (int)w.obs_tiles.size();
    }
    w.leaves.clear();
    for (int g = 0; g < (int)nodes.size(); ++g)
      if (nodes[g].leaf_slot >= 0) w.leaves.push_back(g);
    w.mo_items.clear();  // node-moment items: every node, kMoSlabs x 128 samples each, per d class
    for (int c = 0; c < 2; ++c) {
      w.mo_b[c] = (int)w.mo_items.size();
      for (int g = 0; g < (int)nodes.size(); ++g)
        if (((nodes[g].d > 64) ? 1 : 0) == c)
          for (int r = 0; r < nodes[g].K; r += kMoSlabs * kRows)
            w.mo_items.push_back(MoItem{nodes[g].off_nk + r, g, std::min(nodes[g].K - r, kMoSlabs * kRows), nodes[g].d,
                                        nodes[g].K <= kMoSlabs * kRows ? 1 : 0});
      w.mo_e[c] = (int)w.mo_items.size();
    }
    w.mo_split = false;
    for (const NodeInfo& nd : nodes) w.mo_split = w.mo_split || nd.K > kMoSlabs * kRows;
    if (!w.mo_items.empty()) {
      if (cudaMalloc(&w.d_mo_items, sizeof(MoItem) * w.mo_items.size()) != cudaSuccess) return TMC_ERR_NOMEM;
      cudaMemcpy(w.d_mo_items, w.mo_items.data(), sizeof(MoItem) * w.mo_items.size(), cudaMemcpyHostToDevice);
    }
    w.sample_tiles.clear();
    for (int g = 0; g < (int)nodes.size(); ++g)
      for (int r = 0; r < nodes[g].K; r += sample_rows(nodes[g].d)) w.sample_tiles.push_back(Tile{g, r});
    if (!w.obs_tiles.empty()) {
      if (cudaMalloc(&w.d_obs_tiles, sizeof(Tile) * w.obs_tiles.size()) != cudaSuccess) return TMC_ERR_NOMEM;
      cudaMemcpy(w.d_obs_tiles, w.obs_tiles.data(), sizeof(Tile) * w.obs_tiles.size(), cudaMemcpyHostToDevice);
    }
    if (!w.leaves.empty()) {
      if (cudaMalloc(&w.d_leaves, sizeof(int) * w.leaves.size()) != cudaSuccess) return TMC_ERR_NOMEM;
      cudaMemcpy(w.d_leaves, w.leaves.data(), sizeof(int) * w.leaves.size(), cudaMemcpyHostToDevice);
    }
    {  // leaves grouped by instance (node order keeps each instance's leaves contiguous)
      std::vector<LeafInfo> li(w.leaves.size());
      std::vector<int> off(w.num_inst + 1, 0);
      for (size_t l = 0; l < w.leaves.size(); ++l) {
        const NodeInfo& nd = nodes[w.leaves[l]];
        li[l] = LeafInfo{w.leaves[l], 0, nd.off_q, nd.off_x};
        ++off[nd.b + 1];
      }
      for (int b = 0; b < w.num_inst; ++b) off[b + 1] += off[b];
      if (cudaMalloc(&w.d_leaf_off, sizeof(int) * off.size()) != cudaSuccess) return TMC_ERR_NOMEM;
      cudaMemcpy(w.d_leaf_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice);
      if (!li.empty()) {
        if (cudaMalloc(&w.d_leaf_info, sizeof(LeafInfo) * li.size()) != cudaSuccess) return TMC_ERR_NOMEM;
        cudaMemcpy(w.d_leaf_info, li.data(), sizeof(LeafInfo) * li.size(), cudaMemcpyHostToDevice);
      }
      w.t.leaf_info = w.d_leaf_info;
      w.t.leaf_off = w.d_leaf_off;
    }
    if (!w.sample_tiles.empty()) {
      if (cudaMalloc(&w.d_sample_tiles, sizeof(Tile) * w.sample_tiles.size()) != cudaSuccess) return TMC_ERR_NOMEM;
      cudaMemcpy(w.d_sample_tiles, w.sample_tiles.data(), sizeof(Tile) * w.sample_tiles.size(),
                 cudaMemcpyHostToDevice);
    }
    cudaMemset(w.t.CH, 0, (size_t)w.c_rows * kLdp * sizeof(__half));
    cudaMemset(w.t.CL, 0, (size_t)w.c_rows * kLdp * sizeof(__half));
  }
  int maxlevel = 0;
  for (const NodeInfo& nd : nodes) maxlevel = std::max(maxlevel, nd.level);
  w.maxlevel = maxlevel;
  w.inst_dp.assign(w.num_inst, 64);
  for (const NodeInfo& nd : nodes)
    if (nd.d > 64) w.inst_dp[nd.b] = 128;
  build_items(w, nodes, 0);
  cudaDeviceGetAttribute(&w.num_sms, cudaDevAttrMultiProcessorCount, 0);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&w.num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  w.nonroot.clear();
  w.n_pack_w = 0;
  for (int g = 0; g < (int)nodes.size(); ++g)
    if (nodes[g].parent >= 0) {
      w.nonroot.push_back(g);
      // shared parameters: instance 0's edges hold every distinct W (they come first)
      if (!w.t.shared || nodes[g].b == 0) ++w.n_pack_w;
    }
  if (!w.tiles.empty()) {
    if (cudaMalloc(&w.d_tiles, sizeof(Tile) * w.tiles.size()) != cudaSuccess) return TMC_ERR_NOMEM;
    cudaMemcpy(w.d_tiles, w.tiles.data(), sizeof(Tile) * w.tiles.size(), cudaMemcpyHostToDevice);
  }
  if (!w.nonroot.empty()) {
    if (cudaMalloc(&w.d_nonroot, sizeof(int) * w.nonroot.size()) != cudaSuccess) return TMC_ERR_NOMEM;
    cudaMemcpy(w.d_nonroot, w.nonroot.data(), sizeof(int) * w.nonroot.size(), cudaMemcpyHostToDevice);
  }
  // zero the packed operand arrays once: padding columns / spare rows are read by the MMAs
  cudaMemset(w.t.ZH, 0, (size_t)w.rows * kLdp * sizeof(__half));
  cudaMemset(w.t.ZL, 0, (size_t)w.rows * kLdp * sizeof(__half));
  for (__half* a : {w.t.WH, w.t.WL, w.t.WTH, w.t.WTL}) cudaMemset(a, 0, (size_t)w.num_slots * kLdp * kLdp * sizeof(__half));
  const size_t f64 = fwd_smem<64>(maxK), f128 = fwd_smem<128>(maxK);
  cudaFuncSetAttribute(k_edge_fwd_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f64);
  cudaFuncSetAttribute(k_edge_fwd_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f128);
  cudaFuncSetAttribute(k_edge_bwd_tc<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem<64>(maxK));
  cudaFuncSetAttribute(k_edge_bwd_tc<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem<128>(maxK));
  cudaFuncSetAttribute(k_edge_bwd_tc<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem<64>(maxK));
  cudaFuncSetAttribute(k_edge_bwd_tc<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem<128>(maxK));
  cudaFuncSetAttribute(k_sample_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSampleSmem);
  cudaFuncSetAttribute(k_moments_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MoCfg<64>::smem);
  cudaFuncSetAttribute(k_moments_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MoCfg<128>::smem);
  cudaFuncSetAttribute(k_obs_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)obs_smem<64>());
  cudaFuncSetAttribute(k_obs_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)obs_smem<128>());
  if (cudaGetLastError() != cudaSuccess) return TMC_ERR_CUDA;
  return prepare_dz(w, nodes);
}

tmc_status instance_times(TcWork& w, int B, double* fwd_us, double* bwd_us) {
  if (cudaDeviceSynchronize() != cudaSuccess) return TMC_ERR_CUDA;
  std::vector<unsigned long long> t(2 * (size_t)B), st(2);
  if (cudaMemcpy(t.data(), w.t.inst_t, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(st.data(), w.t.t_start, sizeof(unsigned long long) * 2, cudaMemcpyDeviceToHost) != cudaSuccess)
    return TMC_ERR_CUDA;
  for (int b = 0; b < B; ++b) {
    if (fwd_us) fwd_us[b] = t[b] >= st[0] ? (double)(t[b] - st[0]) * 1e-3 : 0.0;
    if (bwd_us) bwd_us[b] = t[B + b] >= st[1] ? (double)(t[B + b] - st[1]) * 1e-3 : 0.0;
  }
  return TMC_OK;
}

void release(TcWork& w) {
  release_dz(w);
  cudaFree(w.d_tiles);
  cudaFree(w.d_nonroot);
  cudaFree(w.d_obs_tiles);
  cudaFree(w.d_leaves);
  cudaFree(w.d_leaf_info);
  cudaFree(w.d_leaf_off);
  cudaFree(w.d_mo_items);
  cudaFree(w.d_sample_tiles);
  w.d_tiles = nullptr;
  w.d_nonroot = nullptr;
  w.d_obs_tiles = nullptr;
  w.d_leaves = nullptr;
  w.d_leaf_info = nullptr;
  w.d_leaf_off = nullptr;
  w.d_mo_items = nullptr;
  w.d_sample_tiles = nullptr;
}

void launch_sample(TcWork& w, const Dev& D, cudaStream_t s) {
  const int n = (int)w.sample_tiles.size();
  if (n) k_sample_tc<<<std::min(n, 2 * w.num_sms), kSampleThreads, kSampleSmem, s>>>(D, w.t, w.d_sample_tiles, n);
}

void launch_pack(TcWork& w, const Dev& D, cudaStream_t s) {
  const int n = (int)w.nonroot.size();
  if (!n) return;
  if (w.n_pack_w) k_pack_w<<<dim3(w.n_pack_w, w.maxdp / 32, w.maxdp / 32), 256, 0, s>>>(D, w.t, w.d_nonroot);
  if (n > kManyNodes) k_pack_c<4><<<(n + 3) / 4, 128, 0, s>>>(D, w.t, w.d_nonroot, n);
  else k_pack_c<1><<<n, 128, 0, s>>>(D, w.t, w.d_nonroot, n);
}

void launch_obs(TcWork& w, const Dev& D, cudaStream_t s) {
  if (w.obs_tiles.empty()) return;
  const int nl = (int)w.leaves.size();
  if (nl > kManyNodes) k_obs_center<4><<<(nl + 3) / 4, 128, 0, s>>>(D, w.t, w.d_leaves, nl);
  else k_obs_center<1><<<nl, 128, 0, s>>>(D, w.t, w.d_leaves, nl);
  k_pack_cobs<<<dim3(w.num_c, (w.maxobs + 7) / 8), 256, 0, s>>>(D, w.t);
  for (int c = 0; c < 2; ++c) {
    const int b = w.ob_b[c], n = w.ob_e[c] - b;
    if (!n) continue;
    // persistent: as many CTAs as fit at once (shared memory bounds them to 3 / 1 per SM)
    if (c == 0)
      k_obs_tc<64><<<std::min(n, 3 * w.num_sms), 128, obs_smem<64>(), s>>>(D, w.t, w.d_obs_tiles + b, n, w.mZH,
                                                                            w.mZL, w.mCH, w.mCL);
    else
      k_obs_tc<128><<<std::min(n, w.num_sms), 128, obs_smem<128>(), s>>>(D, w.t, w.d_obs_tiles + b, n, w.mZH,
                                                                          w.mZL, w.mCH, w.mCL);
  }
}

// CTAs of a persistent edge launch of n items: one per SM, or the tuned count
static int edge_grid(const TcWork& w, int n) {
  int g = w.grid_ctas > 0 && w.grid_ctas < w.num_sms ? w.grid_ctas : w.num_sms;
  return n < g ? n : g;
}
void launch_edge_fwd(TcWork& w, const Dev& D, cudaStream_t s) {
  cudaMemsetAsync(w.t.done, 0, (size_t)w.num_nodes * sizeof(int), s);
  cudaMemsetAsync(w.t.claim, 0, 2 * sizeof(int), s);
  cudaMemsetAsync(w.t.inst_t, 0, sizeof(unsigned long long) * w.num_inst, s);
  cudaMemsetAsync(w.t.t_start, 0xFF, sizeof(unsigned long long), s);
  for (int c = 0; c < 2; ++c) {
    const int b = w.it_b[0][c], n = w.it_e[0][c] - b;
    if (!n) continue;
    const int grid = edge_grid(w, n);
    int ncb = 1, cbk = 0;
    if (c == 0) {
      const size_t sm = fwd_smem<64>(w.maxK, &ncb, &cbk);
      k_edge_fwd_tc<64><<<grid, kThreadsTc, sm, s>>>(D, w.t, w.d_tiles + b, n, w.t.done, w.t.claim + c, w.pro_lead,
                                                      ncb, cbk, w.mZH, w.mZL,
                                                      w.mWH, w.mWL);
    } else {
      const size_t sm = fwd_smem<128>(w.maxK, &ncb, &cbk);
      k_edge_fwd_tc<128><<<grid, kThreadsTc, sm, s>>>(D, w.t, w.d_tiles + b, n, w.t.done, w.t.claim + c, w.pro_lead,
                                                       ncb, cbk, w.mZH, w.mZL,
                                                       w.mWH, w.mWL);
    }
  }
}

void launch_edge_bwd(TcWork& w, const Dev& D, cudaStream_t s) {
  if (w.num_nodes > kManyNodes) k_zero_dd<4><<<(w.num_nodes + 3) / 4, 256, 0, s>>>(D, w.t.G);
  else k_zero_dd<1><<<w.num_nodes, 256, 0, s>>>(D, w.t.G);
  cudaMemsetAsync(w.t.done, 0, (size_t)w.num_nodes * sizeof(int), s);
  cudaMemsetAsync(w.t.claim + 2, 0, 2 * sizeof(int), s);
  cudaMemsetAsync(w.t.inst_t + w.num_inst, 0, sizeof(unsigned long long) * w.num_inst, s);
  cudaMemsetAsync(w.t.t_start + 1, 0xFF, sizeof(unsigned long long), s);
  for (int c = 0; c < 2; ++c) {
    const int b = w.it_b[1][c], n = w.it_e[1][c] - b;
    if (!n) continue;
    const int grid = edge_grid(w, n);
    if (c == 0)
      k_edge_bwd_tc<64, false><<<grid, kThreadsTc, bwd_smem<64>(w.maxK), s>>>(D, w.t, w.d_tiles + b, n, w.t.done,
                                                                     w.t.claim + 2 + c, w.mZH, w.mZL,
                                                                     w.mWTH, w.mWTL, w.mG);
    else
      k_edge_bwd_tc<128, false><<<grid, kThreadsTc, bwd_smem<128>(w.maxK), s>>>(D, w.t, w.d_tiles + b, n, w.t.done,
                                                                       w.t.claim + 2 + c, w.mZH,
                                                                       w.mZL, w.mWTH, w.mWTL, w.mG);
  }
}

void launch_edge_rows(TcWork& w, const Dev& D, cudaStream_t s) {
  cudaMemsetAsync(w.t.claim + 4, 0, 2 * sizeof(int), s);
  // tile r of edge p -> i names parent rows r .. r + 127; no item depends on another
  for (int c = 0; c < 2; ++c) {
    const int b = w.it_b[2][c], n = w.it_e[2][c] - b;
    if (!n) continue;
    const int grid = edge_grid(w, n);
    if (c == 0)
      k_edge_bwd_tc<64, true><<<grid, kThreadsTc, bwd_smem<64>(w.maxK), s>>>(D, w.t, w.d_tiles + b, n, w.t.done,
                                                                           w.t.claim + 4 + c, w.mZH,
                                                                           w.mZL, w.mWH, w.mWL, w.mG);
    else
      k_edge_bwd_tc<128, true><<<grid, kThreadsTc, bwd_smem<128>(w.maxK), s>>>(D, w.t, w.d_tiles + b, n, w.t.done,
                                                                             w.t.claim + 4 + c, w.mZH, w.mZL, w.mWH, w.mWL, w.mG);
  }
}

void launch_unpack_grads(TcWork& w, const Dev& D, cudaStream_t s) {
  const int nr = (int)w.nonroot.size();
  if (w.mo_split) {  // a node split over several moment items accumulates with atomics
    cudaMemsetAsync(w.t.M2, 0, (size_t)w.num_nodes * kLdp * kLdp * sizeof(float), s);
    cudaMemsetAsync(w.t.zbar, 0, (size_t)w.num_nodes * kLdp * sizeof(float), s);
  }
  for (int c = 0; c < 2; ++c) {  // node moments M2, zbar of every node (roots included)
    const int b = w.mo_b[c], n = w.mo_e[c] - b;
    if (!n) continue;
    const MoItem* it = w.d_mo_items + b;
    if (c == 0)
      k_moments_tc<64><<<std::min(n, w.num_sms), kMoThreads, MoCfg<64>::smem, s>>>(D, w.t, it, n, w.mZH64, w.mZL64);
    else
      k_moments_tc<128><<<std::min(n, w.num_sms), kMoThreads, MoCfg<128>::smem, s>>>(D, w.t, it, n, w.mZH64,
                                                                                   w.mZL64);
  }

  cudaMemsetAsync(w.t.CtC, 0, (size_t)(D.shared ? 1 : D.num_inst) * kLdp * kLdp * sizeof(float), s);
  k_ctc<<<dim3(D.shared ? 1 : D.num_inst, w.maxdp > 64 ? 4 : 1, (w.maxobs + kTile - 1) / kTile), kThreads, 0, s>>>(D, w.t);
  cudaMemsetAsync(w.t.tgP, 0, (size_t)w.num_nodes * kLdp * sizeof(float), s);
  cudaMemsetAsync(w.t.tgC, 0, (size_t)w.num_nodes * kLdp * sizeof(float), s);
  if (nr) {
    k_asm_edge_vec<<<nr, 128, 0, s>>>(D, w.t, w.d_nonroot);
    const int ty = w.maxdp > 64 ? 4 : 1;
    if (D.shared) {  // one W_c per position: no d x d x d product per instance
      const int np = w.num_slots - 1;
      k_wtw<<<dim3(np, ty), kThreads, 0, s>>>(D, w.t);
      k_asm_shared<<<dim3(np, ty, w.asm_groups), kThreads, 0, s>>>(D, w.t, w.shared_nW, w.shared_nS);
    } else {
      k_asm_edge_mat<<<dim3(nr, ty), kThreads, 0, s>>>(D, w.t, w.d_nonroot);
    }
  }
  if (w.maxdp > 64) k_asm_node<4><<<D.num_nodes, 4 * kTcMaxD, 0, s>>>(D, w.t);
  else k_asm_node<1><<<D.num_nodes, kTcMaxD, 0, s>>>(D, w.t);
  k_leaf_S<<<dim3(D.num_inst, w.maxdp > 64 ? 4 : 1), kThreads, 0, s>>>(D, w.t);
  k_asm_dC<<<dim3(D.num_inst, (w.maxobs + kTile - 1) / kTile, w.maxdp / kTile), kThreads, 0, s>>>(D, w.t);
  if (!D.shared) return;
  // shared parameters: every sum over instances (groups) in one launch, then the two products
  // with the shared W_c and C
  RowSeg segs[kMaxRowSegs];
  int n = 0;
  const long long nw = w.shared_nW - w.shared_rootW;
  const long long nC = (long long)w.obs0 * w.leaf_d, nS = (long long)w.leaf_d * w.leaf_d;
  if (D.dW && nr) {
    segs[n++] = RowSeg{w.t.Ppart + w.shared_rootW, w.t.P + w.shared_rootW, w.asm_groups, nw, w.shared_nW};
    segs[n++] = RowSeg{w.t.Spart, w.t.S2, w.asm_groups, w.shared_nS, w.shared_nS};
  }
  if (D.dC) {
    segs[n++] = RowSeg{D.pC, D.dC, w.num_inst, nC, nC};
    segs[n++] = RowSeg{w.t.S, w.t.Ssum, w.num_inst, nS, nS};
  }
  if (D.dbias && D.pbias) segs[n++] = RowSeg{D.pbias, D.dbias, w.num_inst, w.shared_nb, w.shared_nb};
  rows_sum_batch(segs, n, D.rsum, s);
  if (D.dW && nr) k_shared_dw<<<dim3(w.num_slots - 1, w.maxdp > 64 ? 4 : 1), kThreads, 0, s>>>(D, w.t);
  if (D.dC)  // one product of C with the instance sum of S
    k_shared_dC<<<dim3((w.obs0 + kTile - 1) / kTile, (w.leaf_d + kTile - 1) / kTile), kThreads, 0, s>>>(D, w.t);
}

}  // namespace tc
}  // namespace tmc
