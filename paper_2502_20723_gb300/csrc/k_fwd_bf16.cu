// BF16 tensor-core forward of the ansatz (architecture appendix) on sm_103a: tcgen05.mma with FP32
// accumulators in tensor memory, weights streamed into shared memory by cp.async.bulk (TMA engine),
// softmax attention by warp-level MMAs (N <= 16; CUDA cores otherwise), the MLP's GELU in packed FP16
// arithmetic feeding an FP16 GEMM, residual stream and head in FP32.
//
// Tile: 128 token rows (TS sequences of N tokens, TS*N <= 128), one CTA of 256 threads.  TMEM lane r
// holds row r; warps w and w+4 share lane quarter w%4 and split the columns in two halves, so thread
// (w, lane) owns row 32*(w%4)+lane and column half w/4.  The residual stream X stays in FP32 registers;
// GEMM A operands are BF16 copies in shared memory.  All operands use the canonical no-swizzle K-major
// layout: element (row, k) of a [rows][K] tile at byte (row/8)*16K + (k/8)*128 + (row%8)*16 + (k%8)*2
// (core matrices of 8 rows x 16 bytes; LBO = 128 B between core matrices along K, SBO = 16K bytes
// between 8-row groups).
//
// Per layer (D = d_model, F = hidden width, HC = hidden chunk):
//   QKV:  [128 x D] x [D x 3D]      -> TMEM cols [0, 3D)
//   O:    [128 x D] x [D x D]       -> TMEM cols [0, D)
//   MLP1: [128 x D] x [D x HC]      -> TMEM cols [0, HC)      per chunk
//   MLP2: [128 x HC] x [HC x D]     -> TMEM cols [HC, HC + D) accumulated over chunks
// Every mbarrier wait is bounded; on timeout the kernel sets *err, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <type_traits>

#include "attn_mma.cuh"
#include "tdo_device.cuh"
#include "tcgen05.cuh"

// TDO_F16 = 1 compiles the same kernels with FP16 operand images and weights (k_fwd_f16.cu), in their own
// namespace and with launcher names ending in _f16; the default build uses BF16 operands.  TDO_F8 = 1
// (k_fwd_f8.cu) compiles them with E4M3 GEMM operands (tcgen05.mma kind::f8f6f4, FP32 accumulation):
// 8-bit canonical images, one power-of-two scale per weight matrix, one per tile for each activation
// image (from the tile's largest magnitude), dequantised in the epilogue; used for evaluation only
// (no parked activations).
#ifndef TDO_F16
#define TDO_F16 0
#endif
#ifndef TDO_F8
#define TDO_F8 0
#endif
#if TDO_F8
#define TDO_OPNS f8op
#define TDO_OPFN(name) name##_f8
#elif TDO_F16
#define TDO_OPNS f16op
#define TDO_OPFN(name) name##_f16
#else
#define TDO_OPNS bf16
#define TDO_OPFN(name) name
#endif

namespace tdo {
namespace TDO_OPNS {

constexpr bool kF16 = TDO_F16 != 0;   // operand type of every tensor-core GEMM image and weight
constexpr bool kF8 = TDO_F8 != 0;     // E4M3 images and weights instead
constexpr int kEB = kF8 ? 1 : 2;      // bytes per GEMM operand element

constexpr int kThreads = 256;
constexpr int kRows = 128;
constexpr int kTmemCols = 256;

template <int D>
struct Geo {
  static constexpr int HC = (4 * D < 128) ? 4 * D : 128;        // hidden chunk (max mlp_ratio 4)
  static constexpr int A_OFF = 0;                                // BF16 / FP16 / E4M3 [128][D]
  static constexpr int A_BYTES = kRows * D * kEB;
  static constexpr int KS = D + 1;                               // K/V/pool row stride (floats): no bank conflicts
  static constexpr int KV_OFF = A_OFF + A_BYTES;                 // FP32 K [128][KS], V [128][KS]
  static constexpr int KV_BYTES = 2 * kRows * KS * 4;            // (G [128][HC] BF16, pool [128][KS] alias)
  static constexpr int W_OFF = KV_OFF + KV_BYTES;                // weights of the current GEMM
  static constexpr int W_BYTES = ((3 * D * D > HC * D) ? 3 * D * D : HC * D) * kEB;
  static constexpr int M_OFF = W_OFF + W_BYTES;                  // misc
  // misc layout (bytes from M_OFF): mbar_mma 8, mbar_w 8, tmem holder 4, flag 4, configs 2x64x4,
  // F [128][2] floats, results [64] float2, scale reductions [2][8] floats
  static constexpr int RED_OFF = M_OFF + 16 + 8 + 512 + 1024 + 512;
  static constexpr int BYTES = RED_OFF + 64;
  static_assert(kRows * HC * kEB <= KV_BYTES, "hidden chunk fits the K/V region");
  // warp-MMA attention (N <= 16): FP16 Q, K [128][LDH] and V transposed [D][LDT] in the K/V region,
  // sequence s's keys at columns 16 s .. 16 s + 15 of V^T
  static constexpr int LDH = D + 8;                              // halves; conflict-free fragment rows
  static constexpr int QH_OFF = KV_OFF, KH_OFF = QH_OFF + kRows * LDH * 2, VT_OFF = KH_OFF + kRows * LDH * 2;
  static constexpr int LDT = ((KV_BYTES - 2 * kRows * LDH * 2) / (D * 2)) & ~7;
  __host__ __device__ static constexpr bool mma_attention(int n, int ts) { return n <= 16 && ts * 16 + 8 <= LDT; }
  // warp-MMA attention for 17 <= N <= 32: FP16 Q, K, V row-major [LROWS][LDH] each in the K/V region; a
  // unit reads 32 rows from its sequence's first row, at most row (ts - 1) N + 31 <= 136 of the tile
  static constexpr int LROWS = 137;
  static constexpr int QL_OFF = KV_OFF, KL_OFF = QL_OFF + LROWS * LDH * 2, VL_OFF = KL_OFF + LROWS * LDH * 2;
  static_assert(3 * LROWS * LDH * 2 <= KV_BYTES, "long-sequence attention operands fit the K/V region");
  static_assert((LROWS * LDH * 2) % 16 == 0, "16-byte-aligned regions");
};

using namespace tdo::tc;

// Activations parked by the forward for the tensor-core backward (all null = no stores).
struct FwdStore {
  uint8_t *X;      // [L][tiles] images of each layer's BF16 input (canonical [128][D], 2*128*D bytes)
  uint8_t *Xmid;   // [L][tiles] images of each MLP input (null without MLP)
  float *H;        // [tiles][ts][D] pooled vectors of the tile's sequences
  float *F;        // [tiles][ts][2] head outputs (F0, F1)
  size_t tiles;
  const int64_t *dB;   // row count on the device, read at launch (null: the launch's B); B is then a bound
};

struct Ctl {
  uint32_t bar_mma, bar_w;   // smem addresses
  uint32_t ph_mma, ph_w;     // parities to wait for next
  uint32_t tmem;             // TMEM base address (lane 0, first column)
  bool mma_thread;
  int *err;
  bool bad;
  long long spin;            // polls of every mbarrier wait before it gives up (kSpinLimit)
};

// Issue the MMAs of one GEMM: D[tmem + col] (+)= A[128 x K] * B^T, B stored [N][K]; commit to bar_mma.
// Every MMA covers 32 bytes of K (16 16-bit or 32 E4M3 elements): the next one starts 256 B later.
__device__ __forceinline__ void gemm(Ctl &c, uint32_t a_addr, uint32_t b_addr, int K, int N, uint32_t col,
                                     bool accumulate, bool f16 = false) {
  if (c.mma_thread) {
    tc_fence_after();
    // descriptor of addr + 256 kk = descriptor of addr + 16 kk (address field addr >> 4, below 256 KB)
    if constexpr (kF8) {
      const uint32_t id = idesc_e4m3(kRows, N);
      const uint64_t ad = sdesc(a_addr, 128, K * 8), bd = sdesc(b_addr, 128, K * 8);
      for (int kk = 0; kk < K / 32; ++kk)
        mma_e4m3(c.tmem + col, ad + 16 * kk, bd + 16 * kk, id, (accumulate || kk > 0) ? 1u : 0u);
    } else {
      const uint32_t id = f16 ? idesc_f16(kRows, N) : idesc16<kF16>(kRows, N);
      const uint64_t ad = sdesc(a_addr, 128, K * 16), bd = sdesc(b_addr, 128, K * 16);
      for (int kk = 0; kk < K / 16; ++kk)
        mma_bf16(c.tmem + col, ad + 16 * kk, bd + 16 * kk, id, (accumulate || kk > 0) ? 1u : 0u);
    }
    mma_commit(c.bar_mma);
  }
}

// Image element addressing and stores for the build's operand type.
__device__ __forceinline__ uint32_t canonE(int row, int k, int K) {
  if constexpr (kF8) return canon8(row, k, K);
  else return canon(row, k, K);
}
// 8 consecutive k values (k0 % 8 == 0) of one row, times s (E4M3 only; the 16-bit images are unscaled).
__device__ __forceinline__ void put_row8(uint8_t *base, int row, int k0, int K, const float *v, float s) {
  if constexpr (kF8) {
    uint2 q;
    q.x = (uint32_t)pack_e4m3(v[0] * s, v[1] * s) | ((uint32_t)pack_e4m3(v[2] * s, v[3] * s) << 16);
    q.y = (uint32_t)pack_e4m3(v[4] * s, v[5] * s) | ((uint32_t)pack_e4m3(v[6] * s, v[7] * s) << 16);
    *reinterpret_cast<uint2 *>(base + canon8(row, k0, K)) = q;
  } else {
    st_row8<kF16>(base, row, k0, K, v);
  }
}
// Two consecutive k values (k even) of one row, times s (E4M3 only).
__device__ __forceinline__ void put_pair(uint8_t *base, int row, int k, int K, float v0, float v1, float s) {
  if constexpr (kF8) *reinterpret_cast<uint16_t *>(base + canon8(row, k, K)) = pack_e4m3(v0 * s, v1 * s);
  else *reinterpret_cast<uint32_t *>(base + canon(row, k, K)) = pack16<kF16>(v0, v1);
}

// Power-of-two scale for an E4M3 image of the tile: every thread passes the largest magnitude it will
// store; the CTA's largest m in [2^e, 2^(e+1)) gives 2^(7 - e), so scaled magnitudes stay below 256 (E4M3
// saturates at 448).  1 for an all-zero image.  A block barrier; red alternates between two 8-float halves
// so that consecutive calls need no second barrier.  Returns 1 without a barrier in the 16-bit builds.
__device__ __forceinline__ float tile_scale(float amax, float *red, int &par) {
  if constexpr (!kF8) {
    return 1.0f;
  } else {
#pragma unroll
    for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    float *r = red + 8 * par;
    par ^= 1;
    if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = amax;
    __syncthreads();
    float m = r[0];
#pragma unroll
    for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, r[w]);
    if (!(m >= 1.17549435e-38f)) return 1.0f;                   // zero (or subnormal) image
    int f = 127 + 7 - ((int)((__float_as_uint(m) >> 23) & 0xffu) - 127);
    f = f < 1 ? 1 : (f > 254 ? 254 : f);                        // a normal power of two
    return __uint_as_float((uint32_t)f << 23);
  }
}

__device__ __forceinline__ bool wait_mma(Ctl &c) {
  const bool ok = mbar_wait(c.bar_mma, c.ph_mma, c.spin);
  c.ph_mma ^= 1u;
  tc_fence_after();
  return ok;
}

// Start the bulk copy of `bytes` of packed weights into the W region (thread 0), to be waited by all.
__device__ __forceinline__ void stage_w(Ctl &c, uint32_t w_addr, const void *src, uint32_t bytes) {
  if (c.mma_thread) {
    mbar_expect_tx(c.bar_w, bytes);
    bulk_g2s(w_addr, src, bytes, c.bar_w);
  }
}
__device__ __forceinline__ bool wait_w(Ctl &c) {
  const bool ok = mbar_wait(c.bar_w, c.ph_w, c.spin);
  c.ph_w ^= 1u;
  return ok;
}

// GELU (tanh form) of a pair of FP16 values, in packed half2 arithmetic: 0.5 u (1 + tanh(k0 (u + k1 u^3))).
// Two results per instruction; the MLP's hidden activations feed an FP16 GEMM, so they never pass
// through FP32 after the bias add.
__device__ __forceinline__ uint32_t gelu_h2(uint32_t x) {
  const __half2 k1 = __float2half2_rn(0.044715f), k0 = __float2half2_rn(0.7978845608028654f);
  const __half2 one = __float2half2_rn(1.0f), hf = __float2half2_rn(0.5f);
  const __half2 h = *reinterpret_cast<const __half2 *>(&x);
  const __half2 s = __hmul2(__hmul2(h, __hfma2(__hmul2(h, h), k1, one)), k0);
  uint32_t sb = *reinterpret_cast<const uint32_t *>(&s), tb;
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(tb) : "r"(sb));
  const __half2 hh = __hmul2(h, hf);
  const __half2 g = __hfma2(hh, *reinterpret_cast<const __half2 *>(&tb), hh);
  return *reinterpret_cast<const uint32_t *>(&g);
}

// v *= f (E4M3 dequantisation; nothing in the 16-bit builds)
__device__ __forceinline__ void scale16(float (&v)[16], float f) {
  if constexpr (kF8) {
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] *= f;
  }
}
// Zero 8 consecutive k values (k0 % 8 == 0) of one image row.
__device__ __forceinline__ void zero_row8(uint8_t *base, int row, int k0, int K) {
  if constexpr (kF8) *reinterpret_cast<uint2 *>(base + canon8(row, k0, K)) = make_uint2(0u, 0u);
  else *reinterpret_cast<uint4 *>(base + canon(row, k0, K)) = make_uint4(0u, 0u, 0u, 0u);
}
// Packed weights `elems` elements past p (p points at the build's operand type).
__device__ __forceinline__ const uint8_t *wchunk(const uint16_t *p, size_t elems) {
  return reinterpret_cast<const uint8_t *>(p) + elems * kEB;
}

// Agree across the CTA on failure; returns true if any thread saw a timeout.
__device__ __forceinline__ bool sync_fail(Ctl &c, bool ok) {
  const int any = __syncthreads_or(ok ? 0 : 1);
  if (any) c.bad = true;
  return any != 0;
}

// The whole ansatz on one tile; configurations in cfg_s / cfg_p [ts/2], results to res [ts/2].
// Returns false on a (bounded) wait timeout.
// Copy the A image (BF16 [128][D], complete: callers are past a barrier) to global memory.
template <int D>
__device__ __forceinline__ void park_image(const uint8_t *A, uint8_t *dst) {
  constexpr int N16 = Geo<D>::A_BYTES / 16;
  for (int i = threadIdx.x; i < N16; i += kThreads)
    reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(A)[i];
}

// n_tile > 0: the tile's chain length (the ragged batch), else the model's.
template <int D, int HD>
__device__ bool eval_tile(const DevModel &m, const DevModelBF16 &mb, uint8_t *sm, Ctl &c, int ts,
                          const uint32_t *cfg_s, const uint32_t *cfg_p, float2 *res,
                          const FwdStore *store = nullptr, size_t tile = 0, int n_tile = 0) {
  using G = Geo<D>;
  constexpr int DH = D / 2;   // columns per thread (half)
  constexpr int KS = G::KS;
  const int n = n_tile > 0 ? n_tile : m.n_sites;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (warp & 3) + lane;
  const int half = warp >> 2;
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  uint8_t *A = sm + G::A_OFF;
  float *Ks = reinterpret_cast<float *>(sm + G::KV_OFF);
  float *Vs = Ks + kRows * KS;
  uint8_t *Gs = sm + G::KV_OFF;                     // hidden chunk (aliases K/V)
  const uint32_t a_addr = smem_u32(A), w_addr = smem_u32(sm + G::W_OFF), g_addr = smem_u32(Gs);
  const bool valid = row < ts * n;
  const int s = valid ? row / n : 0;

  // ---- embedding: X (FP32, registers) for this thread's row and column half
  float X[DH];
  {
    int pat = 0;
    if (valid) {
      const int cfg = s >> 1, i = row % n;
      const uint32_t w1 = (s & 1) ? cfg_p[cfg] : cfg_s[cfg];
      const uint32_t w2 = (s & 1) ? cfg_s[cfg] : cfg_p[cfg];
      pat = embed_pattern(m.embed, w1, w2, i, n);
    }
    const float4 *e4 = reinterpret_cast<const float4 *>(m.etab + pat * D + half * DH);
#pragma unroll
    for (int j = 0; j < DH; j += 4) {
      const float4 q = valid ? __ldg(e4 + j / 4) : make_float4(0.f, 0.f, 0.f, 0.f);
      X[j] = q.x; X[j + 1] = q.y; X[j + 2] = q.z; X[j + 3] = q.w;
    }
  }
  stage_w(c, w_addr, mb.Wqkv[0], 3 * D * D * kEB);
  float *red = reinterpret_cast<float *>(sm + G::RED_OFF);
  int rpar = 0;
  float ia = 1.f;   // 1 / the scale of the A image's E4M3 values (1 in the 16-bit builds)
  auto put_x = [&]() {   // X -> the A image
    float amx = 0.f;
    if constexpr (kF8) {
#pragma unroll
      for (int j = 0; j < DH; ++j) amx = fmaxf(amx, fabsf(X[j]));
    }
    const float sx = tile_scale(amx, red, rpar);
#pragma unroll
    for (int j = 0; j < DH; j += 8) put_row8(A, row, half * DH + j, D, X + j, sx);
    ia = 1.f / sx;
  };
  put_x();

  const int heads = m.heads;
  const float qscale = rsqrtf((float)HD) * 1.4426950408889634f;   // softmax in base 2
  for (int l = 0; l < m.layers; ++l) {
    // ---------------- QKV (TMEM reads of the previous sub-layer done before the MMA overwrites them)
    tc_fence_before();
    fence_proxy_async();
    bool ok = wait_w(c);
    if (sync_fail(c, ok)) return false;
    gemm(c, a_addr, w_addr, D, 3 * D, 0, false);
    if (store) park_image<D>(A, store->X + ((size_t)l * store->tiles + tile) * (size_t)G::A_BYTES);
    ok = wait_mma(c);
    if (sync_fail(c, ok)) return false;
    stage_w(c, w_addr, mb.Wo[l], D * D * kEB);   // W is free: the QKV MMAs have completed
    // E4M3: dequantisation of Q, K, V (the image's scale times each weight matrix's), and the scale of the
    // attention output's image from max |V| (each output row is a convex combination of V rows)
    const float *wsc = kF8 ? mb.wscale + 6 * l : nullptr;
    const float fq = kF8 ? ia * __ldg(wsc + 0) : 1.f, fk = kF8 ? ia * __ldg(wsc + 1) : 1.f,
                fv = kF8 ? ia * __ldg(wsc + 2) : 1.f;
    const float qs = qscale * fq;
    float so = 1.f;
    if constexpr (kF8) {
      float amx = 0.f;
#pragma unroll
      for (int j = 0; j < DH; j += 16) {
        float vv[16];
        tmem_ld16(c.tmem + lane_addr + 2 * D + half * DH + j, vv);
#pragma unroll
        for (int e = 0; e < 16; ++e) amx = fmaxf(amx, fabsf(vv[e]));
      }
      so = tile_scale(amx * fv, red, rpar);
    }
    if (G::mma_attention(n, ts)) {
      // ---------------- attention by warp-level MMAs, one warp per (sequence, head): FP16 Q (scaled), K
      // and V^T to shared memory, output -> A (BF16)
      __half *Qh = reinterpret_cast<__half *>(sm + G::QH_OFF), *Kh = reinterpret_cast<__half *>(sm + G::KH_OFF);
      __half *Vt = reinterpret_cast<__half *>(sm + G::VT_OFF);
      {   // TMEM loads are warp-collective: every lane loads, valid rows store
        const int sq = valid ? row / n : 0, i = valid ? row % n : 0;
#pragma unroll
        for (int j = 0; j < DH; j += 16) {
          float v[16];
          tmem_ld16(c.tmem + lane_addr + half * DH + j, v);
          if (valid) {   // 16-byte stores: rows 144 bytes apart land on distinct bank groups
            uint4 *dst = reinterpret_cast<uint4 *>(Qh + row * G::LDH + half * DH + j);
            dst[0] = make_uint4(amma::h2(v[0] * qs, v[1] * qs), amma::h2(v[2] * qs, v[3] * qs),
                                amma::h2(v[4] * qs, v[5] * qs), amma::h2(v[6] * qs, v[7] * qs));
            dst[1] = make_uint4(amma::h2(v[8] * qs, v[9] * qs), amma::h2(v[10] * qs, v[11] * qs),
                                amma::h2(v[12] * qs, v[13] * qs), amma::h2(v[14] * qs, v[15] * qs));
          }
          tmem_ld16(c.tmem + lane_addr + D + half * DH + j, v);
          scale16(v, fk);
          if (valid) {
            uint4 *dst = reinterpret_cast<uint4 *>(Kh + row * G::LDH + half * DH + j);
            dst[0] = make_uint4(amma::h2(v[0], v[1]), amma::h2(v[2], v[3]), amma::h2(v[4], v[5]), amma::h2(v[6], v[7]));
            dst[1] = make_uint4(amma::h2(v[8], v[9]), amma::h2(v[10], v[11]), amma::h2(v[12], v[13]),
                                amma::h2(v[14], v[15]));
          }
          tmem_ld16(c.tmem + lane_addr + 2 * D + half * DH + j, v);
          scale16(v, fv);
          if (n == 16) {   // full sequences: V row-major like K (the attention reads it by ldmatrix.trans)
            uint4 *dst = reinterpret_cast<uint4 *>(Vt + row * G::LDH + half * DH + j);
            dst[0] = make_uint4(amma::h2(v[0], v[1]), amma::h2(v[2], v[3]), amma::h2(v[4], v[5]), amma::h2(v[6], v[7]));
            dst[1] = make_uint4(amma::h2(v[8], v[9]), amma::h2(v[10], v[11]), amma::h2(v[12], v[13]),
                                amma::h2(v[14], v[15]));
          } else if (valid) {
#pragma unroll
            for (int e = 0; e < 16; ++e) Vt[(half * DH + j + e) * G::LDT + 16 * sq + i] = __float2half_rn(v[e]);
          }
        }
      }
      if (n < 16)   // keys n .. 15 of every sequence: zero (their probabilities are zero, V must be finite)
        for (int idx = threadIdx.x; idx < D * ts * (16 - n); idx += kThreads) {
          const int f = idx / (ts * (16 - n)), r = idx % (ts * (16 - n));
          Vt[f * G::LDT + 16 * (r / (16 - n)) + n + r % (16 - n)] = __float2half_rn(0.f);
        }
      for (int idx = threadIdx.x; idx < (kRows - ts * n) * (D / 8); idx += kThreads)   // padding rows: O = 0
        zero_row8(A, ts * n + idx / (D / 8), 8 * (idx % (D / 8)), D);
      __syncthreads();
      auto units = [&](auto full) {
        constexpr int H = D / HD;   // heads (d_model = heads x head dimension)
        for (int u = warp; u < ts * H; u += kThreads / 32) {
          const int sq = u / H, h = u % H, rb = sq * (decltype(full)::value ? 16 : n);
          constexpr bool FULL = decltype(full)::value;
          amma::attn_fwd_h<HD, FULL>(
              Qh + rb * G::LDH + h * HD, Kh + rb * G::LDH + h * HD,
              FULL ? Vt + rb * G::LDH + h * HD : Vt + h * HD * G::LDT + 16 * sq, G::LDH, FULL ? G::LDH : G::LDT, n,
              [&](int r, int cc, float v0, float v1) { put_pair(A, rb + r, h * HD + cc, D, v0, v1, so); });
        }
      };
      if (n == 16) units(std::true_type{});
      else units(std::false_type{});
    } else if (n > 16) {
      // ---------------- attention of 17 to 32 tokens by warp-level MMAs, one warp per (sequence, head,
      // block of 16 queries): FP16 Q (scaled), K, V row-major to shared memory, output -> A
      __half *Ql = reinterpret_cast<__half *>(sm + G::QL_OFF), *Kl = reinterpret_cast<__half *>(sm + G::KL_OFF);
      __half *Vl = reinterpret_cast<__half *>(sm + G::VL_OFF);
#pragma unroll
      for (int j = 0; j < DH; j += 16) {   // TMEM loads are warp-collective: every lane loads, valid rows store
        float v[16];
        tmem_ld16(c.tmem + lane_addr + half * DH + j, v);
        if (valid) {
          uint4 *dst = reinterpret_cast<uint4 *>(Ql + row * G::LDH + half * DH + j);
          dst[0] = make_uint4(amma::h2(v[0] * qs, v[1] * qs), amma::h2(v[2] * qs, v[3] * qs),
                              amma::h2(v[4] * qs, v[5] * qs), amma::h2(v[6] * qs, v[7] * qs));
          dst[1] = make_uint4(amma::h2(v[8] * qs, v[9] * qs), amma::h2(v[10] * qs, v[11] * qs),
                              amma::h2(v[12] * qs, v[13] * qs), amma::h2(v[14] * qs, v[15] * qs));
        }
        tmem_ld16(c.tmem + lane_addr + D + half * DH + j, v);
        scale16(v, fk);
        if (valid) {
          uint4 *dst = reinterpret_cast<uint4 *>(Kl + row * G::LDH + half * DH + j);
          dst[0] = make_uint4(amma::h2(v[0], v[1]), amma::h2(v[2], v[3]), amma::h2(v[4], v[5]), amma::h2(v[6], v[7]));
          dst[1] = make_uint4(amma::h2(v[8], v[9]), amma::h2(v[10], v[11]), amma::h2(v[12], v[13]),
                              amma::h2(v[14], v[15]));
        }
        tmem_ld16(c.tmem + lane_addr + 2 * D + half * DH + j, v);
        scale16(v, fv);
        if (valid) {
          uint4 *dst = reinterpret_cast<uint4 *>(Vl + row * G::LDH + half * DH + j);
          dst[0] = make_uint4(amma::h2(v[0], v[1]), amma::h2(v[2], v[3]), amma::h2(v[4], v[5]), amma::h2(v[6], v[7]));
          dst[1] = make_uint4(amma::h2(v[8], v[9]), amma::h2(v[10], v[11]), amma::h2(v[12], v[13]),
                              amma::h2(v[14], v[15]));
        }
      }
      {   // rows past the tile's sequences: zero (finite values for the masked keys' V and the unused queries)
        const int zr = G::LROWS - ts * n, per = D / 8;
        for (int idx = threadIdx.x; idx < 3 * zr * per; idx += kThreads) {
          const int reg = idx / (zr * per), r = ts * n + (idx % (zr * per)) / per, c8 = idx % per;
          __half *base = reg == 0 ? Ql : (reg == 1 ? Kl : Vl);
          *reinterpret_cast<uint4 *>(base + r * G::LDH + 8 * c8) = make_uint4(0, 0, 0, 0);
        }
      }
      for (int idx = threadIdx.x; idx < (kRows - ts * n) * (D / 8); idx += kThreads)   // padding rows: O = 0
        zero_row8(A, ts * n + idx / (D / 8), 8 * (idx % (D / 8)), D);
      __syncthreads();
      constexpr int H = D / HD;
      for (int u = warp; u < ts * H * 2; u += kThreads / 32) {
        const int sq = u / (2 * H), h = (u >> 1) % H, qb = u & 1, rb = sq * n;
        amma::attn_fwd_h32<HD>(Ql + rb * G::LDH + h * HD, Kl + rb * G::LDH + h * HD, Vl + rb * G::LDH + h * HD,
                               G::LDH, n, 16 * qb, [&](int r, int cc, float v0, float v1) {
                                 put_pair(A, rb + r, h * HD + cc, D, v0, v1, so);
                               });
      }
    } else {
    // K, V (FP32) to shared memory, this thread's column half
#pragma unroll
    for (int j = 0; j < DH; j += 16) {
      float v[16];
      tmem_ld16(c.tmem + lane_addr + D + half * DH + j, v);
      scale16(v, fk);
#pragma unroll
      for (int e = 0; e < 16; ++e) Ks[row * KS + half * DH + j + e] = v[e];
      tmem_ld16(c.tmem + lane_addr + 2 * D + half * DH + j, v);
      scale16(v, fv);
#pragma unroll
      for (int e = 0; e < 16; ++e) Vs[row * KS + half * DH + j + e] = v[e];
    }
    __syncthreads();
    // ---------------- attention: this thread's row, heads of its column half, single-pass (online)
    // softmax in base 2; output -> A (BF16)
    {
      const int h0 = half * (heads / 2), h1 = h0 + heads / 2;
      for (int h = h0; h < h1; ++h) {
        float q[HD], o[HD];
        {
          float t8[8];
#pragma unroll
          for (int e8 = 0; e8 < HD; e8 += 8) {
            tmem_ld8(c.tmem + lane_addr + h * HD + e8, t8);
#pragma unroll
            for (int e = 0; e < 8; ++e) q[e8 + e] = t8[e] * qs;
          }
        }
#pragma unroll
        for (int e = 0; e < HD; ++e) o[e] = 0.f;
        if (valid) {
          const float *kr = Ks + s * n * KS + h * HD;
          const float *vr = Vs + s * n * KS + h * HD;
          float mx = -INFINITY, l = 0.f;
#pragma unroll 2
          for (int j = 0; j < n; ++j, kr += KS, vr += KS) {
            float sc = 0.f;
#pragma unroll
            for (int e = 0; e < HD; ++e) sc = fmaf(q[e], kr[e], sc);
            if (sc > mx) {
              const float cr = ex2_fast(mx - sc);
              l *= cr;
#pragma unroll
              for (int e = 0; e < HD; ++e) o[e] *= cr;
              mx = sc;
            }
            const float p = ex2_fast(sc - mx);
            l += p;
#pragma unroll
            for (int e = 0; e < HD; ++e) o[e] = fmaf(p, vr[e], o[e]);
          }
          const float inv = 1.0f / l;
#pragma unroll
          for (int e = 0; e < HD; ++e) o[e] *= inv;
        }
#pragma unroll
        for (int e8 = 0; e8 < HD; e8 += 8) put_row8(A, row, h * HD + e8, D, o + e8, so);
      }
    }
    }
    tc_fence_before();
    fence_proxy_async();
    ok = wait_w(c);
    if (sync_fail(c, ok)) return false;
    gemm(c, a_addr, w_addr, D, D, 0, false);
    ok = wait_mma(c);
    if (sync_fail(c, ok)) return false;
    const bool mlp = m.ffn > 0;
    if (mlp) stage_w(c, w_addr, mb.W1[l], G::HC * D * kEB);
    else if (l + 1 < m.layers) stage_w(c, w_addr, mb.Wqkv[l + 1], 3 * D * D * kEB);
    // X += attention block output
    const float fo = kF8 ? __ldg(wsc + 3) / so : 1.f;
#pragma unroll
    for (int j = 0; j < DH; j += 16) {
      float v[16];
      tmem_ld16(c.tmem + lane_addr + half * DH + j, v);
      scale16(v, fo);
#pragma unroll
      for (int e = 0; e < 16; ++e) X[j + e] += v[e];
    }
    put_x();
    if (mlp) {
      const int nch = m.ffn / G::HC;
      // E4M3: U's dequantisation, and 1 / the scale of each hidden chunk's image (at most two chunks: the
      // chunks' W2 products sit in their own TMEM columns HC + ch D, so that no sum mixes scales)
      const float f1 = kF8 ? ia * __ldg(wsc + 4) : 1.f;
      float ig0 = 1.f, ig1 = 1.f;
      for (int ch = 0; ch < nch; ++ch) {
        tc_fence_before();
        fence_proxy_async();
        ok = wait_w(c);
        if (sync_fail(c, ok)) return false;
        gemm(c, a_addr, w_addr, D, G::HC, 0, false);                 // U chunk -> cols [0, HC)
        if (store && ch == 0)
          park_image<D>(A, store->Xmid + ((size_t)l * store->tiles + tile) * (size_t)G::A_BYTES);
        ok = wait_mma(c);
        if (sync_fail(c, ok)) return false;
        stage_w(c, w_addr, wchunk(mb.W2[l], (size_t)ch * G::HC * D), G::HC * D * kEB);
        constexpr int HH = G::HC / 2;
        if constexpr (kF8) {   // GELU(U + b1) in FP32 -> G (E4M3), scaled from max |U + b1| (|GELU(u)| <= max(|u|, 0.17))
          float amx = 0.f;
#pragma unroll
          for (int j = 0; j < HH; j += 16) {
            float v[16];
            tmem_ld16(c.tmem + lane_addr + half * HH + j, v);
            const float *b1 = m.L[l].b1 + ch * G::HC + half * HH + j;
#pragma unroll
            for (int e = 0; e < 16; ++e) amx = fmaxf(amx, fabsf(fmaf(v[e], f1, __ldg(b1 + e))));
          }
          const float sg = tile_scale(fmaxf(amx, 0.17f), red, rpar);
          if (ch == 0) ig0 = 1.f / sg;
          else ig1 = 1.f / sg;
#pragma unroll
          for (int j = 0; j < HH; j += 16) {
            float v[16];
            tmem_ld16(c.tmem + lane_addr + half * HH + j, v);
            const float *b1 = m.L[l].b1 + ch * G::HC + half * HH + j;
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = gelu_fast(fmaf(v[e], f1, __ldg(b1 + e)));
            put_row8(Gs, row, half * HH + j, G::HC, v, sg);
            put_row8(Gs, row, half * HH + j + 8, G::HC, v + 8, sg);
          }
        } else {
        // GELU(U + b1) -> G (FP16, packed half2 arithmetic), this thread's half of the chunk columns
#pragma unroll
        for (int j = 0; j < HH; j += 16) {
          float v[16];
          tmem_ld16(c.tmem + lane_addr + half * HH + j, v);
          const int c0 = ch * G::HC + half * HH + j;
          const float4 *b4 = reinterpret_cast<const float4 *>(m.L[l].b1 + c0);
#pragma unroll
          for (int e8 = 0; e8 < 2; ++e8) {   // 8 columns (one 16-byte row segment of the image) at a time
            const float4 ba = __ldg(b4 + 2 * e8), bb = __ldg(b4 + 2 * e8 + 1);
            const float *w = v + 8 * e8;
            *reinterpret_cast<uint4 *>(Gs + canon(row, half * HH + j + 8 * e8, G::HC)) =
                make_uint4(gelu_h2(amma::h2(w[0] + ba.x, w[1] + ba.y)), gelu_h2(amma::h2(w[2] + ba.z, w[3] + ba.w)),
                           gelu_h2(amma::h2(w[4] + bb.x, w[5] + bb.y)), gelu_h2(amma::h2(w[6] + bb.z, w[7] + bb.w)));
          }
        }
        }
        tc_fence_before();
        fence_proxy_async();
        ok = wait_w(c);
        if (sync_fail(c, ok)) return false;
        if constexpr (kF8) gemm(c, g_addr, w_addr, G::HC, D, G::HC + ch * D, false);   // chunk ch's own columns
        else gemm(c, g_addr, w_addr, G::HC, D, G::HC, ch > 0, true);      // out -> cols [HC, HC + D), FP16
        ok = wait_mma(c);
        if (sync_fail(c, ok)) return false;
        if (ch + 1 < nch) stage_w(c, w_addr, wchunk(mb.W1[l], (size_t)(ch + 1) * G::HC * D), G::HC * D * kEB);
        else if (l + 1 < m.layers) stage_w(c, w_addr, mb.Wqkv[l + 1], 3 * D * D * kEB);
      }
      const float f2a = kF8 ? ig0 * __ldg(wsc + 5) : 1.f, f2b = kF8 ? ig1 * __ldg(wsc + 5) : 1.f;
      const float4 *b2 = reinterpret_cast<const float4 *>(m.L[l].b2 + half * DH);
#pragma unroll
      for (int j = 0; j < DH; j += 16) {
        float v[16];
        tmem_ld16(c.tmem + lane_addr + G::HC + half * DH + j, v);
        if constexpr (kF8) {
          scale16(v, f2a);
          if (nch > 1) {
            float v2[16];
            tmem_ld16(c.tmem + lane_addr + G::HC + D + half * DH + j, v2);
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = fmaf(v2[e], f2b, v[e]);
          }
        }
#pragma unroll
        for (int e = 0; e < 16; e += 4) {
          const float4 bq = __ldg(b2 + (j + e) / 4);
          X[j + e] += v[e] + bq.x;
          X[j + e + 1] += v[e + 1] + bq.y;
          X[j + e + 2] += v[e + 2] + bq.z;
          X[j + e + 3] += v[e + 3] + bq.w;
        }
      }
      put_x();
    }
  }
  // ---------------- pooling, head, symmetrisation (FP32)
  tc_fence_before();
  __syncthreads();   // all K/V/G reads done before the pool buffer overwrites them
  float *Pool = reinterpret_cast<float *>(sm + G::KV_OFF);
#pragma unroll
  for (int j = 0; j < DH; ++j) Pool[row * KS + half * DH + j] = X[j];
  __syncthreads();
  float *Fs = reinterpret_cast<float *>(sm + G::M_OFF + 16 + 8 + 512);
  for (int p = warp; p < ts * 2; p += kThreads / 32) {
    const int sq = p >> 1, o = p & 1;
    float acc = 0.f;
    for (int cc = lane; cc < D; cc += 32) {
      float hsum = 0.f;
      for (int i = 0; i < n; ++i) hsum += Pool[(sq * n + i) * KS + cc];
      acc = fmaf(hsum, __ldg(m.Wh + 2 * cc + o), acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) Fs[p] = acc / (float)n + __ldg(m.bh + o);
  }
  __syncthreads();
  for (int cc = threadIdx.x; cc < ts / 2; cc += kThreads)
    res[cc] = symmetrise(Fs[4 * cc], Fs[4 * cc + 1], Fs[4 * cc + 2], Fs[4 * cc + 3], nullptr, nullptr);
  if (store) {
    for (int p = threadIdx.x; p < 2 * ts; p += kThreads) store->F[tile * (size_t)(2 * ts) + p] = Fs[p];
    const float inv_n = 1.0f / (float)n;
    for (int idx = threadIdx.x; idx < ts * D; idx += kThreads) {
      const int sq = idx / D, cc = idx % D;
      float hsum = 0.f;
      for (int i = 0; i < n; ++i) hsum += Pool[(sq * n + i) * KS + cc];
      store->H[(tile * (size_t)ts + sq) * D + cc] = hsum * inv_n;
    }
  }
  __syncthreads();
  return true;
}

// Barriers at misc[0, 16), the TMEM address at misc[16, 20); TMEM allocated by warp 0.
__device__ __forceinline__ void ctl_init_misc(Ctl &c, uint8_t *misc, int *err) {
  c.bar_mma = smem_u32(misc);
  c.bar_w = smem_u32(misc + 8);
  c.ph_mma = 0;
  c.ph_w = 0;
  c.mma_thread = threadIdx.x == 0;
  c.err = err;
  c.bad = false;
  c.spin = kSpinLimit;
  if (threadIdx.x == 0) {
    mbar_init(c.bar_mma, 1);
    mbar_init(c.bar_w, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(misc + 16)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tmem = *reinterpret_cast<volatile uint32_t *>(misc + 16);
}

template <int D>
__device__ __forceinline__ void ctl_init(Ctl &c, uint8_t *sm, int *err) {
  ctl_init_misc(c, sm + Geo<D>::M_OFF, err);
}

// Free TMEM; after a timeout, first give in-flight MMAs / copies a bounded chance to finish.
__device__ __forceinline__ void ctl_finish(Ctl &c) {
  if (c.bad) {
    if (threadIdx.x == 0) atomicExch(c.err, 1);
    // bounded drain of whatever the barriers still expect
    mbar_wait(c.bar_mma, c.ph_mma, c.spin);
    mbar_wait(c.bar_w, c.ph_w, c.spin);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem), "r"(kTmemCols));
  }
}

#if !TDO_F16 && !TDO_F8
// Self-test of the bounded waits: the control block of the forward (its two mbarriers and its TMEM
// allocation) with a spin limit given by the caller; the kernel waits for an MMA completion that nothing
// will signal (no copy and no MMA is ever issued), so the wait gives up after `spin` polls, and the
// teardown sets *err, drains the barriers (bounded) and frees the TMEM, as after a real timeout.
__global__ void __launch_bounds__(128) k_wait_probe(int *err, long long spin) {
  __shared__ __align__(16) uint8_t misc[32];
  Ctl c;
  ctl_init_misc(c, misc, err);
  c.spin = spin;
  if (!wait_mma(c)) c.bad = true;
  c.bad = __syncthreads_or(c.bad ? 1 : 0) != 0;
  ctl_finish(c);
}
#endif

template <int D, int HD>
__global__ void __launch_bounds__(kThreads, 2) k_fwd_bf16(DevModel m, DevModelBF16 mb, const uint32_t *__restrict__ sig,
                                                          const uint32_t *__restrict__ sigp, size_t B,
                                                          float2 *__restrict__ out, int *err, FwdStore st) {
  extern __shared__ __align__(1024) uint8_t sm[];
  using G = Geo<D>;
  Ctl c;
  ctl_init<D>(c, sm, err);
  uint32_t *cs = reinterpret_cast<uint32_t *>(sm + G::M_OFF + 24);
  uint32_t *cp = cs + 64;
  float2 *res = reinterpret_cast<float2 *>(sm + G::M_OFF + 16 + 8 + 512 + 1024);
  const int ts = seqs_per_tile(m.n_sites), tc = ts / 2;
  if (st.dB) B = min(B, (size_t)*st.dB);
  const size_t ntiles = (B + tc - 1) / tc;
  for (size_t tile = blockIdx.x; tile < ntiles && !c.bad; tile += gridDim.x) {
    if (threadIdx.x < tc) {
      const size_t b = tile * tc + threadIdx.x;
      cs[threadIdx.x] = b < B ? sig[b] : 0u;
      cp[threadIdx.x] = b < B ? sigp[b] : 0u;
    }
    __syncthreads();
    if (!eval_tile<D, HD>(m, mb, sm, c, ts, cs, cp, res, st.X ? &st : nullptr, tile)) break;
    if (threadIdx.x < tc) {
      const size_t b = tile * tc + threadIdx.x;
      if (b < B) out[b] = res[threadIdx.x];
    }
    __syncthreads();
  }
  ctl_finish(c);
}

// Chains of different lengths in one persistent launch (the ansatz takes any N with the same theta):
// configurations sorted by N into buckets, tiles of each bucket numbered consecutively in the bucket
// order of tab; a CTA takes its next tile from the work counter `next` (dynamic), or tiles blockIdx.x +
// k gridDim.x (next = null, static).  Results go back to the callers' positions through perm.
template <int D, int HD>
__global__ void __launch_bounds__(kThreads, 2)
    k_fwd_ragged(DevModel m, DevModelBF16 mb, const uint32_t *__restrict__ ssig, const uint32_t *__restrict__ ssigp,
                 const uint32_t *__restrict__ perm, RaggedTab tab, unsigned long long *next, float2 *__restrict__ out,
                 int *err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  using G = Geo<D>;
  __shared__ long long s_tile;
  Ctl c;
  ctl_init<D>(c, sm, err);
  uint32_t *cs = reinterpret_cast<uint32_t *>(sm + G::M_OFF + 24);
  uint32_t *cp = cs + 64;
  float2 *res = reinterpret_cast<float2 *>(sm + G::M_OFF + 16 + 8 + 512 + 1024);
  const long long total = tab.tile0[tab.nb];
  for (long long it = 0;; ++it) {
    if (threadIdx.x == 0) s_tile = next ? (long long)atomicAdd(next, 1ull) : blockIdx.x + it * (long long)gridDim.x;
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= total || c.bad) break;
    int k = 0;
    while (k + 1 < tab.nb && tile >= tab.tile0[k + 1]) ++k;
    const int n = tab.n[k], ts = seqs_per_tile(n), tc = ts / 2;
    const long long i0 = tab.base[k] + (tile - tab.tile0[k]) * tc, end = tab.base[k] + tab.count[k];
    const long long idx = i0 + threadIdx.x;
    if (threadIdx.x < tc) {
      cs[threadIdx.x] = idx < end ? ssig[idx] : 0u;
      cp[threadIdx.x] = idx < end ? ssigp[idx] : 0u;
    }
    __syncthreads();
    if (!eval_tile<D, HD>(m, mb, sm, c, ts, cs, cp, res, nullptr, 0, n)) break;
    if (threadIdx.x < tc && idx < end) out[perm[idx]] = res[threadIdx.x];
    __syncthreads();
  }
  ctl_finish(c);
}

// Metropolis chains on the BF16 forward (same proposal stream and acceptance rule as the FP32 sampler,
// including its diagonal mode).
template <int D, int HD>
__global__ void __launch_bounds__(kThreads, 2)
    k_sample_bf16(DevModel m, DevModelBF16 mb, size_t n_chains, size_t n_sweeps, uint64_t seed, uint64_t counter,
                  uint32_t *__restrict__ sig, uint32_t *__restrict__ sigp, uint32_t *__restrict__ ssig,
                  uint32_t *__restrict__ ssigp, unsigned long long *accepted, int *err, int diag,
                  const uint64_t *dcounter) {
  extern __shared__ __align__(1024) uint8_t sm[];
  using G = Geo<D>;
  Ctl c;
  ctl_init<D>(c, sm, err);
  uint32_t *cs = reinterpret_cast<uint32_t *>(sm + G::M_OFF + 24);
  uint32_t *cp = cs + 64;
  float2 *res = reinterpret_cast<float2 *>(sm + G::M_OFF + 16 + 8 + 512 + 1024);
  const int n = m.n_sites;
  const int ts = seqs_per_tile(n), tc = ts / 2;
  const size_t ntiles = (n_chains + tc - 1) / tc;
  if (dcounter) counter += *dcounter;   // a replayed graph: the step's counter is in device memory
  unsigned long long acc_count = 0;
  for (size_t tile = blockIdx.x; tile < ntiles && !c.bad; tile += gridDim.x) {
    const size_t ch = tile * tc + threadIdx.x;
    const bool mine = threadIdx.x < tc && ch < n_chains;
    uint32_t s0 = 0, s1 = 0, p0 = 0, p1 = 0;
    float lcur = 0.f, u = 0.f;
    if (mine) { s0 = sig[ch]; s1 = sigp[ch]; }
    if (threadIdx.x < tc) { cs[threadIdx.x] = s0; cp[threadIdx.x] = s1; }
    __syncthreads();
    if (!eval_tile<D, HD>(m, mb, sm, c, ts, cs, cp, res)) break;
    if (threadIdx.x < tc) lcur = res[threadIdx.x].x;
    bool stop = false;
    const int per = diag ? n : 2 * n;   // proposals per sweep
    for (size_t sw = 0; sw < n_sweeps && !stop; ++sw) {
      for (int j = 0; j < per; ++j) {
        const uint64_t t = counter + (uint64_t)sw * (uint64_t)per + (uint64_t)j;
        if (threadIdx.x < tc) {
          int bit;
          metropolis_draw(seed, (uint32_t)ch, t, per, &bit, &u);
          p0 = s0;
          p1 = s1;
          if (diag) { p0 ^= 1u << bit; p1 ^= 1u << bit; }
          else if (bit < n) p0 ^= 1u << bit;
          else p1 ^= 1u << (bit - n);
          cs[threadIdx.x] = p0;
          cp[threadIdx.x] = p1;
        }
        __syncthreads();
        if (!eval_tile<D, HD>(m, mb, sm, c, ts, cs, cp, res)) { stop = true; break; }
        if (threadIdx.x < tc) {
          const float lnew = res[threadIdx.x].x;
          if (u < expf(fminf(0.0f, (diag ? 1.0f : 2.0f) * (lnew - lcur)))) {
            s0 = p0; s1 = p1; lcur = lnew;
            if (mine) ++acc_count;
          }
        }
      }
      if (!stop && mine && ssig) { ssig[sw * n_chains + ch] = s0; ssigp[sw * n_chains + ch] = s1; }
    }
    if (stop) break;
    if (mine) { sig[ch] = s0; sigp[ch] = s1; }
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    unsigned long long v = acc_count;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0 && accepted) atomicAdd(accepted, v);
  }
  ctl_finish(c);
}

// ------------------------------------------------------------------ packing of BF16 weights
// dst element (n, k) of W^T ([N][K] canonical) = W[k][n] for an FP32 W [K][N] (row stride ldw, col off).
__global__ void k_pack(const float *__restrict__ W, int ldw, int col0, int K, int N, uint8_t *__restrict__ dst,
                       int f16) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * K) return;
  const int n = i / K, k = i % K;
  const float w = W[(size_t)k * ldw + col0 + n];
  if (f16) *reinterpret_cast<__half *>(dst + canon(n, k, K)) = __float2half_rn(w);
  else *reinterpret_cast<__nv_bfloat16 *>(dst + canon(n, k, K)) = __float2bfloat16_rn(w);
}

#if TDO_F8
// Scale of one weight matrix (the K x N block W[k][col0 + n], row stride ldw) for E4M3: its largest
// magnitude in [2^e, 2^(e+1)) gives s = 2^(7 - e); sc[0] = s, sinv[0] = 1 / s (1 for an all-zero block).
__global__ void __launch_bounds__(256) k_wscale(const float *__restrict__ W, int ldw, int col0, int K, int N,
                                                float *__restrict__ sc, float *__restrict__ sinv) {
  __shared__ float red[8];
  float m = 0.f;
  for (int i = threadIdx.x; i < K * N; i += 256) m = fmaxf(m, fabsf(W[(size_t)(i / N) * ldw + col0 + i % N]));
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
    float s = 1.f;
    if (m >= 1.17549435e-38f) {
      int f = 127 + 7 - ((int)((__float_as_uint(m) >> 23) & 0xffu) - 127);
      f = f < 1 ? 1 : (f > 254 ? 254 : f);
      s = __uint_as_float((uint32_t)f << 23);
    }
    sc[0] = s;
    sinv[0] = 1.f / s;
  }
}
// dst element (n, k) of the 8-bit canonical image of W^T ([N][K]) = E4M3(W[k][col0 + n] * sc[0]).
__global__ void k_pack8(const float *__restrict__ W, int ldw, int col0, int K, int N, uint8_t *__restrict__ dst,
                        const float *__restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * K) return;
  const int n = i / K, k = i % K;
  const uint16_t two = pack_e4m3(W[(size_t)k * ldw + col0 + n] * sc[0], 0.f);
  dst[canon8(n, k, K)] = (uint8_t)(two & 0xffu);
}
#endif

}  // namespace TDO_OPNS
}  // namespace tdo

#if !TDO_F16 && !TDO_F8   // operand-independent
bool bf16_supported(const DevModel &m) {
  return (m.d == 64 || m.d == 32) && (m.dh == 8 || m.dh == 16) && m.heads % 2 == 0 && (m.ffn == 0 || m.ffn % (m.d * 4 < 128 ? m.d * 4 : 128) == 0) &&
         m.embed == 0;
}

size_t bf16_packed_bytes(const DevModel &m) {
  const size_t D = m.d, F = m.ffn;
  return (size_t)m.layers * (3 * D * D + D * D + 2 * F * D) * 2;
}

// E4M3 images (1 byte per weight), then per layer the six scales (q, k, v, o, w1, w2) and their inverses.
size_t f8_packed_bytes(const DevModel &m) {
  const size_t D = m.d, F = m.ffn;
  return (size_t)m.layers * (3 * D * D + D * D + 2 * F * D) + (size_t)m.layers * 12 * sizeof(float) + 16;
}
#endif

// Packs every layer's weights into dst and fills the device views.
cudaError_t TDO_OPFN(launch_pack_bf16)(const DevModel &m, uint16_t *dst16, DevModelBF16 *views, cudaStream_t st) {
  using namespace tdo::TDO_OPNS;
#if TDO_F8
  {   // E4M3: every weight matrix with its own power-of-two scale (kernel k_wscale), then its image
    uint8_t *dst = reinterpret_cast<uint8_t *>(dst16);
    const int D = m.d, F = m.ffn;
    const int HC = (4 * D < 128) ? 4 * D : 128;
    size_t off = 0;
    for (int l = 0; l < m.layers; ++l) off += (size_t)(3 * D * D + D * D + 2 * F * D);
    off = (off + 15) / 16 * 16;
    float *sc = reinterpret_cast<float *>(dst + off), *sinv = sc + 6 * m.layers;
    views->wscale = sinv;
    off = 0;
    for (int l = 0; l < m.layers; ++l) {
      const DevLayer &L = m.L[l];
      float *s6 = sc + 6 * l, *i6 = sinv + 6 * l;
      k_wscale<<<1, 256, 0, st>>>(L.Wq, D, 0, D, D, s6 + 0, i6 + 0);
      k_wscale<<<1, 256, 0, st>>>(L.Wk, D, 0, D, D, s6 + 1, i6 + 1);
      k_wscale<<<1, 256, 0, st>>>(L.Wv, D, 0, D, D, s6 + 2, i6 + 2);
      k_wscale<<<1, 256, 0, st>>>(L.Wo, D, 0, D, D, s6 + 3, i6 + 3);
      uint8_t *q = dst + off;
      views->Wqkv[l] = reinterpret_cast<const uint16_t *>(q);
      k_pack8<<<(D * D + 255) / 256, 256, 0, st>>>(L.Wq, D, 0, D, D, q, s6 + 0);
      k_pack8<<<(D * D + 255) / 256, 256, 0, st>>>(L.Wk, D, 0, D, D, q + (size_t)D * D, s6 + 1);
      k_pack8<<<(D * D + 255) / 256, 256, 0, st>>>(L.Wv, D, 0, D, D, q + (size_t)2 * D * D, s6 + 2);
      off += (size_t)3 * D * D;
      views->Wo[l] = reinterpret_cast<const uint16_t *>(dst + off);
      k_pack8<<<(D * D + 255) / 256, 256, 0, st>>>(L.Wo, D, 0, D, D, dst + off, s6 + 3);
      off += (size_t)D * D;
      if (F > 0) {
        k_wscale<<<1, 256, 0, st>>>(L.W1, F, 0, D, F, s6 + 4, i6 + 4);
        k_wscale<<<1, 256, 0, st>>>(L.W2, D, 0, F, D, s6 + 5, i6 + 5);
        views->W1[l] = reinterpret_cast<const uint16_t *>(dst + off);
        for (int c = 0; c < F / HC; ++c)
          k_pack8<<<(HC * D + 255) / 256, 256, 0, st>>>(L.W1, F, c * HC, D, HC, dst + off + (size_t)c * HC * D, s6 + 4);
        off += (size_t)F * D;
        views->W2[l] = reinterpret_cast<const uint16_t *>(dst + off);
        for (int c = 0; c < F / HC; ++c)
          k_pack8<<<(HC * D + 255) / 256, 256, 0, st>>>(L.W2 + (size_t)c * HC * D, D, 0, HC, D,
                                                        dst + off + (size_t)c * HC * D, s6 + 5);
        off += (size_t)F * D;
      } else {
        views->W1[l] = views->W2[l] = nullptr;
      }
    }
    return cudaGetLastError();
  }
#endif
  uint8_t *dst = reinterpret_cast<uint8_t *>(dst16);
  const int D = m.d, F = m.ffn;
  const int HC = (4 * D < 128) ? 4 * D : 128;
  size_t off = 0;
  auto pack = [&](const float *W, int ldw, int col0, int K, int N, uint8_t *out, int f16 = kF16 ? 1 : 0) {
    k_pack<<<(N * K + 255) / 256, 256, 0, st>>>(W, ldw, col0, K, N, out, f16);
  };
  for (int l = 0; l < m.layers; ++l) {
    const DevLayer &L = m.L[l];
    // Wqkv^T [3D][D]: rows 0..D-1 from Wq, D..2D-1 from Wk, 2D..3D-1 from Wv; one canonical tile
    uint8_t *q = dst + off;
    views->Wqkv[l] = reinterpret_cast<const uint16_t *>(q);
    pack(L.Wq, D, 0, D, D, q);
    pack(L.Wk, D, 0, D, D, q + (size_t)D * D * 2);   // 8-row groups D/8.. continue at D*16*D/8 bytes = D*D*2
    pack(L.Wv, D, 0, D, D, q + (size_t)2 * D * D * 2);
    off += (size_t)3 * D * D * 2;
    views->Wo[l] = reinterpret_cast<const uint16_t *>(dst + off);
    pack(L.Wo, D, 0, D, D, dst + off);
    off += (size_t)D * D * 2;
    if (F > 0) {
      // W1^T chunks: [HC][D] each (rows = hidden units c*HC..), contiguous
      views->W1[l] = reinterpret_cast<const uint16_t *>(dst + off);
      for (int c = 0; c < F / HC; ++c) pack(L.W1, F, c * HC, D, HC, dst + off + (size_t)c * HC * D * 2);
      off += (size_t)F * D * 2;
      // W2^T chunks: [D][HC] each (K = hidden units c*HC..c*HC+HC-1), FP16 (the GEMM with the FP16 GELU output)
      views->W2[l] = reinterpret_cast<const uint16_t *>(dst + off);
      for (int c = 0; c < F / HC; ++c)
        pack(L.W2 + (size_t)c * HC * D, D, 0, HC, D, dst + off + (size_t)c * HC * D * 2, 1);
      off += (size_t)F * D * 2;
    } else {
      views->W1[l] = views->W2[l] = nullptr;
    }
  }
  return cudaGetLastError();
}

// CTAs of the forward / sampler resident per SM: two (2 x 256 TMEM columns, 2 x 128 registers x 256
// threads = the register file, 2 x 110.7 KB of the 228 KB shared memory) unless the kernel's attributes
// say that one does not fit.  Every CTA runs its own tiles, so a launch of two per SM is correct however
// many are resident.
template <typename K>
static int ctas_per_sm(K kernel, int bytes) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) { cudaGetLastError(); return 1; }
  int dev = 0, regs = 0, smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const long long per_cta_regs = (long long)fa.numRegs * tdo::TDO_OPNS::kThreads;
  const long long per_cta_smem = (long long)bytes + (long long)fa.sharedSizeBytes + 1024;
  return (2 * per_cta_regs <= regs && 2 * per_cta_smem <= smem) ? 2 : 1;
}

template <int D, int HD>
static cudaError_t fwd_bf16_impl(const DevModel &m, const DevModelBF16 &mb, const uint32_t *sig,
                                 const uint32_t *sigp, size_t B, float2 *out, int *err, int n_sm, cudaStream_t st,
                                 const tdo::TDO_OPNS::FwdStore &store) {
  using namespace tdo::TDO_OPNS;
  const int bytes = Geo<D>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_fwd_bf16<D, HD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fwd_bf16<D, HD>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  const int per_sm = ctas_per_sm(k_fwd_bf16<D, HD>, bytes);
  const int tc = tdo::seqs_per_tile(m.n_sites) / 2;
  const size_t ntiles = (B + tc - 1) / tc;
  size_t grid = (size_t)n_sm * per_sm;
  if (grid > ntiles) grid = ntiles;
  k_fwd_bf16<D, HD><<<(unsigned)grid, kThreads, bytes, st>>>(m, mb, sig, sigp, B, out, err, store);
  return cudaGetLastError();
}

cudaError_t TDO_OPFN(launch_fwd_bf16_store)(const DevModel &m, const DevModelBF16 &mb, const uint32_t *sig,
                                  const uint32_t *sigp, size_t B, float2 *logrho, int *err_flag, int n_sm,
                                  cudaStream_t st, uint8_t *x_img, uint8_t *xmid_img, float *h, float *f,
                                  size_t tiles, const int64_t *dB) {
  if (B == 0) return cudaSuccess;
  tdo::TDO_OPNS::FwdStore fs{x_img, xmid_img, h, f, tiles, dB};
  if (m.d == 64 && m.dh == 8) return fwd_bf16_impl<64, 8>(m, mb, sig, sigp, B, logrho, err_flag, n_sm, st, fs);
  if (m.d == 64 && m.dh == 16) return fwd_bf16_impl<64, 16>(m, mb, sig, sigp, B, logrho, err_flag, n_sm, st, fs);
  if (m.d == 32 && m.dh == 8) return fwd_bf16_impl<32, 8>(m, mb, sig, sigp, B, logrho, err_flag, n_sm, st, fs);
  if (m.d == 32 && m.dh == 16) return fwd_bf16_impl<32, 16>(m, mb, sig, sigp, B, logrho, err_flag, n_sm, st, fs);
  return cudaErrorInvalidValue;
}

#if !TDO_F16 && !TDO_F8
cudaError_t launch_wait_probe(int *err_flag, long long spin, cudaStream_t st) {
  tdo::bf16::k_wait_probe<<<1, 128, 0, st>>>(err_flag, spin);
  return cudaGetLastError();
}
#endif

cudaError_t TDO_OPFN(launch_fwd_bf16)(const DevModel &m, const DevModelBF16 &mb, const uint32_t *sig, const uint32_t *sigp,
                            size_t B, float2 *logrho, int *err_flag, int n_sm, cudaStream_t st) {
  return TDO_OPFN(launch_fwd_bf16_store)(m, mb, sig, sigp, B, logrho, err_flag, n_sm, st, nullptr, nullptr, nullptr,
                                         nullptr, 0, nullptr);
}

template <int D, int HD>
static cudaError_t fwd_ragged_impl(const DevModel &m, const DevModelBF16 &mb, const uint32_t *ssig,
                                   const uint32_t *ssigp, const uint32_t *perm, const RaggedTab &tab,
                                   unsigned long long *next, float2 *out, int *err, int n_sm, int ctas_per_sm_req,
                                   cudaStream_t st) {
  using namespace tdo::TDO_OPNS;
  const int bytes = Geo<D>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_fwd_ragged<D, HD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fwd_ragged<D, HD>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  const int fit = ctas_per_sm(k_fwd_ragged<D, HD>, bytes);
  const int per_sm = ctas_per_sm_req < fit ? ctas_per_sm_req : fit;
  const long long total = tab.tile0[tab.nb];
  long long grid = (long long)n_sm * (per_sm < 1 ? 1 : per_sm);
  if (grid > total) grid = total;
  if (grid < 1) return cudaSuccess;
  if (next && (e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
  k_fwd_ragged<D, HD><<<(unsigned)grid, kThreads, bytes, st>>>(m, mb, ssig, ssigp, perm, tab, next, out, err);
  return cudaGetLastError();
}

cudaError_t TDO_OPFN(launch_fwd_ragged)(const DevModel &m, const DevModelBF16 &mb, const uint32_t *ssig,
                                        const uint32_t *ssigp, const uint32_t *perm, const RaggedTab &tab,
                                        unsigned long long *next, float2 *out, int *err_flag, int n_sm,
                                        int ctas_per_sm_req, cudaStream_t st) {
  if (m.d == 64 && m.dh == 8) return fwd_ragged_impl<64, 8>(m, mb, ssig, ssigp, perm, tab, next, out, err_flag, n_sm, ctas_per_sm_req, st);
  if (m.d == 64 && m.dh == 16) return fwd_ragged_impl<64, 16>(m, mb, ssig, ssigp, perm, tab, next, out, err_flag, n_sm, ctas_per_sm_req, st);
  if (m.d == 32 && m.dh == 8) return fwd_ragged_impl<32, 8>(m, mb, ssig, ssigp, perm, tab, next, out, err_flag, n_sm, ctas_per_sm_req, st);
  if (m.d == 32 && m.dh == 16) return fwd_ragged_impl<32, 16>(m, mb, ssig, ssigp, perm, tab, next, out, err_flag, n_sm, ctas_per_sm_req, st);
  return cudaErrorInvalidValue;
}

template <int D, int HD>
static cudaError_t sample_bf16_impl(const DevModel &m, const DevModelBF16 &mb, size_t n_chains, size_t n_sweeps,
                                    uint64_t seed, uint64_t counter, uint32_t *sig, uint32_t *sigp, uint32_t *ssig,
                                    uint32_t *ssigp, unsigned long long *accepted, int *err, int diag, int n_sm,
                                    cudaStream_t st, const uint64_t *dcounter) {
  using namespace tdo::TDO_OPNS;
  const int bytes = Geo<D>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_sample_bf16<D, HD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sample_bf16<D, HD>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  const int per_sm = ctas_per_sm(k_sample_bf16<D, HD>, bytes);
  const int tc = tdo::seqs_per_tile(m.n_sites) / 2;
  const size_t ntiles = (n_chains + tc - 1) / tc;
  size_t grid = (size_t)n_sm * per_sm;
  if (grid > ntiles) grid = ntiles;
  k_sample_bf16<D, HD><<<(unsigned)grid, kThreads, bytes, st>>>(m, mb, n_chains, n_sweeps, seed, counter, sig, sigp,
                                                               ssig, ssigp, accepted, err, diag, dcounter);
  return cudaGetLastError();
}

cudaError_t TDO_OPFN(launch_sample_bf16)(const DevModel &m, const DevModelBF16 &mb, size_t n_chains, size_t n_sweeps,
                               uint64_t seed, uint64_t counter, uint32_t *sig, uint32_t *sigp, uint32_t *ssig,
                               uint32_t *ssigp, unsigned long long *accepted, int *err_flag, int diag, int n_sm,
                               cudaStream_t st, const uint64_t *dcounter) {
  if (n_chains == 0) return cudaSuccess;
#define TDO_SAMPLE_BF16(DD, HH)                                                                                   \
  if (m.d == DD && m.dh == HH)                                                                                     \
    return sample_bf16_impl<DD, HH>(m, mb, n_chains, n_sweeps, seed, counter, sig, sigp, ssig, ssigp, accepted,     \
                                    err_flag, diag, n_sm, st, dcounter);
  TDO_SAMPLE_BF16(64, 8)
  TDO_SAMPLE_BF16(64, 16)
  TDO_SAMPLE_BF16(32, 8)
  TDO_SAMPLE_BF16(32, 16)
#undef TDO_SAMPLE_BF16
  return cudaErrorInvalidValue;
}
