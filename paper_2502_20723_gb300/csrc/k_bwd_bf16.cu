// Tensor-core (tcgen05, BF16) backward of the ansatz: the cost gradient as one vector-Jacobian product
// over every connected row (derivative of Eq. lossnetk through Eq. log_sum_exp_conjugate, the head,
// the mean pooling and every layer of the architecture appendix).
//
// The forward (k_fwd_bf16 with stores) parks, per tile of 128 token rows, the BF16 image of each layer's
// input and of each MLP input (canonical K-major [128][D] layout), the pooled vectors and the head
// outputs.  The backward then runs sub-layer by sub-layer over all tiles, so that the weight
// gradients of one sub-layer stay in tensor memory for all the tiles a CTA processes and leave it once
// per CTA (float atomics into 16 accumulator copies), instead of once per tile:
//   head:      k_head_bwd (dF, dWh, dbh); the dX at the last layer output, (1/N) Wh dF per row, is formed
//              inside that layer's MLP passes (k_head_dx writes it out only for models without an MLP)
//   per layer: k_bwd_mlp  x2 (one pass per 128-wide half of the hidden layer):
//                U = Xmid W1, dG = dX W2^T (MMA), dU = dG gelu'(U) (CUDA cores),
//                dX' = dX + dU W1^T, dW1^T += dU^T Xmid, dW2 += G^T dX, db1 += dU^T 1, db2 += dX^T 1
//                (MMA, MN-major operands); the second pass adds its dX' part onto the first's output
//              k_bwd_attn1: QKV = X Wqkv, dH = dX' Wo^T (MMA); softmax attention forward and backward
//                per (sequence, head) by warp-level MMAs on FP16 copies -> dQ, dK, dV (BF16 images);
//                dWo += H^T dX'  (sequences of up to 32 tokens)
//              k_bwd_attn2: dWqkv += X^T [dQ dK dV], dX = dX' + [dQ dK dV] Wqkv^T (MMA)
//   then:      k_embed_grad, the token-embedding gradient from dX at the first layer's input (in the
//              per-configuration mode attention pass 2 of the first layer sums it per configuration)
// Weight-gradient MMAs read the row-major activation images as MN-major operands: M or N = the
// image's feature dimension, K = the 128 rows of the tile.
#include <cuda_bf16.h>

#include <type_traits>

#include "attn_mma.cuh"
#include "tcgen05.cuh"
#include "tdo_device.cuh"

// TDO_F16 = 1 compiles the same kernels with FP16 operand images and weights (k_bwd_f16.cu), in their own
// namespace and with launcher names ending in _f16; the default build uses BF16 operands.
#ifndef TDO_F16
#define TDO_F16 0
#endif
#if TDO_F16
#define TDO_BWNS bwdtc16
#define TDO_OPFN(name) name##_f16
#else
#define TDO_BWNS bwdtc
#define TDO_OPFN(name) name
#endif

namespace tdo {
namespace TDO_BWNS {

using namespace tdo::tc;
constexpr bool kF16 = TDO_F16 != 0;   // operand type of every tensor-core GEMM image and weight

constexpr int kRows = 128;
constexpr int kCopiesMax = 16;

// Descriptors. K-major image [rows][K]: LBO 128 B (next 8 k), SBO 16K B (next 8 rows), 256 B per 16 k.
// The start address sits in the low 14 bits as addr >> 4 and shared addresses stay below 256 KB, so the
// descriptor of addr + delta is the descriptor of addr plus delta >> 4.
// The same image read MN-major (the stored K is the MMA's M or N, the rows are the MMA's K):
// 8-element MN groups 128 B apart, 8-row K groups 16K B apart, 32K B per 16 rows.
__device__ __forceinline__ uint64_t dk(uint32_t addr, int K) { return sdesc(addr, 128, K * 16); }
__device__ __forceinline__ uint64_t dmn(uint32_t addr, int Kimg) { return sdesc(addr, Kimg * 16, 128); }

struct Sync {
  uint32_t bar_mma, bar_ld;
  uint32_t ph_mma, ph_ld;
  uint32_t tmem;
  bool bad;
  int *err;
};

__device__ __forceinline__ bool sync_ok(Sync &s, bool ok) {
  const int any = __syncthreads_or(ok ? 0 : 1);
  if (any) s.bad = true;
  return any == 0;
}
__device__ __forceinline__ bool wait_mma(Sync &s) {
  const bool ok = mbar_wait(s.bar_mma, s.ph_mma);
  s.ph_mma ^= 1u;
  tc_fence_after();
  return ok;
}
__device__ __forceinline__ bool wait_ld(Sync &s) {
  const bool ok = mbar_wait(s.bar_ld, s.ph_ld);
  s.ph_ld ^= 1u;
  return ok;
}

// K-major x K-major: D[tmem + col] (+)= A[128 x K] B[N x K]^T
__device__ __forceinline__ void mma_kk(const Sync &s, uint32_t a, uint32_t b, int K, int N, uint32_t col, bool acc) {
  const uint32_t id = idesc16<kF16>(kRows, N);
  const uint64_t da = dk(a, K), db = dk(b, K);
  for (int kk = 0; kk < K / 16; ++kk)
    mma_bf16(s.tmem + col, da + kk * 16, db + kk * 16, id, (acc || kk > 0) ? 1u : 0u);
}
// MN-major x MN-major over the 128 rows: D[tmem + col][M = Ka][N = Kb] (+)= A_img^T B_img
__device__ __forceinline__ void mma_mm(const Sync &s, uint32_t a, int Ka, uint32_t b, int Kb, int N, uint32_t col,
                                       bool acc) {
  const uint32_t id = idesc16_major<kF16>(kRows, N, 1, 1);
  const uint64_t da = dmn(a, Ka), db = dmn(b, Kb);
  for (int kk = 0; kk < kRows / 16; ++kk)
    mma_bf16(s.tmem + col, da + kk * Ka * 2, db + kk * Kb * 2, id, (acc || kk > 0) ? 1u : 0u);
}

// The same products with an explicit operand type (F16: FP16, else BF16) and, for mma_kk_range, a K range
// [k0, k1) of both K-major images (multiples of 16).
template <bool F16>
__device__ __forceinline__ void mma_kk_range(const Sync &s, uint32_t a, uint32_t b, int K, int k0, int k1, int N,
                                             uint32_t col, bool acc) {
  const uint32_t id = idesc16<F16>(kRows, N);
  const uint64_t da = dk(a, K), db = dk(b, K);
  for (int kk = k0 / 16; kk < k1 / 16; ++kk)
    mma_bf16(s.tmem + col, da + kk * 16, db + kk * 16, id, (acc || kk > k0 / 16) ? 1u : 0u);
}
template <bool F16>
__device__ __forceinline__ void mma_mm_t(const Sync &s, uint32_t a, int Ka, uint32_t b, int Kb, int N, uint32_t col,
                                         bool acc) {
  const uint32_t id = idesc16_major<F16>(kRows, N, 1, 1);
  const uint64_t da = dmn(a, Ka), db = dmn(b, Kb);
  for (int kk = 0; kk < kRows / 16; ++kk)
    mma_bf16(s.tmem + col, da + kk * Ka * 2, db + kk * Kb * 2, id, (acc || kk > 0) ? 1u : 0u);
}

__device__ __forceinline__ void sync_init(Sync &s, uint8_t *misc, int *err) {
  s.bar_mma = smem_u32(misc);
  s.bar_ld = smem_u32(misc + 8);
  s.ph_mma = s.ph_ld = 0;
  s.bad = false;
  s.err = err;
  if (threadIdx.x == 0) {
    mbar_init(s.bar_mma, 1);
    mbar_init(s.bar_ld, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(misc + 16)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  s.tmem = *reinterpret_cast<volatile uint32_t *>(misc + 16);
}

__device__ __forceinline__ void sync_finish(Sync &s) {
  if (s.bad) {
    if (threadIdx.x == 0) atomicExch(s.err, 1);
    mbar_wait(s.bar_mma, s.ph_mma);
    mbar_wait(s.bar_ld, s.ph_ld);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "r"(512));
  }
}

// Thread 0 starts bulk copies (sizes multiples of 16) completing on bar_ld.
__device__ __forceinline__ void load2(Sync &s, uint32_t d0, const void *s0, uint32_t n0, uint32_t d1, const void *s1,
                                      uint32_t n1) {
  if (threadIdx.x == 0) {
    mbar_expect_tx(s.bar_ld, n0 + n1);
    bulk_g2s(d0, s0, n0, s.bar_ld);
    if (n1) bulk_g2s(d1, s1, n1, s.bar_ld);
  }
}

// GELU (tanh form) at u into *g and its derivative, from one tanh.approx: with s = u^2,
// t = tanh(u (k0 + k0 k1 s)) and h = (1 + t) / 2, gelu = u h and gelu' = h + (k0 / 2) u (1 - t^2)(1 + 3 k1 s).
__device__ __forceinline__ float gelu_grad_fast(float u, float *g) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float s = u * u;
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u * fmaf(k0 * k1, s, k0)));
  const float h = fmaf(0.5f, t, 0.5f);
  *g = u * h;
  return fmaf(0.5f * k0, u * (fmaf(-t, t, 1.0f) * fmaf(3.0f * k1, s, 1.0f)), h);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Flush a TMEM accumulator block [128 lanes][N cols] (this thread: lane m, its half of the columns) to
// the gradient accumulator with index(m, n) (negative = skip).
// NQ = threads / 128 column groups (warp >> 2); N / NQ must be a multiple of 16.
template <typename IDX, int NQ = 2>
__device__ __forceinline__ void flush_block(const Sync &s, uint32_t col, int N, float *g, IDX idx) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = 32 * (warp & 3) + lane, cg = warp >> 2;
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  for (int j = 0; j < N / NQ; j += 16) {
    float v[16];
    tmem_ld16(s.tmem + lane_addr + col + cg * (N / NQ) + j, v);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const long long k = idx(m, cg * (N / NQ) + j + e);
      if (k >= 0) atomicAdd(g + k, v[e]);
    }
  }
}

// ---- per-configuration (log-derivative) mode.  The rows are virtual configurations v = 2 b + seed
// (sample b, cotangent (1, 0) for seed 0 and (0, -1) for seed 1), 2N rows (two sequences of N tokens)
// each: a tile holds cpt = ts / 2 of them, the two seeds of cpt / 2 samples (4 at N = 16, 2 at N = 24
// or 32; the N this mode takes make 2N a multiple of the MMAs' 16-row K step).  Weight gradients are then
// MMAs over each configuration's 2N rows (2N / 16 K steps) into their own TMEM columns, written to O[b][k]
// as the pair (seed 0, seed 1) = (d Re log rho, d Im log rho): FP32, or BF16 of O - oref.
struct JacOut {
  float *o32;            // [nvirt / 2][ldo] float2, or
  uint16_t *o16;         // [nvirt / 2][ldo] BF16 pairs of O - oref
  const float2 *oref;
  size_t ldo;
  size_t nvirt;          // virtual configurations (0: the kernels run in VJP mode)
  const float *iscale;   // inverse of the seeds' power-of-two scale (null: 1), applied to every output
  int cpt;               // virtual configurations per tile (even)
  int rpc;               // rows per virtual configuration (2N, a multiple of 16)
};

__device__ __forceinline__ float jac_unscale(const JacOut &j) { return j.iscale ? *j.iscale : 1.0f; }

// A replayed step graph keeps its row count in device memory (dB): a launch's B, Bpad and tiles are then
// bounds (buffers and grids sized for the most rows the step can have) and each kernel reads the count.
__device__ __forceinline__ size_t rows_now(const int64_t *dB, size_t B) {
  return dB ? min(B, (size_t)*dB) : B;
}
__device__ __forceinline__ size_t tiles_now(const int64_t *dB, size_t tiles, int tc) {
  return dB ? min(tiles, ((size_t)*dB + tc - 1) / tc) : tiles;
}

__device__ __forceinline__ void jac_put2(const JacOut &j, size_t b, long long k, float re, float im) {
  const size_t i = b * j.ldo + (size_t)k;
  const float u = jac_unscale(j);
  re *= u;
  im *= u;
  if (j.o16) {
    const float2 r = j.oref[k];
    reinterpret_cast<uint32_t *>(j.o16)[i] = pack_bf16(re - r.x, im - r.y);
  } else {
    reinterpret_cast<float2 *>(j.o32)[i] = make_float2(re, im);
  }
}
__device__ __forceinline__ void jac_put1(const JacOut &j, size_t v, long long k, float x) {
  const size_t i = ((v >> 1) * j.ldo + (size_t)k) * 2 + (v & 1);
  x *= jac_unscale(j);
  if (j.o16) j.o16[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x - ((v & 1) ? j.oref[k].y : j.oref[k].x)));
  else j.o32[i] = x;
}

// MN-major x MN-major over rows [r0, r0 + 16 nsteps) of the images: D[tmem + col] = A_img^T B_img
// (operand type F16: FP16, else BF16)
template <bool F16 = kF16>
__device__ __forceinline__ void mma_mm_rows(const Sync &s, uint32_t a, int Ka, uint32_t b, int Kb, int N,
                                            uint32_t col, int r0, int nsteps) {
  const uint32_t id = idesc16_major<F16>(kRows, N, 1, 1);
  const uint64_t da = dmn(a, Ka), db = dmn(b, Kb);
  for (int kk = 0; kk < nsteps; ++kk) {
    const int r = r0 / 16 + kk;
    mma_bf16(s.tmem + col, da + r * Ka * 2, db + r * Kb * 2, id, kk > 0 ? 1u : 0u);
  }
}

// Flush per-configuration TMEM blocks [lanes M][N cols] at columns col0 + c * N for the tile's cpt virtual
// configurations: each thread (lane quarter, column group of NQ) pairs the two seeds of a sample.
// idx(m, n) < 0 skips an element.
template <typename IDX, int NQ>
__device__ __forceinline__ void jac_flush(const Sync &s, const JacOut &j, size_t tile, uint32_t col0, int N, IDX idx) {
  const float u = jac_unscale(j);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = 32 * (warp & 3) + lane, cg = warp >> 2;
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  for (int jj = 0; jj < N / NQ; jj += 16) {
    // the reference values of this thread's 16 columns, shared by both samples of the tile
    float2 rf[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const long long k = idx(m, cg * (N / NQ) + jj + e);
      rf[e] = (j.o16 && k >= 0) ? j.oref[k] : make_float2(0.f, 0.f);
    }
    for (int pr = 0; pr < 2 && pr < j.cpt / 2; ++pr) {   // configurations 2 pr (seed 0) and 2 pr + 1 of the tile
      const size_t v0 = tile * j.cpt + 2 * pr;
      float re[16], im[16];
      tmem_ld16x2(s.tmem + lane_addr + col0 + (2 * pr) * N + cg * (N / NQ) + jj, re,
                  s.tmem + lane_addr + col0 + (2 * pr + 1) * N + cg * (N / NQ) + jj, im);
      if (v0 + 1 < j.nvirt) {
        const size_t b = v0 >> 1;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const long long k = idx(m, cg * (N / NQ) + jj + e);
          if (k < 0) continue;
          const size_t i = b * j.ldo + (size_t)k;
          if (j.o16) reinterpret_cast<uint32_t *>(j.o16)[i] = pack_bf16(u * re[e] - rf[e].x, u * im[e] - rf[e].y);
          else reinterpret_cast<float2 *>(j.o32)[i] = make_float2(u * re[e], u * im[e]);
        }
      }
    }
  }
}

// The same for blocks whose output index is contiguous along the columns (k = off + m * ld + n, rows
// m < mlim) when O is stored in BF16: each warp stages 32 rows x 8 columns of (seed 0, seed 1) pairs in
// shared memory (2 KB per warp at stage + 512 floats * warp) and writes them back 4 rows x 8 columns per
// instruction, so a warp store covers 4 contiguous 32-byte pieces instead of 32 scattered elements.
// NPR = cpt / 2 samples per tile.
template <int NQ, int NPR>
__device__ __noinline__ void jac_flush_rows_n(const Sync &s, const JacOut &j, size_t tile, uint32_t col0, int N,
                                               long long off, int ld, int mlim, float *stage) {
  const float u = jac_unscale(j);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cg = warp >> 2, mb = 32 * (warp & 3);
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  float2 *st = reinterpret_cast<float2 *>(stage) + warp * 256;   // [32 rows][8 columns]
  for (int jj = 0; jj < N / NQ; jj += 16) {
    // reference values of the 16 elements this lane writes back, shared by both samples of the tile
    float2 rf[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int m = mb + 4 * it + (lane >> 3);
        rf[h][it] = m < mlim ? j.oref[off + (long long)m * ld + cg * (N / NQ) + jj + 8 * h + (lane & 7)]
                             : make_float2(0.f, 0.f);
      }
    for (int pr = 0; pr < NPR; ++pr) {
      const size_t v0 = tile * (2 * NPR) + 2 * pr;
      const bool ok = v0 + 1 < j.nvirt;
      const size_t b = v0 >> 1;
      float re[16], im[16];
      tmem_ld16x2(s.tmem + lane_addr + col0 + (2 * pr) * N + cg * (N / NQ) + jj, re,
                  s.tmem + lane_addr + col0 + (2 * pr + 1) * N + cg * (N / NQ) + jj, im);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int e = 0; e < 8; ++e) st[lane * 8 + e] = make_float2(re[8 * h + e], im[8 * h + e]);
        __syncwarp();
        if (ok) {
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            const int r = 4 * it + (lane >> 3), c = lane & 7, m = mb + r;
            if (m < mlim) {
              const long long k = off + (long long)m * ld + cg * (N / NQ) + jj + 8 * h + c;
              const float2 v = st[r * 8 + c];
              reinterpret_cast<uint32_t *>(j.o16)[b * j.ldo + (size_t)k] =
                  pack_bf16(u * v.x - rf[h][it].x, u * v.y - rf[h][it].y);
            }
          }
        }
        __syncwarp();
      }
    }
  }
}

template <int NQ>
__device__ __forceinline__ void jac_flush_rows(const Sync &s, const JacOut &j, size_t tile, uint32_t col0, int N,
                                               long long off, int ld, int mlim, float *stage) {
  if (j.cpt == 4) jac_flush_rows_n<NQ, 2>(s, j, tile, col0, N, off, ld, mlim, stage);
  else jac_flush_rows_n<NQ, 1>(s, j, tile, col0, N, off, ld, mlim, stage);
}

// ====================================================================================== head
struct HeadArgs {
  const float2 *cot;   // [B] cotangents of log rho
  const float *cscale; // power-of-two factor applied to every cotangent (null: 1)
  const float *F;      // [B][4] head outputs (F0, F1 of both orders)
  const float *H;      // [2B][D] pooled vectors
  const float *Wh;     // [D][2]
  float *dF;           // [Bpad][4]
  size_t B, Bpad;
  const int64_t *dB;   // device row count (null: B); Bpad then shrinks to its tiles
  int tc;              // configurations per tile
  float *g;            // gradient accumulator copies
  size_t g_stride;
  long long off_wh, off_bh;
  int D;
  JacOut jac;
};

// dF of one configuration: (Re, Im) cotangent times the symmetrisation's weights of both orders.
__device__ __forceinline__ float4 head_df(const HeadArgs &a, size_t b) {
  float2 pw, pv;
  symmetrise(a.F[4 * b], a.F[4 * b + 1], a.F[4 * b + 2], a.F[4 * b + 3], &pw, &pv);
  float2 c = a.cot[b];
  if (a.cscale) {
    const float k = *a.cscale;
    c.x *= k;
    c.y *= k;
  }
  const float cwr = c.x * pw.x - c.y * pw.y, cwi = c.x * pw.y + c.y * pw.x;
  const float cvr = c.x * pv.x - c.y * pv.y, cvi = c.x * pv.y + c.y * pv.x;
  return make_float4(cwr, -cwi, cvr, cvi);
}

// VJP mode (D = 64): one warp per configuration at a time, lane k owns features k and k + 32 of dWh in
// registers (coalesced reads of the pooled vectors, no shared-memory atomics in the loop); one block
// reduction and one set of global atomics per block at the end.
__global__ void __launch_bounds__(256) k_head_bwd_vjp(HeadArgs a) {
  __shared__ float red[8][130];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float w0[2] = {0.f, 0.f}, w1[2] = {0.f, 0.f}, bb0 = 0.f, bb1 = 0.f;
  const size_t B = rows_now(a.dB, a.B), Bpad = tiles_now(a.dB, a.Bpad / a.tc, a.tc) * a.tc;
  for (size_t b = blockIdx.x * (size_t)8 + warp; b < Bpad; b += gridDim.x * (size_t)8) {
    float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
    if (b < B) {
      d = head_df(a, b);
      const float *hA = a.H + (2 * b) * 64, *hB = hA + 64;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float xa = hA[lane + 32 * h], xb = hB[lane + 32 * h];
        w0[h] = fmaf(xa, d.x, fmaf(xb, d.z, w0[h]));
        w1[h] = fmaf(xa, d.y, fmaf(xb, d.w, w1[h]));
      }
      bb0 += d.x + d.z;
      bb1 += d.y + d.w;
    }
    if (lane == 0) reinterpret_cast<float4 *>(a.dF)[b] = d;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    red[warp][2 * (lane + 32 * h)] = w0[h];
    red[warp][2 * (lane + 32 * h) + 1] = w1[h];
  }
  if (lane == 0) { red[warp][128] = bb0; red[warp][129] = bb1; }
  __syncthreads();
  float *g = a.g + (size_t)(blockIdx.x % kCopiesMax) * a.g_stride;
  for (int i = threadIdx.x; i < 130; i += blockDim.x) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += red[w][i];
    atomicAdd(g + (i < 128 ? a.off_wh + i : a.off_bh + (i - 128)), v);
  }
}

__global__ void k_head_bwd(HeadArgs a) {
  extern __shared__ float acc[];   // [2D + 2]
  const int nacc = 2 * a.D + 2;
  for (int i = threadIdx.x; i < nacc; i += blockDim.x) acc[i] = 0.f;
  __syncthreads();
  for (size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x; b < a.Bpad; b += gridDim.x * (size_t)blockDim.x) {
    float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
    if (b < a.B) {
      float2 pw, pv;
      symmetrise(a.F[4 * b], a.F[4 * b + 1], a.F[4 * b + 2], a.F[4 * b + 3], &pw, &pv);
      const float4 d = head_df(a, b);
      d0 = d.x; d1 = d.y; d2 = d.z; d3 = d.w;
      const float *hA = a.H + (2 * b) * a.D, *hB = hA + a.D;
      if (a.jac.nvirt) {   // this configuration's own head gradient
        for (int k = 0; k < a.D; ++k) {
          jac_put1(a.jac, b, a.off_wh + 2 * k, hA[k] * d0 + hB[k] * d2);
          jac_put1(a.jac, b, a.off_wh + 2 * k + 1, hA[k] * d1 + hB[k] * d3);
        }
        jac_put1(a.jac, b, a.off_bh, d0 + d2);
        jac_put1(a.jac, b, a.off_bh + 1, d1 + d3);
      } else {
        for (int k = 0; k < a.D; ++k) {
          atomicAdd(&acc[2 * k], hA[k] * d0 + hB[k] * d2);
          atomicAdd(&acc[2 * k + 1], hA[k] * d1 + hB[k] * d3);
        }
        atomicAdd(&acc[2 * a.D], d0 + d2);
        atomicAdd(&acc[2 * a.D + 1], d1 + d3);
      }
    }
    reinterpret_cast<float4 *>(a.dF)[b] = make_float4(d0, d1, d2, d3);
  }
  __syncthreads();
  if (a.jac.nvirt) return;
  float *g = a.g + (size_t)(blockIdx.x % kCopiesMax) * a.g_stride;
  for (int i = threadIdx.x; i < nacc; i += blockDim.x) {
    const long long k = i < 2 * a.D ? a.off_wh + i : a.off_bh + (i - 2 * a.D);
    atomicAdd(g + k, acc[i]);
  }
}

// dX at the last layer output: (1/N) sum_o Wh[c][o] dF[seq(r)][o] for valid rows, 0 for padding.
__global__ void k_head_dx(const float *__restrict__ dF, const float *__restrict__ Wh, int D, int n, int ts,
                          size_t tiles, float *__restrict__ dX, const int64_t *dB) {
  const int tc = ts / 2;
  const size_t total = tiles_now(dB, tiles, tc) * kRows * (size_t)D;
  const float inv_n = 1.0f / (float)n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += gridDim.x * (size_t)blockDim.x) {
    const size_t rowg = i / D;
    const int c = (int)(i % D);
    const size_t tile = rowg / kRows;
    const int r = (int)(rowg % kRows);
    float v = 0.f;
    if (r < ts * n) {
      const int s = r / n;
      const size_t b = tile * tc + (s >> 1);
      const float f0 = dF[4 * b + 2 * (s & 1)], f1 = dF[4 * b + 2 * (s & 1) + 1];
      v = (Wh[2 * c] * f0 + Wh[2 * c + 1] * f1) * inv_n;
    }
    dX[i] = v;
  }
}

// ====================================================================================== MLP pass
template <int D>
struct MlpGeo {
  static constexpr int HC = 128;
  static constexpr int IMG = kRows * D * 2;            // [128][D] BF16 image
  static constexpr int W1T_OFF = 0;                    // [HC][D]  (U = Xmid W1_c)
  static constexpr int W2_OFF = W1T_OFF + HC * D * 2;  // [HC][D]  (dG = dX W2_c^T)
  static constexpr int W1_OFF = W2_OFF + HC * D * 2;   // [D][HC]  (dX' = dU W1_c^T)
  static constexpr int X_OFF = W1_OFF + HC * D * 2;    // Xmid images [2][128][D] (tile t and t + 1)
  static constexpr int DX_OFF = X_OFF + 2 * IMG;       // dX (BF16) images [2][128][D] (tile t and t + 1)
  static constexpr int G_OFF = DX_OFF + 2 * IMG;       // G  [128][HC]
  static constexpr int DU_OFF = G_OFF + kRows * HC * 2;  // dU [128][HC]
  static constexpr int ONE_OFF = DU_OFF + kRows * HC * 2;  // all-ones [128][16] (row sums by MMA)
  static constexpr int M_OFF = ONE_OFF + kRows * 16 * 2;    // misc: bars, holder, b1 of the chunk [HC], Wh [D][2]
  static constexpr int BYTES = M_OFF + 64 + 4 * HC + 8 * D;
  // TMEM columns (C_B1: db1 = dU^T 1, C_B2: db2 = dX^T 1; every one of their 16 columns holds the same sums)
  static constexpr int C_U = 0, C_DG = 128, C_DX = 256, C_W1 = 320, C_W2 = 384, C_B1 = 448, C_B2 = 464;
  // per-configuration mode: 4 x 16 db1 and 4 x 16 db2 columns (dW1/dW2 blocks in [0, 256))
  static constexpr int C_JB1 = 320, C_JB2 = 384;
};

struct MlpArgs {
  const uint8_t *w1t, *w2, *w1;   // packed images of this half: W1^T [HC][D], W2 rows [HC][D], W1 rows [D][HC]
  const float *b1;                // b1 of this half
  const uint8_t *xmid;            // [tiles] images
  const float *dxo;               // FP32 [tiles*128][D]: dX at the MLP output
  float *dxm;                     // FP32 out: dX' (first pass: dxo + its part; second pass: += its part)
  // last layer: dX at the MLP output formed from the head instead of read from dxo (dF non-null):
  // dX[row][c] = (1/N) sum_o Wh[c][o] dF[seq(row)][o] for valid rows, 0 for padding rows
  const float *dF, *Wh;
  int n, ts;
  size_t tiles;
  const int64_t *dB;              // device row count (null: every tile); tiles is then a bound
  int do_db2;
  float *g;
  size_t g_stride;
  long long off_w1, off_b1, off_w2, off_b2;   // flat offsets (off_w1 / off_b1 / off_w2 already at this half)
  int F;
  int *err;
  JacOut jac;
};

// 512 threads: thread (row, cg) owns a quarter of the hidden chunk's and of dX's columns; 16 warps hide
// the latency of the CUDA-core phases.  Two tiles are in flight: the products U, dG of tile t + 1 (MMA1,
// barrier bar_mma) are issued while the backward products of tile t (MMA2, barrier bar2) run and its dX'
// is written out; the Xmid and dX images are double-buffered and the incoming dX is read one tile early.
// In the per-configuration mode MMA2 also fills TMEM columns [0, 256), so MMA1 of the next tile waits
// for the end of the tile.
constexpr int kMlpThreads = 512;

// ADD: the dX' part is added onto dxm (the first pass's output) by one vector reduction per element, with
// no read of it here.
template <int D, bool ADD>
__global__ void __launch_bounds__(kMlpThreads, 1) k_bwd_mlp(MlpArgs a) {
  using G = MlpGeo<D>;
  extern __shared__ __align__(1024) uint8_t sm[];
  constexpr int NQ = kMlpThreads / 128;
  constexpr int QD = D / NQ, QH = G::HC / NQ;   // dX columns and hidden columns per thread
  static_assert(QD % 16 == 0 && QH % 16 == 0, "column groups of 16");
  const uint32_t bar2 = smem_u32(sm + G::M_OFF + 24);
  uint32_t ph2 = 0;
  if (threadIdx.x == 0) mbar_init(bar2, 1);   // made visible by the fence and barrier in sync_init
  Sync s;
  sync_init(s, sm + G::M_OFF, a.err);
  float *b1s = reinterpret_cast<float *>(sm + G::M_OFF + 64);
  float *whs = b1s + G::HC;
  const bool head = a.dF != nullptr;
  for (int i = threadIdx.x; i < G::HC; i += kMlpThreads) b1s[i] = a.b1[i];
  if (head)
    for (int i = threadIdx.x; i < 2 * D; i += kMlpThreads) whs[i] = a.Wh[i];
  for (int i = threadIdx.x; i < kRows * 16 / 8; i += kMlpThreads)   // 1.0 in the operand type
    reinterpret_cast<uint4 *>(sm + G::ONE_OFF)[i] = make_uint4(kOnePair<kF16>, kOnePair<kF16>, kOnePair<kF16>, kOnePair<kF16>);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (warp & 3) + lane, cg = warp >> 2;
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t w1t = smem_u32(sm + G::W1T_OFF), w2 = smem_u32(sm + G::W2_OFF), w1 = smem_u32(sm + G::W1_OFF);
  const uint32_t xs0 = smem_u32(sm + G::X_OFF), dxs0 = smem_u32(sm + G::DX_OFF), gs = smem_u32(sm + G::G_OFF),
                 dus = smem_u32(sm + G::DU_OFF), ones = smem_u32(sm + G::ONE_OFF);
  const bool jac = a.jac.nvirt != 0;
  fence_proxy_async();   // the ones image is read by the tensor cores
  // weights once per kernel
  if (threadIdx.x == 0) {
    mbar_expect_tx(s.bar_ld, 3 * G::HC * D * 2);
    bulk_g2s(w1t, a.w1t, G::HC * D * 2, s.bar_ld);
    bulk_g2s(w2, a.w2, G::HC * D * 2, s.bar_ld);
    bulk_g2s(w1, a.w1, G::HC * D * 2, s.bar_ld);
  }
  bool ok = wait_ld(s);
  bool first = true;
  const size_t t0 = blockIdx.x, step = gridDim.x, ntl = tiles_now(a.dB, a.tiles, a.ts / 2);
  if (sync_ok(s, ok) && t0 < ntl) {
    // head mode: this row's (dF0, dF1) / N of tile t, zero for padding rows
    const bool hvalid = head && row < a.ts * a.n;
    const float inv_n = head ? 1.0f / (float)a.n : 0.f;
    auto head_f = [&](size_t t) -> float2 {
      if (!hvalid) return make_float2(0.f, 0.f);
      const int sq = row / a.n;
      const float2 f = *reinterpret_cast<const float2 *>(a.dF + 4 * (t * (a.ts / 2) + (sq >> 1)) + 2 * (sq & 1));
      return make_float2(f.x * inv_n, f.y * inv_n);
    };
    auto head_dx = [&](float2 f, float (&v)[QD]) {
#pragma unroll
      for (int j = 0; j < QD; ++j) {
        const float2 w = *reinterpret_cast<const float2 *>(whs + 2 * (cg * QD + j));
        v[j] = fmaf(w.x, f.x, w.y * f.y);
      }
    };
    float4 nx[QD / 4];   // this thread's incoming dX of a coming tile (head mode: its (dF0, dF1) / N in nx[0])
    auto load_nx = [&](size_t t) {
      if (head) {
        const float2 f = head_f(t);
        nx[0] = make_float4(f.x, f.y, 0.f, 0.f);
        return;
      }
      const float4 *src = reinterpret_cast<const float4 *>(a.dxo + (t * kRows + row) * (size_t)D + cg * QD);
#pragma unroll
      for (int j = 0; j < QD / 4; ++j) nx[j] = src[j];
    };
    // dX image of tile t (BF16, buffer b) from nx
    auto put_dx = [&](int b) {
      float dxo[QD];
      if (head) {
        head_dx(make_float2(nx[0].x, nx[0].y), dxo);
      } else {
#pragma unroll
        for (int j = 0; j < QD; j += 4) {
          const float4 v = nx[j / 4];
          dxo[j] = v.x; dxo[j + 1] = v.y; dxo[j + 2] = v.z; dxo[j + 3] = v.w;
        }
      }
#pragma unroll
      for (int j = 0; j < QD; j += 8) st_row8<kF16>(sm + G::DX_OFF + b * G::IMG, row, cg * QD + j, D, dxo + j);
    };
    // MMA1 of tile t from buffer b, once its Xmid image has landed and its dX image is written
    auto issue_mma1 = [&](int b) -> bool {
      const bool okl = wait_ld(s);
      fence_proxy_async();
      tc_fence_before();
      if (!sync_ok(s, okl)) return false;
      if (threadIdx.x == 0) {
        tc_fence_after();
        mma_kk(s, xs0 + b * G::IMG, w1t, D, G::HC, G::C_U, false);    // U  = Xmid W1_c
        mma_kk(s, dxs0 + b * G::IMG, w2, D, G::HC, G::C_DG, false);   // dG = dX W2_c^T
        mma_commit(s.bar_mma);
      }
      return true;
    };
    // prologue: tile t0 in buffer 0, then the Xmid image of t0 + step into buffer 1
    load2(s, xs0, a.xmid + t0 * (size_t)G::IMG, G::IMG, 0, nullptr, 0);
    load_nx(t0);
    put_dx(0);
    if (t0 + step < ntl) load_nx(t0 + step);
    bool live = issue_mma1(0);
    if (live && t0 + step < ntl) load2(s, xs0 + G::IMG, a.xmid + (t0 + step) * (size_t)G::IMG, G::IMG, 0, nullptr, 0);
    int buf = 0;
    for (size_t tile = t0; live && tile < ntl; tile += step, buf ^= 1) {
      const uint32_t xs = xs0 + buf * G::IMG, dxs = dxs0 + buf * G::IMG;
      const size_t rg = (tile * kRows + row) * (size_t)D + cg * QD;
      const bool has_next = tile + step < ntl;
      ok = wait_mma(s);   // U, dG of this tile; also MMA2 of the previous tile (G, dU images free)
      if (!sync_ok(s, ok)) break;
      // dU = dG gelu'(U + b1), G = gelu(U + b1) -> shared images
#pragma unroll
      for (int j = 0; j < QH; j += 16) {
        float u[16], dg[16];
        tmem_ld16x2(s.tmem + lane_addr + G::C_U + cg * QH + j, u, s.tmem + lane_addr + G::C_DG + cg * QH + j, dg);
        float gl[16], du[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float uu = u[e] + b1s[cg * QH + j + e];
          du[e] = dg[e] * gelu_grad_fast(uu, &gl[e]);
        }
        st_row8<kF16>(sm + G::G_OFF, row, cg * QH + j, G::HC, gl);
        st_row8<kF16>(sm + G::G_OFF, row, cg * QH + j + 8, G::HC, gl + 8);
        st_row8<kF16>(sm + G::DU_OFF, row, cg * QH + j, G::HC, du);
        st_row8<kF16>(sm + G::DU_OFF, row, cg * QH + j + 8, G::HC, du + 8);
      }
      tc_fence_before();
      fence_proxy_async();
      if (!sync_ok(s, true)) break;
      if (threadIdx.x == 0) {
        tc_fence_after();
        mma_kk(s, dus, w1, G::HC, D, G::C_DX, false);              // dX' part = dU W1_c^T
        if (!jac) {
          mma_mm(s, dus, G::HC, xs, D, D, G::C_W1, !first);          // dW1_c^T += dU^T Xmid
          mma_mm(s, gs, G::HC, dxs, D, D, G::C_W2, !first);          // dW2_c   += G^T dX
          mma_mm(s, dus, G::HC, ones, 16, 16, G::C_B1, !first);       // db1_c   += dU^T 1
          // db2 += dX^T 1: M = 128 reads the D-wide image as 128 features; lanes >= D hold unused sums
          if (a.do_db2) mma_mm(s, dxs, D, ones, 16, 16, G::C_B2, !first);
        } else {   // per configuration: dW1_c^T into columns [64 c, 64 c + 64) (U and dG are consumed)
          const int rpc = a.jac.rpc, ks = rpc / 16;
          for (int c = 0; c < 4 && c < a.jac.cpt; ++c) {
            mma_mm_rows(s, dus, G::HC, xs, D, D, 64 * c, rpc * c, ks);
            mma_mm_rows(s, dus, G::HC, ones, 16, 16, G::C_JB1 + 16 * c, rpc * c, ks);
            if (a.do_db2) mma_mm_rows(s, dxs, D, ones, 16, 16, G::C_JB2 + 16 * c, rpc * c, ks);
          }
        }
        mma_commit(bar2);
      }
      // while MMA2 runs: this tile's residual base (first pass: dX again, from L2; the loads are pinned
      // here), the next tile's dX image (the other buffer, last read by the previous tile's MMA2) and, in
      // VJP mode, the next tile's MMA1
      float4 base[ADD ? 1 : QD / 4];
      if constexpr (!ADD) {
        if (head) {
          float v[QD];
          head_dx(head_f(tile), v);
#pragma unroll
          for (int j = 0; j < QD / 4; ++j) base[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < QD / 4; ++j) base[j] = ld_pinned_f4(a.dxo + rg + 4 * j);
        }
      }
      if (has_next) {
        put_dx(buf ^ 1);
        if (tile + 2 * step < ntl) load_nx(tile + 2 * step);
        if (!jac && !issue_mma1(buf ^ 1)) break;
      }
      ok = mbar_wait(bar2, ph2);
      ph2 ^= 1u;
      tc_fence_after();
      if (!sync_ok(s, ok)) break;
      // MMA2 has read this tile's Xmid buffer: the Xmid image two tiles ahead goes there (in the
      // per-configuration mode after the next tile's image has been waited for)
      if (!jac && tile + 2 * step < ntl)
        load2(s, xs, a.xmid + (tile + 2 * step) * (size_t)G::IMG, G::IMG, 0, nullptr, 0);
      if (jac) {
        const int F = a.F;
        auto i1 = [&](int m, int nn) -> long long { return a.off_w1 + (long long)nn * F + m; };
        jac_flush<decltype(i1), NQ>(s, a.jac, tile, 0, D, i1);
        if (cg == 0) {   // db1 (lane m = hidden unit) and db2 (lane m < D = feature) per configuration:
                         // column 0 of each 16-column block
          float re[16], im[16];
          for (int pr = 0; pr < 2 && pr < a.jac.cpt / 2; ++pr) {
            const size_t v0 = tile * a.jac.cpt + 2 * pr;
            tmem_ld16x2(s.tmem + lane_addr + G::C_JB1 + 16 * (2 * pr), re,
                        s.tmem + lane_addr + G::C_JB1 + 16 * (2 * pr + 1), im);
            if (v0 + 1 < a.jac.nvirt) jac_put2(a.jac, v0 >> 1, a.off_b1 + row, re[0], im[0]);
            if (a.do_db2) {
              tmem_ld16x2(s.tmem + lane_addr + G::C_JB2 + 16 * (2 * pr), re,
                          s.tmem + lane_addr + G::C_JB2 + 16 * (2 * pr + 1), im);
              if (row < D && v0 + 1 < a.jac.nvirt) jac_put2(a.jac, v0 >> 1, a.off_b2 + row, re[0], im[0]);
            }
          }
        }
        tc_fence_before();
        if (!sync_ok(s, true)) break;
        if (threadIdx.x == 0) {
          tc_fence_after();
          for (int c = 0; c < 4 && c < a.jac.cpt; ++c)   // dW2_c per config
            mma_mm_rows(s, gs, G::HC, dxs, D, D, 64 * c, a.jac.rpc * c, a.jac.rpc / 16);
          mma_commit(bar2);
        }
        ok = mbar_wait(bar2, ph2);
        ph2 ^= 1u;
        tc_fence_after();
        if (!sync_ok(s, ok)) break;
        if (a.jac.o16) {   // dU image region (32 KB): free, its MMAs have completed
          jac_flush_rows<NQ>(s, a.jac, tile, 0, D, a.off_w2, D, G::HC, reinterpret_cast<float *>(sm + G::DU_OFF));
        } else {
          auto i2 = [&](int m, int nn) -> long long { return a.off_w2 + (long long)m * D + nn; };
          jac_flush<decltype(i2), NQ>(s, a.jac, tile, 0, D, i2);
        }
      }
#pragma unroll
      for (int j = 0; j < QD; j += 16) {
        float v[16];
        tmem_ld16(s.tmem + lane_addr + G::C_DX + cg * QD + j, v);
#pragma unroll
        for (int e = 0; e < 16; e += 4) {
          float4 *dst = reinterpret_cast<float4 *>(a.dxm + rg + j + e);
          if constexpr (ADD) {
            atomicAdd(dst, make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]));
          } else {
            const float4 b = base[(j + e) / 4];
            *dst = make_float4(b.x + v[e], b.y + v[e + 1], b.z + v[e + 2], b.w + v[e + 3]);
          }
        }
      }
      first = false;
      if (jac && has_next) {   // TMEM [0, 256) read out: the next tile's MMA1, then its successor's Xmid load
        if (!issue_mma1(buf ^ 1)) break;
        if (tile + 2 * step < ntl) load2(s, xs, a.xmid + (tile + 2 * step) * (size_t)G::IMG, G::IMG, 0, nullptr, 0);
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  if (!s.bad && !first && !jac) {
    float *g = a.g + (size_t)(blockIdx.x % kCopiesMax) * a.g_stride;
    const int F = a.F;
    // dW1_c^T block: lane m = hidden unit (of this half), column n = input feature i
    auto i1 = [&](int m, int n) -> long long { return a.off_w1 + (long long)n * F + m; };
    auto i2 = [&](int m, int n) -> long long { return a.off_w2 + (long long)m * D + n; };
    flush_block<decltype(i1), NQ>(s, G::C_W1, D, g, i1);
    flush_block<decltype(i2), NQ>(s, G::C_W2, D, g, i2);
    if (cg == 0) {   // lane m of the db1 accumulator = hidden unit m of this half; of db2 = feature m < D
      float v[16], w[16];
      tmem_ld16x2(s.tmem + lane_addr + G::C_B1, v, s.tmem + lane_addr + G::C_B2, w);
      atomicAdd(g + a.off_b1 + row, v[0]);
      if (a.do_db2 && row < D) atomicAdd(g + a.off_b2 + row, w[0]);
    }
  }
  if (s.bad) mbar_wait(bar2, ph2);   // bounded: the error path waits out a product still in flight
  sync_finish(s);
}

// ====================================================================================== attention pass 1
// One warp per (sequence, head) does the softmax attention forward and backward with warp-level MMAs on
// FP16 copies of Q, K, V, dH (row stride D + 8 halves: ldmatrix rows on distinct banks): one 16-row block
// for N <= 16, two query and two key blocks for 17 <= N <= 32.  The 16 zero rows after the tile keep every
// block in bounds: a sequence's blocks reach row (ts - 1) N + 31 <= 136 for N >= 17.
template <int D>
struct A1Geo {
  static constexpr int IMG = kRows * D * 2;
  static constexpr int LDH = D + 8;
  static constexpr int HROWS = kRows + 16;
  static constexpr int W_OFF = 0;                      // Wqkv^T [3D][D] (the forward's image), kept
  static constexpr int W_BYTES = 3 * D * D * 2;
  static constexpr int WO_OFF = W_OFF + W_BYTES;       // Wo rows [D][D], kept
  static constexpr int X_OFF = WO_OFF + D * D * 2;     // X images [2][128][D] (the next tile's early)
  static constexpr int DX_OFF = X_OFF + 2 * IMG;       // dX' BF16 images [2][128][D] (read by dWo of the tile)
  static constexpr int H_OFF = DX_OFF + 2 * IMG;       // head outputs [128][128] BF16 (upper half zero)
  static constexpr int F_OFF = H_OFF + kRows * 128 * 2;   // Q, K, V, dH FP16 [HROWS][LDH] each
  static constexpr int F_BYTES = HROWS * LDH * 2;
  static constexpr int M_OFF = F_OFF + 4 * F_BYTES;
  static constexpr int BYTES = M_OFF + 64;
  static constexpr int C_QKV = 0, C_DH = 3 * D, C_WO = 256;
  static constexpr int C_JWO = 256;   // per-configuration mode: 4 x D dWo columns
};

struct A1Args {
  const uint8_t *wqkvT, *wo;      // packed: Wqkv^T [3D][D] (forward image), Wo rows [D][D]
  const uint8_t *x;               // [tiles] layer-input images
  const float *dxm;               // FP32 [tiles*128][D]
  uint8_t *dqkv;                  // out [tiles] images [128][3D]
  size_t tiles;
  const int64_t *dB;              // device row count (null: every tile); tiles is then a bound
  int n, ts, heads;
  float *g;
  size_t g_stride;
  long long off_wo;
  int *err;
  JacOut jac;
};

// 512 threads: thread (row, quarter) stages a quarter of the columns; 16 warps share the tile's
// (sequence, head) attention units.  The next tile's dX' rows are read during this tile; in VJP mode the
// dWo product of a tile (barrier bar2) completes behind the next tile's loads and products.
constexpr int kA1Threads = 512;

template <int D, int HD>
__global__ void __launch_bounds__(kA1Threads, 1) k_bwd_attn1(A1Args a) {
  using G = A1Geo<D>;
  extern __shared__ __align__(1024) uint8_t sm[];
  constexpr int NQ = kA1Threads / 128, QC = D / NQ, LDH = G::LDH;
  static_assert(QC % 16 == 0, "column groups of 16");
  const uint32_t bar2 = smem_u32(sm + G::M_OFF + 24);
  uint32_t ph2 = 0;
  bool pend2 = false;
  if (threadIdx.x == 0) mbar_init(bar2, 1);   // made visible by the fence and barrier in sync_init
  Sync s;
  sync_init(s, sm + G::M_OFF, a.err);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (warp & 3) + lane, quarter = warp >> 2;
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t wr = smem_u32(sm + G::W_OFF), wo = smem_u32(sm + G::WO_OFF), xs0 = smem_u32(sm + G::X_OFF),
                 dxs0 = smem_u32(sm + G::DX_OFF), hs = smem_u32(sm + G::H_OFF), f16 = smem_u32(sm + G::F_OFF);
  __half *Fh = reinterpret_cast<__half *>(sm + G::F_OFF);   // Q, K, V, dH at multiples of HROWS * LDH
  for (int i = threadIdx.x; i < kRows * 128 * 2 / 16; i += kA1Threads)
    reinterpret_cast<uint4 *>(sm + G::H_OFF)[i] = make_uint4(0, 0, 0, 0);
  for (int i = threadIdx.x; i < 4 * 16 * LDH / 8; i += kA1Threads) {   // the 16 rows after each tile block
    const int arr = i / (16 * LDH / 8), k = i % (16 * LDH / 8);
    reinterpret_cast<uint4 *>(Fh + arr * G::HROWS * LDH + kRows * LDH)[k] = make_uint4(0, 0, 0, 0);
  }
  const int n = a.n, nvalid = a.ts * n;
  const bool valid = row < nvalid;
  const float qscale = rsqrtf((float)HD) * 1.4426950408889634f;   // scores in base 2
  const float scale = rsqrtf((float)HD);
  if (threadIdx.x == 0) {   // both weight images once per kernel
    mbar_expect_tx(s.bar_ld, G::W_BYTES + D * D * 2);
    bulk_g2s(wr, a.wqkvT, G::W_BYTES, s.bar_ld);
    bulk_g2s(wo, a.wo, D * D * 2, s.bar_ld);
  }
  bool ok = wait_ld(s);
  bool first = true;
  const size_t ntl = tiles_now(a.dB, a.tiles, a.ts / 2);
  if (sync_ok(s, ok)) {
    if ((size_t)blockIdx.x < ntl) load2(s, xs0, a.x + blockIdx.x * (size_t)G::IMG, G::IMG, 0, nullptr, 0);
    float4 nx[QC / 4];   // this thread's dX' of the coming tile
    auto load_nx = [&](size_t t) {
      const float4 *src = reinterpret_cast<const float4 *>(a.dxm + (t * kRows + row) * (size_t)D + quarter * QC);
#pragma unroll
      for (int j = 0; j < QC / 4; ++j) nx[j] = src[j];
    };
    if ((size_t)blockIdx.x < ntl) load_nx(blockIdx.x);
    int buf = 0;
    for (size_t tile = blockIdx.x; tile < ntl; tile += gridDim.x, buf ^= 1) {
      const uint32_t xs = xs0 + buf * G::IMG, dxs = dxs0 + buf * G::IMG;
      {   // this buffer was last read by the dWo product two tiles back, waited for in the previous tile
        float v[QC];
#pragma unroll
        for (int j = 0; j < QC; j += 4) {
          const float4 q = nx[j / 4];
          v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
        }
#pragma unroll
        for (int j = 0; j < QC; j += 8) st_row8<kF16>(sm + G::DX_OFF + buf * G::IMG, row, quarter * QC + j, D, v + j);
      }
      if (tile + gridDim.x < ntl) load_nx(tile + gridDim.x);
      ok = wait_ld(s);   // this tile's X image
      fence_proxy_async();
      if (!sync_ok(s, ok)) break;
      {   // the other X buffer was last read by the previous tile's MMAs, which have completed
        const size_t nxt = tile + gridDim.x;
        if (nxt < ntl) load2(s, xs0 + (buf ^ 1) * G::IMG, a.x + nxt * (size_t)G::IMG, G::IMG, 0, nullptr, 0);
      }
      if (threadIdx.x == 0) {
        tc_fence_after();
        mma_kk(s, xs, wr, D, 3 * D, G::C_QKV, false);   // Q, K, V
        mma_kk(s, dxs, wo, D, D, G::C_DH, false);       // dH = dX' Wo^T
        mma_commit(s.bar_mma);
      }
      ok = wait_mma(s);
      if (pend2) {   // the previous tile's dWo product: complete, the products just waited for came after it
        ok = mbar_wait(bar2, ph2) && ok;
        ph2 ^= 1u;
        pend2 = false;
      }
      if (!sync_ok(s, ok)) break;
      // Q, K, V, dH -> FP16 rows (TMEM loads are warp-collective; rows past the tile's sequences stay)
      static_assert(QC == 16, "one 16-column group per part");
#pragma unroll
      for (int pp = 0; pp < 2; ++pp) {   // parts (Q, K) then (V, dH): two TMEM loads per wait
        float v[2][16];
        tmem_ld16x2(s.tmem + lane_addr + G::C_QKV + (2 * pp) * D + quarter * QC, v[0],
                    s.tmem + lane_addr + (pp == 0 ? G::C_QKV + D : G::C_DH) + quarter * QC, v[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          __half *dst = Fh + (2 * pp + h) * G::HROWS * LDH + row * LDH + quarter * QC;
          const float *w = v[h];
          reinterpret_cast<uint4 *>(dst)[0] = make_uint4(amma::h2(w[0], w[1]), amma::h2(w[2], w[3]),
                                                         amma::h2(w[4], w[5]), amma::h2(w[6], w[7]));
          reinterpret_cast<uint4 *>(dst)[1] = make_uint4(amma::h2(w[8], w[9]), amma::h2(w[10], w[11]),
                                                         amma::h2(w[12], w[13]), amma::h2(w[14], w[15]));
        }
      }
      (void)valid;
      __syncthreads();   // every row's Q, K, V, dH visible
      uint8_t *dq_img = a.dqkv + tile * (size_t)(kRows * 3 * D * 2);
      for (int i = threadIdx.x; i < (kRows - nvalid) * (3 * D / 8); i += kA1Threads) {   // padding rows: dQKV = 0
        const int r = nvalid + i / (3 * D / 8), c8 = i % (3 * D / 8);
        *reinterpret_cast<uint4 *>(dq_img + canon(r, 8 * c8, 3 * D)) = make_uint4(0, 0, 0, 0);
      }
      auto units = [&](auto full) {
        constexpr int H = D / HD;   // heads (d_model = heads x head dimension)
        for (int u = warp; u < a.ts * H; u += kA1Threads / 32) {
          const int sq = u / H, h = u % H, rb = sq * (decltype(full)::value ? 16 : n);
          const uint32_t off = (uint32_t)(rb * LDH + h * HD) * 2;
          amma::attn_fwd_bwd_h<HD, decltype(full)::value>(
              f16 + off, f16 + G::F_BYTES + off, f16 + 2 * G::F_BYTES + off, f16 + 3 * G::F_BYTES + off, LDH, n,
              qscale, scale, [&](int kind, int r, int c, float v0, float v1) {
                const int rr = rb + r, col = h * HD + c;
                if (kind == 0)
                  *reinterpret_cast<uint32_t *>(sm + G::H_OFF + canon(rr, col, 128)) = pack16<kF16>(v0, v1);
                else   // dQ, dK: BF16 (FP32's exponent range; they sit decades below dV); dV: the operand type
                  *reinterpret_cast<uint32_t *>(dq_img + canon(rr, (kind - 1) * D + col, 3 * D)) =
                      kind < 3 ? pack_bf16(v0, v1) : pack16<kF16>(v0, v1);
              });
        }
      };
      if (n == 16) {
        units(std::true_type{});
      } else if (n <= 16) {
        units(std::false_type{});
      } else {   // 17 to 32 tokens: one warp per (sequence, head), both 16-query blocks
        constexpr int H = D / HD;
        for (int u = warp; u < a.ts * H; u += kA1Threads / 32) {
          const int sq = u / H, h = u % H, rb = sq * n;
          const uint32_t off = (uint32_t)(rb * LDH + h * HD) * 2;
          amma::attn_fwd_bwd_h32<HD>(
              f16 + off, f16 + G::F_BYTES + off, f16 + 2 * G::F_BYTES + off, f16 + 3 * G::F_BYTES + off, LDH, n,
              qscale, scale, [&](int kind, int r, int c, float v0, float v1) {
                const int rr = rb + r, col = h * HD + c;
                if (kind == 0)
                  *reinterpret_cast<uint32_t *>(sm + G::H_OFF + canon(rr, col, 128)) = pack16<kF16>(v0, v1);
                else
                  *reinterpret_cast<uint32_t *>(dq_img + canon(rr, (kind - 1) * D + col, 3 * D)) =
                      kind < 3 ? pack_bf16(v0, v1) : pack16<kF16>(v0, v1);
              });
        }
      }
      fence_proxy_async();
      if (!sync_ok(s, true)) break;
      if (threadIdx.x == 0) {
        tc_fence_after();
        if (!a.jac.nvirt) {
          mma_mm(s, hs, 128, dxs, D, D, G::C_WO, !first);   // dWo += H^T dX'   (rows of H beyond D are zero)
          mma_commit(bar2);
        } else {
          for (int c = 0; c < 4 && c < a.jac.cpt; ++c)
            mma_mm_rows(s, hs, 128, dxs, D, D, G::C_JWO + 64 * c, a.jac.rpc * c, a.jac.rpc / 16);
          mma_commit(s.bar_mma);
        }
      }
      first = false;
      ok = true;
      if (!a.jac.nvirt) {
        pend2 = true;
      } else {
        ok = wait_mma(s);
        if (!sync_ok(s, ok)) break;
        if (a.jac.o16) {   // FP16 attention copies (free after the attention)
          jac_flush_rows<NQ>(s, a.jac, tile, G::C_JWO, D, a.off_wo, D, D, reinterpret_cast<float *>(sm + G::F_OFF));
        } else {
          auto iwo = [&](int m, int nn) -> long long { return m < D ? a.off_wo + (long long)m * D + nn : -1; };
          jac_flush<decltype(iwo), NQ>(s, a.jac, tile, G::C_JWO, D, iwo);
        }
      }
      tc_fence_before();
      if (!sync_ok(s, ok)) break;
    }
  }
  if (pend2) {   // the last tile's dWo product (bounded wait, also on the error path)
    const bool okw = mbar_wait(bar2, ph2);
    ph2 ^= 1u;
    tc_fence_after();
    sync_ok(s, okw);
  }
  if (!s.bad && !first && !a.jac.nvirt) {
    float *g = a.g + (size_t)(blockIdx.x % kCopiesMax) * a.g_stride;
    auto iwo = [&](int m, int nn) -> long long { return m < D ? a.off_wo + (long long)m * D + nn : -1; };
    flush_block<decltype(iwo), NQ>(s, G::C_WO, D, g, iwo);
  }
  sync_finish(s);
}

// ====================================================================================== attention pass 2
template <int D>
struct A2Geo {
  static constexpr int IMG = kRows * D * 2;
  static constexpr int QIMG = kRows * 3 * D * 2;
  static constexpr int W_OFF = 0;                       // Wqkv rows [D][3D]
  static constexpr int W_BYTES = 3 * D * D * 2;
  static constexpr int XR_OFF = W_OFF + W_BYTES;        // X images as stored [2][128][D] (next tile early)
  static constexpr int ST_OFF = XR_OFF + 2 * IMG;       // per-configuration mode: flush staging, 2 KB per warp
  static constexpr int DQ_OFF = ST_OFF + 16 * 2048;     // [dQ dK dV] images [2][128][3D]
  static constexpr int XB_OFF = DQ_OFF + 2 * QIMG;      // FP16 operands: a BF16 copy of the tile's X image
  static constexpr int M_OFF = XB_OFF + IMG;             // misc: bars, holder, dE [4][4][D]
  static constexpr int BYTES = M_OFF + 64 + 4 * 4 * 4 * D;
  static constexpr int C_W = 0, C_DX = 256;
};

struct A2Args {
  const uint8_t *wqkv;            // packed Wqkv rows [D][3D]
  const uint8_t *x, *dqkv;        // [tiles] images
  const float *dxm;               // FP32 [tiles*128][D] (dX')
  float *dxo;                     // FP32 out: dX at the layer input
  size_t tiles;
  const int64_t *dB;              // device row count (null: B and every tile); B and tiles are then bounds
  int n, ts, embed_grad;
  const uint32_t *sig, *sigp;     // configurations (for the embedding gradient)
  size_t B;
  float *g;
  size_t g_stride;
  long long off_wq, off_wk, off_wv, off_e;
  int *err;
  JacOut jac;
};

// 512 threads: thread (row, quarter) owns a quarter of dX's columns; the next tile's dX' rows are read
// during this tile.  The weight-gradient MMAs read the stored X image MN-major with M = 128: TMEM lanes
// >= D then hold sums of unrelated image bytes and are never read.
constexpr int kA2Threads = 512;

template <int D>
__global__ void __launch_bounds__(kA2Threads, 1) k_bwd_attn2(A2Args a) {
  using G = A2Geo<D>;
  extern __shared__ __align__(1024) uint8_t sm[];
  constexpr int NQ = kA2Threads / 128, QC = D / NQ;
  static_assert(QC % 16 == 0, "column groups of 16");
  Sync s;
  sync_init(s, sm + G::M_OFF, a.err);
  float *dE = reinterpret_cast<float *>(sm + G::M_OFF + 64);   // [4][D], or [4 configurations][4][D]
  for (int i = threadIdx.x; i < 4 * 4 * D; i += kA2Threads) dE[i] = 0.f;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (warp & 3) + lane, quarter = warp >> 2;
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t wq = smem_u32(sm + G::W_OFF), xr0 = smem_u32(sm + G::XR_OFF), dq0 = smem_u32(sm + G::DQ_OFF);
  // the dQ, dK block of the [dQ dK dV] image is BF16: with FP16 operands its products take a BF16 copy of X
  // and BF16 rows of Wq, Wk (packed so); with BF16 operands everything is BF16 already
  const uint32_t xb = kF16 ? smem_u32(sm + G::XB_OFF) : 0u;
  if (threadIdx.x == 0) {
    mbar_expect_tx(s.bar_ld, G::W_BYTES);
    bulk_g2s(wq, a.wqkv, G::W_BYTES, s.bar_ld);
  }
  bool ok = wait_ld(s);
  const int n = a.n, nvalid = a.ts * n, tc = a.ts / 2;
  const size_t ntl = tiles_now(a.dB, a.tiles, tc), Bn = rows_now(a.dB, a.B);
  bool first = true;
  if (sync_ok(s, ok)) {
    if ((size_t)blockIdx.x < ntl)
      load2(s, xr0, a.x + blockIdx.x * (size_t)G::IMG, G::IMG, dq0, a.dqkv + blockIdx.x * (size_t)G::QIMG, G::QIMG);
    float4 nx[QC / 4];   // this thread's dX' of the coming tile
    auto load_nx = [&](size_t t) {
      const float4 *src = reinterpret_cast<const float4 *>(a.dxm + (t * kRows + row) * (size_t)D + quarter * QC);
#pragma unroll
      for (int j = 0; j < QC / 4; ++j) nx[j] = src[j];
    };
    if ((size_t)blockIdx.x < ntl) load_nx(blockIdx.x);
    int buf = 0;
    for (size_t tile = blockIdx.x; tile < ntl; tile += gridDim.x, buf ^= 1) {
      const uint32_t dq = dq0 + buf * G::QIMG, xr = xr0 + buf * G::IMG;
      const size_t rg = (tile * kRows + row) * (size_t)D + quarter * QC;
      float base[QC];
#pragma unroll
      for (int j = 0; j < QC; j += 4) {
        const float4 q = nx[j / 4];
        base[j] = q.x; base[j + 1] = q.y; base[j + 2] = q.z; base[j + 3] = q.w;
      }
      if (tile + gridDim.x < ntl) load_nx(tile + gridDim.x);
      ok = wait_ld(s);   // this tile's X and [dQ dK dV] images
      if (!sync_ok(s, ok)) break;
      if (kF16) {   // BF16 copy of the X image (same canonical layout); its last reader, the previous tile's
                    // MMAs, has completed
        const uint4 *src = reinterpret_cast<const uint4 *>(sm + G::XR_OFF + buf * G::IMG);
        uint4 *dst = reinterpret_cast<uint4 *>(sm + G::XB_OFF);
        for (int i = threadIdx.x; i < G::IMG / 16; i += kA2Threads) {
          const uint4 q = src[i];
          const uint32_t w[4] = {q.x, q.y, q.z, q.w};
          uint32_t o[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[e]));
            o[e] = pack_bf16(f.x, f.y);
          }
          dst[i] = make_uint4(o[0], o[1], o[2], o[3]);
        }
        fence_proxy_async();
        __syncthreads();
      }
      {   // the other buffers were last read by the previous tile's MMAs, which have completed
        const size_t nxt = tile + gridDim.x;
        if (nxt < ntl)
          load2(s, xr0 + (buf ^ 1) * G::IMG, a.x + nxt * (size_t)G::IMG, G::IMG, dq0 + (buf ^ 1) * G::QIMG,
                a.dqkv + nxt * (size_t)G::QIMG, G::QIMG);
      }
      if (threadIdx.x == 0) {
        tc_fence_after();
        if (kF16) {
          if (!a.jac.nvirt) {   // dWq, dWk += X^T [dQ dK] (BF16); dWv += X^T dV (FP16)
            mma_mm_t<false>(s, xb, D, dq, 3 * D, 2 * D, G::C_W, !first);
            mma_mm_t<true>(s, xr, D, dq + (2 * D / 8) * 128, 3 * D, D, G::C_W + 2 * D, !first);
          }
          mma_kk_range<false>(s, dq, wq, 3 * D, 0, 2 * D, D, G::C_DX, false);   // [dQ dK] [Wq Wk]^T
          mma_kk_range<true>(s, dq, wq, 3 * D, 2 * D, 3 * D, D, G::C_DX, true);  // + dV Wv^T
        } else {
          if (!a.jac.nvirt) mma_mm(s, xr, D, dq, 3 * D, 3 * D, G::C_W, !first);   // dWqkv += X^T [dQ dK dV]
          mma_kk(s, dq, wq, 3 * D, D, G::C_DX, false);            // [dQ dK dV] Wqkv^T
        }
        mma_commit(s.bar_mma);
      }
      ok = wait_mma(s);
      if (!sync_ok(s, ok)) break;
      float out[QC];   // dX = dX' + [dQ dK dV] Wqkv^T, read out first (its TMEM columns are reused below)
#pragma unroll
      for (int j = 0; j < QC; j += 16) {
        float v[16];
        tmem_ld16(s.tmem + lane_addr + G::C_DX + quarter * QC + j, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) out[j + e] = base[j + e] + v[e];
      }
      if (a.jac.nvirt) {   // dWq, dWk, dWv per configuration: 4 x D column blocks, alternately at TMEM
                           // columns 0 and 256, the next part's MMAs running under this part's flush
        tc_fence_before();
        if (!sync_ok(s, true)) break;
        auto issue_part = [&](int part) {
          if (threadIdx.x == 0) {
            tc_fence_after();
            // columns [D part, D part + D) of the [dQ dK dV] image start (D / 8) MN groups (128 B each) in
            const int rpc = a.jac.rpc, ks = rpc / 16;
            for (int c = 0; c < 4 && c < a.jac.cpt; ++c) {
              if (kF16 && part < 2)   // dQ, dK parts: BF16
                mma_mm_rows<false>(s, xb, D, dq + part * (D / 8) * 128, 3 * D, D, 256 * (part & 1) + 64 * c, rpc * c, ks);
              else
                mma_mm_rows(s, xr, D, dq + part * (D / 8) * 128, 3 * D, D, 256 * (part & 1) + 64 * c, rpc * c, ks);
            }
            mma_commit(s.bar_mma);
          }
        };
        issue_part(0);
        bool fine = true;
        for (int part = 0; part < 3 && fine; ++part) {
          fine = wait_mma(s);
          if (!sync_ok(s, fine)) break;
          if (part + 1 < 3) issue_part(part + 1);   // into the other column half, free since part - 1's flush
          const long long off = part == 0 ? a.off_wq : part == 1 ? a.off_wk : a.off_wv;
          const uint32_t col0 = 256 * (part & 1);
          if (a.jac.o16) {
            jac_flush_rows<NQ>(s, a.jac, tile, col0, D, off, D, D, reinterpret_cast<float *>(sm + G::ST_OFF));
          } else {
            auto iw = [&](int m, int nn) -> long long { return m < D ? off + (long long)m * D + nn : -1; };
            jac_flush<decltype(iw), NQ>(s, a.jac, tile, col0, D, iw);
          }
          tc_fence_before();
          if (!sync_ok(s, true)) break;
        }
        if (s.bad) break;
      }
#pragma unroll
      for (int j = 0; j < QC; j += 4)
        *reinterpret_cast<float4 *>(a.dxo + rg + j) = make_float4(out[j], out[j + 1], out[j + 2], out[j + 3]);
      if (a.embed_grad && a.jac.nvirt && row < nvalid) {   // VJP mode: k_embed_grad after the launch
        const int sqn = row / n, i = row % n;
        const size_t b = tile * tc + (sqn >> 1);
        if (b < Bn) {
          const uint32_t w1 = (sqn & 1) ? a.sigp[b] : a.sig[b];
          const uint32_t w2 = (sqn & 1) ? a.sig[b] : a.sigp[b];
          const int pat = embed_pattern(0, w1, w2, i, n);
          // one [4][D] block per virtual configuration (sqn >> 1) of the tile
          float *dst = dE + (sqn >> 1) * 4 * D;
#pragma unroll
          for (int j = 0; j < QC; ++j) atomicAdd(&dst[pat * D + quarter * QC + j], out[j]);
        }
      }
      if (a.jac.nvirt && a.embed_grad) {
        __syncthreads();
        for (int i = threadIdx.x; i < a.jac.cpt * 4 * D; i += kA2Threads) {
          const size_t v = tile * a.jac.cpt + i / (4 * D);
          if (v < a.jac.nvirt) jac_put1(a.jac, v, a.off_e + i % (4 * D), dE[i]);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < a.jac.cpt * 4 * D; i += kA2Threads) dE[i] = 0.f;
      }
      first = false;
      tc_fence_before();
      __syncthreads();
    }
  }
  if (!s.bad && !first && !a.jac.nvirt) {
    float *g = a.g + (size_t)(blockIdx.x % kCopiesMax) * a.g_stride;
    auto iw = [&](int m, int nn) -> long long {
      if (m >= D) return -1;
      if (nn < D) return a.off_wq + (long long)m * D + nn;
      if (nn < 2 * D) return a.off_wk + (long long)m * D + (nn - D);
      return a.off_wv + (long long)m * D + (nn - 2 * D);
    };
    flush_block<decltype(iw), NQ>(s, G::C_W, 3 * D, g, iw);
  }
  sync_finish(s);
}

// Non-transposed 16-bit packing: dst canonical [N][Ktot], element (n, koff + k) = W[n * ldw + col0 + k].
__global__ void k_pack_nt(const float *__restrict__ W, int ldw, int col0, int K, int N, int Ktot, int koff,
                          uint8_t *__restrict__ dst, int f16) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * K) return;
  const int nn = i / K, k = i % K;
  const float w = W[(size_t)nn * ldw + col0 + k];
  if (f16) *reinterpret_cast<__half *>(dst + canon(nn, koff + k, Ktot)) = __float2half_rn(w);
  else *reinterpret_cast<__nv_bfloat16 *>(dst + canon(nn, koff + k, Ktot)) = __float2bfloat16_rn(w);
}

// Power-of-two scale of the backward's cotangents (the VJP's, or the +-1 seeds of the log-derivatives):
// with m = max_b max(|Re c_b|, |Im c_b|) and h = max_c (|Wh[c][0]| + |Wh[c][1]|), the last layer's dX is
// at most B = 2 m h / N per element; scale[0] = 2^(11 - e) with B = f 2^e, f in [0.5, 1) (1 when B is zero
// or not finite), scale[1] = 1 / scale[0].  It puts the largest gradient signal of the last layer near
// 2^11, so that the backward's FP16 images hold the bulk of the signals (whose median sits three to five
// decades below the largest) above FP16's subnormals, with 2^5 of headroom for their growth towards the
// first layer; the exact power of two is undone on every output.
__global__ void __launch_bounds__(1024) k_cot_scale(const float2 *__restrict__ cot, size_t B,
                                                     const float *__restrict__ Wh, int D, int n,
                                                     float *__restrict__ scale, const int64_t *dB) {
  __shared__ float red[32];
  float m = 0.f, h = 0.f;
  B = rows_now(dB, B);
  for (size_t b = threadIdx.x; b < B; b += blockDim.x) {
    const float2 c = cot[b];
    m = fmaxf(m, fmaxf(fabsf(c.x), fabsf(c.y)));   // a NaN operand is dropped by fmaxf; caught downstream
  }
  for (int c = threadIdx.x; c < D; c += blockDim.x) h = fmaxf(h, fabsf(Wh[2 * c]) + fabsf(Wh[2 * c + 1]));
  m *= 2.0f;   // (both orders of the doubled configuration)
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  float mh = 0.f;
  if (threadIdx.x < 32) {
    mh = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) mh = fmaxf(mh, __shfl_xor_sync(0xffffffffu, mh, o));
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = h;
  __syncthreads();
  if (threadIdx.x < 32) {
    h = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
    if (threadIdx.x == 0) {
      const float bound = mh * h / (float)n;
      int e = 0;
      if (bound > 0.f && isfinite(bound)) frexpf(bound, &e);
      int k = 11 - e;
      k = k < -100 ? -100 : (k > 100 ? 100 : k);
      scale[0] = ldexpf(1.0f, k);
      scale[1] = ldexpf(1.0f, -k);
    }
  }
}

}  // namespace TDO_BWNS
}  // namespace tdo

// ------------------------------------------------------------------------------------- host side
#include "../../include/tdo.h"

struct BwdTcLayer {
  const uint8_t *w1t[2], *w2r[2], *w1r[2];   // per hidden half
  const uint8_t *wqkvT, *wor, *wqkvr;
};

#if !TDO_F16   // operand-independent
size_t bwdtc_packed_bytes(const DevModel &m) {
  const size_t D = m.d, F = m.ffn;
  return (size_t)m.layers * (2 * F * D + D * D + 3 * D * D) * 2;
}
#endif

// Row-major (non-transposed) 16-bit images for the backward; views per layer into dst.
cudaError_t TDO_OPFN(launch_pack_bwdtc)(const DevModel &m, uint8_t *dst, BwdTcLayer *views, cudaStream_t st) {
  using namespace tdo::TDO_BWNS;
  const int D = m.d, F = m.ffn;
  size_t off = 0;
  auto pack = [&](const float *W, int ldw, int col0, int K, int N, int Ktot, int koff, uint8_t *out,
                  int f16 = kF16 ? 1 : 0) {
    k_pack_nt<<<(N * K + 255) / 256, 256, 0, st>>>(W, ldw, col0, K, N, Ktot, koff, out, f16);
  };
  for (int l = 0; l < m.layers; ++l) {
    const DevLayer &L = m.L[l];
    BwdTcLayer &v = views[l];
    if (F > 0) {
      for (int hb = 0; hb < F / 128; ++hb) {
        v.w2r[hb] = dst + off;    // W2 rows hb*128.. : [128][D]
        pack(L.W2 + (size_t)hb * 128 * D, D, 0, D, 128, D, 0, dst + off);
        off += (size_t)128 * D * 2;
        v.w1r[hb] = dst + off;    // W1 rows, columns hb*128.. : [D][128]
        pack(L.W1, F, hb * 128, 128, D, 128, 0, dst + off);
        off += (size_t)128 * D * 2;
      }
    }
    v.wor = dst + off;
    pack(L.Wo, D, 0, D, D, D, 0, dst + off);
    off += (size_t)D * D * 2;
    v.wqkvr = dst + off;
    pack(L.Wq, D, 0, D, D, 3 * D, 0, dst + off, 0);   // the rows multiplying the BF16 dQ, dK block
    pack(L.Wk, D, 0, D, D, 3 * D, D, dst + off, 0);
    pack(L.Wv, D, 0, D, D, 3 * D, 2 * D, dst + off);
    off += (size_t)3 * D * D * 2;
  }
  return cudaGetLastError();
}

#if !TDO_F16
bool bwdtc_supported(const DevModel &m) {
  return m.d == 64 && (m.dh == 8 || m.dh == 16) && m.heads % 2 == 0 && m.heads <= 16 &&
         (m.ffn == 0 || m.ffn == 128 || m.ffn == 256) && m.embed == 0 && m.n_sites <= 32;
}
#endif

struct BwdTcBuffers {
  uint8_t *x, *xmid, *dqkv;
  float *h, *f, *dF, *dxa, *dxb;
  size_t tiles;
  float *cscale;   // [2]: cotangent scale and its inverse (VJP mode)
};

// Token-embedding gradient of the VJP: dE[p][c] = sum over the rows whose token is p of dX[row][c], dX the
// gradient at the first layer's input ([tiles * 128][D] FP32, tile-major rows).  Thread = (row slot,
// 4 columns); 4 x 4 register sums per thread (no shared-memory atomics on the 4 hot rows of dE), one
// block reduction, then float atomics into the block's gradient copy.
namespace tdo {
namespace TDO_BWNS {
__global__ void __launch_bounds__(256) k_embed_grad(const float *__restrict__ dX, const uint32_t *__restrict__ sig,
                                                    const uint32_t *__restrict__ sigp, size_t B, int n, int ts,
                                                    size_t tiles, float *__restrict__ g, size_t g_stride,
                                                    long long off_e, const int64_t *dB) {
  constexpr int D = 64, CG = D / 4, SLOTS = 256 / CG;
  __shared__ float4 red[SLOTS][4][CG];
  const int cg = threadIdx.x % CG, slot = threadIdx.x / CG, tc = ts / 2, nvalid = ts * n;
  float4 acc[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) acc[p] = make_float4(0.f, 0.f, 0.f, 0.f);
  const size_t rows = tiles_now(dB, tiles, tc) * kRows;
  B = rows_now(dB, B);
  // each block streams one contiguous range of rows (UNR * SLOTS rows = 16 KB per iteration); UNR rows per
  // thread and iteration, all loads first: enough bytes in flight to stream dX
  constexpr int UNR = 4;
  const size_t per = (rows + gridDim.x - 1) / gridDim.x;
  const size_t r_begin = (size_t)blockIdx.x * per, r_end = r_begin + per < rows ? r_begin + per : rows;
  for (size_t r0 = r_begin + slot; r0 < r_end; r0 += UNR * SLOTS) {
    float4 v[UNR];
    int pat[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const size_t r = r0 + u * SLOTS;
      pat[u] = -1;
      v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r >= r_end) continue;
      const int rt = (int)(r % kRows);
      if (rt >= nvalid) continue;
      const int sq = rt / n, i = rt % n;
      const size_t b = (r / kRows) * tc + (sq >> 1);
      if (b >= B) continue;
      const uint32_t w1 = (sq & 1) ? sigp[b] : sig[b];
      const uint32_t w2 = (sq & 1) ? sig[b] : sigp[b];
      pat[u] = embed_pattern(0, w1, w2, i, n);
      v[u] = __ldcs(reinterpret_cast<const float4 *>(dX + r * D) + cg);
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u)
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const float m = p == pat[u] ? 1.f : 0.f;
        acc[p].x = fmaf(m, v[u].x, acc[p].x); acc[p].y = fmaf(m, v[u].y, acc[p].y);
        acc[p].z = fmaf(m, v[u].z, acc[p].z); acc[p].w = fmaf(m, v[u].w, acc[p].w);
      }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) red[slot][p][cg] = acc[p];
  __syncthreads();
  if (threadIdx.x < 4 * CG) {
    const int p = threadIdx.x / CG, c = threadIdx.x % CG;
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = 0; q < SLOTS; ++q) {
      const float4 u = red[q][p][c];
      t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
    }
    float *dst = g + (size_t)(blockIdx.x % kCopiesMax) * g_stride + off_e + p * D + 4 * c;
    atomicAdd(dst, t.x); atomicAdd(dst + 1, t.y); atomicAdd(dst + 2, t.z); atomicAdd(dst + 3, t.w);
  }
}
}  // namespace TDO_BWNS
}  // namespace tdo

// Output of the per-configuration mode (log-derivatives); nvirt = 0 selects the VJP.
struct BwdTcJac {
  float *o32;
  uint16_t *o16;
  const float2 *oref;
  size_t ldo, nvirt;
};

#if !TDO_F16
// The per-configuration mode needs 2N rows per configuration in whole 16-row K steps and at most 4
// configurations per tile (their TMEM column blocks): N = 16, 24 or 32.
bool bwdtc_jac_supported(const DevModel &m) {
  return bwdtc_supported(m) && (m.n_sites == 16 || m.n_sites == 24 || m.n_sites == 32);
}
#endif

namespace tdo {
namespace TDO_BWNS {
// VJP-mode db2 of a layer: the column sums of the FP32 dX at its MLP output, dX [rows][D] (padding rows
// zero).  A thread owns 4 columns (float4 loads, D / 4 threads per row, coalesced rows) and sums its rows in
// FP32 runs of 64, added in FP64 between runs (GB300 issues about two FP64 adds per SM and cycle: a
// dependent FP64 chain over every row took 8 ms per launch); one float atomic per column and block into
// the block's gradient copy.  (A sum over every connected row cancels heavily: summing the 16-bit image
// would leave the rounding of single rows in it.)
__global__ void __launch_bounds__(256) k_db2_rows(const float *__restrict__ dX, size_t rows, int D, float *g,
                                                  size_t g_stride, long long off, const int64_t *dB, int tc) {
  __shared__ double red[256][4];
  rows = tiles_now(dB, rows / kRows, tc) * kRows;
  const int tpr = D / 4, groups = 256 / tpr, c4 = threadIdx.x % tpr, grp = threadIdx.x / tpr;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  if (grp < groups) {
    const size_t stride = gridDim.x * (size_t)groups;
    size_t r = blockIdx.x * (size_t)groups + grp;
    while (r < rows) {
      float f[4] = {0.f, 0.f, 0.f, 0.f};
      for (int k = 0; k < 64 && r < rows; ++k, r += stride) {
        const float4 v = __ldcs(reinterpret_cast<const float4 *>(dX + r * D) + c4);
        f[0] += v.x; f[1] += v.y; f[2] += v.z; f[3] += v.w;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) a[e] += (double)f[e];
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) red[threadIdx.x][e] = a[e];
  __syncthreads();
  if (threadIdx.x < tpr) {
    for (int e = 0; e < 4; ++e) {
      double t = 0.0;
      for (int k = 0; k < groups; ++k) t += red[k * tpr + threadIdx.x][e];
      atomicAdd(g + (size_t)(blockIdx.x % kCopiesMax) * g_stride + off + 4 * threadIdx.x + e, (float)t);
    }
  }
}

// The last layer's db2, whose dX is formed from the head: every sequence has N rows, each carrying
// (1/N) Wh dF of its sequence, so db2[c] = sum_o Wh[c][o] S_o with S_o = sum over configurations of the
// F_o cotangents of both orders, dF [Bpad][4] (zero beyond B).  A grid of blocks, each summing its range
// of configurations in FP32 runs of 64 added in FP64, then adding its own Wh S into copy blockIdx % 16.
__global__ void __launch_bounds__(256) k_db2_head(const float *__restrict__ dF, size_t Bpad, const float *__restrict__ Wh,
                                                  int D, float *g, size_t g_stride, long long off, const int64_t *dB,
                                                  int tc) {
  __shared__ double red[2][256];
  Bpad = tiles_now(dB, Bpad / tc, tc) * tc;
  double s0 = 0.0, s1 = 0.0;
  const size_t stride = gridDim.x * (size_t)blockDim.x;
  size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  while (b < Bpad) {
    float f0 = 0.f, f1 = 0.f;
    for (int k = 0; k < 64 && b < Bpad; ++k, b += stride) {
      const float4 q = __ldcs(reinterpret_cast<const float4 *>(dF) + b);
      f0 += q.x + q.z;
      f1 += q.y + q.w;
    }
    s0 += (double)f0;
    s1 += (double)f1;
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = 128; w; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  float *gc = g + (size_t)(blockIdx.x % kCopiesMax) * g_stride;
  for (int c = threadIdx.x; c < D; c += blockDim.x)
    atomicAdd(gc + off + c, (float)((double)Wh[2 * c] * red[0][0] + (double)Wh[2 * c + 1] * red[1][0]));
}
}  // namespace TDO_BWNS
}  // namespace tdo

// Virtual configurations of the per-configuration mode: v = 2 b + seed, cotangent (1, 0) or (0, -1).
namespace tdo {
namespace TDO_BWNS {
__global__ void k_jac_virtual(const uint32_t *__restrict__ sig, const uint32_t *__restrict__ sigp, size_t Ns,
                              uint32_t *__restrict__ vs, uint32_t *__restrict__ vp, float2 *__restrict__ vc) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 2 * Ns; i += gridDim.x * (size_t)blockDim.x) {
    vs[i] = sig[i >> 1];
    vp[i] = sigp[i >> 1];
    vc[i] = (i & 1) ? make_float2(0.f, -1.f) : make_float2(1.f, 0.f);
  }
}
}  // namespace TDO_BWNS
}  // namespace tdo

#if !TDO_F16
cudaError_t launch_jac_virtual(const uint32_t *sig, const uint32_t *sigp, size_t Ns, uint32_t *vs, uint32_t *vp,
                               float2 *vc, cudaStream_t st) {
  const unsigned grid = (unsigned)((2 * Ns + 255) / 256 < 4096 ? (2 * Ns + 255) / 256 : 4096);
  tdo::TDO_BWNS::k_jac_virtual<<<grid ? grid : 1, 256, 0, st>>>(sig, sigp, Ns, vs, vp, vc);
  return cudaGetLastError();
}
#endif

// The whole tensor-core VJP given the forward's parked activations and the row cotangents; with jac
// (nvirt > 0) the per-configuration log-derivatives of the virtual configurations instead (gacc unused).
cudaError_t TDO_OPFN(launch_bwdtc)(const DevModel &m, const DevModelBF16 &mb, const BwdTcLayer *views, const BwdTcBuffers &bf,
                         const uint32_t *sig, const uint32_t *sigp, size_t B, const float2 *cot, float *gacc,
                         size_t g_stride, const long long *fo, int *err, int n_sm, cudaStream_t st,
                         const BwdTcJac *jac, const int64_t *dB) {
  using namespace tdo::TDO_BWNS;
  const int n_ = m.n_sites, tc_ = tdo::seqs_per_tile(n_) / 2;
  JacOut jo{nullptr, nullptr, nullptr, 0, 0, nullptr, tc_, 2 * n_};
  if (jac) jo = JacOut{jac->o32, jac->o16, jac->oref, jac->ldo, jac->nvirt, bf.cscale + 1, tc_, 2 * n_};
  constexpr int D = 64;
  const int n = m.n_sites, ts = tdo::seqs_per_tile(n), tc = ts / 2;
  const size_t tiles = bf.tiles, Bpad = tiles * tc;
  const long long *Wq = fo + 1, *Wk = Wq + TDO_MAX_LAYERS, *Wv = Wk + TDO_MAX_LAYERS, *Wo = Wv + TDO_MAX_LAYERS,
                  *W1 = Wo + TDO_MAX_LAYERS, *b1 = W1 + TDO_MAX_LAYERS, *W2 = b1 + TDO_MAX_LAYERS,
                  *b2 = W2 + TDO_MAX_LAYERS;
  const long long off_e = fo[0], off_wh = fo[1 + 8 * TDO_MAX_LAYERS], off_bh = fo[2 + 8 * TDO_MAX_LAYERS];
  cudaError_t e;
  {
    k_cot_scale<<<1, 1024, 0, st>>>(cot, B, m.Wh, D, n, bf.cscale, dB);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    HeadArgs h{cot, bf.cscale, bf.f, bf.h, m.Wh, bf.dF, B, Bpad, dB, tc, gacc, g_stride, off_wh, off_bh, D, jo};
    if (jac) {
      const unsigned grid = (unsigned)((Bpad + 255) / 256 < 1024 ? (Bpad + 255) / 256 : 1024);
      k_head_bwd<<<grid ? grid : 1, 256, (2 * D + 2) * sizeof(float), st>>>(h);
    } else {
      const unsigned grid = (unsigned)((Bpad + 7) / 8 < (size_t)4 * n_sm ? (Bpad + 7) / 8 : (size_t)4 * n_sm);
      k_head_bwd_vjp<<<grid ? grid : 1, 256, 0, st>>>(h);
    }
    if (m.ffn == 0)   // with an MLP the last layer's MLP passes form this dX from dF themselves
      k_head_dx<<<(unsigned)(tiles * kRows * D / 256 < 65535 * 8 ? (tiles * kRows * D + 255) / 256 : 65535 * 8), 256,
                  0, st>>>(bf.dF, m.Wh, D, n, ts, tiles, bf.dxa, dB);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int grid = (int)(tiles < (size_t)n_sm ? tiles : (size_t)n_sm);
  const size_t img = (size_t)kRows * D * 2;
#define TDO_COMMA ,
#define TDO_SET_SMEM(K, BYTES)                                                                 \
  if ((e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, BYTES)) != cudaSuccess) return e;
  TDO_SET_SMEM(k_bwd_mlp<D TDO_COMMA false>, MlpGeo<D>::BYTES);
  TDO_SET_SMEM(k_bwd_mlp<D TDO_COMMA true>, MlpGeo<D>::BYTES);
  TDO_SET_SMEM(k_bwd_attn2<D>, A2Geo<D>::BYTES);
  TDO_SET_SMEM(k_bwd_attn1<D TDO_COMMA 8>, A1Geo<D>::BYTES);
  TDO_SET_SMEM(k_bwd_attn1<D TDO_COMMA 16>, A1Geo<D>::BYTES);
#undef TDO_SET_SMEM
#undef TDO_COMMA
  for (int l = m.layers - 1; l >= 0; --l) {
    const BwdTcLayer &v = views[l];
    const float *dxmid = bf.dxa;
    if (m.ffn > 0) {
      for (int hb = 0; hb < m.ffn / 128; ++hb) {
        MlpArgs ma;
        ma.w1t = reinterpret_cast<const uint8_t *>(mb.W1[l]) + (size_t)hb * 128 * D * 2;
        ma.w2 = v.w2r[hb];
        ma.w1 = v.w1r[hb];
        ma.b1 = m.L[l].b1 + hb * 128;
        ma.xmid = bf.xmid + (size_t)l * tiles * img;
        ma.dxo = bf.dxa;
        ma.dxm = bf.dxb;
        ma.tiles = tiles;
        ma.dB = dB;
        ma.do_db2 = hb == 0 && jac;   // VJP mode: db2 from the FP32 dX (below)
        ma.g = gacc;
        ma.g_stride = g_stride;
        ma.off_w1 = W1[l] + hb * 128;
        ma.off_b1 = b1[l] + hb * 128;
        ma.off_w2 = W2[l] + (long long)hb * 128 * D;
        ma.off_b2 = b2[l];
        ma.F = m.ffn;
        ma.err = err;
        ma.jac = jo;
        const bool last = l == m.layers - 1;
        ma.dF = last ? bf.dF : nullptr;
        ma.Wh = last ? m.Wh : nullptr;
        ma.n = n;
        ma.ts = ts;
        if (hb == 0) k_bwd_mlp<D, false><<<grid, kMlpThreads, MlpGeo<D>::BYTES, st>>>(ma);
        else k_bwd_mlp<D, true><<<grid, kMlpThreads, MlpGeo<D>::BYTES, st>>>(ma);
      }
      dxmid = bf.dxb;
      if (!jac) {   // db2 of this layer from FP32 data (its MLP output's dX: the head's for the last layer)
        if (l == m.layers - 1)
          k_db2_head<<<(unsigned)(2 * n_sm), 256, 0, st>>>(bf.dF, Bpad, m.Wh, D, gacc, g_stride, b2[l], dB, tc);
        else
          k_db2_rows<<<(unsigned)(4 * n_sm), 256, 0, st>>>(bf.dxa, tiles * kRows, D, gacc, g_stride, b2[l], dB, tc);
      }
    }
    A1Args a1;
    a1.wqkvT = reinterpret_cast<const uint8_t *>(mb.Wqkv[l]);
    a1.wo = v.wor;
    a1.x = bf.x + (size_t)l * tiles * img;
    a1.dxm = dxmid;
    a1.dqkv = bf.dqkv;
    a1.tiles = tiles;
    a1.dB = dB;
    a1.n = n;
    a1.ts = ts;
    a1.heads = m.heads;
    a1.g = gacc;
    a1.g_stride = g_stride;
    a1.off_wo = Wo[l];
    a1.err = err;
    a1.jac = jo;
    if (m.dh == 8) k_bwd_attn1<D, 8><<<grid, kA1Threads, A1Geo<D>::BYTES, st>>>(a1);
    else k_bwd_attn1<D, 16><<<grid, kA1Threads, A1Geo<D>::BYTES, st>>>(a1);
    A2Args a2;
    a2.wqkv = v.wqkvr;
    a2.x = bf.x + (size_t)l * tiles * img;
    a2.dqkv = bf.dqkv;
    a2.dxm = dxmid;
    a2.dxo = bf.dxa;
    a2.tiles = tiles;
    a2.dB = dB;
    a2.n = n;
    a2.ts = ts;
    a2.embed_grad = l == 0;
    a2.sig = sig;
    a2.sigp = sigp;
    a2.B = B;
    a2.g = gacc;
    a2.g_stride = g_stride;
    a2.off_wq = Wq[l];
    a2.off_wk = Wk[l];
    a2.off_wv = Wv[l];
    a2.off_e = off_e;
    a2.err = err;
    a2.jac = jo;
    k_bwd_attn2<D><<<grid, kA2Threads, A2Geo<D>::BYTES, st>>>(a2);
    if (l == 0 && !jo.nvirt)
      k_embed_grad<<<(unsigned)(2 * n_sm), 256, 0, st>>>(bf.dxa, sig, sigp, B, n, ts, tiles, gacc, g_stride, off_e, dB);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}
