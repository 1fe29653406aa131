// Softmax attention of one (sequence, head) pair on one warp with warp-level tensor-core MMAs
// (mma.sync m16n8k16 / m16n8k8, FP16 operands, FP32 accumulation), for sequences of at most 32
// tokens (16-query blocks) and head dimension HD in {8, 16} (Eq. attn-head-appendix and its derivative).
//
// A 16 x 16 score block is 1/8 of one tcgen05 tile and lives in registers across the whole
// forward-and-backward of the pair, so these blocks use the warp-synchronous MMA, while the
// projections around them use tcgen05.  Fragment layouts (m16n8k16, lane = 4 g + t):
//   A [16][16]: a0 = (g, 2t..2t+1), a1 = (g+8, 2t..), a2 = (g, 8+2t..), a3 = (g+8, 8+2t..)
//   B [16][8] : b0 = (k = 2t..2t+1, n = g), b1 = (k = 8+2t.., n = g)
//   C [16][8] : c0,c1 = (g, 2t..2t+1), c2,c3 = (g+8, 2t..2t+1)
// m16n8k8 uses a0, a1 and b0 only.  The C fragments of the two key halves of a score block are,
// packed pairwise, the A fragment of the same block, and movmatrix transposes an 8 x 8 piece.
#pragma once
#include <cuda_fp16.h>

#include <cstdint>

#include "tcgen05.cuh"

namespace tdo {
namespace amma {

__device__ __forceinline__ uint32_t h2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %2, %1;" : "=r"(r) : "f"(lo), "f"(hi));
  return r;
}

// The warp-level MMA and the 8 x 8 transpose are pure register operations (not volatile: the compiler may
// schedule them among independent work); the shared-memory fragment loads below stay volatile.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma1688(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm(
      "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ uint32_t trans8(uint32_t x) {
  uint32_t r;
  asm("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(r) : "r"(x));
  return r;
}

__device__ __forceinline__ void zero4(float (&d)[4]) { d[0] = d[1] = d[2] = d[3] = 0.f; }

// dS (FP32 C fragments of this warp's 16 x 16 block) to FP16 A fragments, after scaling the block by the
// power of two that puts its largest magnitude in [2^13, 2^14).  dS = P (dA - delta) is a small difference
// times probabilities; unscaled, much of it would fall among FP16's subnormals (below 6.1e-5) or to zero,
// and the dQ, dK weight gradients built from it would be mostly rounding.  Returns the inverse factor,
// applied exactly to the FP32 products dS K and dS^T Q.
__device__ __forceinline__ float ds_pack_scaled(const float (&da)[2][4], uint32_t &x00, uint32_t &x10, uint32_t &x01,
                                                uint32_t &x11) {
  float m = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) m = fmaxf(m, fabsf(da[j][e]));
#pragma unroll
  for (int o = 1; o <= 16; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  int ex = 0;
  if (m > 0.f && isfinite(m)) frexpf(m, &ex);   // m = f 2^ex, f in [0.5, 1)
  int k = 14 - ex;
  k = k > 100 ? 100 : (k < -100 ? -100 : k);
  const float up = ldexpf(1.0f, k);
  x00 = h2(da[0][0] * up, da[0][1] * up);
  x10 = h2(da[0][2] * up, da[0][3] * up);
  x01 = h2(da[1][0] * up, da[1][1] * up);
  x11 = h2(da[1][2] * up, da[1][3] * up);
  return ldexpf(1.0f, -k);
}

// ---- shared-memory fragments by ldmatrix (FP16 row-major blocks, 16-byte-aligned rows)
__device__ __forceinline__ void ldsm2(uint32_t addr, uint32_t &r0, uint32_t &r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void ldsm4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm2t(uint32_t addr, uint32_t &r0, uint32_t &r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void ldsm4t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

// A fragment of the [16][HD] block at M (row stride ldh halves): HD = 8 fills a[0..1], HD = 16 a[0..3].
template <int HD>
__device__ __forceinline__ void frag_a(uint32_t M, int ldh, uint32_t (&a)[4]) {
  const int lane = threadIdx.x & 31;
  const int r = (lane & 7) + 8 * ((lane >> 3) & 1);
  if (HD == 8) {
    ldsm2(M + (uint32_t)(r * ldh) * 2, a[0], a[1]);
    a[2] = a[3] = 0u;
  } else {
    ldsm4(M + (uint32_t)(r * ldh + 8 * (lane >> 4)) * 2, a[0], a[1], a[2], a[3]);
  }
}
// B fragments of X^T for a [16 rows = n][HD cols = k] block X: b[j][kh] = n-tile j (rows 8j..8j+7), k half kh.
template <int HD>
__device__ __forceinline__ void frag_bn(uint32_t M, int ldh, uint32_t (&b)[2][2]) {
  const int lane = threadIdx.x & 31, j = lane >> 3;
  if (HD == 8) {
    ldsm2(M + (uint32_t)(((lane & 7) + 8 * (j & 1)) * ldh) * 2, b[0][0], b[1][0]);
    b[0][1] = b[1][1] = 0u;
  } else {
    ldsm4(M + (uint32_t)(((lane & 7) + 8 * (j >> 1)) * ldh + 8 * (j & 1)) * 2, b[0][0], b[0][1], b[1][0], b[1][1]);
  }
}
// B fragments of a [16 rows = k][HD cols = n] block (transposing load): b[c][kh] = n-tile c, k half kh.
template <int HD>
__device__ __forceinline__ void frag_bk(uint32_t M, int ldh, uint32_t (&b)[HD / 8][2]) {
  const int lane = threadIdx.x & 31, j = lane >> 3;
  if (HD == 8) {
    ldsm2t(M + (uint32_t)(((lane & 7) + 8 * (j & 1)) * ldh) * 2, b[0][0], b[0][1]);
  } else {
    uint32_t r0, r1, r2, r3;
    ldsm4t(M + (uint32_t)(((lane & 7) + 8 * (j & 1)) * ldh + 8 * (j >> 1)) * 2, r0, r1, r2, r3);
    b[0][0] = r0; b[0][1] = r1; b[HD / 8 - 1][0] = r2; b[HD / 8 - 1][1] = r3;
  }
}

// S[16][16] = A B^T over HD features (A, B: [16][HD] blocks as fragments).
template <int HD>
__device__ __forceinline__ void mma_s(const uint32_t (&a)[4], const uint32_t (&b)[2][2], float (&s)[2][4]) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    zero4(s[j]);
    if (HD == 8) mma1688(s[j], a[0], a[1], b[j][0]);
    else mma16816(s[j], a, b[j][0], b[j][1]);
  }
}
// Y[16][HD] = X[16][16] M[16][HD] with X as an A fragment and M's B fragments.
template <int HD>
__device__ __forceinline__ void mma_y(const uint32_t (&x)[4], const uint32_t (&b)[HD / 8][2], float (&y)[HD / 8][4]) {
#pragma unroll
  for (int c = 0; c < HD / 8; ++c) {
    zero4(y[c]);
    mma16816(y[c], x, b[c][0], b[c][1]);
  }
}

// Forward only, operands already FP16 in shared memory (the forward kernel's layout):
//   Qh, Kh: [rows][ldh] halves, this sequence's rows from 0 (Q pre-scaled by 1/sqrt(HD) log2 e),
//   V:      FULL: [rows][ldh] halves like K (16-byte-aligned rows: fragments by ldmatrix.trans);
//           otherwise V transposed, [features][ldv] halves, this sequence's keys at columns 0..15
//           (keys >= n zero),
// all with 4-byte-aligned pairs.  emit(row, col, v0, v1) for the attention output O, row < n.
// FULL: n = 16 at compile time (no masks).
template <int HD, bool FULL = false, typename EMIT>
__device__ __forceinline__ void attn_fwd_h(const __half *Qh, const __half *Kh, const __half *V, int ldh, int ldv,
                                           int n, EMIT emit) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  auto ld2 = [&](const __half *M, int r, int c) -> uint32_t {
    return (FULL || r < n) ? *reinterpret_cast<const uint32_t *>(M + r * ldh + c) : 0u;
  };
  float s[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j) zero4(s[j]);
  if (HD == 8) {
    const uint32_t a0 = ld2(Qh, g, 2 * t), a1 = ld2(Qh, g + 8, 2 * t);
#pragma unroll
    for (int j = 0; j < 2; ++j) mma1688(s[j], a0, a1, ld2(Kh, 8 * j + g, 2 * t));
  } else {
    const uint32_t a[4] = {ld2(Qh, g, 2 * t), ld2(Qh, g + 8, 2 * t), ld2(Qh, g, 8 + 2 * t), ld2(Qh, g + 8, 8 + 2 * t)};
#pragma unroll
    for (int j = 0; j < 2; ++j) mma16816(s[j], a, ld2(Kh, 8 * j + g, 2 * t), ld2(Kh, 8 * j + g, 8 + 2 * t));
  }
  float m0 = -INFINITY, m1 = -INFINITY;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const bool ok = FULL || 8 * j + 2 * t + e < n;
      s[j][e] = ok ? s[j][e] : -INFINITY;
      s[j][2 + e] = ok ? s[j][2 + e] : -INFINITY;
      m0 = fmaxf(m0, s[j][e]);
      m1 = fmaxf(m1, s[j][2 + e]);
    }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
  }
  float l0 = 0.f, l1 = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      s[j][e] = tc::ex2_fast(s[j][e] - m0);
      s[j][2 + e] = tc::ex2_fast(s[j][2 + e] - m1);
      l0 += s[j][e];
      l1 += s[j][2 + e];
    }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    l0 += __shfl_xor_sync(0xffffffffu, l0, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
  }
  const float i0 = tc::rcp_fast(l0), i1 = tc::rcp_fast(l1);
  const uint32_t pa[4] = {h2(s[0][0] * i0, s[0][1] * i0), h2(s[0][2] * i1, s[0][3] * i1),
                          h2(s[1][0] * i0, s[1][1] * i0), h2(s[1][2] * i1, s[1][3] * i1)};
  if constexpr (FULL) {   // O = P V with V's B fragments by transposing ldmatrix
    uint32_t vb[HD / 8][2];
    frag_bk<HD>((uint32_t)__cvta_generic_to_shared(V), ldh, vb);
    float o[HD / 8][4];
    mma_y<HD>(pa, vb, o);
#pragma unroll
    for (int c = 0; c < HD / 8; ++c) {
      emit(g, 8 * c + 2 * t, o[c][0], o[c][1]);
      emit(g + 8, 8 * c + 2 * t, o[c][2], o[c][3]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < HD / 8; ++c) {
      float o[4];
      zero4(o);
      const __half *vr = V + (8 * c + g) * ldv;
      mma16816(o, pa, *reinterpret_cast<const uint32_t *>(vr + 2 * t),
               *reinterpret_cast<const uint32_t *>(vr + 8 + 2 * t));
      if (g < n) emit(g, 8 * c + 2 * t, o[0], o[1]);
      if (g + 8 < n) emit(g + 8, 8 * c + 2 * t, o[2], o[3]);
    }
  }
}

// Forward only, for sequences of 17 to 32 tokens: one warp computes the 16 query rows q0 .. q0 + 15 of one
// (sequence, head) against its 32 keys (keys >= n masked), FP16 operands in shared memory, all row-major
// with row stride ldh halves and 16-byte-aligned rows: Qh (pre-scaled by 1/sqrt(HD) log2 e), Kh and Vh
// point at the sequence's first row; rows up to 31 below them must hold finite values (the next sequence
// or zeros).  Scores in four 16 x 8 key tiles, softmax in base 2 over the 32 keys, O = P V in two k-steps
// of 16 keys with V's B fragments by transposing ldmatrix.  emit(row, col, v0, v1) for rows < n.
template <int HD, typename EMIT>
__device__ __forceinline__ void attn_fwd_h32(const __half *Qh, const __half *Kh, const __half *Vh, int ldh, int n,
                                             int q0, EMIT emit) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  auto ld2 = [&](const __half *M, int r, int c) -> uint32_t {
    return *reinterpret_cast<const uint32_t *>(M + r * ldh + c);
  };
  float s[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) zero4(s[j]);
  if (HD == 8) {
    const uint32_t a0 = ld2(Qh, q0 + g, 2 * t), a1 = ld2(Qh, q0 + g + 8, 2 * t);
#pragma unroll
    for (int j = 0; j < 4; ++j) mma1688(s[j], a0, a1, ld2(Kh, 8 * j + g, 2 * t));
  } else {
    const uint32_t a[4] = {ld2(Qh, q0 + g, 2 * t), ld2(Qh, q0 + g + 8, 2 * t), ld2(Qh, q0 + g, 8 + 2 * t),
                           ld2(Qh, q0 + g + 8, 8 + 2 * t)};
#pragma unroll
    for (int j = 0; j < 4; ++j) mma16816(s[j], a, ld2(Kh, 8 * j + g, 2 * t), ld2(Kh, 8 * j + g, 8 + 2 * t));
  }
  float m0 = -INFINITY, m1 = -INFINITY;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const bool ok = 8 * j + 2 * t + e < n;
      s[j][e] = ok ? s[j][e] : -INFINITY;
      s[j][2 + e] = ok ? s[j][2 + e] : -INFINITY;
      m0 = fmaxf(m0, s[j][e]);
      m1 = fmaxf(m1, s[j][2 + e]);
    }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
  }
  float l0 = 0.f, l1 = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      s[j][e] = tc::ex2_fast(s[j][e] - m0);
      s[j][2 + e] = tc::ex2_fast(s[j][2 + e] - m1);
      l0 += s[j][e];
      l1 += s[j][2 + e];
    }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    l0 += __shfl_xor_sync(0xffffffffu, l0, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
  }
  const float i0 = tc::rcp_fast(l0), i1 = tc::rcp_fast(l1);
  float o[HD / 8][4];
#pragma unroll
  for (int c = 0; c < HD / 8; ++c) zero4(o[c]);
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {   // keys 16 kk .. 16 kk + 15
    const uint32_t pa[4] = {h2(s[2 * kk][0] * i0, s[2 * kk][1] * i0), h2(s[2 * kk][2] * i1, s[2 * kk][3] * i1),
                            h2(s[2 * kk + 1][0] * i0, s[2 * kk + 1][1] * i0),
                            h2(s[2 * kk + 1][2] * i1, s[2 * kk + 1][3] * i1)};
    uint32_t vb[HD / 8][2];
    frag_bk<HD>((uint32_t)__cvta_generic_to_shared(Vh + 16 * kk * ldh), ldh, vb);
#pragma unroll
    for (int c = 0; c < HD / 8; ++c) mma16816(o[c], pa, vb[c][0], vb[c][1]);
  }
#pragma unroll
  for (int c = 0; c < HD / 8; ++c) {
    if (q0 + g < n) emit(q0 + g, 8 * c + 2 * t, o[c][0], o[c][1]);
    if (q0 + g + 8 < n) emit(q0 + g + 8, 8 * c + 2 * t, o[c][2], o[c][3]);
  }
}

// Forward and backward of softmax attention for one (sequence, head) on one warp, FP16 operands in
// shared memory: Qh, Kh, Vh, dHh are u32 shared addresses of this sequence's first row and this head's
// first feature in [rows][ldh] row-major FP16 arrays (Q unscaled), readable 16 rows down (rows >= n
// hold finite values: the next sequence or zero padding).  Keys >= n are masked; query rows >= n get
// zero probabilities, so they add nothing to dK and dV.  emit(kind, row, col, v0, v1): kind 0 = the
// attention output O, 1 = dQ, 2 = dK, 3 = dV at (row, col..col+1), row < n.  FULL: n = 16 at
// compile time (no masks).
template <int HD, bool FULL = false, typename EMIT>
__device__ __forceinline__ void attn_fwd_bwd_h(uint32_t Qh, uint32_t Kh, uint32_t Vh, uint32_t dHh, int ldh, int n,
                                               float qscale, float scale, EMIT emit) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t qa[4], kb[2][2];
  frag_a<HD>(Qh, ldh, qa);
  frag_bn<HD>(Kh, ldh, kb);
  float s[2][4];
  mma_s<HD>(qa, kb, s);
  const bool q0 = FULL || g < n, q1 = FULL || g + 8 < n;
  float m0 = -INFINITY, m1 = -INFINITY;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const bool ok = FULL || 8 * j + 2 * t + e < n;
      s[j][e] = ok ? s[j][e] * qscale : -INFINITY;
      s[j][2 + e] = ok ? s[j][2 + e] * qscale : -INFINITY;
      m0 = fmaxf(m0, s[j][e]);
      m1 = fmaxf(m1, s[j][2 + e]);
    }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
  }
  float l0 = 0.f, l1 = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      s[j][e] = tc::ex2_fast(s[j][e] - m0);
      s[j][2 + e] = tc::ex2_fast(s[j][2 + e] - m1);
      l0 += s[j][e];
      l1 += s[j][2 + e];
    }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    l0 += __shfl_xor_sync(0xffffffffu, l0, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
  }
  const float i0 = q0 ? tc::rcp_fast(l0) : 0.f, i1 = q1 ? tc::rcp_fast(l1) : 0.f;   // invalid query rows: P = 0
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    s[j][0] *= i0; s[j][1] *= i0;
    s[j][2] *= i1; s[j][3] *= i1;
  }
  const uint32_t pa[4] = {h2(s[0][0], s[0][1]), h2(s[0][2], s[0][3]), h2(s[1][0], s[1][1]), h2(s[1][2], s[1][3])};
  {   // O = P V
    uint32_t vb[HD / 8][2];
    frag_bk<HD>(Vh, ldh, vb);
    float o[HD / 8][4];
    mma_y<HD>(pa, vb, o);
#pragma unroll
    for (int c = 0; c < HD / 8; ++c) {
      if (q0) emit(0, g, 8 * c + 2 * t, o[c][0], o[c][1]);
      if (q1) emit(0, g + 8, 8 * c + 2 * t, o[c][2], o[c][3]);
    }
  }
  // dA = dH V^T; delta_i = sum_j P_ij dA_ij; dS = scale P (dA - delta)
  float da[2][4];
  {
    uint32_t ha[4], vn[2][2];
    frag_a<HD>(dHh, ldh, ha);
    frag_bn<HD>(Vh, ldh, vn);
    mma_s<HD>(ha, vn, da);
  }
  float d0 = 0.f, d1 = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    d0 = fmaf(s[j][0], da[j][0], fmaf(s[j][1], da[j][1], d0));
    d1 = fmaf(s[j][2], da[j][2], fmaf(s[j][3], da[j][3], d1));
  }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    d0 += __shfl_xor_sync(0xffffffffu, d0, o);
    d1 += __shfl_xor_sync(0xffffffffu, d1, o);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    da[j][0] = scale * s[j][0] * (da[j][0] - d0);
    da[j][1] = scale * s[j][1] * (da[j][1] - d0);
    da[j][2] = scale * s[j][2] * (da[j][2] - d1);
    da[j][3] = scale * s[j][3] * (da[j][3] - d1);
  }
  uint32_t x00, x10, x01, x11;
  const float ds_down = ds_pack_scaled(da, x00, x10, x01, x11);
  {   // dQ = dS K
    const uint32_t dsa[4] = {x00, x10, x01, x11};
    uint32_t b[HD / 8][2];
    frag_bk<HD>(Kh, ldh, b);
    float y[HD / 8][4];
    mma_y<HD>(dsa, b, y);
#pragma unroll
    for (int c = 0; c < HD / 8; ++c) {
      if (q0) emit(1, g, 8 * c + 2 * t, y[c][0] * ds_down, y[c][1] * ds_down);
      if (q1) emit(1, g + 8, 8 * c + 2 * t, y[c][2] * ds_down, y[c][3] * ds_down);
    }
  }
  {   // dK = dS^T Q
    const uint32_t dst[4] = {trans8(x00), trans8(x01), trans8(x10), trans8(x11)};
    uint32_t b[HD / 8][2];
    frag_bk<HD>(Qh, ldh, b);
    float y[HD / 8][4];
    mma_y<HD>(dst, b, y);
#pragma unroll
    for (int c = 0; c < HD / 8; ++c) {
      if (q0) emit(2, g, 8 * c + 2 * t, y[c][0] * ds_down, y[c][1] * ds_down);
      if (q1) emit(2, g + 8, 8 * c + 2 * t, y[c][2] * ds_down, y[c][3] * ds_down);
    }
  }
  {   // dV = P^T dH
    const uint32_t pt[4] = {trans8(pa[0]), trans8(pa[2]), trans8(pa[1]), trans8(pa[3])};
    uint32_t b[HD / 8][2];
    frag_bk<HD>(dHh, ldh, b);
    float y[HD / 8][4];
    mma_y<HD>(pt, b, y);
#pragma unroll
    for (int c = 0; c < HD / 8; ++c) {
      if (q0) emit(3, g, 8 * c + 2 * t, y[c][0], y[c][1]);
      if (q1) emit(3, g + 8, 8 * c + 2 * t, y[c][2], y[c][3]);
    }
  }
}


// Forward and backward of softmax attention for one (sequence, head) of 17 to 32 tokens on one warp, with
// the operands of attn_fwd_bwd_h, readable 32 rows down from the sequence's first row (rows past the
// sequence hold finite values).  The two 16-query blocks run one after the other; for each, the 16 x 32
// score block is a row of four 8-key C fragments, and its softmax, dA = dH V^T, delta and dS follow as
// for 16 tokens.  dQ of the block is emitted at once; dK and dV sum over both query blocks in FP32
// registers and are emitted at the end.  Each block scales its dS by its own power of two
// (ds_pack_scaled) and its dQ, dK products are unscaled before any sum.  emit(kind, row, col, v0, v1)
// as in attn_fwd_bwd_h, row < n.
template <int HD, typename EMIT>
__device__ __forceinline__ void attn_fwd_bwd_h32(uint32_t Qh, uint32_t Kh, uint32_t Vh, uint32_t dHh, int ldh, int n,
                                                 float qscale, float scale, EMIT emit) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t blk = (uint32_t)(16 * ldh * 2);   // bytes from one 16-row block to the next
  uint32_t kb[2][2][2], vn[2][2][2];                // K and V rows as B fragments (key blocks 0-15, 16-31)
  frag_bn<HD>(Kh, ldh, kb[0]);
  frag_bn<HD>(Kh + blk, ldh, kb[1]);
  frag_bn<HD>(Vh, ldh, vn[0]);
  frag_bn<HD>(Vh + blk, ldh, vn[1]);
  uint32_t kk[2][HD / 8][2], vk[2][HD / 8][2];      // K and V rows as k-major B fragments (for dQ, O)
  frag_bk<HD>(Kh, ldh, kk[0]);
  frag_bk<HD>(Kh + blk, ldh, kk[1]);
  frag_bk<HD>(Vh, ldh, vk[0]);
  frag_bk<HD>(Vh + blk, ldh, vk[1]);
  float dk[2][HD / 8][4], dv[2][HD / 8][4];
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int c = 0; c < HD / 8; ++c) { zero4(dk[b][c]); zero4(dv[b][c]); }
#pragma unroll
  for (int qb = 0; qb < 2; ++qb) {
    const uint32_t qo = (uint32_t)qb * blk;
    const bool q0 = 16 * qb + g < n, q1 = 16 * qb + g + 8 < n;
    uint32_t qa[4];
    frag_a<HD>(Qh + qo, ldh, qa);
    float s[4][4];   // s[j]: keys 8 j .. 8 j + 7
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      zero4(s[j]);
      if (HD == 8) mma1688(s[j], qa[0], qa[1], kb[j >> 1][j & 1][0]);
      else mma16816(s[j], qa, kb[j >> 1][j & 1][0], kb[j >> 1][j & 1][1]);
    }
    float m0 = -INFINITY, m1 = -INFINITY;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const bool ok = 8 * j + 2 * t + e < n;
        s[j][e] = ok ? s[j][e] * qscale : -INFINITY;
        s[j][2 + e] = ok ? s[j][2 + e] * qscale : -INFINITY;
        m0 = fmaxf(m0, s[j][e]);
        m1 = fmaxf(m1, s[j][2 + e]);
      }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
      m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    }
    float l0 = 0.f, l1 = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        s[j][e] = tc::ex2_fast(s[j][e] - m0);
        s[j][2 + e] = tc::ex2_fast(s[j][2 + e] - m1);
        l0 += s[j][e];
        l1 += s[j][2 + e];
      }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      l0 += __shfl_xor_sync(0xffffffffu, l0, o);
      l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    }
    const float i0 = q0 ? tc::rcp_fast(l0) : 0.f, i1 = q1 ? tc::rcp_fast(l1) : 0.f;   // invalid query rows: P = 0
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      s[j][0] *= i0; s[j][1] *= i0;
      s[j][2] *= i1; s[j][3] *= i1;
    }
    uint32_t pa[2][4];   // P of key block kb as an A fragment
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      pa[b][0] = h2(s[2 * b][0], s[2 * b][1]);
      pa[b][1] = h2(s[2 * b][2], s[2 * b][3]);
      pa[b][2] = h2(s[2 * b + 1][0], s[2 * b + 1][1]);
      pa[b][3] = h2(s[2 * b + 1][2], s[2 * b + 1][3]);
    }
    {   // O = P V over both key blocks
      float o[HD / 8][4];
#pragma unroll
      for (int c = 0; c < HD / 8; ++c) {
        zero4(o[c]);
        mma16816(o[c], pa[0], vk[0][c][0], vk[0][c][1]);
        mma16816(o[c], pa[1], vk[1][c][0], vk[1][c][1]);
        if (q0) emit(0, 16 * qb + g, 8 * c + 2 * t, o[c][0], o[c][1]);
        if (q1) emit(0, 16 * qb + g + 8, 8 * c + 2 * t, o[c][2], o[c][3]);
      }
    }
    // dA = dH V^T; delta_i = sum_j P_ij dA_ij; dS = scale P (dA - delta)
    float da[4][4];
    uint32_t ha[4];
    frag_a<HD>(dHh + qo, ldh, ha);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      zero4(da[j]);
      if (HD == 8) mma1688(da[j], ha[0], ha[1], vn[j >> 1][j & 1][0]);
      else mma16816(da[j], ha, vn[j >> 1][j & 1][0], vn[j >> 1][j & 1][1]);
    }
    float d0 = 0.f, d1 = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      d0 = fmaf(s[j][0], da[j][0], fmaf(s[j][1], da[j][1], d0));
      d1 = fmaf(s[j][2], da[j][2], fmaf(s[j][3], da[j][3], d1));
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      d0 += __shfl_xor_sync(0xffffffffu, d0, o);
      d1 += __shfl_xor_sync(0xffffffffu, d1, o);
    }
    float mx = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      da[j][0] = scale * s[j][0] * (da[j][0] - d0);
      da[j][1] = scale * s[j][1] * (da[j][1] - d0);
      da[j][2] = scale * s[j][2] * (da[j][2] - d1);
      da[j][3] = scale * s[j][3] * (da[j][3] - d1);
#pragma unroll
      for (int e = 0; e < 4; ++e) mx = fmaxf(mx, fabsf(da[j][e]));
    }
    // one power of two for the whole 16 x 32 block (ds_pack_scaled's rule), so that both key blocks'
    // fragments share it
#pragma unroll
    for (int o = 1; o <= 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int ex = 0;
    if (mx > 0.f && isfinite(mx)) frexpf(mx, &ex);
    int kx = 14 - ex;
    kx = kx > 100 ? 100 : (kx < -100 ? -100 : kx);
    const float up = ldexpf(1.0f, kx), down = ldexpf(1.0f, -kx);
    uint32_t x[2][4];   // dS of key block b as an A fragment (scaled)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      x[b][0] = h2(da[2 * b][0] * up, da[2 * b][1] * up);
      x[b][1] = h2(da[2 * b][2] * up, da[2 * b][3] * up);
      x[b][2] = h2(da[2 * b + 1][0] * up, da[2 * b + 1][1] * up);
      x[b][3] = h2(da[2 * b + 1][2] * up, da[2 * b + 1][3] * up);
    }
    {   // dQ = dS K over both key blocks
      float y[HD / 8][4];
#pragma unroll
      for (int c = 0; c < HD / 8; ++c) {
        zero4(y[c]);
        mma16816(y[c], x[0], kk[0][c][0], kk[0][c][1]);
        mma16816(y[c], x[1], kk[1][c][0], kk[1][c][1]);
        if (q0) emit(1, 16 * qb + g, 8 * c + 2 * t, y[c][0] * down, y[c][1] * down);
        if (q1) emit(1, 16 * qb + g + 8, 8 * c + 2 * t, y[c][2] * down, y[c][3] * down);
      }
    }
    uint32_t qk[HD / 8][2], hk[HD / 8][2];   // this block's Q and dH rows as k-major B fragments
    frag_bk<HD>(Qh + qo, ldh, qk);
    frag_bk<HD>(dHh + qo, ldh, hk);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      // dK[key block b] += dS^T Q, dV[key block b] += P^T dH (this query block's 16 rows as K = 16)
      const uint32_t dst[4] = {trans8(x[b][0]), trans8(x[b][2]), trans8(x[b][1]), trans8(x[b][3])};
      const uint32_t pt[4] = {trans8(pa[b][0]), trans8(pa[b][2]), trans8(pa[b][1]), trans8(pa[b][3])};
#pragma unroll
      for (int c = 0; c < HD / 8; ++c) {
        float y[4];
        zero4(y);
        mma16816(y, dst, qk[c][0], qk[c][1]);
#pragma unroll
        for (int e = 0; e < 4; ++e) dk[b][c][e] = fmaf(y[e], down, dk[b][c][e]);
        mma16816(dv[b][c], pt, hk[c][0], hk[c][1]);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int c = 0; c < HD / 8; ++c) {
      const int r0 = 16 * b + g, r1 = r0 + 8;
      if (r0 < n) {
        emit(2, r0, 8 * c + 2 * t, dk[b][c][0], dk[b][c][1]);
        emit(3, r0, 8 * c + 2 * t, dv[b][c][0], dv[b][c][1]);
      }
      if (r1 < n) {
        emit(2, r1, 8 * c + 2 * t, dk[b][c][2], dk[b][c][3]);
        emit(3, r1, 8 * c + 2 * t, dv[b][c][2], dv[b][c][3]);
      }
    }
}

}  // namespace amma
}  // namespace tdo
