// FP32 (CUDA-core) evaluation of one tile of sequences through the whole ansatz.
//
// A tile is TS sequences (TS/2 doubled configurations, both orders of each) of N tokens, TS*N <= 128
// rows, processed by one CTA of 256 threads with every activation resident in shared memory:
//   Xs  [128][LDX]  residual stream
//   Qs, Ks, Vs [128][LDX]  projections (Qs is overwritten by the concatenated head outputs, Ks holds
//                          the GELU'd MLP hidden chunk)
//   Ws  [3 D D]     weights of the current GEMM, staged from global (L2-resident) memory
// GEMMs use a 4-row x 8-column register tile per thread (D = 64) with float4 shared-memory loads.
#pragma once
#include "tdo_device.cuh"

namespace tdo {

constexpr int kThreads = 256;
constexpr int kRows = 128;

template <int D, int R = kRows>
struct F32Geom {
  static constexpr int LDX = D + 4;
  static constexpr int TX = D / 8;          // threads across the 8-column groups
  static constexpr int TY = kThreads / TX;  // row groups
  static constexpr int RPT = R / TY;        // rows per thread
  static constexpr int X_OFF = 0;
  static constexpr int Q_OFF = X_OFF + kRows * LDX;
  static constexpr int K_OFF = Q_OFF + kRows * LDX;
  static constexpr int V_OFF = K_OFF + kRows * LDX;
  static constexpr int W_OFF = V_OFF + kRows * LDX;
  static constexpr int F_OFF = W_OFF + 3 * D * D;        // [128 seqs][2] head outputs
  static constexpr int C_OFF = F_OFF + 2 * kRows;        // tile configs: sig[64], sigp[64] (uint32)
  static constexpr int O_OFF = C_OFF + kRows;            // results [64] float2
  static constexpr int FLOATS = O_OFF + kRows;
  static constexpr size_t BYTES = sizeof(float) * FLOATS;
};

// acc[j][0..7] += sum_k A[row_j][k] * W[k][cols], row_j = ty + j*TY, cols {4tx..4tx+3, D/2+4tx..+3}.
template <int D, int R = kRows>
__device__ __forceinline__ void mm_acc(const float *__restrict__ A, int lda,
                                       const float *__restrict__ W, int K,
                                       float (&acc)[F32Geom<D, R>::RPT][8]) {
  using G = F32Geom<D, R>;
  const int tx = threadIdx.x % G::TX, ty = threadIdx.x / G::TX;
  const int c0 = 4 * tx, c1 = D / 2 + 4 * tx;
#pragma unroll 2
  for (int k = 0; k < K; k += 4) {
    float4 a[G::RPT];
#pragma unroll
    for (int j = 0; j < G::RPT; ++j)
      a[j] = *reinterpret_cast<const float4 *>(A + (ty + j * G::TY) * lda + k);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const float4 w0 = *reinterpret_cast<const float4 *>(W + (k + kk) * D + c0);
      const float4 w1 = *reinterpret_cast<const float4 *>(W + (k + kk) * D + c1);
#pragma unroll
      for (int j = 0; j < G::RPT; ++j) {
        const float av = kk == 0 ? a[j].x : kk == 1 ? a[j].y : kk == 2 ? a[j].z : a[j].w;
        acc[j][0] = fmaf(av, w0.x, acc[j][0]);
        acc[j][1] = fmaf(av, w0.y, acc[j][1]);
        acc[j][2] = fmaf(av, w0.z, acc[j][2]);
        acc[j][3] = fmaf(av, w0.w, acc[j][3]);
        acc[j][4] = fmaf(av, w1.x, acc[j][4]);
        acc[j][5] = fmaf(av, w1.y, acc[j][5]);
        acc[j][6] = fmaf(av, w1.z, acc[j][6]);
        acc[j][7] = fmaf(av, w1.w, acc[j][7]);
      }
    }
  }
}

template <int D, int R = kRows>
__device__ __forceinline__ void acc_zero(float (&acc)[F32Geom<D, R>::RPT][8]) {
#pragma unroll
  for (int j = 0; j < F32Geom<D, R>::RPT; ++j)
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[j][e] = 0.f;
}

// Visit the (row, col, value) of every accumulator element of this thread.
template <int D, int R = kRows, typename F>
__device__ __forceinline__ void acc_foreach(float (&acc)[F32Geom<D, R>::RPT][8], F f) {
  using G = F32Geom<D, R>;
  const int tx = threadIdx.x % G::TX, ty = threadIdx.x / G::TX;
#pragma unroll
  for (int j = 0; j < G::RPT; ++j)
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int col = (e < 4) ? (4 * tx + e) : (D / 2 + 4 * tx + e - 4);
      f(ty + j * G::TY, col, acc[j][e]);
    }
}

// Store the accumulator tile to a [128][LDX] shared array (float4 stores).
template <int D, int R = kRows>
__device__ __forceinline__ void acc_store(float (&acc)[F32Geom<D, R>::RPT][8], float *dst) {
  using G = F32Geom<D, R>;
  const int tx = threadIdx.x % G::TX, ty = threadIdx.x / G::TX;
#pragma unroll
  for (int j = 0; j < G::RPT; ++j) {
    float *p = dst + (ty + j * G::TY) * G::LDX;
    *reinterpret_cast<float4 *>(p + 4 * tx) = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
    *reinterpret_cast<float4 *>(p + D / 2 + 4 * tx) =
        make_float4(acc[j][4], acc[j][5], acc[j][6], acc[j][7]);
  }
}

// Copy a rows x D block (global row stride gld floats, starting at column col0) to contiguous smem.
template <int D>
__device__ __forceinline__ void stage_block(const float *__restrict__ g, int gld, int col0, int rows,
                                            float *s) {
  const int n4 = rows * (D / 4);
  for (int i = threadIdx.x; i < n4; i += kThreads) {
    const int r = i / (D / 4), c = (i % (D / 4)) * 4;
    *reinterpret_cast<float4 *>(s + r * D + c) =
        __ldg(reinterpret_cast<const float4 *>(g + (size_t)r * gld + col0 + c));
  }
}

// Per (sequence, head): softmax(Q K^T / sqrt(dh)) V, one lane per query token; the result replaces
// that head's columns of Q (each lane reads its own query row before writing it).
template <int D>
__device__ __forceinline__ void attention_f32(float *Qs, const float *Ks, const float *Vs, int ts,
                                              int n, int heads, int dh, float *Out = nullptr) {
  using G = F32Geom<D>;
  if (Out == nullptr) Out = Qs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = n <= 8 ? 8 : (n <= 16 ? 16 : 32);
  const int upw = 32 / grp;
  const int units = ts * heads;
  const float scale = rsqrtf((float)dh);
  for (int u0 = warp * upw; u0 < units; u0 += (kThreads / 32) * upw) {
    const int u = u0 + lane / grp, i = lane % grp;
    if (u < units && i < n) {
      const int s = u / heads, h = u % heads;
      const int row = s * n + i, base = s * n, col = h * dh;
      float q[16], o[16], sc[TDO_MAX_N];
#pragma unroll
      for (int e = 0; e < 16; ++e) { q[e] = e < dh ? Qs[row * G::LDX + col + e] : 0.f; o[e] = 0.f; }
      float mx = -INFINITY;
#pragma unroll
      for (int j = 0; j < TDO_MAX_N; ++j) {
        if (j < n) {
          const float *kr = Ks + (base + j) * G::LDX + col;
          float dot = 0.f;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (e < dh) dot = fmaf(q[e], kr[e], dot);
          sc[j] = dot * scale;
          mx = fmaxf(mx, sc[j]);
        }
      }
      float sum = 0.f;
#pragma unroll
      for (int j = 0; j < TDO_MAX_N; ++j) {
        if (j < n) {
          const float p = expf(sc[j] - mx);
          sum += p;
          const float *vr = Vs + (base + j) * G::LDX + col;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (e < dh) o[e] = fmaf(p, vr[e], o[e]);
        }
      }
      const float inv = 1.0f / sum;
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (e < dh) Out[row * G::LDX + col + e] = o[e] * inv;
    }
  }
}

// Embedding of the tile's sequences into Xs (padding rows = 0).  Sequence s is configuration s/2 in
// order s%2 (0: channels (sigma, sigma'), 1: (sigma', sigma)).
template <int D, int R = kRows>
__device__ __forceinline__ void embed_f32(const DevModel &m, const uint32_t *csig, const uint32_t *csigp,
                                          int ts, float *Xs) {
  using G = F32Geom<D, R>;
  const int n = m.n_sites;
  for (int idx = threadIdx.x; idx < R * (D / 4); idx += kThreads) {
    const int r = idx / (D / 4), c = (idx % (D / 4)) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < ts * n) {
      const int s = r / n, i = r % n, cfg = s >> 1;
      const uint32_t w1 = (s & 1) ? csigp[cfg] : csig[cfg];
      const uint32_t w2 = (s & 1) ? csig[cfg] : csigp[cfg];
      const int pat = embed_pattern(m.embed, w1, w2, i, n);
      v = __ldg(reinterpret_cast<const float4 *>(m.etab + pat * D + c));
    }
    *reinterpret_cast<float4 *>(Xs + r * G::LDX + c) = v;
  }
}

// One encoder layer on the tile (attention + residual, optional MLP + residual).
template <int D>
__device__ __forceinline__ void layer_f32(const DevModel &m, const DevLayer &L, float *sm, int ts) {
  using G = F32Geom<D>;
  float *Xs = sm + G::X_OFF, *Qs = sm + G::Q_OFF, *Ks = sm + G::K_OFF, *Vs = sm + G::V_OFF,
        *Ws = sm + G::W_OFF;
  stage_block<D>(L.Wq, D, 0, D, Ws);
  stage_block<D>(L.Wk, D, 0, D, Ws + D * D);
  stage_block<D>(L.Wv, D, 0, D, Ws + 2 * D * D);
  __syncthreads();
  {
    float acc[G::RPT][8];
    acc_zero<D>(acc);
    mm_acc<D>(Xs, G::LDX, Ws, D, acc);
    acc_store<D>(acc, Qs);
    acc_zero<D>(acc);
    mm_acc<D>(Xs, G::LDX, Ws + D * D, D, acc);
    acc_store<D>(acc, Ks);
    acc_zero<D>(acc);
    mm_acc<D>(Xs, G::LDX, Ws + 2 * D * D, D, acc);
    acc_store<D>(acc, Vs);
  }
  __syncthreads();
  attention_f32<D>(Qs, Ks, Vs, ts, m.n_sites, m.heads, m.dh);
  stage_block<D>(L.Wo, D, 0, D, Ws);
  __syncthreads();
  {
    float acc[G::RPT][8];
    acc_zero<D>(acc);
    mm_acc<D>(Qs, G::LDX, Ws, D, acc);
    acc_foreach<D>(acc, [&](int r, int c, float v) { Xs[r * G::LDX + c] += v; });
  }
  __syncthreads();
  if (m.ffn > 0) {
    float acc2[G::RPT][8];
    acc_zero<D>(acc2);
    for (int c0 = 0; c0 < m.ffn; c0 += D) {
      stage_block<D>(L.W1, m.ffn, c0, D, Ws);
      stage_block<D>(L.W2 + (size_t)c0 * D, D, 0, D, Ws + D * D);
      __syncthreads();
      float acc[G::RPT][8];
      acc_zero<D>(acc);
      mm_acc<D>(Xs, G::LDX, Ws, D, acc);
      acc_foreach<D>(acc, [&](int r, int c, float v) {
        Ks[r * G::LDX + c] = gelu_f(v + __ldg(L.b1 + c0 + c));
      });
      __syncthreads();
      mm_acc<D>(Ks, G::LDX, Ws + D * D, D, acc2);
      __syncthreads();
    }
    acc_foreach<D>(acc2, [&](int r, int c, float v) { Xs[r * G::LDX + c] += v + __ldg(L.b2 + c); });
    __syncthreads();
  }
}

// Mean pooling, dense head and symmetrisation; results for the tile's configurations in out[ts/2].
template <int D>
__device__ __forceinline__ void head_f32(const DevModel &m, float *sm, int ts, float2 *out) {
  using G = F32Geom<D>;
  float *Xs = sm + G::X_OFF, *Hp = sm + G::Q_OFF, *Fs = sm + G::F_OFF;
  const int n = m.n_sites;
  const float inv_n = 1.0f / (float)n;
  for (int idx = threadIdx.x; idx < ts * D; idx += kThreads) {
    const int s = idx / D, c = idx % D;
    float acc = 0.f;
    for (int i = 0; i < n; ++i) acc += Xs[(s * n + i) * G::LDX + c];
    Hp[s * D + c] = acc * inv_n;
  }
  __syncthreads();
  // one warp per (sequence, output) pair
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int p = warp; p < ts * 2; p += kThreads / 32) {
    const int s = p >> 1, o = p & 1;
    float acc = 0.f;
    for (int c = lane; c < D; c += 32) acc = fmaf(Hp[s * D + c], __ldg(m.Wh + 2 * c + o), acc);
    acc = warp_sum(acc);
    if (lane == 0) Fs[p] = acc + __ldg(m.bh + o);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ts / 2; c += kThreads)
    out[c] = symmetrise(Fs[4 * c], Fs[4 * c + 1], Fs[4 * c + 2], Fs[4 * c + 3], nullptr, nullptr);
  __syncthreads();
}

// Full evaluation of the configurations in smem (C_OFF) -> results in smem (O_OFF).
template <int D>
__device__ __forceinline__ void eval_tile_f32(const DevModel &m, float *sm, int ts) {
  using G = F32Geom<D>;
  const uint32_t *csig = reinterpret_cast<const uint32_t *>(sm + G::C_OFF);
  const uint32_t *csigp = csig + kRows / 2;
  embed_f32<D>(m, csig, csigp, ts, sm + G::X_OFF);
  __syncthreads();
  for (int l = 0; l < m.layers; ++l) layer_f32<D>(m, m.L[l], sm, ts);
  head_f32<D>(m, sm, ts, reinterpret_cast<float2 *>(sm + G::O_OFF));
}

}  // namespace tdo
