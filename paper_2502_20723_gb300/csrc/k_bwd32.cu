// FP32 backward of the ansatz with activation recomputation.
//
// Per tile of configurations the kernel (1) recomputes the forward, saving each layer's input, Q, K, V,
// head outputs and attention-block output to a per-CTA scratch area (L2-resident), (2) back-propagates
// the cotangent of log rho through the Hermitian symmetrisation (Eq. log_sum_exp_conjugate), the head,
// the mean pooling, every layer in reverse (MLP, W^O, softmax attention, Q/K/V) and the embedding.
// Weight gradients are D x D blocks reduced over the rows of the tile:
//   mode 0 (VJP): summed over the tile and added with float4 atomics to one of n_copies FP32 accumulator
//                 vectors (CTA b uses copy b % n_copies; 16 copies stay L2-resident), reduced in FP64,
//   mode 1 (Jacobian): one per (configuration, seed) and written to O[b][k][seed] (row stride ldo >= P),
//                      FP32 or BF16 of O - oref (seed 0: d Re log rho, seed 1: d Im log rho).
#include <cuda_bf16.h>

#include "f32_tile.cuh"

namespace tdo {

struct FlatOffsets {
  long long E;
  long long Wq[TDO_MAX_LAYERS], Wk[TDO_MAX_LAYERS], Wv[TDO_MAX_LAYERS], Wo[TDO_MAX_LAYERS];
  long long W1[TDO_MAX_LAYERS], b1[TDO_MAX_LAYERS], W2[TDO_MAX_LAYERS], b2[TDO_MAX_LAYERS];
  long long Wh, bh;
};

template <int D>
struct BwdGeom {
  static constexpr int R = (D == 64) ? 64 : 128;
  static constexpr int LDX = D + 4;
  static constexpr int BUF = R * LDX;
  static constexpr int W_OFF = 9 * BUF;
  static constexpr int ST_OFF = W_OFF + 3 * D * D;   // max, 1/sum, delta: 3 x [R][16]
  static constexpr int F_OFF = ST_OFF + 3 * R * 16;  // head outputs / their cotangents [R][2]
  static constexpr int C_OFF = F_OFF + 2 * R;        // configs sig[R/2], sigp[R/2]
  static constexpr int T_OFF = C_OFF + R;            // cotangent per virtual configuration [R/2] float2
  static constexpr int FLOATS = T_OFF + R;
  static constexpr size_t BYTES = sizeof(float) * FLOATS;
  static constexpr int TX = D / 8;
  static constexpr int TY = kThreads / TX;
  static constexpr int KPT = (D / TY) > 0 ? (D / TY) : 1;   // weight rows per thread in dW blocks
};

__host__ __device__ __forceinline__ int seqs_for(int n, int rows) {
  int ts = 2 * (rows / (2 * n));
  return ts < 2 ? 2 : ts;
}

struct SinkCtx {
  int mode;
  float *g;          // mode 0: this CTA's accumulator copy [P] (16-byte aligned)
  float *O;          // mode 1: [B][P][2] FP32, or
  uint16_t *O16;     //         [B][P][2] BF16 of O - oref (oref: [P] (re, im))
  const float2 *oref;
  size_t P, ldo;     // parameters; elements per row of O (>= P)
  float *dtab;       // conv embedding: mode 0 [64][D] accumulator; mode 1 [B][2][64][D]
};

__device__ __forceinline__ uint16_t bf16_bits(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Add / write one gradient value at flat parameter index k for virtual configuration v of the tile.
__device__ __forceinline__ void sink1(const SinkCtx &s, long long k, float v, long long b, int seed) {
  if (s.mode == 0) {
    atomicAdd(s.g + k, v);
  } else {
    const size_t i = ((size_t)b * s.ldo + (size_t)k) * 2 + seed;
    if (s.O16) s.O16[i] = bf16_bits(v - (seed ? s.oref[k].y : s.oref[k].x));
    else s.O[i] = v;
  }
}

// Copy a rows x D block of global memory (row stride gld, column offset col0) transposed into smem:
// s[c][r] = g[r][col0 + c].
// Consecutive threads take consecutive r: conflict-free shared stores; the strided global reads of the
// block (16 KB at D = 64) are served from L1 after the first touch of each line.
template <int D>
__device__ __forceinline__ void stage_blockT(const float *__restrict__ g, int gld, int col0, float *s) {
  for (int i = threadIdx.x; i < D * D; i += kThreads) {
    const int r = i % D, c = i / D;
    s[c * D + r] = __ldg(g + (size_t)r * gld + col0 + c);
  }
}

template <int D, int R>
__device__ __forceinline__ void save_block(const float *src, float *dst) {
  constexpr int LDX = D + 4;
  for (int i = threadIdx.x; i < R * (D / 4); i += kThreads) {
    const int r = i / (D / 4), c = (i % (D / 4)) * 4;
    *reinterpret_cast<float4 *>(dst + r * D + c) = *reinterpret_cast<const float4 *>(src + r * LDX + c);
  }
}
template <int D, int R>
__device__ __forceinline__ void load_block(const float *src, float *dst) {
  constexpr int LDX = D + 4;
  for (int i = threadIdx.x; i < R * (D / 4); i += kThreads) {
    const int r = i / (D / 4), c = (i % (D / 4)) * 4;
    *reinterpret_cast<float4 *>(dst + r * LDX + c) = *reinterpret_cast<const float4 *>(src + r * D + c);
  }
}

// dW[k][c] = sum_{r in [r0, r1)} f(A[r][k]) * Bm[r][c] over this thread's (k, c) set:
// k = ty + j*TY (j < KPT, k < D), c in {4tx..4tx+3, D/2+4tx..+3}.
template <int D, bool GELU_A>
__device__ __forceinline__ void mmT_acc(const float *A, const float *Bm, int r0, int r1,
                                        float (&acc)[BwdGeom<D>::KPT][8]) {
  using BG = BwdGeom<D>;
  constexpr int LDX = D + 4;
  const int tx = threadIdx.x % BG::TX, ty = threadIdx.x / BG::TX;
  const int c0 = 4 * tx, c1 = D / 2 + 4 * tx;
#pragma unroll
  for (int j = 0; j < BG::KPT; ++j)
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[j][e] = 0.f;
  if (ty >= D) return;
  for (int r = r0; r < r1; ++r) {
    const float4 b0 = *reinterpret_cast<const float4 *>(Bm + r * LDX + c0);
    const float4 b1 = *reinterpret_cast<const float4 *>(Bm + r * LDX + c1);
#pragma unroll
    for (int j = 0; j < BG::KPT; ++j) {
      float a = A[r * LDX + ty + j * BG::TY];
      if (GELU_A) a = gelu_f(a);
      acc[j][0] = fmaf(a, b0.x, acc[j][0]);
      acc[j][1] = fmaf(a, b0.y, acc[j][1]);
      acc[j][2] = fmaf(a, b0.z, acc[j][2]);
      acc[j][3] = fmaf(a, b0.w, acc[j][3]);
      acc[j][4] = fmaf(a, b1.x, acc[j][4]);
      acc[j][5] = fmaf(a, b1.y, acc[j][5]);
      acc[j][6] = fmaf(a, b1.z, acc[j][6]);
      acc[j][7] = fmaf(a, b1.w, acc[j][7]);
    }
  }
}

// Send a dW block (flat offset off, row stride ld) to the sink.
template <int D>
__device__ __forceinline__ void sink_block(const SinkCtx &s, float (&acc)[BwdGeom<D>::KPT][8],
                                           long long off, long long ld, long long b, int seed) {
  using BG = BwdGeom<D>;
  const int tx = threadIdx.x % BG::TX, ty = threadIdx.x / BG::TX;
  if (ty >= D) return;
#pragma unroll
  for (int j = 0; j < BG::KPT; ++j) {
    const long long k = ty + j * BG::TY;
    if (k >= D) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long base = off + k * ld + (h ? D / 2 : 0) + 4 * tx;
      if (s.mode == 0 && (base & 3) == 0) {
        atomicAdd(reinterpret_cast<float4 *>(s.g + base),
                  make_float4(acc[j][4 * h], acc[j][4 * h + 1], acc[j][4 * h + 2], acc[j][4 * h + 3]));
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) sink1(s, base + e, acc[j][4 * h + e], b, seed);
      }
    }
  }
}

// Column sums of Bm over rows [r0, r1) -> sink at off + c, c < D.
template <int D>
__device__ __forceinline__ void colsum_sink(const SinkCtx &s, const float *Bm, int r0, int r1,
                                            long long off, long long b, int seed) {
  constexpr int LDX = D + 4;
  for (int c = threadIdx.x; c < D; c += kThreads) {
    float acc = 0.f;
    for (int r = r0; r < r1; ++r) acc += Bm[r * LDX + c];
    sink1(s, off + c, acc, b, seed);
  }
}

// Attention backward of one (sequence, head) unit per lane group; see the header comment.
template <int D>
__device__ __forceinline__ void attention_bwd(const float *Qs, const float *Ks, const float *Vs,
                                              const float *dHs, float *dQ, float *dK, float *dV,
                                              float *st, int ts, int n, int heads, int dh) {
  constexpr int LDX = D + 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = n <= 8 ? 8 : (n <= 16 ? 16 : 32);
  const int upw = 32 / grp;
  const int units = ts * heads;
  const float scale = rsqrtf((float)dh);
  const int RS = BwdGeom<D>::R * 16;
  float *smx = st, *sis = st + RS, *sdl = st + 2 * RS;
  for (int u0 = warp * upw; u0 < units; u0 += (kThreads / 32) * upw) {
    const int u = u0 + lane / grp, i = lane % grp;
    const bool act = (u < units && i < n);
    const int s = act ? u / heads : 0, h = act ? u % heads : 0;
    const int base = s * n, col = h * dh;
    if (act) {   // pass 1: lane = query row
      const int row = base + i;
      float q[16], g[16], dq[16], sc[TDO_MAX_N], da[TDO_MAX_N];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        q[e] = e < dh ? Qs[row * LDX + col + e] : 0.f;
        g[e] = e < dh ? dHs[row * LDX + col + e] : 0.f;
        dq[e] = 0.f;
      }
      float mx = -INFINITY;
#pragma unroll
      for (int j = 0; j < TDO_MAX_N; ++j) {
        if (j < n) {
          const float *kr = Ks + (base + j) * LDX + col;
          const float *vr = Vs + (base + j) * LDX + col;
          float dot = 0.f, dd = 0.f;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (e < dh) { dot = fmaf(q[e], kr[e], dot); dd = fmaf(g[e], vr[e], dd); }
          sc[j] = dot * scale;
          da[j] = dd;
          mx = fmaxf(mx, sc[j]);
        }
      }
      float sum = 0.f;
#pragma unroll
      for (int j = 0; j < TDO_MAX_N; ++j)
        if (j < n) { sc[j] = expf(sc[j] - mx); sum += sc[j]; }
      const float is = 1.0f / sum;
      float delta = 0.f;
#pragma unroll
      for (int j = 0; j < TDO_MAX_N; ++j)
        if (j < n) { sc[j] *= is; delta = fmaf(sc[j], da[j], delta); }
#pragma unroll
      for (int j = 0; j < TDO_MAX_N; ++j) {
        if (j < n) {
          const float w = scale * sc[j] * (da[j] - delta);
          const float *kr = Ks + (base + j) * LDX + col;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (e < dh) dq[e] = fmaf(w, kr[e], dq[e]);
        }
      }
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (e < dh) dQ[row * LDX + col + e] = dq[e];
      smx[row * 16 + h] = mx;
      sis[row * 16 + h] = is;
      sdl[row * 16 + h] = delta;
    }
    __syncwarp();
    if (act) {   // pass 2: lane = key row j
      const int jrow = base + i;
      float k[16], v[16], dk[16], dv[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        k[e] = e < dh ? Ks[jrow * LDX + col + e] : 0.f;
        v[e] = e < dh ? Vs[jrow * LDX + col + e] : 0.f;
        dk[e] = 0.f;
        dv[e] = 0.f;
      }
      for (int qi = 0; qi < n; ++qi) {
        const int row = base + qi;
        const float *qr = Qs + row * LDX + col;
        const float *gr = dHs + row * LDX + col;
        float dot = 0.f, dd = 0.f;
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (e < dh) { dot = fmaf(qr[e], k[e], dot); dd = fmaf(gr[e], v[e], dd); }
        const float a = expf(dot * scale - smx[row * 16 + h]) * sis[row * 16 + h];
        const float w = scale * a * (dd - sdl[row * 16 + h]);
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (e < dh) { dv[e] = fmaf(a, gr[e], dv[e]); dk[e] = fmaf(w, qr[e], dk[e]); }
      }
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (e < dh) { dK[jrow * LDX + col + e] = dk[e]; dV[jrow * LDX + col + e] = dv[e]; }
    }
    __syncwarp();
  }
}

template <int D>
__global__ void __launch_bounds__(kThreads, 1)
    k_bwd32(const DevModel m, const int mode, const uint32_t *__restrict__ sig,
            const uint32_t *__restrict__ sigp, const size_t B, const float2 *__restrict__ cot,
            float *__restrict__ gacc, const int n_copies, const size_t g_stride, float *__restrict__ O,
            uint16_t *__restrict__ O16, const float2 *__restrict__ oref, const size_t P, const size_t ldo,
            const FlatOffsets fo, float *__restrict__ scratch, float *__restrict__ dtab) {
  using BG = BwdGeom<D>;
  constexpr int R = BG::R, LDX = BG::LDX;
  using G = F32Geom<D, R>;
  extern __shared__ float4 smem4[];
  float *sm = reinterpret_cast<float *>(smem4);
  float *Bf[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) Bf[i] = sm + i * BG::BUF;
  float *Ws = sm + BG::W_OFF, *st = sm + BG::ST_OFF, *Fs = sm + BG::F_OFF;
  uint32_t *csig = reinterpret_cast<uint32_t *>(sm + BG::C_OFF);
  uint32_t *csigp = csig + R / 2;
  float2 *ccot = reinterpret_cast<float2 *>(sm + BG::T_OFF);

  const int n = m.n_sites;
  const int ts = seqs_for(n, R), tcv = ts / 2, nrows = ts * n;
  const size_t nvirt = mode == 0 ? B : 2 * B;
  const size_t ntiles = (nvirt + tcv - 1) / tcv;
  const size_t blk = (size_t)6 * R * D;
  float *scr = scratch + (size_t)blockIdx.x * (size_t)m.layers * blk;
  SinkCtx sk;
  sk.mode = mode;
  sk.g = gacc ? gacc + (size_t)(blockIdx.x % n_copies) * g_stride : nullptr;   // g_stride % 4 == 0
  sk.O = O;
  sk.O16 = O16;
  sk.oref = oref;
  sk.P = P;
  sk.ldo = ldo;
  sk.dtab = dtab;
  const int nranges = mode == 0 ? 1 : tcv;

  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (threadIdx.x < tcv) {
      const size_t vg = tile * tcv + threadIdx.x;
      const bool valid = vg < nvirt;
      const size_t b = mode == 0 ? vg : vg / 2;
      csig[threadIdx.x] = valid ? sig[b] : 0u;
      csigp[threadIdx.x] = valid ? sigp[b] : 0u;
      float2 c = make_float2(0.f, 0.f);
      if (valid) c = mode == 0 ? cot[b] : ((vg & 1) ? make_float2(0.f, -1.f) : make_float2(1.f, 0.f));
      ccot[threadIdx.x] = c;
    }
    __syncthreads();
    // virtual configuration v of this tile -> (global configuration, seed) for mode-1 sinks
    auto vb = [&](int v) -> long long { return (long long)((tile * tcv + v) / 2); };
    auto vs = [&](int v) -> int { return (int)((tile * tcv + v) & 1); };
    auto vvalid = [&](int v) -> bool { return tile * tcv + v < nvirt; };

    // ---------------- forward recompute, saving activations per layer
    embed_f32<D, R>(m, csig, csigp, ts, Bf[0]);
    __syncthreads();
    for (int l = 0; l < m.layers; ++l) {
      const DevLayer &L = m.L[l];
      float *sl = scr + (size_t)l * blk;
      save_block<D, R>(Bf[0], sl);
      stage_block<D>(L.Wq, D, 0, D, Ws);
      stage_block<D>(L.Wk, D, 0, D, Ws + D * D);
      stage_block<D>(L.Wv, D, 0, D, Ws + 2 * D * D);
      __syncthreads();
      {
        float acc[G::RPT][8];
#pragma unroll
        for (int w = 0; w < 3; ++w) {
          acc_zero<D, R>(acc);
          mm_acc<D, R>(Bf[0], LDX, Ws + w * D * D, D, acc);
          acc_store<D, R>(acc, Bf[1 + w]);
        }
      }
      __syncthreads();
      attention_f32<D>(Bf[1], Bf[2], Bf[3], ts, n, m.heads, m.dh, Bf[4]);
      stage_block<D>(L.Wo, D, 0, D, Ws);
      __syncthreads();
      save_block<D, R>(Bf[1], sl + 1 * R * D);
      save_block<D, R>(Bf[2], sl + 2 * R * D);
      save_block<D, R>(Bf[3], sl + 3 * R * D);
      save_block<D, R>(Bf[4], sl + 4 * R * D);
      {
        float acc[G::RPT][8];
        acc_zero<D, R>(acc);
        mm_acc<D, R>(Bf[4], LDX, Ws, D, acc);
        acc_foreach<D, R>(acc, [&](int r, int c, float v) { Bf[0][r * LDX + c] += v; });
      }
      __syncthreads();
      if (m.ffn > 0) {
        save_block<D, R>(Bf[0], sl + 5 * R * D);
        float acc2[G::RPT][8];
        acc_zero<D, R>(acc2);
        for (int c0 = 0; c0 < m.ffn; c0 += D) {
          stage_block<D>(L.W1, m.ffn, c0, D, Ws);
          stage_block<D>(L.W2 + (size_t)c0 * D, D, 0, D, Ws + D * D);
          __syncthreads();
          float acc[G::RPT][8];
          acc_zero<D, R>(acc);
          mm_acc<D, R>(Bf[0], LDX, Ws, D, acc);
          acc_foreach<D, R>(acc, [&](int r, int c, float v) {
            Bf[7][r * LDX + c] = gelu_f(v + __ldg(L.b1 + c0 + c));
          });
          __syncthreads();
          mm_acc<D, R>(Bf[7], LDX, Ws + D * D, D, acc2);
          __syncthreads();
        }
        acc_foreach<D, R>(acc2, [&](int r, int c, float v) { Bf[0][r * LDX + c] += v + __ldg(L.b2 + c); });
        __syncthreads();
      }
    }
    // ---------------- head: pooling, dense layer, symmetrisation weights, cotangents of F
    float *Hp = Bf[7];
    {
      const float inv_n = 1.0f / (float)n;
      for (int idx = threadIdx.x; idx < ts * D; idx += kThreads) {
        const int s = idx / D, c = idx % D;
        float a = 0.f;
        for (int i = 0; i < n; ++i) a += Bf[0][(s * n + i) * LDX + c];
        Hp[s * D + c] = a * inv_n;
      }
      __syncthreads();
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int p = warp; p < ts * 2; p += kThreads / 32) {
        const int s = p >> 1, o = p & 1;
        float a = 0.f;
        for (int c = lane; c < D; c += 32) a = fmaf(Hp[s * D + c], __ldg(m.Wh + 2 * c + o), a);
        a = warp_sum(a);
        if (lane == 0) Fs[p] = a + __ldg(m.bh + o);
      }
      __syncthreads();
      for (int v = threadIdx.x; v < tcv; v += kThreads) {
        float2 pw, pv;
        symmetrise(Fs[4 * v], Fs[4 * v + 1], Fs[4 * v + 2], Fs[4 * v + 3], &pw, &pv);
        const float2 c = ccot[v];
        const float cwr = c.x * pw.x - c.y * pw.y, cwi = c.x * pw.y + c.y * pw.x;
        const float cvr = c.x * pv.x - c.y * pv.y, cvi = c.x * pv.y + c.y * pv.x;
        Fs[4 * v] = cwr;
        Fs[4 * v + 1] = -cwi;
        Fs[4 * v + 2] = cvr;
        Fs[4 * v + 3] = cvi;
      }
      __syncthreads();
      // dWh[k][o] = sum_s h[s][k] dF[s][o], dbh[o] = sum_s dF[s][o]
      for (int rg = 0; rg < nranges; ++rg) {
        const int s0 = mode == 0 ? 0 : 2 * rg, s1 = mode == 0 ? ts : 2 * rg + 2;
        if (mode == 1 && !vvalid(rg)) continue;
        for (int idx = threadIdx.x; idx < 2 * D + 2; idx += kThreads) {
          float a = 0.f;
          if (idx < 2 * D) {
            const int k = idx >> 1, o = idx & 1;
            for (int s = s0; s < s1; ++s) a = fmaf(Hp[s * D + k], Fs[2 * s + o], a);
            sink1(sk, fo.Wh + idx, a, vb(rg), vs(rg));
          } else {
            const int o = idx - 2 * D;
            for (int s = s0; s < s1; ++s) a += Fs[2 * s + o];
            sink1(sk, fo.bh + o, a, vb(rg), vs(rg));
          }
        }
      }
      // dX_L[r][k] = (1/N) sum_o Wh[k][o] dF[s(r)][o]
      for (int idx = threadIdx.x; idx < R * D; idx += kThreads) {
        const int r = idx / D, k = idx % D;
        float v = 0.f;
        if (r < nrows) {
          const int s = r / n;
          v = (__ldg(m.Wh + 2 * k) * Fs[2 * s] + __ldg(m.Wh + 2 * k + 1) * Fs[2 * s + 1]) * inv_n;
        }
        Bf[6][r * LDX + k] = v;
      }
      __syncthreads();
    }
    // ---------------- layers in reverse
    for (int l = m.layers - 1; l >= 0; --l) {
      const DevLayer &L = m.L[l];
      const float *sl = scr + (size_t)l * blk;
      load_block<D, R>(sl, Bf[0]);
      load_block<D, R>(sl + 1 * R * D, Bf[1]);
      load_block<D, R>(sl + 2 * R * D, Bf[2]);
      load_block<D, R>(sl + 3 * R * D, Bf[3]);
      load_block<D, R>(sl + 4 * R * D, Bf[4]);
      if (m.ffn > 0) load_block<D, R>(sl + 5 * R * D, Bf[5]);
      __syncthreads();
      if (m.ffn > 0) {
        float adx[G::RPT][8];
        acc_zero<D, R>(adx);
        acc_foreach<D, R>(adx, [&](int r, int c, float &v) { v = Bf[6][r * LDX + c]; });
        for (int c0 = 0; c0 < m.ffn; c0 += D) {
          stage_block<D>(L.W1, m.ffn, c0, D, Ws);                  // W1_c [in][hid]
          stage_blockT<D>(L.W1, m.ffn, c0, Ws + D * D);            // W1_c^T [hid][in]
          stage_blockT<D>(L.W2 + (size_t)c0 * D, D, 0, Ws + 2 * D * D);   // W2_c^T [out][hid]
          __syncthreads();
          {
            float au[G::RPT][8], ag[G::RPT][8];
            acc_zero<D, R>(au);
            mm_acc<D, R>(Bf[5], LDX, Ws, D, au);
            acc_zero<D, R>(ag);
            mm_acc<D, R>(Bf[6], LDX, Ws + 2 * D * D, D, ag);
            acc_foreach<D, R>(au, [&](int r, int c, float &v) {
              v += __ldg(L.b1 + c0 + c);
              Bf[7][r * LDX + c] = v;     // U (pre-activation)
            });
            // dU = dG * gelu'(U): both accumulators share the (row, col) map
            const int tx = threadIdx.x % G::TX, ty = threadIdx.x / G::TX;
#pragma unroll
            for (int j = 0; j < G::RPT; ++j)
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int col = (e < 4) ? (4 * tx + e) : (D / 2 + 4 * tx + e - 4);
                Bf[8][(ty + j * G::TY) * LDX + col] = ag[j][e] * gelu_grad_f(au[j][e]);
              }
          }
          __syncthreads();
          for (int rg = 0; rg < nranges; ++rg) {
            if (mode == 1 && !vvalid(rg)) continue;
            const int r0 = mode == 0 ? 0 : rg * 2 * n, r1 = mode == 0 ? nrows : r0 + 2 * n;
            float dw[BG::KPT][8];
            mmT_acc<D, true>(Bf[7], Bf[6], r0, r1, dw);
            sink_block<D>(sk, dw, fo.W2[l] + (long long)c0 * D, D, vb(rg), vs(rg));
            mmT_acc<D, false>(Bf[5], Bf[8], r0, r1, dw);
            sink_block<D>(sk, dw, fo.W1[l] + c0, m.ffn, vb(rg), vs(rg));
            colsum_sink<D>(sk, Bf[8], r0, r1, fo.b1[l] + c0, vb(rg), vs(rg));
          }
          mm_acc<D, R>(Bf[8], LDX, Ws + D * D, D, adx);
          __syncthreads();
        }
        for (int rg = 0; rg < nranges; ++rg) {
          if (mode == 1 && !vvalid(rg)) continue;
          const int r0 = mode == 0 ? 0 : rg * 2 * n, r1 = mode == 0 ? nrows : r0 + 2 * n;
          colsum_sink<D>(sk, Bf[6], r0, r1, fo.b2[l], vb(rg), vs(rg));
        }
        __syncthreads();
        acc_store<D, R>(adx, Bf[6]);   // dX at the attention-block output
        __syncthreads();
      }
      // attention block: X' = concat(heads) Wo + X
      stage_blockT<D>(L.Wo, D, 0, Ws);
      __syncthreads();
      {
        float acc[G::RPT][8];
        acc_zero<D, R>(acc);
        mm_acc<D, R>(Bf[6], LDX, Ws, D, acc);
        acc_store<D, R>(acc, Bf[7]);   // dH
      }
      for (int rg = 0; rg < nranges; ++rg) {
        if (mode == 1 && !vvalid(rg)) continue;
        const int r0 = mode == 0 ? 0 : rg * 2 * n, r1 = mode == 0 ? nrows : r0 + 2 * n;
        float dw[BG::KPT][8];
        mmT_acc<D, false>(Bf[4], Bf[6], r0, r1, dw);
        sink_block<D>(sk, dw, fo.Wo[l], D, vb(rg), vs(rg));
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < (R - nrows) * D; idx += kThreads) {
        const int r = nrows + idx / D, c = idx % D;
        Bf[4][r * LDX + c] = 0.f;
        Bf[5][r * LDX + c] = 0.f;
        Bf[8][r * LDX + c] = 0.f;
      }
      attention_bwd<D>(Bf[1], Bf[2], Bf[3], Bf[7], Bf[4], Bf[5], Bf[8], st, ts, n, m.heads, m.dh);
      stage_blockT<D>(L.Wq, D, 0, Ws);
      stage_blockT<D>(L.Wk, D, 0, Ws + D * D);
      stage_blockT<D>(L.Wv, D, 0, Ws + 2 * D * D);
      __syncthreads();
      for (int rg = 0; rg < nranges; ++rg) {
        if (mode == 1 && !vvalid(rg)) continue;
        const int r0 = mode == 0 ? 0 : rg * 2 * n, r1 = mode == 0 ? nrows : r0 + 2 * n;
        float dw[BG::KPT][8];
        mmT_acc<D, false>(Bf[0], Bf[4], r0, r1, dw);
        sink_block<D>(sk, dw, fo.Wq[l], D, vb(rg), vs(rg));
        mmT_acc<D, false>(Bf[0], Bf[5], r0, r1, dw);
        sink_block<D>(sk, dw, fo.Wk[l], D, vb(rg), vs(rg));
        mmT_acc<D, false>(Bf[0], Bf[8], r0, r1, dw);
        sink_block<D>(sk, dw, fo.Wv[l], D, vb(rg), vs(rg));
      }
      {
        float acc[G::RPT][8];
        acc_zero<D, R>(acc);
        acc_foreach<D, R>(acc, [&](int r, int c, float &v) { v = Bf[6][r * LDX + c]; });
        mm_acc<D, R>(Bf[4], LDX, Ws, D, acc);
        mm_acc<D, R>(Bf[5], LDX, Ws + D * D, D, acc);
        mm_acc<D, R>(Bf[8], LDX, Ws + 2 * D * D, D, acc);
        __syncthreads();
        acc_store<D, R>(acc, Bf[6]);
      }
      __syncthreads();
    }
    // ---------------- embedding: gradient of the table row each token read (4 token rows, or the 64
    // conv patterns whose table is back-propagated to the conv parameters by k_conv_vjp).  The layer-0
    // input buffer is dead here and holds each row's pattern.
    {
      const int npat = m.embed == 0 ? 4 : 64;
      int *rpat = reinterpret_cast<int *>(Bf[0]);
      for (int r = threadIdx.x; r < nrows; r += kThreads) {
        const int s = r / n, i = r % n, cfg = s >> 1;
        const uint32_t w1 = (s & 1) ? csigp[cfg] : csig[cfg];
        const uint32_t w2 = (s & 1) ? csig[cfg] : csigp[cfg];
        rpat[r] = embed_pattern(m.embed, w1, w2, i, n);
      }
      __syncthreads();
      float *dcopy = (m.embed != 0 && mode == 0) ? sk.dtab + (size_t)(blockIdx.x % n_copies) * (64 * D) : nullptr;
      for (int rg = 0; rg < nranges; ++rg) {
        if (mode == 1 && !vvalid(rg)) continue;
        const int r0 = mode == 0 ? 0 : rg * 2 * n, r1 = mode == 0 ? nrows : r0 + 2 * n;
        for (int idx = threadIdx.x; idx < npat * D; idx += kThreads) {
          const int pat = idx / D, c = idx % D;
          float a = 0.f;
          for (int r = r0; r < r1; ++r)
            if (rpat[r] == pat) a += Bf[6][r * LDX + c];
          if (m.embed == 0) sink1(sk, fo.E + idx, a, vb(rg), vs(rg));
          else if (mode == 0) { if (a != 0.f) atomicAdd(dcopy + idx, a); }
          else sk.dtab[((size_t)vb(rg) * 2 + vs(rg)) * (64 * D) + idx] = a;
        }
      }
    }
    __syncthreads();
  }
}

template <int D>
static cudaError_t bwd_impl(const DevModel &m, int mode, const uint32_t *sig, const uint32_t *sigp,
                            size_t B, const float2 *cot, float *gacc, int n_copies, size_t g_stride, float *O,
                            uint16_t *O16, const float2 *oref, size_t P, size_t ldo, const FlatOffsets &fo,
                            float *scratch, float *dtab, int grid, cudaStream_t st) {
  const size_t bytes = BwdGeom<D>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_bwd32<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_bwd32<D><<<grid, kThreads, bytes, st>>>(m, mode, sig, sigp, B, cot, gacc, n_copies, g_stride, O, O16, oref, P,
                                            ldo, fo, scratch, dtab);
  return cudaGetLastError();
}

}  // namespace tdo

size_t bwd32_scratch_floats(const DevModel &m, int grid) {
  const int R = m.d == 64 ? 64 : 128;
  return (size_t)grid * (size_t)m.layers * 6 * (size_t)R * (size_t)m.d;
}

int bwd32_grid(const DevModel &m, size_t B, int mode, int n_sm) {
  const int R = m.d == 64 ? 64 : 128;
  const int tcv = tdo::seqs_for(m.n_sites, R) / 2;
  const size_t nvirt = mode == 0 ? B : 2 * B;
  const size_t ntiles = (nvirt + tcv - 1) / tcv;
  size_t grid = (size_t)n_sm;
  if (m.d < 64) grid *= 1;   // one CTA per SM (shared memory bound)
  if (grid > ntiles) grid = ntiles;
  return (int)(grid ? grid : 1);
}

cudaError_t launch_bwd32_impl(const DevModel &m, int mode, const uint32_t *sig, const uint32_t *sigp,
                              size_t B, const float2 *cot, float *gacc, int n_copies, size_t g_stride,
                              float *O, uint16_t *O16, const float2 *oref, size_t P, size_t ldo,
                              const long long *flat_offsets, float *scratch, float *dtab, int grid, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  tdo::FlatOffsets fo;
  static_assert(sizeof(tdo::FlatOffsets) == sizeof(long long) * (3 + 8 * TDO_MAX_LAYERS), "layout");
  memcpy(&fo, flat_offsets, sizeof(fo));
  switch (m.d) {
    case 16: return tdo::bwd_impl<16>(m, mode, sig, sigp, B, cot, gacc, n_copies, g_stride, O, O16, oref, P, ldo, fo, scratch,
                                      dtab, grid, st);
    case 32: return tdo::bwd_impl<32>(m, mode, sig, sigp, B, cot, gacc, n_copies, g_stride, O, O16, oref, P, ldo, fo, scratch,
                                      dtab, grid, st);
    case 64: return tdo::bwd_impl<64>(m, mode, sig, sigp, B, cot, gacc, n_copies, g_stride, O, O16, oref, P, ldo, fo, scratch,
                                      dtab, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------------- conv embedding VJP
// Back-propagates per-pattern table gradients dT[p][e] through the conv embedding table
//   a1[p][o2][f] = bc1[f] + sum_{o1,ch} Wc1[o1][ch][f] x[p][o2+o1][ch],  h1 = gelu(a1)
//   a2[p][e]     = bc2[e] + sum_{o2,f} Wc2[o2][f][e] h1[p][o2][f],        T  = gelu(a2)
// (two kernel-2 circular convolutions over sites i, i+1, i+2; x = +-1 spins of both channels).
// One block per table-gradient set (the sum of ncopy consecutive [64][d] copies); mode 0 adds into the
// accumulator g at the flat offsets, mode 1 writes O[set/2][k][set%2].
namespace tdo {
__global__ void k_conv_vjp(int d, int c1, const float *__restrict__ Wc1, const float *__restrict__ bc1,
                           const float *__restrict__ Wc2, const float *__restrict__ bc2,
                           const float *__restrict__ dT, int nsets, int ncopy, int mode, float *__restrict__ g,
                           float *__restrict__ O, uint16_t *__restrict__ O16, const float2 *__restrict__ oref,
                           size_t ldo, long long o_wc1, long long o_bc1, long long o_wc2, long long o_bc2) {
  extern __shared__ float sh[];
  float *a1 = sh;                       // [64][2][c1]
  float *dh = a1 + 64 * 2 * c1;         // [64][2][c1] (da1 in place)
  float *a2 = dh + 64 * 2 * c1;         // [64][d]     (da2 in place)
  for (int set = blockIdx.x; set < nsets; set += gridDim.x) {
    const float *dts = dT + (size_t)set * ncopy * 64 * d;
    for (int i = threadIdx.x; i < 64 * 2 * c1; i += blockDim.x) {
      const int p = i / (2 * c1), o2 = (i / c1) % 2, f = i % c1;
      float acc = bc1[f];
      for (int o1 = 0; o1 < 2; ++o1)
        for (int ch = 0; ch < 2; ++ch) {
          const int bit = (p >> (ch * 3 + o2 + o1)) & 1;
          acc = fmaf(Wc1[(o1 * 2 + ch) * c1 + f], 1.0f - 2.0f * (float)bit, acc);
        }
      a1[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * d; i += blockDim.x) {
      const int p = i / d, e = i % d;
      float acc = bc2[e];
      for (int o2 = 0; o2 < 2; ++o2)
        for (int f = 0; f < c1; ++f) acc = fmaf(Wc2[(o2 * c1 + f) * d + e], gelu_f(a1[(p * 2 + o2) * c1 + f]), acc);
      float dt = 0.f;
      for (int k = 0; k < ncopy; ++k) dt += dts[(size_t)k * 64 * d + i];
      a2[i] = dt * gelu_grad_f(acc);   // da2
    }
    __syncthreads();
    auto put = [&](long long k, float v) {
      if (mode == 0) {
        atomicAdd(g + k, v);
      } else {
        const size_t i = ((size_t)(set >> 1) * ldo + (size_t)k) * 2 + (set & 1);
        if (O16) O16[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v - ((set & 1) ? oref[k].y : oref[k].x)));
        else O[i] = v;
      }
    };
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
      float acc = 0.f;
      for (int p = 0; p < 64; ++p) acc += a2[p * d + e];
      put(o_bc2 + e, acc);
    }
    for (int i = threadIdx.x; i < 2 * c1 * d; i += blockDim.x) {
      const int o2 = i / (c1 * d), f = (i / d) % c1, e = i % d;
      float acc = 0.f;
      for (int p = 0; p < 64; ++p) acc = fmaf(a2[p * d + e], gelu_f(a1[(p * 2 + o2) * c1 + f]), acc);
      put(o_wc2 + i, acc);
    }
    for (int i = threadIdx.x; i < 64 * 2 * c1; i += blockDim.x) {
      const int p = i / (2 * c1), o2 = (i / c1) % 2, f = i % c1;
      float acc = 0.f;
      for (int e = 0; e < d; ++e) acc = fmaf(Wc2[(o2 * c1 + f) * d + e], a2[p * d + e], acc);
      dh[i] = acc * gelu_grad_f(a1[i]);   // da1
    }
    __syncthreads();
    for (int f = threadIdx.x; f < c1; f += blockDim.x) {
      float acc = 0.f;
      for (int p = 0; p < 64; ++p) acc += dh[(p * 2) * c1 + f] + dh[(p * 2 + 1) * c1 + f];
      put(o_bc1 + f, acc);
    }
    for (int i = threadIdx.x; i < 4 * c1; i += blockDim.x) {
      const int o1 = i / (2 * c1), ch = (i / c1) % 2, f = i % c1;
      float acc = 0.f;
      for (int p = 0; p < 64; ++p)
        for (int o2 = 0; o2 < 2; ++o2) {
          const int bit = (p >> (ch * 3 + o2 + o1)) & 1;
          acc = fmaf(dh[(p * 2 + o2) * c1 + f], 1.0f - 2.0f * (float)bit, acc);
        }
      put(o_wc1 + i, acc);
    }
    __syncthreads();
  }
}
}  // namespace tdo

cudaError_t launch_conv_vjp(int d, int c1, const float *Wc1, const float *bc1, const float *Wc2, const float *bc2,
                            const float *dT, int nsets, int ncopy, int mode, float *g, float *O, uint16_t *O16,
                            const float2 *oref, size_t ldo, long long o_wc1, long long o_bc1, long long o_wc2,
                            long long o_bc2, cudaStream_t st) {
  if (nsets <= 0) return cudaSuccess;
  const size_t bytes = sizeof(float) * (2 * 64 * 2 * c1 + 64 * d);
  cudaError_t e = cudaFuncSetAttribute(tdo::k_conv_vjp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  const int grid = nsets < 1024 ? nsets : 1024;
  tdo::k_conv_vjp<<<grid, 256, bytes, st>>>(d, c1, Wc1, bc1, Wc2, bc2, dT, nsets, ncopy, mode, g, O, O16, oref, ldo,
                                            o_wc1, o_bc1, o_wc2, o_bc2);
  return cudaGetLastError();
}

// oref[k] = mean over the n rows of O32 ([n][P] complex FP32): the shift removed from BF16-stored O.
namespace tdo {
__global__ void k_oref(const float2 *__restrict__ O32, int n, size_t P, float2 *__restrict__ oref) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    float ar = 0.f, ai = 0.f;
    for (int r = 0; r < n; ++r) {
      const float2 o = O32[(size_t)r * P + k];
      ar += o.x;
      ai += o.y;
    }
    oref[k] = make_float2(ar / (float)n, ai / (float)n);
  }
}
}  // namespace tdo

cudaError_t launch_oref(const float *O32, int n, size_t P, float *oref, cudaStream_t st) {
  const unsigned grid = (unsigned)((P + 255) / 256 < 4096 ? (P + 255) / 256 : 4096);
  tdo::k_oref<<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(O32), n, P, reinterpret_cast<float2 *>(oref));
  return cudaGetLastError();
}
