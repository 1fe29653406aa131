// Device helpers shared by the kernels of libtdo.so: counter RNG, activation, the Hermitian
// symmetrisation, the embedding pattern of a token, and the FP32 tile geometry.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "tdo_internal.cuh"

namespace tdo {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (c0,c1,c2,c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)), key += (W0, W1)
// between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += W0; k.y += W1; }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Proposal of Metropolis step t of chain c: which of the 2N bits to flip, and the uniform u.
// choices = 2N for the |rho|^2 chains (bit k < N flips sigma_k, else sigma'_{k-N}), N for the chains on
// the diagonal |rho(alpha, alpha)| (bit k flips site k of alpha).
__device__ __forceinline__ void metropolis_draw(uint64_t seed, uint32_t chain, uint64_t t, int choices,
                                                int *bit, float *u) {
  const uint4 x = philox4x32_10(make_uint4(chain, (uint32_t)t, (uint32_t)(t >> 32), 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  *bit = (int)(((uint64_t)(x.x >> 8) * (uint64_t)choices) >> 24);
  *u = (float)(x.y >> 8) * (1.0f / 16777216.0f);
}

// GELU, tanh form: 0.5 u (1 + tanh(sqrt(2/pi) (u + 0.044715 u^3))).
__device__ __forceinline__ float gelu_f(float u) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  return 0.5f * u * (1.0f + tanhf(k0 * (u + k1 * u * u * u)));
}
// d gelu / du
__device__ __forceinline__ float gelu_grad_f(float u) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float t = tanhf(k0 * (u + k1 * u * u * u));
  return 0.5f * (1.0f + t) + 0.5f * u * (1.0f - t * t) * k0 * (1.0f + 3.0f * k1 * u * u);
}

// Hermitian symmetrisation: w = z(s,s') = (a0, a1), v = conj z(s',s) = (b0, -b1);
// log rho = log(e^w + e^v) on the principal branch, evaluated with the larger real part factored out.
// Also returns the holomorphic weights pw = e^w / (e^w + e^v), pv = e^v / (e^w + e^v) (complex).
__device__ __forceinline__ float2 symmetrise(float a0, float a1, float b0, float b1, float2 *pw,
                                             float2 *pv) {
  const float vr = b0, vi = -b1;
  const float m = fmaxf(a0, vr);
  const float ea = expf(a0 - m), eb = expf(vr - m);
  float sa, ca, sb, cb;
  sincosf(a1, &sa, &ca);
  sincosf(vi, &sb, &cb);
  const float wr = ea * ca, wi = ea * sa, xr = eb * cb, xi = eb * sb;
  const float sr = wr + xr, si = wi + xi;
  const float n2 = sr * sr + si * si;
  if (pw) {
    const float inv = 1.0f / n2;   // (w_e / s) = w_e conj(s) / |s|^2
    *pw = make_float2((wr * sr + wi * si) * inv, (wi * sr - wr * si) * inv);
    *pv = make_float2((xr * sr + xi * si) * inv, (xi * sr - xr * si) * inv);
  }
  return make_float2(m + 0.5f * logf(n2), atan2f(si, sr));
}

// Embedding-table row of token i of a sequence whose first channel is word w1 and second w2.
// Token embedding: 2*bit(w1,i) + bit(w2,i).  Conv embedding: the 6 bits of sites i, i+1, i+2 (mod N)
// of both channels (the receptive field of two kernel-2 circular convolutions).
__device__ __forceinline__ int embed_pattern(int embed, uint32_t w1, uint32_t w2, int i, int n) {
  if (embed == 0) return (int)(((w1 >> i) & 1u) * 2u + ((w2 >> i) & 1u));
  const int i1 = (i + 1) % n, i2 = (i + 2) % n;
  return (int)(((w1 >> i) & 1u) | (((w1 >> i1) & 1u) << 1) | (((w1 >> i2) & 1u) << 2) |
               (((w2 >> i) & 1u) << 3) | (((w2 >> i1) & 1u) << 4) | (((w2 >> i2) & 1u) << 5));
}

// Sequences per 128-row tile (even: both orders of a configuration sit in one tile).
__host__ __device__ __forceinline__ int seqs_per_tile(int n) {
  int ts = 2 * (128 / (2 * n));
  return ts < 2 ? 2 : ts;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace tdo
