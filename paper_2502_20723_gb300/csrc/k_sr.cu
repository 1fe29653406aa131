// Stochastic reconfiguration solve (metric-tensor and regularisation sections):
//   (Re S + lambda I) x = rhs,  S_ij = <O_i^* O_j> - <O_i^*><O_j>  over Ns samples,
// by Jacobi-preconditioned conjugate gradients, matrix-free: with Obar = O - mean(O),
//   S v = (1/Ns) Re[Obar^H (Obar v)],
// O stored as FP32 (re, im) [Ns][P], or as BF16 pairs of O - oref (a per-parameter shift that the
// centring removes exactly; it keeps the BF16 rounding at the scale of O's spread, not of its mean).
// One iteration streams O twice from HBM (t = Obar v per sample,
// then w = Obar^H t per parameter) and is HBM-bound; both passes keep many independent loads in flight.
// Two optional products read O once (k_sr_fused on thread-block clusters, k_sr_grid over the whole grid).
// Products are formed in FP32 over runs of 32 terms and accumulated in FP64 (GB300's FP64 rate is far
// below its FP32 rate); CG vectors and scalars are FP64 and stay on the device: a device flag ends the
// iteration, the host looks at it between groups of iterations only.
#include "tdo_internal.cuh"
#include "tdo_device.cuh"
#include "tcgen05.cuh"

namespace tdo {

constexpr int kSrBlock = 256;
constexpr int kRun = 32;     // FP32 products per FP64 accumulation

// One complex element of O: FP32 (re, im) or a BF16 pair (re in the low half).
__device__ __forceinline__ float2 cplx(float2 v) { return v; }
__device__ __forceinline__ float2 cplx(uint32_t v) {
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}
// Four consecutive elements from a 16-byte-aligned address.
__device__ __forceinline__ void load4(const float2 *p, float2 (&c)[4]) {
  const float4 a = __ldcs(reinterpret_cast<const float4 *>(p)), b = __ldcs(reinterpret_cast<const float4 *>(p) + 1);
  c[0] = make_float2(a.x, a.y); c[1] = make_float2(a.z, a.w);
  c[2] = make_float2(b.x, b.y); c[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void load4(const uint32_t *p, float2 (&c)[4]) {
  const uint4 q = __ldcs(reinterpret_cast<const uint4 *>(p));
  c[0] = cplx(q.x); c[1] = cplx(q.y); c[2] = cplx(q.z); c[3] = cplx(q.w);
}

enum {
  S_RZ = 0, S_BN, S_AL, S_RN, S_DONE, S_IT, S_TOL, S_PAP, S_CR, S_CI, S_TR, S_TI, S_TT, S_RESTART, S_COUNT
};
// S_RESTART (graph mode): 0 none, 1 a restart from x = 0 is pending, 2 the solve was restarted
// S_DONE: 1 converged, 2 breakdown (p . S' p not positive: p = 0 before convergence), 3 a non-finite value
// (in the right-hand side, the log-derivatives' moments or a product)
enum { SR_CONVERGED = 1, SR_BREAKDOWN = 2, SR_NONFINITE = 3 };

__device__ __forceinline__ double block_sum_d(double v, double *sh) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum_d(t);
  }
  __syncthreads();
  return t;   // valid in thread 0
}

__device__ __forceinline__ double sum_parts(const double *part, int n, double *sh) {
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
  return block_sum_d(a, sh);
}

// vf = (float) v; block partials of mean . vf (re, im).  The centring term takes the same rounded copy
// as the t-pass, so t = (O - mean) vf holds up to the products' rounding.
// (zero, nzero: 16-byte words the next launch needs at zero, or NULL)
__global__ void k_sr_vprep(size_t P, const double *__restrict__ v, const double2 *__restrict__ mean,
                           float *__restrict__ vf, double *__restrict__ part, double *__restrict__ part2,
                           const double *__restrict__ sc, uint4 *__restrict__ zero = nullptr, size_t nzero = 0) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  if (zero)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nzero; i += gridDim.x * (size_t)blockDim.x)
      zero[i] = make_uint4(0u, 0u, 0u, 0u);
  double cr = 0.0, ci = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    const float xf = (float)v[k];
    vf[k] = xf;
    cr += mean[k].x * (double)xf;
    ci += mean[k].y * (double)xf;
  }
  const double a = block_sum_d(cr, sh);
  const double b = block_sum_d(ci, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = a; part2[blockIdx.x] = b; }
}

__global__ void k_sr_cfin(const double *__restrict__ part, const double *__restrict__ part2, int nb,
                          double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  const double a = sum_parts(part, nb, sh);
  const double b = sum_parts(part2, nb, sh);
  if (threadIdx.x == 0) { sc[S_CR] = a; sc[S_CI] = b; }
}

// Partial dot products of the rows of O with v over one chunk of parameters: block (chunk, sg) streams
// the chunk of every sample row of sample group sg (8 KB contiguous), one warp per row at a time,
// 16-byte loads per lane when every row starts on a 16-byte boundary, with the chunk of v in shared
// memory.  part[chunk][s] = sum_{k in chunk} O[s][k] v[k].
constexpr int kChunk = 1024;   // the smaller chunk (the most chunks: buffer sizes)
constexpr int kSampleGroups = 8;
// Parameters per chunk: 1024 for FP32 pairs, 2048 for BF16 pairs, so that a block reads 8 KB contiguous
// runs of a row either way (4 KB runs left BF16 passes at 71-83 % of the copy bandwidth); chunk / 4
// threads per block.
template <typename OT>
struct SrChunk {
  static constexpr int value = sizeof(OT) == 4 ? 2 * kChunk : kChunk;
};

template <typename OT, bool VEC>
__global__ void __launch_bounds__(SrChunk<OT>::value / 4) k_sr_tpart(const OT *__restrict__ O, size_t Ns, size_t P,
                                                                      size_t ldo, const float *__restrict__ vf,
                                                                      double2 *__restrict__ part,
                                                                      const double *__restrict__ sc) {
  constexpr int CH = SrChunk<OT>::value;
  __shared__ float4 vs4[CH / 4];
  float *vs = reinterpret_cast<float *>(vs4);
  if (sc[S_DONE] != 0.0) return;
  const size_t k0 = (size_t)blockIdx.x * CH;
  const int kn = (int)((P - k0) < (size_t)CH ? (P - k0) : (size_t)CH);
  for (int i = threadIdx.x; i < CH; i += blockDim.x) vs[i] = i < kn ? vf[k0 + i] : 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const size_t per = (Ns + kSampleGroups - 1) / kSampleGroups;
  const size_t s_begin = (size_t)blockIdx.y * per;
  const size_t s_end = s_begin + per < Ns ? s_begin + per : Ns;
  for (size_t s = s_begin + warp; s < s_end; s += nw) {
    const OT *row = O + s * ldo + k0;
    float ar = 0.f, ai = 0.f;
    if (VEC) {   // 4 elements per lane and load, then the chunk's last kn % 4 one by one
#pragma unroll 4
      for (int i4 = lane; i4 < kn / 4; i4 += 32) {
        float2 c[4];
        load4(row + 4 * i4, c);
        const float4 x = vs4[i4];
        ar = fmaf(c[0].x, x.x, fmaf(c[1].x, x.y, fmaf(c[2].x, x.z, fmaf(c[3].x, x.w, ar))));
        ai = fmaf(c[0].y, x.x, fmaf(c[1].y, x.y, fmaf(c[2].y, x.z, fmaf(c[3].y, x.w, ai))));
      }
      for (int i = (kn & ~3) + lane; i < kn; i += 32) {
        const float2 o = cplx(__ldg(row + i));
        ar = fmaf(o.x, vs[i], ar);
        ai = fmaf(o.y, vs[i], ai);
      }
    } else {
#pragma unroll 8
      for (int i = lane; i < kn; i += 32) {
        const float2 o = cplx(__ldg(row + i));
        const float x = vs[i];
        ar = fmaf(o.x, x, ar);
        ai = fmaf(o.y, x, ai);
      }
    }
    ar = warp_sum(ar);
    ai = warp_sum(ai);
    if (lane == 0) part[(size_t)blockIdx.x * Ns + s] = make_double2(ar, ai);
  }
}

// t[s] = sum_chunks part[chunk][s] - mean . v   (thread per sample, FP64)
__global__ void k_sr_tred(const double2 *__restrict__ part, int nchunks, size_t Ns, float2 *__restrict__ t,
                          const double *__restrict__ sc) {
  if (sc[S_DONE] != 0.0) return;
  const double cr = sc[S_CR], ci = sc[S_CI];
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < Ns; s += gridDim.x * (size_t)blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int c = 0; c < nchunks; ++c) { const double2 q = part[(size_t)c * Ns + s]; a += q.x; b += q.y; }
    t[s] = make_float2((float)(a - cr), (float)(b - ci));
  }
}

// T = sum_s t[s] (zero in exact arithmetic; subtracted explicitly below) and sum_s |t[s]|^2, from which
// p . S' p = (1/Ns) sum_s |t_s - T/Ns|^2 + shift |p|^2 is formed: non-negative by construction, where
// the dot product of p with the rounded S' p is not once |O| is large against the shift.
__global__ void k_sr_tsum(const float2 *__restrict__ t, size_t Ns, double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  double a = 0.0, b = 0.0, q = 0.0;
  for (size_t s = threadIdx.x; s < Ns; s += blockDim.x) {
    const double x = t[s].x, y = t[s].y;
    a += x;
    b += y;
    q += x * x + y * y;
  }
  a = block_sum_d(a, sh);
  b = block_sum_d(b, sh);
  q = block_sum_d(q, sh);
  if (threadIdx.x == 0) { sc[S_TR] = a; sc[S_TI] = b; sc[S_TT] = q; }
}

// Partial products w = Re(O^H t) over one chunk of parameters and one sample group: block
// (chunk, sg) streams the chunk (8 KB contiguous) of every sample row of its
// group, each thread owning 4 consecutive parameters (16-byte loads when every row starts on a 16-byte
// boundary), with the group's t in shared memory.  FP32 runs of kRun rows, FP64 across runs.
// wpart[sg][k] = sum_{s in group sg} Re(conj(O[s][k]) t[s]).
constexpr int kWRows = 2048;   // t values of a sample group staged at a time (16 KB)
template <typename OT, bool VEC>
__global__ void __launch_bounds__(SrChunk<OT>::value / 4) k_sr_wpart(const OT *__restrict__ O, size_t Ns, size_t P,
                                                                      size_t ldo, const float2 *__restrict__ t,
                                                                      double *__restrict__ wpart,
                                                                      const double *__restrict__ sc) {
  __shared__ float2 ts[kWRows];
  if (sc[S_DONE] != 0.0) return;
  const size_t k = (size_t)blockIdx.x * SrChunk<OT>::value + 4 * threadIdx.x;
  const int kn = k < P ? (int)(P - k < 4 ? P - k : 4) : 0;
  const size_t per = (Ns + kSampleGroups - 1) / kSampleGroups;
  const size_t s_begin = (size_t)blockIdx.y * per;
  const size_t s_end = s_begin + per < Ns ? s_begin + per : Ns;
  double w[4] = {0.0, 0.0, 0.0, 0.0};
  for (size_t g0 = s_begin; g0 < s_end; g0 += kWRows) {
    const int gn = (int)(s_end - g0 < (size_t)kWRows ? s_end - g0 : (size_t)kWRows);
    __syncthreads();
    for (int i = threadIdx.x; i < gn; i += blockDim.x) ts[i] = t[g0 + i];
    __syncthreads();
    if (kn == 0) continue;
    for (int r0 = 0; r0 < gn; r0 += kRun) {
      const int r1 = r0 + kRun < gn ? r0 + kRun : gn;
      float f[4] = {0.f, 0.f, 0.f, 0.f};
      if (VEC && kn == 4) {
        int r = r0;
        if constexpr (sizeof(OT) == 4) {   // BF16 pairs: 8 rows (8 x 16 bytes) in flight per thread
          for (; r + 8 <= r1; r += 8) {
            uint4 q[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) q[u] = __ldcs(reinterpret_cast<const uint4 *>(O + (g0 + r + u) * ldo + k));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const float2 tv = ts[r + u];
              const float2 c0 = cplx(q[u].x), c1 = cplx(q[u].y), c2 = cplx(q[u].z), c3 = cplx(q[u].w);
              f[0] = fmaf(c0.x, tv.x, fmaf(c0.y, tv.y, f[0]));
              f[1] = fmaf(c1.x, tv.x, fmaf(c1.y, tv.y, f[1]));
              f[2] = fmaf(c2.x, tv.x, fmaf(c2.y, tv.y, f[2]));
              f[3] = fmaf(c3.x, tv.x, fmaf(c3.y, tv.y, f[3]));
            }
          }
        }
        for (; r + 4 <= r1; r += 4) {
          float2 c[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u) load4(O + (g0 + r + u) * ldo + k, c[u]);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 tv = ts[r + u];
#pragma unroll
            for (int e = 0; e < 4; ++e) f[e] = fmaf(c[u][e].x, tv.x, fmaf(c[u][e].y, tv.y, f[e]));
          }
        }
        for (; r < r1; ++r) {
          float2 c[4];
          load4(O + (g0 + r) * ldo + k, c);
          const float2 tv = ts[r];
#pragma unroll
          for (int e = 0; e < 4; ++e) f[e] = fmaf(c[e].x, tv.x, fmaf(c[e].y, tv.y, f[e]));
        }
      } else {
        for (int r = r0; r < r1; ++r) {
          const float2 tv = ts[r];
          const OT *row = O + (g0 + r) * ldo + k;
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (e < kn) {
              const float2 o = cplx(__ldcs(row + e));
              f[e] = fmaf(o.x, tv.x, fmaf(o.y, tv.y, f[e]));
            }
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) w[e] += (double)f[e];
    }
  }
  for (int e = 0; e < kn; ++e) wpart[(size_t)blockIdx.y * P + k + e] = w[e];
}

// Moments of O in one pass, with the w-pass's access shape (a block owns one chunk of parameters, 8 KB
// contiguous per row, of one of kSampleGroups sample groups; each thread 4 consecutive parameters):
// mpart[q][sg][k] = sum over group sg of Re O[s][k] (q = 0), Im O[s][k] (q = 1), |O[s][k]|^2 (q = 2), in
// FP32 runs of kRun samples accumulated in FP64.
template <typename OT, bool VEC>
__global__ void __launch_bounds__(SrChunk<OT>::value / 4) k_sr_mpart(const OT *__restrict__ O, size_t Ns, size_t P,
                                                                      size_t ldo, double *__restrict__ mpart) {
  const size_t k = (size_t)blockIdx.x * SrChunk<OT>::value + 4 * threadIdx.x;
  const int kn = k < P ? (int)(P - k < 4 ? P - k : 4) : 0;
  if (kn == 0) return;
  const size_t per = (Ns + kSampleGroups - 1) / kSampleGroups;
  const size_t s_begin = (size_t)blockIdx.y * per;
  const size_t s_end = s_begin + per < Ns ? s_begin + per : Ns;
  double ar[4] = {0.0, 0.0, 0.0, 0.0}, ai[4] = {0.0, 0.0, 0.0, 0.0}, aa[4] = {0.0, 0.0, 0.0, 0.0};
  auto acc = [](float2 o, float &fr, float &fi, float &fa) {
    fr += o.x;
    fi += o.y;
    fa = fmaf(o.x, o.x, fmaf(o.y, o.y, fa));
  };
  for (size_t r0 = s_begin; r0 < s_end; r0 += kRun) {
    const size_t r1 = r0 + kRun < s_end ? r0 + kRun : s_end;
    float fr[4] = {0.f, 0.f, 0.f, 0.f}, fi[4] = {0.f, 0.f, 0.f, 0.f}, fa[4] = {0.f, 0.f, 0.f, 0.f};
    size_t r = r0;
    if (VEC && kn == 4) {
      if constexpr (sizeof(OT) == 4) {   // BF16 pairs: 8 rows (8 x 16 bytes) in flight per thread
        for (; r + 8 <= r1; r += 8) {
          uint4 q[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) q[u] = __ldcs(reinterpret_cast<const uint4 *>(O + (r + u) * ldo + k));
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            acc(cplx(q[u].x), fr[0], fi[0], fa[0]);
            acc(cplx(q[u].y), fr[1], fi[1], fa[1]);
            acc(cplx(q[u].z), fr[2], fi[2], fa[2]);
            acc(cplx(q[u].w), fr[3], fi[3], fa[3]);
          }
        }
      }
      for (; r + 4 <= r1; r += 4) {
        float2 c[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) load4(O + (r + u) * ldo + k, c[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc(c[u][e], fr[e], fi[e], fa[e]);
      }
      for (; r < r1; ++r) {
        float2 c[4];
        load4(O + r * ldo + k, c);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc(c[e], fr[e], fi[e], fa[e]);
      }
    } else {
      for (; r < r1; ++r) {
        const OT *row = O + r * ldo + k;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (e < kn) acc(cplx(__ldcs(row + e)), fr[e], fi[e], fa[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ar[e] += (double)fr[e];
      ai[e] += (double)fi[e];
      aa[e] += (double)fa[e];
    }
  }
  const size_t g = (size_t)blockIdx.y * P;
  for (int e = 0; e < kn; ++e) {
    mpart[g + k + e] = ar[e];
    mpart[(size_t)kSampleGroups * P + g + k + e] = ai[e];
    mpart[2 * (size_t)kSampleGroups * P + g + k + e] = aa[e];
  }
}

// mean[k] = (1/Ns) sum_s O[s][k] and the Jacobi preconditioner diag[k] = (1/Ns) sum_s |O[s][k]|^2 -
// |mean[k]|^2 + shift (the variance of O_k floored at 0; 1 where that sum is 0), from the group sums.
// The preconditioner only sets the CG's convergence rate, so the one-pass variance formula is accurate
// enough for it.
__global__ void k_sr_mfin(size_t Ns, size_t P, double shift, const double *__restrict__ mpart,
                          double2 *__restrict__ mean, double *__restrict__ diag) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    double ar = 0.0, ai = 0.0, aa = 0.0;
#pragma unroll
    for (int g = 0; g < kSampleGroups; ++g) {
      ar += mpart[(size_t)g * P + k];
      ai += mpart[(size_t)(kSampleGroups + g) * P + k];
      aa += mpart[(size_t)(2 * kSampleGroups + g) * P + k];
    }
    const double mr = ar / (double)Ns, mi = ai / (double)Ns;
    mean[k] = make_double2(mr, mi);
    const double var = aa / (double)Ns - (mr * mr + mi * mi);
    const double dk = (var > 0.0 ? var : 0.0) + shift;
    diag[k] = dk > 0.0 ? dk : 1.0;   // a constant O_k with no shift: leave that coordinate unscaled
  }
}

// Ap[k] = (1/Ns) [sum_g wpart[g][k] - Re(conj(mean[k]) T)] + shift p[k] over ng partial rows; partials
// of p . p.
__global__ void k_sr_wfin(size_t Ns, size_t P, const double2 *__restrict__ mean, const double *__restrict__ wpart,
                          int ng, const double *__restrict__ p, double shift, double *__restrict__ Ap,
                          double *__restrict__ part, const double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  const double Tr = sc[S_TR], Ti = sc[S_TI];
  double loc = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    double a = 0.0;
    for (int g = 0; g < ng; ++g) a += wpart[(size_t)g * P + k];
    const double2 m = mean[k];
    const double v = (a - (m.x * Tr + m.y * Ti)) / (double)Ns + shift * p[k];
    Ap[k] = v;
    loc += p[k] * p[k];
  }
  const double b = block_sum_d(loc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// ---------------------------------------------------------------- one-pass product (BF16 pairs)
// S' v with O read from HBM once.  Thread-block clusters of C CTAs share a range of sample rows; CTA q of a
// cluster owns the parameter slice [q SL, q SL + SL) of each of those rows.  Per row:
//   - the slice arrives by one bulk copy into a ring of kFusedRing shared-memory buffers;
//   - the CTA forms its partial of t_s = O_s . v over the slice and sends it to every other CTA of the
//     cluster by an asynchronous store into the peer's shared memory that also counts its 16 bytes on the
//     peer's mbarrier (st.async ... complete_tx); its own partial goes to its own slot by a plain store;
//   - once all C partials of the row are in, warp 1 forms t_s (centred as in k_sr_tred) and publishes it
//     in shared memory, and every thread adds Re(conj(O_sk) t_s) to its parameters' FP32 run sums from the
//     same buffer.
// The partials of rows s + 1 and s + 2 are sent before row s's are awaited, so the exchange overlaps the
// stream; with a lookahead of kFusedLook rows, 2 kFusedLook + 2 exchange slots keep a CTA that runs ahead
// from overwriting a slot (or counting bytes on a barrier phase) that a peer has not finished with.  A
// slot's barrier is armed for (C - 1) x 16 bytes by its own CTA before any peer can send into that phase
// (at the start, and after the slot's previous row was consumed), so its byte count never goes negative.
// Arithmetic: GB300's FP64 rate is a small fraction of its FP32 rate, so no FP64 operation is on the
// per-row path.  A CTA's partial is an FP32 sum (per thread, per warp, then a 16-lane tree over the warps:
// one chunk sum, as in k_sr_tpart); the sum over the cluster's C partials is double-float (an FP32 pair
// hi + lo combined by Knuth's TwoSum, about 48 significant bits, in the role of k_sr_tred's FP64 sum) in a
// fixed xor-butterfly tree, so every CTA of a cluster gets the same bits of t_s.  Runs of kRun rows of
// FP32 products per parameter are added into the cluster's double-float partial row wpart[cluster][P]
// (L2-resident; each element has one owner thread, the first run writes instead of adding); k_sr_wfin_dd
// sums the partial rows in FP64.  Every wait is bounded: on a timeout the CTA flags *err and goes on, so
// that every CTA of the cluster still reaches each exchange and the final cluster barrier.
constexpr int kFusedThreads = 512;
constexpr int kFusedGroups = 8;   // 4-element groups per thread
constexpr int kFusedRing = 4, kFusedLook = 2, kFusedSlots = 2 * kFusedLook + 2;
constexpr int kFusedMaxSlice = 4 * kFusedGroups * kFusedThreads;
constexpr int kFusedMaxClusters = 3 * kSampleGroups;   // partial rows kept in the moments' buffer

struct FusedLayout {
  int slots, wsum, tbuf, bars, bytes;   // byte offsets in dynamic shared memory (ring at 0) and the total
};
__host__ __device__ inline FusedLayout fused_layout(int SL, int C) {
  FusedLayout L;
  L.slots = kFusedRing * SL * 4;   // SL is a multiple of 4: every buffer starts on a 16-byte boundary
  L.wsum = L.slots + kFusedSlots * C * 16;
  L.tbuf = L.wsum + 2 * (kFusedThreads / 32) * 8;   // per-warp partials, double-buffered by row parity
  L.bars = L.tbuf + 2 * 8;                          // t of the row, double-buffered by row parity
  L.bytes = L.bars + (kFusedRing + kFusedSlots) * 8;
  return L;
}

// Double-float value hi + lo (|lo| <= ulp(hi) / 2 after renormalisation).
struct DF {
  float hi, lo;
};
// (a + b) exactly as s + e (Knuth's TwoSum, symmetric in a and b)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  DF r;
  r.hi = s + e;
  r.lo = e - (r.hi - s);
  return r;
}
// Sum over lanes 0-15 of a warp (the only lanes that call it) by an xor butterfly: each ends with the same
// bits.
__device__ __forceinline__ DF df_half_sum(DF v) {
#pragma unroll
  for (int o = 8; o; o >>= 1) {
    DF w;
    w.hi = __shfl_xor_sync(0x0000ffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0x0000ffffu, v.lo, o);
    v = df_add(v, w);
  }
  return v;
}

__device__ __forceinline__ uint32_t cl_special(int which) {
  uint32_t r;
  if (which == 0) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  else if (which == 1) asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  else if (which == 2) asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  else asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// The shared::cluster address of local shared address a in the CTA of rank r.
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t r) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(r));
  return d;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// 16 bytes into a peer's shared memory (cluster address a), counted on the peer's mbarrier (cluster
// address bar) as completed transaction bytes.
__device__ __forceinline__ void cl_put_async(uint32_t a, float4 v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(a),
               "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
               : "memory");
}
// Bounded wait on a local mbarrier that peers of the cluster complete (acquire at cluster scope).
__device__ __forceinline__ bool cl_wait(uint32_t a, uint32_t parity) {
  for (long long i = 0; i < tc::kSpinLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}
__global__ void __launch_bounds__(kFusedThreads, 1)
    k_sr_fused(const uint32_t *__restrict__ O, size_t Ns, size_t P, size_t ldo, int SL, const float *__restrict__ vf,
               float2 *__restrict__ t, float2 *__restrict__ wpart, const double *__restrict__ sc, int *err) {
  extern __shared__ __align__(16) uint8_t sm[];
  if (sc[S_DONE] != 0.0) return;   // the same value for every CTA: all of them leave here together
  const int C = (int)cl_special(1), q = (int)cl_special(0);
  const size_t g = cl_special(2), G = cl_special(3);
  const FusedLayout L = fused_layout(SL, C);
  const uint32_t base = tc::smem_u32(sm);
  const uint32_t full = base + L.bars, recv = full + 8 * kFusedRing, slots = base + L.slots;
  const float4 *slot = reinterpret_cast<const float4 *>(sm + L.slots);
  float2 *wsum = reinterpret_cast<float2 *>(sm + L.wsum);
  float2 *tbuf = reinterpret_cast<float2 *>(sm + L.tbuf);
  const size_t per = (Ns + G - 1) / G;
  const size_t s0 = g * per < Ns ? g * per : Ns;
  const int nr = (int)((s0 + per < Ns ? s0 + per : Ns) - s0);
  const size_t k0 = (size_t)q * SL;
  const int kn = k0 < P ? (int)(P - k0 < (size_t)SL ? P - k0 : (size_t)SL) : 0;
  const int ngr = (kn + 3) / 4;
  const uint32_t bytes = 16u * (uint32_t)ngr;   // inside the row: ldo and k0 are multiples of 4
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  DF ncr, nci;   // -(mean . v) as double-float pairs: the kernel's only FP64 arithmetic
  {
    const double cr = sc[S_CR], ci = sc[S_CI];
    ncr.hi = (float)(-cr);
    ncr.lo = (float)(-cr - (double)ncr.hi);
    nci.hi = (float)(-ci);
    nci.lo = (float)(-ci - (double)nci.hi);
  }
  float4 vr[kFusedGroups], f[kFusedGroups];
#pragma unroll
  for (int i = 0; i < kFusedGroups; ++i) {
    const int k = 4 * (tid + kFusedThreads * i);
    float x[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) x[e] = k + e < kn ? vf[k0 + k + e] : 0.f;
    vr[i] = make_float4(x[0], x[1], x[2], x[3]);
    f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (tid == 0) {
    for (int b = 0; b < kFusedRing; ++b) tc::mbar_init(full + 8 * b, 1);
    for (int b = 0; b < kFusedSlots; ++b) tc::mbar_init(recv + 8 * b, 1);
    for (int b = 0; b < kFusedSlots; ++b) tc::mbar_expect_tx(recv + 8 * b, 16u * (uint32_t)(C - 1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cl_sync();   // every CTA's barriers exist and are armed before a peer stores into its slots
  auto issue = [&](int r) {   // thread 0: row r's slice into buffer r % kFusedRing
    const uint32_t bar = full + 8 * (r % kFusedRing);
    tc::mbar_expect_tx(bar, bytes);
    tc::bulk_g2s(base + (uint32_t)((r % kFusedRing) * SL * 4), O + (s0 + r) * ldo + k0, bytes, bar);
  };
  if (tid == 0 && ngr > 0)
    for (int r = 0; r < kFusedRing && r < nr; ++r) issue(r);
  bool ok = true;
  // the four elements of group gi from a row buffer (zero past the slice: padding columns are never data)
  auto elems = [&](const uint4 &u, int gi, float2 (&c)[4]) {
    c[0] = cplx(u.x); c[1] = cplx(u.y); c[2] = cplx(u.z); c[3] = cplx(u.w);
    if (4 * gi + 4 > kn)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (4 * gi + e >= kn) c[e] = make_float2(0.f, 0.f);
  };
  // row r: this CTA's partial of O_s . v to every CTA of the cluster
  auto send = [&](int r) {
    float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};   // independent chains per element slot
    if (ngr > 0) {
      ok = tc::mbar_wait(full + 8 * (r % kFusedRing), (uint32_t)((r / kFusedRing) & 1)) && ok;
      const uint4 *buf = reinterpret_cast<const uint4 *>(sm + (size_t)(r % kFusedRing) * SL * 4);
#pragma unroll
      for (int i = 0; i < kFusedGroups; ++i) {
        const int gi = tid + kFusedThreads * i;
        if (gi < ngr) {
          float2 c[4];
          elems(buf[gi], gi, c);
          const float vv[4] = {vr[i].x, vr[i].y, vr[i].z, vr[i].w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            ar[e] = fmaf(c[e].x, vv[e], ar[e]);
            ai[e] = fmaf(c[e].y, vv[e], ai[e]);
          }
        }
      }
    }
    float pr = (ar[0] + ar[1]) + (ar[2] + ar[3]), pi = (ai[0] + ai[1]) + (ai[2] + ai[3]);
    pr = warp_sum(pr);
    pi = warp_sum(pi);
    float2 *ws = wsum + (r & 1) * (kFusedThreads / 32);
    if (lane == 0) ws[warp] = make_float2(pr, pi);
    __syncthreads();
    if (warp == 0 && lane < 16) {   // the CTA's partial: FP32 tree over the 16 warps (as one chunk sum)
      float a = ws[lane].x, b = ws[lane].y;
#pragma unroll
      for (int o = 8; o; o >>= 1) {
        a += __shfl_xor_sync(0x0000ffffu, a, o);
        b += __shfl_xor_sync(0x0000ffffu, b, o);
      }
      if (lane < C) {   // lane p: the partial into slot q of CTA p
        const int sl = r % kFusedSlots;
        const float4 msg = make_float4(a, 0.f, b, 0.f);
        if (lane == q)   // read by warp 1 after the block barriers between this send and the row's turn
          *reinterpret_cast<float4 *>(sm + L.slots + (sl * C + q) * 16) = msg;
        else
          cl_put_async(cl_map(slots + (uint32_t)((sl * C + q) * 16), (uint32_t)lane), msg,
                       cl_map(recv + 8 * sl, (uint32_t)lane));
      }
    }
  };
  // warp 1 (lanes 0-15), row r: t_s from the C partials, centred, to tbuf[r & 1] (and to t by the
  // cluster's CTA 0)
  auto form_t = [&](int r) {
    const int sl = r % kFusedSlots;
    ok = cl_wait(recv + 8 * sl, (uint32_t)((r / kFusedSlots) & 1)) && ok;
    DF a = {0.f, 0.f}, b = {0.f, 0.f};
    if (lane < C) {
      const float4 m = slot[sl * C + lane];
      a.hi = m.x; a.lo = m.y; b.hi = m.z; b.lo = m.w;
    }
    a = df_add(df_half_sum(a), ncr);
    b = df_add(df_half_sum(b), nci);
    if (lane == 0) {
      const float2 tv = make_float2(a.hi + a.lo, b.hi + b.lo);
      tbuf[r & 1] = tv;
      if (q == 0) t[s0 + r] = tv;
    }
  };
  for (int r = 0; r < kFusedLook && r < nr; ++r) send(r);
  __syncthreads();   // own-slot stores of the first rows before warp 1 reads them
  bool first = true;
  for (int r = 0; r < nr; ++r) {
    if (warp == 1 && lane < 16) form_t(r);
    if (r + kFusedLook < nr) send(r + kFusedLook);   // its block barrier also publishes tbuf[r & 1]
    else __syncthreads();
    const float2 tv = tbuf[r & 1];
    if (ngr > 0) {
      const uint4 *buf = reinterpret_cast<const uint4 *>(sm + (size_t)(r % kFusedRing) * SL * 4);
#pragma unroll
      for (int i = 0; i < kFusedGroups; ++i) {
        const int gi = tid + kFusedThreads * i;
        if (gi < ngr) {
          float2 c[4];
          elems(buf[gi], gi, c);
          f[i].x = fmaf(c[0].x, tv.x, fmaf(c[0].y, tv.y, f[i].x));
          f[i].y = fmaf(c[1].x, tv.x, fmaf(c[1].y, tv.y, f[i].y));
          f[i].z = fmaf(c[2].x, tv.x, fmaf(c[2].y, tv.y, f[i].z));
          f[i].w = fmaf(c[3].x, tv.x, fmaf(c[3].y, tv.y, f[i].w));
        }
      }
    }
    if ((r + 1) % kRun == 0 || r + 1 == nr) {   // the run into the cluster's double-float partial row
#pragma unroll
      for (int i = 0; i < kFusedGroups; ++i) {
        const int k = 4 * (tid + kFusedThreads * i);
        const float fe[4] = {f[i].x, f[i].y, f[i].z, f[i].w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (k + e < kn) {
            float2 *w = wpart + g * P + k0 + k + e;
            DF acc = {0.f, 0.f};
            if (!first) { const float2 o = *w; acc.hi = o.x; acc.lo = o.y; }
            acc = df_add(acc, DF{fe[e], 0.f});
            *w = make_float2(acc.hi, acc.lo);
          }
        f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      first = false;
    }
    __syncthreads();   // buffer r % kFusedRing, slot r % kFusedSlots and tbuf are done with
    if (tid == 0) {
      tc::mbar_expect_tx(recv + 8 * (r % kFusedSlots), 16u * (uint32_t)(C - 1));   // for row r + kFusedSlots
      if (ngr > 0 && r + kFusedRing < nr) {
        tc::fence_proxy_async();
        issue(r + kFusedRing);
      }
    }
  }
  if (nr == 0)
    for (int k = tid; k < kn; k += kFusedThreads) wpart[g * P + k0 + k] = make_float2(0.f, 0.f);
  const bool bad = __syncthreads_or(ok ? 0 : 1) != 0;
  if (bad && tid == 0 && ngr > 0)   // copies still in flight after a timeout: wait for them (bounded)
    for (int r = nr - kFusedRing > 0 ? nr - kFusedRing : 0; r < nr; ++r)
      tc::mbar_wait(full + 8 * (r % kFusedRing), (uint32_t)((r / kFusedRing) & 1));
  cl_sync();   // no CTA leaves while a peer may still store into its slots
  if (bad && tid == 0 && err) atomicExch(err, 1);
}

// Ap[k] = (1/Ns) [sum_g (hi + lo)(wpart[g][k]) - Re(conj(mean[k]) T)] + shift p[k] over ng double-float
// partial rows (FP64 sums); partials of p . p.
__global__ void k_sr_wfin_dd(size_t Ns, size_t P, const double2 *__restrict__ mean, const float2 *__restrict__ wpart,
                             int ng, const double *__restrict__ p, double shift, double *__restrict__ Ap,
                             double *__restrict__ part, const double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  const double Tr = sc[S_TR], Ti = sc[S_TI];
  double loc = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    double a = 0.0;
    for (int g = 0; g < ng; ++g) {
      const float2 w = wpart[(size_t)g * P + k];
      a += (double)w.x + (double)w.y;
    }
    const double2 m = mean[k];
    const double v = (a - (m.x * Tr + m.y * Ti)) / (double)Ns + shift * p[k];
    Ap[k] = v;
    loc += p[k] * p[k];
  }
  const double b = block_sum_d(loc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// ---------------------------------------------------------------- one-pass product over the whole grid
// S' v with O read from HBM once, without clusters.  G co-resident CTAs (one per SM) each own the
// parameter slab [q SL, q SL + SL) of every row; rows go in blocks of kGR.  Warp roles in a CTA:
//   - warp 0 (lane 0): bulk-copies the slab of every row of a block from HBM into the t ring (ns1
//     shared-memory stages), for the partials of t;
//   - warp 1 (lane 0): bulk-copies the same slab again, kGLook blocks later, into the w ring (ns2
//     stages).  Between the two reads the GPU streams about kGLook blocks (8 x 6.3 MB at the headline
//     shape), far less than the 129 MB L2, so the second copy is served from L2 (evict-first hint: the
//     line is not needed again) and DRAM sees O once;
//   - the compute warps (4 parameters per thread and group): at step b they form their partials of
//     t_s = O_s . v for the rows of block b from the t ring and leave them in shared memory, then add
//     Re(conj(O_sk) t_s) for the rows of block b - kGLook from the w ring;
//   - warp 2 ("publisher"): sums the compute warps' partials of block b and stores this CTA's 16 values
//     (re, im of 8 rows) to the block's exchange slot in global memory, each as one 64-bit word with the
//     block's tag in its high half, so a reader that sees the tag sees the value (no fence, no counter);
//   - warps 3 .. 2 + kGExch ("exchange"): block b belongs to one of them in turn.  Once its own CTA has
//     published kGAhead blocks further (an mbarrier: the warp sleeps, it does not spin), it reads the G
//     CTAs' words of block b, again after a pause until every tag is there, sums them in a fixed order (every CTA gets the same bits of t_s), centres them as k_sr_tred
//     does and hands t of the block to the compute warps through a shared-memory ring.
// So the exchange of a block has kGLook steps of streaming to complete before its t is needed, and the
// compute warps never wait on global memory.  At the headline shape shared memory holds three HBM
// stages and two L2 stages of 42 KB.  The exchange slots are cleared before the launch (tag 0;
// tags are b + 1) and reused every kGPB blocks: a CTA publishes block b' only after its own w-part of
// block b' - 1 - kGLook, which needed every CTA's words of that block, which each CTA published only
// after its w-part of b' - 2 - 2 kGLook, i.e. after it had read every block up to there; kGPB >= 2 kGLook
// + 2 keeps a slot from being overwritten while a CTA may still read it.
// Arithmetic: FP32 products and sums up to the CTA partial (per thread, a 32-lane tree, then the
// compute warps in order), an FP32 sum over the G partials (G / 32 per lane, then a 32-lane tree), the
// centring in FP64; w in FP32 runs of kRun rows accumulated in FP64 per parameter.
// Every wait is bounded and watches the device error flag: a wait that gives up sets it, and every other
// wait of every CTA then returns at once, so the launch ends (its results invalid) instead of hanging.
constexpr int kGR = 8;               // sample rows per block
constexpr int kGV = 2 * kGR;         // exchanged values per block: re, im of each row
constexpr int kGLook = 8, kGExch = 6;   // blocks between a block's t-part and its w-part; exchange warps
constexpr int kGAhead = 2;           // blocks this CTA has published beyond the one an exchange warp reads
constexpr int kGPB = 32;             // exchange slots (G x kGV tagged words each)
constexpr int kGTB = 16;             // t slots in shared memory
constexpr int kGRB = 4;              // slots of the compute warps' partials in shared memory
constexpr int kGMaxStages = 6;       // stages of either ring at most
constexpr int kGMaxCompute = 16;     // compute warps at most (800 threads in all)
constexpr int kGRoles = 3 + kGExch;  // copiers, publisher, exchange warps
constexpr unsigned long long kGridWaitNs = 1000000000ull;   // a wait gives up after 1 s
static_assert(kGPB >= 2 * kGLook + 2 && kGTB >= kGLook + kGExch && kRun % kGR == 0, "grid product rings");

struct GridLayout {
  int stage, wring, tb, red, bars, bytes;   // bytes of one stage; byte offsets of the w ring, the t slots,
                                            // the warp partials and the mbarriers; total
};
__host__ __device__ inline GridLayout grid_layout(int ngr, int ns1, int ns2, int nw) {
  GridLayout L;
  L.stage = kGR * 16 * ngr;   // kGR slab rows of 16 ngr bytes (every row on a 16-byte boundary)
  L.wring = ns1 * L.stage;
  L.tb = L.wring + ns2 * L.stage;
  L.red = L.tb + kGTB * kGR * 8;
  L.bars = L.red + kGRB * nw * kGV * 4;
  L.bytes = L.bars + (2 * ns1 + 2 * ns2 + 3 * kGTB + 2 * kGRB) * 8;
  return L;
}

__device__ __forceinline__ bool grid_aborted(const int *err) { return *reinterpret_cast<const volatile int *>(err) != 0; }
__device__ __forceinline__ void mbar_arrive1(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on a local mbarrier phase: false at once when the error flag is up (abort = true), and
// false with the flag raised after `limit` ns.
__device__ __forceinline__ bool grid_wait(uint32_t bar, uint32_t parity, int *err,
                                          unsigned long long limit = kGridWaitNs, bool abort = true) {
  if (tc::mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer_ns();
  for (unsigned i = 1;; ++i) {
    if (tc::mbar_try(bar, parity)) return true;
    if ((i & 31) == 0) {
      if (abort && grid_aborted(err)) return false;
      if (gtimer_ns() - t0 > limit) {
        atomicExch(err, 1);
        return false;
      }
      __nanosleep(64);
    }
  }
}
// Sum over the 32 lanes of each of NV values (NV = 2, 4, ..., 32) by recursive halving (NV - 1 + 5 -
// log2 NV shuffles): afterwards lane l holds the warp's sum of value l / (32 / NV), the same bits in all
// 32 / NV lanes that hold it.
template <int NV>
__device__ __forceinline__ float xreduce(float (&a)[NV], int lane) {
#pragma unroll
  for (int h = NV / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float send = up ? a[j] : a[j + h];
      const float keep = up ? a[j + h] : a[j];
      a[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float x = a[0];
#pragma unroll
  for (int o = 16 / NV; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
// The four elements of group gi (columns 4 gi .. 4 gi + 3 of the slab), zero at and past kn: padding
// columns are never data.
__device__ __forceinline__ void grid_elems(const uint4 &u, int gi, int kn, float2 (&c)[4]) {
  c[0] = cplx(u.x); c[1] = cplx(u.y); c[2] = cplx(u.z); c[3] = cplx(u.w);
  if (4 * gi + 4 > kn)
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (4 * gi + e >= kn) c[e] = make_float2(0.f, 0.f);
}

// One row's slab into shared memory with an L2 evict-first policy (a copy whose lines are not read again).
__device__ __forceinline__ void bulk_g2s_evict_first(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar,
                                                     uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(pol)
      : "memory");
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ ulonglong2 ld_relaxed_u64x2(const unsigned long long *p) {
  ulonglong2 v;
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
  return v;
}

// w[k] = sum_s Re(conj(O[s][k]) t_s) for k < P and t (the centred O v, written by CTA 0).  xw:
// [kGPB][G][kGV] tagged exchange words, all zero at the launch.
template <int GPT>
__global__ void __launch_bounds__(32 * (kGRoles + kGMaxCompute), 1)
    k_sr_grid(const uint32_t *__restrict__ O, size_t Ns, size_t P, size_t ldo, int SL, int ns1, int ns2,
              const float *__restrict__ vf, float2 *__restrict__ t, double *__restrict__ w,
              unsigned long long *__restrict__ xw, const double *__restrict__ sc, int *err) {
  extern __shared__ __align__(16) uint8_t sm[];
  if (sc[S_DONE] != 0.0) return;   // the same value for every CTA: all of them leave here together
  const int G = (int)gridDim.x, q = (int)blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = (int)(blockDim.x >> 5) - kGRoles;
  const int ngr_max = SL / 4;
  const GridLayout L = grid_layout(ngr_max, ns1, ns2, nw);
  const size_t k0 = (size_t)q * SL;
  const int kn = k0 < P ? (int)(P - k0 < (size_t)SL ? P - k0 : (size_t)SL) : 0;
  const int ngr = (kn + 3) / 4;
  const int nb = (int)((Ns + kGR - 1) / kGR);
  const uint32_t base = tc::smem_u32(sm);
  // mbarriers: t ring full / empty, w ring full / empty, t slots full / empty, partial slots full / empty,
  // block b published (slot b % kGTB)
  const uint32_t tf = base + L.bars, te = tf + 8 * ns1, wf = te + 8 * ns1, we = wf + 8 * ns2, xf = we + 8 * ns2,
                 xe = xf + 8 * kGTB, pf = xe + 8 * kGTB, pe = pf + 8 * kGRB, pb = pe + 8 * kGRB;
  float2 *tb = reinterpret_cast<float2 *>(sm + L.tb);
  float *red = reinterpret_cast<float *>(sm + L.red);
  if (tid == 0) {
    for (int i = 0; i < ns1; ++i) { tc::mbar_init(tf + 8 * i, 1); tc::mbar_init(te + 8 * i, (uint32_t)nw); }
    for (int i = 0; i < ns2; ++i) { tc::mbar_init(wf + 8 * i, 1); tc::mbar_init(we + 8 * i, (uint32_t)nw); }
    for (int i = 0; i < kGTB; ++i) { tc::mbar_init(xf + 8 * i, 1); tc::mbar_init(xe + 8 * i, (uint32_t)nw); }
    for (int i = 0; i < kGRB; ++i) { tc::mbar_init(pf + 8 * i, (uint32_t)nw); tc::mbar_init(pe + 8 * i, 1); }
    for (int i = 0; i < kGTB; ++i) tc::mbar_init(pb + 8 * i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto rows_of = [&](int b) {
    const size_t r0 = (size_t)b * kGR;
    return (int)(Ns - r0 < (size_t)kGR ? Ns - r0 : (size_t)kGR);
  };
  if (warp <= 1) {
    if (lane == 0) {   // a copier: warp 0 fills the t ring, warp 1 the w ring
      const int ns = warp == 0 ? ns1 : ns2;
      const uint32_t full = warp == 0 ? tf : wf, empty = warp == 0 ? te : we;
      const uint32_t ring = base + (uint32_t)(warp == 0 ? 0 : L.wring);
      uint64_t pol = 0;
      if (warp == 1) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
      int fills[kGMaxStages];
      for (int i = 0; i < kGMaxStages; ++i) fills[i] = 0;
      const uint32_t rb = 16u * (uint32_t)ngr;   // bytes of one row's slab (inside the row: ldo, k0 multiples of 4)
      for (int b = 0; b < nb; ++b) {
        const int st = b % ns, m = b / ns;
        if (m > 0) {   // the stage's previous block is done with; stop issuing once anything gave up
          if (!grid_wait(empty + 8 * st, (uint32_t)((m - 1) & 1), err) || grid_aborted(err)) break;
          tc::fence_proxy_async();
        }
        const int nr = rows_of(b);
        tc::mbar_expect_tx(full + 8 * st, rb * (uint32_t)nr);
        if (ngr > 0)
          for (int r = 0; r < nr; ++r) {
            const uint32_t dst = ring + (uint32_t)(st * L.stage + r * 16 * ngr_max);
            const uint32_t *src = O + ((size_t)b * kGR + r) * ldo + k0;
            if (warp == 0) tc::bulk_g2s(dst, src, rb, full + 8 * st);
            else bulk_g2s_evict_first(dst, src, rb, full + 8 * st, pol);
          }
        fills[st] = m + 1;
      }
      for (int st = 0; st < ns && st < kGMaxStages; ++st)   // no copy is still landing when the CTA exits
        if (fills[st] > 0) grid_wait(full + 8 * st, (uint32_t)((fills[st] - 1) & 1), err, kGridWaitNs / 2, false);
    }
    __syncwarp();
  } else if (warp == 2) {   // the publisher
    for (int b = 0; b < nb; ++b) {
      const int rs = b % kGRB;
      grid_wait(pf + 8 * rs, (uint32_t)((b / kGRB) & 1), err);
      if (lane < kGV) {
        const float *rb = red + rs * nw * kGV;
        float x = 0.f;
        for (int u = 0; u < nw; ++u) x += rb[u * kGV + lane];
        st_relaxed_u64(xw + ((size_t)(b % kGPB) * G + q) * kGV + lane,
                       (unsigned long long)__float_as_uint(x) | ((unsigned long long)(unsigned)(b + 1) << 32));
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive1(pe + 8 * rs);
        mbar_arrive1(pb + 8 * (b % kGTB));
      }
    }
  } else if (warp < kGRoles) {   // an exchange warp
    const double cr = sc[S_CR], ci = sc[S_CI];
    for (int b = warp - 3; b < nb; b += kGExch) {
      const int j = b % kGTB, m = b / kGTB, slot = b % kGPB;
      if (m > 0) grid_wait(xe + 8 * j, (uint32_t)((m - 1) & 1), err);
      // this CTA has published block c (the other CTAs are about as far): the words of b are likely in
      const int c = b + kGAhead < nb ? b + kGAhead : nb - 1;
      grid_wait(pb + 8 * (c % kGTB), (uint32_t)((c / kGTB) & 1), err);
      const unsigned tag = (unsigned)(b + 1);
      const unsigned long long *src = xw + (size_t)slot * G * kGV;
      float a[kGV];
      const unsigned long long t0 = gtimer_ns();
      for (unsigned it = 0;; ++it) {   // every word of the block, in a fixed order, until all tags are in
        bool ready = true;
#pragma unroll
        for (int x = 0; x < kGV; ++x) a[x] = 0.f;
        for (int g = lane; g < G; g += 32) {
#pragma unroll
          for (int u = 0; u < kGV / 2; ++u) {
            const ulonglong2 x = ld_relaxed_u64x2(src + (size_t)g * kGV + 2 * u);
            ready = ready && (unsigned)(x.x >> 32) == tag && (unsigned)(x.y >> 32) == tag;
            a[2 * u] += __uint_as_float((unsigned)x.x);
            a[2 * u + 1] += __uint_as_float((unsigned)x.y);
          }
        }
        if (__all_sync(0xffffffffu, ready)) break;
        if (__any_sync(0xffffffffu, grid_aborted(err))) break;
        if (__shfl_sync(0xffffffffu, gtimer_ns() - t0 > kGridWaitNs ? 1 : 0, 0)) {
          if (lane == 0) atomicExch(err, 1);
          break;
        }
        __nanosleep(256);
      }
      const float s = xreduce<kGV>(a, lane);
      constexpr int span = 32 / kGV;   // lanes holding each value
      const int idx = lane / span, r = idx >> 1, nr = rows_of(b);
      if (lane % span == 0) {
        const float tv = r < nr ? (float)((double)s - ((idx & 1) ? ci : cr)) : 0.f;
        reinterpret_cast<float *>(tb + j * kGR)[idx] = tv;
        if (q == 0 && r < nr) reinterpret_cast<float *>(t + (size_t)b * kGR + r)[idx & 1] = tv;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive1(xf + 8 * j);
    }
  } else {   // a compute warp
    const int ct = tid - 32 * kGRoles, cw = ct >> 5, nct = 32 * nw;
    float v[GPT][4], f[GPT][4];
    double wacc[GPT][4];
#pragma unroll
    for (int i = 0; i < GPT; ++i) {
      const int gi = ct + nct * i;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int kk = 4 * gi + e;
        v[i][e] = (gi < ngr && kk < kn) ? vf[k0 + kk] : 0.f;
        f[i][e] = 0.f;
        wacc[i][e] = 0.0;
      }
    }
    for (int b = 0; b < nb + kGLook; ++b) {
      if (b < nb) {   // this warp's partials of t for block b, from the t ring, to the publisher
        const int st = b % ns1, nr = rows_of(b);
        grid_wait(tf + 8 * st, (uint32_t)((b / ns1) & 1), err);
        const uint4 *buf = reinterpret_cast<const uint4 *>(sm + (size_t)st * L.stage);
        float a[kGV];
#pragma unroll
        for (int x = 0; x < kGV; ++x) a[x] = 0.f;
#pragma unroll
        for (int i = 0; i < GPT; ++i) {
          const int gi = ct + nct * i;
          if (gi < ngr) {
#pragma unroll
            for (int r = 0; r < kGR; ++r)
              if (r < nr) {
                float2 c[4];
                grid_elems(buf[r * ngr_max + gi], gi, kn, c);
                a[2 * r] = fmaf(c[0].x, v[i][0], fmaf(c[1].x, v[i][1], fmaf(c[2].x, v[i][2], fmaf(c[3].x, v[i][3], a[2 * r]))));
                a[2 * r + 1] =
                    fmaf(c[0].y, v[i][0], fmaf(c[1].y, v[i][1], fmaf(c[2].y, v[i][2], fmaf(c[3].y, v[i][3], a[2 * r + 1]))));
              }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive1(te + 8 * st);   // this warp is done with the stage
        const float s = xreduce<kGV>(a, lane);
        const int rs = b % kGRB;
        if (b >= kGRB) grid_wait(pe + 8 * rs, (uint32_t)((b / kGRB - 1) & 1), err);
        if (lane % (32 / kGV) == 0) red[(rs * nw + cw) * kGV + lane / (32 / kGV)] = s;
        __syncwarp();
        if (lane == 0) mbar_arrive1(pf + 8 * rs);
      }
      const int bw = b - kGLook;
      if (bw >= 0) {   // w over block bw, from the w ring
        const int st = bw % ns2, j = bw % kGTB, nr = rows_of(bw);
        grid_wait(xf + 8 * j, (uint32_t)((bw / kGTB) & 1), err);
        grid_wait(wf + 8 * st, (uint32_t)((bw / ns2) & 1), err);
        const uint4 *buf = reinterpret_cast<const uint4 *>(sm + (size_t)L.wring + (size_t)st * L.stage);
#pragma unroll
        for (int r = 0; r < kGR; ++r)
          if (r < nr) {
            const float2 tv = tb[j * kGR + r];
#pragma unroll
            for (int i = 0; i < GPT; ++i) {
              const int gi = ct + nct * i;
              if (gi < ngr) {
                float2 c[4];
                grid_elems(buf[r * ngr_max + gi], gi, kn, c);
#pragma unroll
                for (int e = 0; e < 4; ++e) f[i][e] = fmaf(c[e].x, tv.x, fmaf(c[e].y, tv.y, f[i][e]));
              }
            }
          }
        if ((bw + 1) % (kRun / kGR) == 0 || bw + 1 == nb)
#pragma unroll
          for (int i = 0; i < GPT; ++i)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              wacc[i][e] += (double)f[i][e];
              f[i][e] = 0.f;
            }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive1(we + 8 * st);
          mbar_arrive1(xe + 8 * j);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < GPT; ++i) {
      const int gi = ct + nct * i;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (gi < ngr && 4 * gi + e < kn) w[k0 + 4 * gi + e] = wacc[i][e];
    }
  }
  __syncthreads();
}

// alpha = r.z / p.S'p with p.S'p = (1/Ns) sum_s |t_s - tbar|^2 + shift p.p (the partials hold p.p)
__global__ void k_sr_alpha(const double *__restrict__ part, int nb, size_t Ns, double shift, double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  const double pp = sum_parts(part, nb, sh);
  if (threadIdx.x == 0) {
    const double n = (double)Ns, Tr = sc[S_TR], Ti = sc[S_TI];
    const double var = sc[S_TT] - (Tr * Tr + Ti * Ti) / n;   // sum_s |t_s - tbar|^2
    const double pap = (var > 0.0 ? var : 0.0) / n + shift * pp;
    sc[S_PAP] = pap;
    if (!isfinite(pap) || !isfinite(sc[S_RZ])) {
      sc[S_AL] = 0.0;
      sc[S_DONE] = SR_NONFINITE;
    } else if (!(pap > 0.0)) {
      sc[S_AL] = 0.0;
      sc[S_DONE] = SR_BREAKDOWN;
    } else {
      sc[S_AL] = sc[S_RZ] / pap;
    }
  }
}

// x += alpha p; r -= alpha Ap; z = r / diag; partials of r.r (part) and r.z (part2)
__global__ void k_sr_xr(size_t P, double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
                        const double *__restrict__ p, const double *__restrict__ Ap,
                        const double *__restrict__ diag, double *__restrict__ part,
                        double *__restrict__ part2, const double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  const double al = sc[S_AL];
  double rr = 0.0, rz = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    x[k] += al * p[k];
    const double rk = r[k] - al * Ap[k];
    r[k] = rk;
    const double zk = rk / diag[k];
    z[k] = zk;
    rr += rk * rk;
    rz += rk * zk;
  }
  const double a = block_sum_d(rr, sh);
  const double b = block_sum_d(rz, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = a; part2[blockIdx.x] = b; }
}

__global__ void k_sr_beta(const double *__restrict__ part, const double *__restrict__ part2, int nb,
                          double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  const double rr = sum_parts(part, nb, sh);
  const double rz = sum_parts(part2, nb, sh);
  if (threadIdx.x == 0) {
    sc[S_IT] += 1.0;
    sc[S_RN] = rr;
    sc[S_AL] = (sc[S_RZ] != 0.0) ? rz / sc[S_RZ] : 0.0;   // beta (alpha slot reused)
    sc[S_RZ] = rz;
    if (!isfinite(rr) || !isfinite(rz)) sc[S_DONE] = SR_NONFINITE;
    else if (rr <= sc[S_TOL] * sc[S_BN]) sc[S_DONE] = SR_CONVERGED;
  }
}

__global__ void k_sr_p(size_t P, double *__restrict__ p, const double *__restrict__ z, const double *__restrict__ sc) {
  if (sc[S_DONE] != 0.0) return;
  const double be = sc[S_AL];
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x)
    p[k] = z[k] + be * p[k];
}

// Initial state.  Without x0: x = 0, r = rhs.  With x0 (Ap holds S' x0): x = x0, r = rhs - Ap.
// Then z = r/diag, p = z; partials of r.r, r.z and rhs.rhs.
__global__ void k_sr_init(size_t P, const double *__restrict__ rhs, const double *__restrict__ x0,
                          const double *__restrict__ Ap, double *__restrict__ x, double *__restrict__ r,
                          double *__restrict__ z, double *__restrict__ p, const double *__restrict__ diag,
                          double *__restrict__ part, double *__restrict__ part2, double *__restrict__ part3,
                          const double *gate) {
  __shared__ double sh[32];
  if (gate && gate[S_RESTART] != 1.0) return;   // graph mode: only a pending restart runs it
  double rr = 0.0, rz = 0.0, bb = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    const double b = rhs[k];
    const double rk = x0 ? b - Ap[k] : b;
    x[k] = x0 ? x0[k] : 0.0;
    r[k] = rk;
    const double zk = rk / diag[k];
    z[k] = zk;
    p[k] = zk;
    rr += rk * rk;
    rz += rk * zk;
    bb += b * b;
  }
  const double a = block_sum_d(rr, sh);
  const double b2 = block_sum_d(rz, sh);
  const double c = block_sum_d(bb, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = a; part2[blockIdx.x] = b2; part3[blockIdx.x] = c; }
}

__global__ void k_sr_init_scalars(const double *__restrict__ part, const double *__restrict__ part2,
                                  const double *__restrict__ part3, int nb, double tol, double *__restrict__ sc,
                                  int gated) {
  __shared__ double sh[32];
  if (gated && sc[S_RESTART] != 1.0) return;
  const double rr = sum_parts(part, nb, sh);
  const double rz = sum_parts(part2, nb, sh);
  const double bb = sum_parts(part3, nb, sh);
  if (threadIdx.x == 0) {
    sc[S_RZ] = rz;
    sc[S_BN] = bb;
    sc[S_RN] = rr;
    sc[S_AL] = 0.0;
    sc[S_IT] = 0.0;
    sc[S_TOL] = tol * tol;
    sc[S_PAP] = 0.0;
    if (!isfinite(rr) || !isfinite(rz) || !isfinite(bb)) sc[S_DONE] = SR_NONFINITE;
    else sc[S_DONE] = (rr <= tol * tol * bb) ? SR_CONVERGED : 0.0;
    if (gated) sc[S_RESTART] = 2.0;
  }
}

// Last kernel of a CG iteration in graph mode: another iteration while the solve is neither done nor at
// max_iter.  A breakdown or a non-finite value with a warm start (*warm != 0) and no restart yet marks a
// restart from x = 0 as pending and asks for one more pass, whose first kernels re-initialise.
__global__ void k_sr_cond(cudaGraphConditionalHandle h, double *__restrict__ sc, int max_iter, const int *warm) {
  if (threadIdx.x != 0) return;
  const double done = sc[S_DONE];
  bool more = done == 0.0 && sc[S_IT] < (double)max_iter;
  if ((done == SR_BREAKDOWN || done == SR_NONFINITE) && *warm && sc[S_RESTART] == 0.0) {
    sc[S_RESTART] = 1.0;
    more = true;
  }
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void k_sr_clear(double *__restrict__ sc) {
  if (threadIdx.x < S_COUNT) sc[threadIdx.x] = 0.0;
}


struct SrPtrs {
  double2 *mean;
  double *diag, *r, *z, *p, *Ap, *part, *part2, *part3, *sc;
  float *vf;
  float2 *t;
  double2 *tpart;
  double *wpart;
  double *mpart;   // [3][kSampleGroups][P] group sums of the moments pass
};

// Carves the workspace; every region starts on a 16-byte boundary (double2 / float2 / float4 access).
static SrPtrs sr_carve(double *work, size_t Ns, size_t P) {
  char *b = reinterpret_cast<char *>(work);
  size_t off = 0;
  auto take = [&](size_t bytes) { char *p = b + off; off += (bytes + 15) / 16 * 16; return p; };
  SrPtrs q;
  q.mean = reinterpret_cast<double2 *>(take(16 * P));
  q.diag = reinterpret_cast<double *>(take(8 * P));
  q.r = reinterpret_cast<double *>(take(8 * P));
  q.z = reinterpret_cast<double *>(take(8 * P));
  q.p = reinterpret_cast<double *>(take(8 * P));
  q.Ap = reinterpret_cast<double *>(take(8 * P));
  q.part = reinterpret_cast<double *>(take(8 * 1024));
  q.part2 = reinterpret_cast<double *>(take(8 * 1024));
  q.part3 = reinterpret_cast<double *>(take(8 * 1024));
  q.sc = reinterpret_cast<double *>(take(8 * 32));
  q.vf = reinterpret_cast<float *>(take(4 * P));
  q.t = reinterpret_cast<float2 *>(take(8 * Ns));
  q.tpart = reinterpret_cast<double2 *>(take(16 * ((P + kChunk - 1) / kChunk) * Ns));
  q.wpart = reinterpret_cast<double *>(take(8 * kSampleGroups * P));
  q.mpart = reinterpret_cast<double *>(take(3 * 8 * kSampleGroups * P));
  return q;
}

// S' v -> Ap (and the partials of v . Ap in q.part), all on the device: 7 launches, O streamed twice.
template <typename OT>
static void matvec(const OT *O, size_t Ns, size_t P, size_t ldo, const double *v, double shift, SrPtrs &q,
                   int nb, cudaStream_t st) {
  constexpr int CH = SrChunk<OT>::value, TB = CH / 4;
  const int nchunks = (int)((P + CH - 1) / CH);
  constexpr size_t align = 16 / sizeof(OT);   // elements per 16 bytes
  k_sr_vprep<<<nb, kSrBlock, 0, st>>>(P, v, q.mean, q.vf, q.part, q.part2, q.sc);
  k_sr_cfin<<<1, 1024, 0, st>>>(q.part, q.part2, nb, q.sc);
  const bool vec = ldo % align == 0 && reinterpret_cast<uintptr_t>(O) % 16 == 0;   // 16-byte-aligned rows
  if (vec)
    k_sr_tpart<OT, true><<<dim3(nchunks, kSampleGroups), TB, 0, st>>>(O, Ns, P, ldo, q.vf, q.tpart, q.sc);
  else
    k_sr_tpart<OT, false><<<dim3(nchunks, kSampleGroups), TB, 0, st>>>(O, Ns, P, ldo, q.vf, q.tpart, q.sc);
  k_sr_tred<<<(unsigned)((Ns + 255) / 256), 256, 0, st>>>(q.tpart, nchunks, Ns, q.t, q.sc);
  k_sr_tsum<<<1, 1024, 0, st>>>(q.t, Ns, q.sc);
  if (vec)
    k_sr_wpart<OT, true><<<dim3(nchunks, kSampleGroups), TB, 0, st>>>(O, Ns, P, ldo, q.t, q.wpart, q.sc);
  else
    k_sr_wpart<OT, false><<<dim3(nchunks, kSampleGroups), TB, 0, st>>>(O, Ns, P, ldo, q.t, q.wpart, q.sc);
  k_sr_wfin<<<nb, kSrBlock, 0, st>>>(Ns, P, q.mean, q.wpart, kSampleGroups, v, shift, q.Ap, q.part, q.sc);
}

// The one-pass product's shape for this O: the smallest cluster (so the most clusters) whose three row
// slices fit in shared memory, and as many clusters as the device runs at once (at most
// kFusedMaxClusters).  C = 0: not available (FP32 storage, unaligned rows, no cluster launch).
struct FusedPlan {
  int C = 0, G = 0, SL = 0, bytes = 0;
};
static FusedPlan fused_plan(const void *O, size_t Ns, size_t P, size_t ldo) {
  FusedPlan pl;
  if (ldo % 4 != 0 || reinterpret_cast<uintptr_t>(O) % 16 != 0 || Ns == 0) return pl;
  int dev = 0, smax = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return pl;
  for (int C = 1; C <= 16; C *= 2) {
    const size_t sl = ((P + C - 1) / C + 3) / 4 * 4;
    if (sl > (size_t)kFusedMaxSlice) continue;
    const FusedLayout L = fused_layout((int)sl, C);
    if (L.bytes > smax) continue;
    if (cudaFuncSetAttribute(k_sr_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, L.bytes) != cudaSuccess ||
        (C > 8 && cudaFuncSetAttribute(k_sr_fused, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess))
      break;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = L.bytes;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int G = 0;
    if (cudaOccupancyMaxActiveClusters(&G, k_sr_fused, &cfg) != cudaSuccess || G <= 0) break;
    if (G > kFusedMaxClusters) G = kFusedMaxClusters;
    if ((size_t)G > Ns) G = (int)Ns;
    pl.C = C;
    pl.G = G;
    pl.SL = (int)sl;
    pl.bytes = L.bytes;
    break;
  }
  cudaGetLastError();   // a refused attribute or query leaves the two-pass product in use
  return pl;
}

// S' v -> Ap by the one-pass product: 5 launches, O streamed once.
static cudaError_t matvec_fused(const uint32_t *O, size_t Ns, size_t P, size_t ldo, const double *v, double shift,
                                SrPtrs &q, int nb, const FusedPlan &pl, int *err, cudaStream_t st) {
  k_sr_vprep<<<nb, kSrBlock, 0, st>>>(P, v, q.mean, q.vf, q.part, q.part2, q.sc);
  k_sr_cfin<<<1, 1024, 0, st>>>(q.part, q.part2, nb, q.sc);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = pl.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(pl.C * pl.G);
  cfg.blockDim = dim3(kFusedThreads);
  cfg.dynamicSmemBytes = pl.bytes;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  float2 *wp = reinterpret_cast<float2 *>(q.mpart);   // G double-float rows of P in the moments' buffer
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_sr_fused, O, Ns, P, ldo, pl.SL, (const float *)q.vf, q.t, wp,
                                           (const double *)q.sc, err);
  if (e != cudaSuccess) return e;
  k_sr_tsum<<<1, 1024, 0, st>>>(q.t, Ns, q.sc);
  k_sr_wfin_dd<<<nb, kSrBlock, 0, st>>>(Ns, P, q.mean, wp, pl.G, v, shift, q.Ap, q.part, q.sc);
  return cudaSuccess;
}


// The grid product's shape for this O: G CTAs (one per SM, fewer when P is small), slab SL, compute
// warps, stages.  G = 0: not available (unaligned rows, no error flag, a slab too wide, or no room).
struct GridPlan {
  int G = 0, SL = 0, gpt = 0, threads = 0, ns1 = 0, ns2 = 0, bytes = 0;
};
static GridPlan grid_plan(const void *O, size_t Ns, size_t P, size_t ldo, const int *err) {
  GridPlan pl;
  if (!err || ldo % 4 != 0 || reinterpret_cast<uintptr_t>(O) % 16 != 0 || Ns == 0 || P == 0) return pl;
  int dev = 0, smax = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return pl;
  }
  size_t G = (P + 255) / 256;
  if (G > (size_t)nsm) G = (size_t)nsm;
  if (G < 1) G = 1;
  const size_t SL = ((P + G - 1) / G + 3) / 4 * 4;
  const size_t ngr = SL / 4;
  const int gpt = ngr <= 32u * kGMaxCompute ? 1 : (ngr <= 64u * kGMaxCompute ? 2 : 0);
  if (gpt == 0) return pl;
  const int nw = (int)((ngr + 32 * gpt - 1) / (32 * gpt));
  // t ring: the block being read and at least one landing; w ring: the same
  static const int shapes[][2] = {{6, 4}, {5, 4}, {5, 3}, {4, 3}, {3, 2}, {2, 2}};
  int ns1 = 0, ns2 = 0;
  for (const auto &sh : shapes)
    if (grid_layout((int)ngr, sh[0], sh[1], nw).bytes <= smax) {
      ns1 = sh[0];
      ns2 = sh[1];
      break;
    }
  if (ns1 == 0) return pl;
  // the exchange words live in the moments' buffer (3 kSampleGroups P doubles), free during the solve
  if (sizeof(unsigned long long) * kGPB * G * kGV > 8 * 3 * (size_t)kSampleGroups * P) return pl;
  const int bytes = grid_layout((int)ngr, ns1, ns2, nw).bytes, threads = 32 * (kGRoles + nw);
  const void *fn = gpt == 1 ? (const void *)k_sr_grid<1> : (const void *)k_sr_grid<2>;
  int occ = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, bytes) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return pl;
  }
  pl.G = (int)G;
  pl.SL = (int)SL;
  pl.gpt = gpt;
  pl.threads = threads;
  pl.ns1 = ns1;
  pl.ns2 = ns2;
  pl.bytes = bytes;
  return pl;
}

// S' v -> Ap by the grid product: 5 launches, O streamed once.
static cudaError_t matvec_grid(const uint32_t *O, size_t Ns, size_t P, size_t ldo, const double *v, double shift,
                               SrPtrs &q, int nb, const GridPlan &pl, int *err, cudaStream_t st) {
  unsigned long long *xw = reinterpret_cast<unsigned long long *>(q.mpart);
  const size_t nx = (size_t)kGPB * pl.G * kGV;
  // also clears the exchange words (tag 0) for the grid kernel
  k_sr_vprep<<<nb, kSrBlock, 0, st>>>(P, v, q.mean, q.vf, q.part, q.part2, q.sc, reinterpret_cast<uint4 *>(xw),
                                      nx / 2);
  k_sr_cfin<<<1, 1024, 0, st>>>(q.part, q.part2, nb, q.sc);
  if (pl.gpt == 1)
    k_sr_grid<1><<<pl.G, pl.threads, pl.bytes, st>>>(O, Ns, P, ldo, pl.SL, pl.ns1, pl.ns2, q.vf, q.t, q.wpart, xw, q.sc, err);
  else
    k_sr_grid<2><<<pl.G, pl.threads, pl.bytes, st>>>(O, Ns, P, ldo, pl.SL, pl.ns1, pl.ns2, q.vf, q.t, q.wpart, xw, q.sc, err);
  k_sr_tsum<<<1, 1024, 0, st>>>(q.t, Ns, q.sc);
  k_sr_wfin<<<nb, kSrBlock, 0, st>>>(Ns, P, q.mean, q.wpart, 1, v, shift, q.Ap, q.part, q.sc);
  return cudaGetLastError();
}

}  // namespace tdo

size_t sr_work_doubles(size_t Ns, size_t P) {
  // the regions carved by sr_carve, each rounded up to 16 bytes, plus slack
  const size_t nchunks = (P + tdo::kChunk - 1) / tdo::kChunk;
  const size_t bytes = 16 * P + 5 * (8 * P + 16) + 3 * 8 * 1024 + 8 * 32 + (4 * P + 16) + (8 * Ns + 16) +
                       16 * nchunks * Ns + 16 + 8 * tdo::kSampleGroups * P + 16 + 3 * 8 * tdo::kSampleGroups * P + 16 +
                       64;
  return (bytes + 7) / 8;
}

namespace tdo {
// mean and Jacobi diagonal of O (one pass over O)
template <typename OT>
static void moments(const OT *O2, size_t Ns, size_t P, size_t ldo, double shift, SrPtrs &q, int nb, cudaStream_t st) {
  constexpr int CH = SrChunk<OT>::value;
  const int nchunks = (int)((P + CH - 1) / CH);
  const bool vec = ldo % (16 / sizeof(OT)) == 0 && reinterpret_cast<uintptr_t>(O2) % 16 == 0;
  if (vec)
    k_sr_mpart<OT, true><<<dim3(nchunks, kSampleGroups), CH / 4, 0, st>>>(O2, Ns, P, ldo, q.mpart);
  else
    k_sr_mpart<OT, false><<<dim3(nchunks, kSampleGroups), CH / 4, 0, st>>>(O2, Ns, P, ldo, q.mpart);
  k_sr_mfin<<<nb, kSrBlock, 0, st>>>(Ns, P, shift, q.mpart, q.mean, q.diag);
}

static int sr_blocks(size_t P) {
  int nb = (int)((P + kSrBlock - 1) / kSrBlock);
  return nb > 1024 ? 1024 : (nb < 1 ? 1 : nb);
}

// One product (Re S + shift I) v -> Ap outside the CG loop (BF16-pair storage).
static cudaError_t sr_apply_t(const uint32_t *O2, size_t Ns, size_t P, size_t ldo, const double *v, double shift,
                              double *Ap, double *work, int product_mode, int *err, int *shape, cudaStream_t st) {
  SrPtrs q = sr_carve(work, Ns, P);
  const int nb = sr_blocks(P);
  FusedPlan pl;
  GridPlan gp;
  if (product_mode == 1) pl = fused_plan(O2, Ns, P, ldo);
  if (product_mode == 2) gp = grid_plan(O2, Ns, P, ldo, err);
  if (shape) {
    shape[0] = gp.G > 0 ? 2 : (pl.C > 0 ? 1 : 0);
    shape[1] = gp.G > 0 ? 1 : pl.C;
    shape[2] = gp.G > 0 ? gp.G : pl.G;
  }
  moments(O2, Ns, P, ldo, shift, q, nb, st);
  k_sr_clear<<<1, 32, 0, st>>>(q.sc);
  if (gp.G > 0) {
    const cudaError_t e = matvec_grid(O2, Ns, P, ldo, v, shift, q, nb, gp, err, st);
    if (e != cudaSuccess) return e;
  } else if (pl.C > 0) {
    const cudaError_t e = matvec_fused(O2, Ns, P, ldo, v, shift, q, nb, pl, err, st);
    if (e != cudaSuccess) return e;
  } else {
    matvec(O2, Ns, P, ldo, v, shift, q, nb, st);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(Ap, q.Ap, sizeof(double) * P, cudaMemcpyDeviceToDevice, st);
}

template <typename OT>
static cudaError_t sr_cg_t(const OT *O2, size_t Ns, size_t P, size_t ldo, const double *rhs, const double *x0,
                           double shift,
                           double tol, int max_iter, double *x, double *work, int *iters, double *resid,
                           int *outcome, double *last_pap,
                           long long *launches, cudaEvent_t *mv_ev, int mv_cap, int *mv_used, int product_mode,
                           int *err, int *shape, cudaStream_t st) {
  SrPtrs q = sr_carve(work, Ns, P);
  FusedPlan pl;
  GridPlan gp;
  if constexpr (sizeof(OT) == 4) {
    if (product_mode == 1) pl = fused_plan(O2, Ns, P, ldo);
    if (product_mode == 2) gp = grid_plan(O2, Ns, P, ldo, err);
  }
  if (shape) {
    shape[0] = gp.G > 0 ? 2 : (pl.C > 0 ? 1 : 0);
    shape[1] = gp.G > 0 ? 1 : pl.C;
    shape[2] = gp.G > 0 ? gp.G : pl.G;
  }
  const int nb = sr_blocks(P);
  long long nl = 0;
  int nmv = 0;
  if (mv_used) *mv_used = 0;
  auto mv = [&](const double *v) -> cudaError_t {
    const bool rec = mv_ev && nmv < mv_cap;
    if (rec) cudaEventRecord(mv_ev[2 * nmv], st);
    if constexpr (sizeof(OT) == 4) {
      if (gp.G > 0) {
        const cudaError_t e = matvec_grid(O2, Ns, P, ldo, v, shift, q, nb, gp, err, st);
        if (e != cudaSuccess) return e;
        nl += 5;
      } else if (pl.C > 0) {
        const cudaError_t e = matvec_fused(O2, Ns, P, ldo, v, shift, q, nb, pl, err, st);
        if (e != cudaSuccess) return e;
        nl += 5;
      } else {
        matvec(O2, Ns, P, ldo, v, shift, q, nb, st);
        nl += 7;
      }
    } else {
      matvec(O2, Ns, P, ldo, v, shift, q, nb, st);
      nl += 7;
    }
    if (rec) {
      cudaEventRecord(mv_ev[2 * nmv + 1], st);
      ++nmv;
      if (mv_used) *mv_used = nmv;
    }
    return cudaSuccess;
  };
  moments(O2, Ns, P, ldo, shift, q, nb, st);
  k_sr_clear<<<1, 32, 0, st>>>(q.sc);
  nl += 3;
  cudaError_t e;
  if (x0 && (e = mv(x0)) != cudaSuccess) return e;
  k_sr_init<<<nb, kSrBlock, 0, st>>>(P, rhs, x0, q.Ap, x, q.r, q.z, q.p, q.diag, q.part, q.part2, q.part3, nullptr);
  k_sr_init_scalars<<<1, 1024, 0, st>>>(q.part, q.part2, q.part3, nb, tol, q.sc, 0);
  nl += 2;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // Iterations are launched in groups; the done flag on the device makes the rest of a group a no-op,
  // and the host looks at it between groups only.
  const int group = 8;
  double h[S_COUNT];
  bool fetched = false;
  for (int it = 0; it < max_iter;) {
    const int end = it + group < max_iter ? it + group : max_iter;
    for (; it < end; ++it) {
      if ((e = mv(q.p)) != cudaSuccess) return e;
      k_sr_alpha<<<1, 1024, 0, st>>>(q.part, nb, Ns, shift, q.sc);
      k_sr_xr<<<nb, kSrBlock, 0, st>>>(P, x, q.r, q.z, q.p, q.Ap, q.diag, q.part, q.part2, q.sc);
      k_sr_beta<<<1, 1024, 0, st>>>(q.part, q.part2, nb, q.sc);
      k_sr_p<<<nb, kSrBlock, 0, st>>>(P, q.p, q.z, q.sc);
      nl += 4;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(h, q.sc, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    fetched = true;
    if (h[S_DONE] != 0.0) break;
  }
  if (!fetched) {
    e = cudaMemcpyAsync(h, q.sc, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
  }
  if (iters) *iters = (int)h[S_IT];
  if (mv_used) {   // launches after convergence returned at once: keep the pairs of real products only
    const int real = (x0 ? 1 : 0) + (int)h[S_IT] + (h[S_DONE] == (double)SR_CONVERGED ? 0 : 1);
    if (*mv_used > real) *mv_used = real;
  }
  if (resid) *resid = h[S_BN] > 0 ? sqrt(h[S_RN] / h[S_BN]) : 0.0;
  if (launches) *launches = nl;
  if (outcome) *outcome = (int)h[S_DONE];
  if (last_pap) *last_pap = h[S_PAP];
  return cudaSuccess;
}

// Records a while loop into the graph being captured on st: a conditional node (its condition 1 at every
// launch of the graph when `initial`, else 0), whose body `body(stream, handle)` records on a stream of its
// own; the capture on st then continues after the node.
template <typename F>
static cudaError_t capture_while(cudaStream_t st, unsigned initial, F &&body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureUnmatched;
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, initial, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np)) != cudaSuccess) return e;
  cudaStream_t side;
  if ((e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking)) != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(side, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    const cudaError_t eb = body(side, h);
    cudaGraph_t out;
    e = cudaStreamEndCapture(side, &out);
    if (eb != cudaSuccess) e = eb;
  }
  cudaStreamDestroy(side);
  if (e != cudaSuccess) return e;
  return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// The CG solve recorded into the graph being captured on st.  The same launches as sr_cg_t with a warm
// start from x (zero when there is no previous solution), the iterations in a while node: each pass runs
// the restart kernels (no-ops unless a restart from x = 0 is pending), one iteration, and k_sr_cond.
// *warm (device int) allows the restart, as a warm start does in sr_cg_t's caller.
template <typename OT>
static cudaError_t sr_cg_capture_t(const OT *O2, size_t Ns, size_t P, size_t ldo, const double *rhs, double *x,
                                   double shift, double tol, int max_iter, double *work, int product_mode,
                                   const int *warm, int *err, int *shape, cudaStream_t st) {
  SrPtrs q = sr_carve(work, Ns, P);
  FusedPlan pl;
  GridPlan gp;
  if constexpr (sizeof(OT) == 4) {
    if (product_mode == 1) pl = fused_plan(O2, Ns, P, ldo);
    if (product_mode == 2) gp = grid_plan(O2, Ns, P, ldo, err);
  }
  if (shape) {
    shape[0] = gp.G > 0 ? 2 : (pl.C > 0 ? 1 : 0);
    shape[1] = gp.G > 0 ? 1 : pl.C;
    shape[2] = gp.G > 0 ? gp.G : pl.G;
  }
  const int nb = sr_blocks(P);
  auto mv = [&](const double *v, cudaStream_t s) -> cudaError_t {
    if constexpr (sizeof(OT) == 4) {
      if (gp.G > 0) return matvec_grid(O2, Ns, P, ldo, v, shift, q, nb, gp, err, s);
      if (pl.C > 0) return matvec_fused(O2, Ns, P, ldo, v, shift, q, nb, pl, err, s);
    }
    matvec(O2, Ns, P, ldo, v, shift, q, nb, s);
    return cudaSuccess;
  };
  moments(O2, Ns, P, ldo, shift, q, nb, st);
  k_sr_clear<<<1, 32, 0, st>>>(q.sc);
  cudaError_t e;
  if ((e = mv(x, st)) != cudaSuccess) return e;
  k_sr_init<<<nb, kSrBlock, 0, st>>>(P, rhs, x, q.Ap, x, q.r, q.z, q.p, q.diag, q.part, q.part2, q.part3, nullptr);
  k_sr_init_scalars<<<1, 1024, 0, st>>>(q.part, q.part2, q.part3, nb, tol, q.sc, 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return capture_while(st, max_iter > 0 ? 1u : 0u, [&](cudaStream_t s, cudaGraphConditionalHandle h) -> cudaError_t {
    k_sr_init<<<nb, kSrBlock, 0, s>>>(P, rhs, nullptr, q.Ap, x, q.r, q.z, q.p, q.diag, q.part, q.part2, q.part3, q.sc);
    k_sr_init_scalars<<<1, 1024, 0, s>>>(q.part, q.part2, q.part3, nb, tol, q.sc, 1);
    cudaError_t ei = mv(q.p, s);
    if (ei != cudaSuccess) return ei;
    k_sr_alpha<<<1, 1024, 0, s>>>(q.part, nb, Ns, shift, q.sc);
    k_sr_xr<<<nb, kSrBlock, 0, s>>>(P, x, q.r, q.z, q.p, q.Ap, q.diag, q.part, q.part2, q.sc);
    k_sr_beta<<<1, 1024, 0, s>>>(q.part, q.part2, nb, q.sc);
    k_sr_p<<<nb, kSrBlock, 0, s>>>(P, q.p, q.z, q.sc);
    k_sr_cond<<<1, 32, 0, s>>>(h, q.sc, max_iter, warm);
    return cudaGetLastError();
  });
}
}  // namespace tdo

// mv_ev (optional): mv_cap event pairs recorded around the S' v launches; *mv_used = pairs recorded.
// o_bf16: O holds BF16 pairs (uint32 per element) instead of FP32 (re, im); ldo >= P: elements per row.
// *outcome: 0 stopped at max_iter, 1 converged, 2 breakdown (p . S'p not positive), 3 a non-finite value;
// *last_pap: the last p . S'p.  product_mode 0: two passes; 1: the one-pass product on clusters, 2: the
// one-pass product over the whole grid, each where O's storage and shape allow it (BF16 pairs; the grid
// product also needs err), else two passes.  err (device int, may be NULL): set when a bounded wait of a
// one-pass product gave up.  shape (may be NULL): {product used (0, 1, 2), cluster size (1 for the grid
// product), clusters or CTAs}.  The return value reports CUDA errors only.
cudaError_t sr_cg_impl(const void *O, int o_bf16, size_t Ns, size_t P, size_t ldo, const double *rhs, const double *x0,
                       double shift, double tol, int max_iter, double *x, double *work, int n_sm, int *iters,
                       double *resid, int *outcome, double *last_pap, long long *launches, cudaEvent_t *mv_ev,
                       int mv_cap, int *mv_used, int product_mode, int *err, int *shape, cudaStream_t st) {
  (void)n_sm;
  if (o_bf16)
    return tdo::sr_cg_t(reinterpret_cast<const uint32_t *>(O), Ns, P, ldo, rhs, x0, shift, tol, max_iter, x, work, iters,
                        resid, outcome, last_pap, launches, mv_ev, mv_cap, mv_used, product_mode, err, shape, st);
  return tdo::sr_cg_t(reinterpret_cast<const float2 *>(O), Ns, P, ldo, rhs, x0, shift, tol, max_iter, x, work, iters,
                      resid, outcome, last_pap, launches, mv_ev, mv_cap, mv_used, product_mode, err, shape, st);
}

// Graph mode: the solve of sr_cg_impl recorded into the graph being captured on st (see sr_cg_capture_t);
// warm start from x, restart from x = 0 after a breakdown or a non-finite value when *warm.  The result
// is read after a launch of the graph by sr_cg_result.
cudaError_t sr_cg_capture(const void *O, int o_bf16, size_t Ns, size_t P, size_t ldo, const double *rhs, double *x,
                          double shift, double tol, int max_iter, double *work, int product_mode, const int *warm,
                          int *err, int *shape, cudaStream_t st) {
  if (o_bf16)
    return tdo::sr_cg_capture_t(reinterpret_cast<const uint32_t *>(O), Ns, P, ldo, rhs, x, shift, tol, max_iter, work,
                                product_mode, warm, err, shape, st);
  return tdo::sr_cg_capture_t(reinterpret_cast<const float2 *>(O), Ns, P, ldo, rhs, x, shift, tol, max_iter, work,
                              product_mode, warm, err, shape, st);
}

// The outcome of the last solve on work, as sr_cg_impl reports it, and whether it was restarted
// (synchronises st).
cudaError_t sr_cg_result(double *work, size_t Ns, size_t P, int *iters, double *resid, int *outcome,
                         double *last_pap, int *restarted, cudaStream_t st) {
  tdo::SrPtrs q = tdo::sr_carve(work, Ns, P);
  double h[tdo::S_COUNT];
  cudaError_t e = cudaMemcpyAsync(h, q.sc, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (iters) *iters = (int)h[tdo::S_IT];
  if (resid) *resid = h[tdo::S_BN] > 0 ? sqrt(h[tdo::S_RN] / h[tdo::S_BN]) : 0.0;
  if (outcome) *outcome = (int)h[tdo::S_DONE];
  if (last_pap) *last_pap = h[tdo::S_PAP];
  if (restarted) *restarted = h[tdo::S_RESTART] == 2.0 ? 1 : 0;
  return cudaSuccess;
}

// Device address of the solve's outcome slot on work (0 max_iter, 1 converged, 2 breakdown, 3 non-finite).
const double *sr_outcome_slot(double *work, size_t Ns, size_t P) {
  return tdo::sr_carve(work, Ns, P).sc + tdo::S_DONE;
}

// One product (Re S + shift I) v with O as BF16 pairs [Ns][ldo] (ldo >= P), v and Ap FP64 [P] on the device.
cudaError_t sr_apply_impl(const uint32_t *O, size_t Ns, size_t P, size_t ldo, const double *v, double shift, double *Ap,
                          double *work, int product_mode, int *err, int *shape, cudaStream_t st) {
  return tdo::sr_apply_t(O, Ns, P, ldo, v, shift, Ap, work, product_mode, err, shape, st);
}
