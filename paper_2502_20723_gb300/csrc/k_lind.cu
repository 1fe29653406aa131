// Rows of the vectorised Lindbladian (Eq. VecLin), the local estimator L_loc and the cost (Eq. lossnetk),
// the gradient cotangents, and the FP64 reductions.  All ALU / latency bound and small next to the
// transformer; FP64 is used for the coefficient sums and every reduction over samples.
#include "tdo_device.cuh"

namespace tdo {

// One warp per sample; lanes take the connection patterns in groups of 32 and compact the nonzero ones
// (pattern 0, the diagonal, is always kept) with a ballot, preserving the pattern order.
__global__ void k_connections(const ConnPattern *__restrict__ pat, int n_pat,
                              const ConnContrib *__restrict__ con, const uint32_t *__restrict__ sig,
                              const uint32_t *__restrict__ sigp, size_t Ns, int32_t *__restrict__ count,
                              uint32_t *__restrict__ csig, uint32_t *__restrict__ csigp,
                              float2 *__restrict__ ccoef) {
  const int lane = threadIdx.x & 31;
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = (gridDim.x * (size_t)blockDim.x) >> 5;
  for (size_t smp = warp; smp < Ns; smp += nwarps) {
    const uint32_t s = sig[smp], p = sigp[smp];
    int pos = 0;
    for (int base = 0; base < n_pat; base += 32) {
      const int q = base + lane;
      double vr = 0.0, vi = 0.0;
      bool keep = false;
      uint32_t ys = 0, yp = 0;
      if (q < n_pat) {
        const ConnPattern P = pat[q];
        for (int c = P.c_begin; c < P.c_end; ++c) {
          const ConnContrib &C = con[c];
          const int a = C.sel_l >= 0 ? (int)((s >> C.sel_l) & 1u) : 0;
          const int b = C.sel_r >= 0 ? (int)((p >> C.sel_r) & 1u) : 0;
          const double sgn = ((__popc(s & C.m1) + __popc(p & C.m2)) & 1) ? -1.0 : 1.0;
          vr += sgn * C.tab[2 * a + b][0];
          vi += sgn * C.tab[2 * a + b][1];
        }
        keep = (q == 0) || vr != 0.0 || vi != 0.0;
        ys = s ^ P.lmask;
        yp = p ^ P.rmask;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const size_t at = smp * (size_t)n_pat + pos + __popc(mask & ((1u << lane) - 1u));
        csig[at] = ys;
        csigp[at] = yp;
        ccoef[at] = make_float2((float)vr, (float)vi);
      }
      pos += __popc(mask);
    }
    if (lane == 0) count[smp] = pos;
  }
}

// Exclusive scan of the counts (one block, fixed order: deterministic).
__global__ void k_scan(const int32_t *__restrict__ count, size_t Ns, int64_t *__restrict__ offs) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const size_t per = (Ns + blockDim.x - 1) / blockDim.x;
  const size_t a = t * per, b = (a + per < Ns) ? a + per : Ns;
  int64_t loc = 0;
  for (size_t i = a; i < b; ++i) loc += count[i];
  part[t] = loc;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) { const int64_t v = part[i]; part[i] = run; run += v; }
    offs[Ns] = run;
  }
  __syncthreads();
  int64_t run = part[t];
  for (size_t i = a; i < b; ++i) { offs[i] = run; run += count[i]; }
}

__global__ void k_compact(const int32_t *__restrict__ count, const int64_t *__restrict__ offs, size_t Ns,
                          int M, const uint32_t *__restrict__ csig, const uint32_t *__restrict__ csigp,
                          const float2 *__restrict__ ccoef, uint32_t *__restrict__ fsig,
                          uint32_t *__restrict__ fsigp, float2 *__restrict__ fcoef) {
  const size_t total = Ns * (size_t)M;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += gridDim.x * (size_t)blockDim.x) {
    const size_t s = i / M;
    const int j = (int)(i % M);
    if (j < count[s]) {
      const size_t o = offs[s] + j;
      fsig[o] = csig[i];
      fsigp[o] = csigp[i];
      fcoef[o] = ccoef[i];
    }
  }
}

// rho_y / rho_x from the two log values: exp of the log-ratio in FP32.
__device__ __forceinline__ float2 ratio_f32(float2 ly, float2 lx) {
  const float e = expf(ly.x - lx.x);
  float sn, cs;
  sincosf(ly.y - lx.y, &sn, &cs);
  return make_float2(e * cs, e * sn);
}

// L_loc(x) = sum_j coef_j rho(y_j)/rho(x): warp per sample, FP32 terms summed in FP64.
__global__ void k_lloc(const int64_t *__restrict__ offs, size_t Ns, const float2 *__restrict__ fcoef,
                       const float2 *__restrict__ flr, double2 *__restrict__ lloc,
                       double *__restrict__ l2, int *nonfinite) {
  const int lane = threadIdx.x & 31;
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = (gridDim.x * (size_t)blockDim.x) >> 5;
  for (size_t s = warp; s < Ns; s += nwarps) {
    const int64_t o = offs[s], cnt = offs[s + 1] - o;
    const float2 lx = flr[o];
    double ar = 0.0, ai = 0.0;
    for (int64_t j = lane; j < cnt; j += 32) {
      const float2 r = ratio_f32(flr[o + j], lx);
      const float2 c = fcoef[o + j];
      ar += (double)(c.x * r.x - c.y * r.y);
      ai += (double)(c.x * r.y + c.y * r.x);
    }
    ar = warp_sum_d(ar);
    ai = warp_sum_d(ai);
    if (lane == 0) {
      lloc[s] = make_double2(ar, ai);
      const double a2 = ar * ar + ai * ai;
      l2[s] = a2;
      if (!isfinite(a2) || !isfinite(lx.x) || !isfinite(lx.y)) atomicOr(nonfinite, 1);
    }
  }
}

// Deterministic single-block sums of l2[] and l2[]^2 -> stats[0], stats[1].
__global__ void k_cost_stats(const double *__restrict__ l2, size_t Ns, double *__restrict__ stats) {
  __shared__ double s1[1024], s2[1024];
  double a = 0.0, b = 0.0;
  for (size_t i = threadIdx.x; i < Ns; i += blockDim.x) { a += l2[i]; b += l2[i] * l2[i]; }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) { s1[threadIdx.x] += s1[threadIdx.x + w]; s2[threadIdx.x] += s2[threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { stats[0] = s1[0]; stats[1] = s2[0]; }
}

// Cotangent per row: (2/Ns) conj(L_loc(x)) coef rho_y/rho_x, and -(2/Ns) Cost on the diagonal row.
__global__ void k_cotangent(const int64_t *__restrict__ offs, size_t Ns, const float2 *__restrict__ fcoef,
                            const float2 *__restrict__ flr, const double2 *__restrict__ lloc,
                            const double *__restrict__ stats, float2 *__restrict__ cot) {
  const int lane = threadIdx.x & 31;
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = (gridDim.x * (size_t)blockDim.x) >> 5;
  const double scale = 2.0 / (double)Ns;
  const double cost = stats[0] / (double)Ns;
  for (size_t s = warp; s < Ns; s += nwarps) {
    const int64_t o = offs[s], cnt = offs[s + 1] - o;
    const float2 lx = flr[o];
    const double2 L = lloc[s];
    for (int64_t j = lane; j < cnt; j += 32) {
      const float2 r = ratio_f32(flr[o + j], lx);
      const float2 c = fcoef[o + j];
      const double tr = (double)(c.x * r.x - c.y * r.y), ti = (double)(c.x * r.y + c.y * r.x);
      // conj(L) * t
      double vr = L.x * tr + L.y * ti, vi = L.x * ti - L.y * tr;
      if (j == 0) vr -= cost;
      cot[o + j] = make_float2((float)(scale * vr), (float)(scale * vi));
    }
  }
}

__global__ void k_reduce_copies(const float *__restrict__ acc, int n_copies, size_t stride, size_t P,
                                double *__restrict__ out, int accumulate, const float *__restrict__ scale) {
  const double f = scale ? (double)*scale : 1.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    double a = 0.0;
    for (int c = 0; c < n_copies; ++c) a += (double)acc[(size_t)c * stride + k];
    out[k] = (accumulate ? out[k] : 0.0) + f * a;
  }
}

__global__ void k_f64_to_f32(const double *__restrict__ src, float *__restrict__ dst, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += gridDim.x * (size_t)blockDim.x)
    dst[k] = (float)src[k];
}

// Conv embedding as a table over the 64 patterns of (sigma, sigma') bits at sites i, i+1, i+2: two
// kernel-2 circular convolutions, each followed by GELU (Eq. circ-conv and the next equation).
// Spins enter as +-1 (bit 0 -> +1).  Thread per (pattern, output channel).
__global__ void k_conv_table(int d, int c1, const float *__restrict__ Wc1, const float *__restrict__ bc1,
                             const float *__restrict__ Wc2, const float *__restrict__ bc2,
                             float *__restrict__ table) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 64 * d) return;
  const int pat = idx / d, e = idx % d;
  float x[3][2];
  for (int o = 0; o < 3; ++o) {
    x[o][0] = 1.0f - 2.0f * (float)((pat >> o) & 1);
    x[o][1] = 1.0f - 2.0f * (float)((pat >> (3 + o)) & 1);
  }
  float acc = bc2[e];
  for (int o2 = 0; o2 < 2; ++o2)        // second conv reads first-conv outputs at sites i, i+1
    for (int f = 0; f < c1; ++f) {
      float h = bc1[f];
      for (int o1 = 0; o1 < 2; ++o1)
        for (int ch = 0; ch < 2; ++ch) h = fmaf(Wc1[(o1 * 2 + ch) * c1 + f], x[o2 + o1][ch], h);
      acc = fmaf(Wc2[(o2 * c1 + f) * d + e], gelu_f(h), acc);
    }
  table[idx] = gelu_f(acc);
}

// FP64 flat parameters -> FP32 copy whose tensors start on 16-float boundaries (tab: flat, pad, size).
__global__ void k_params_f32(const double *__restrict__ theta, size_t P, const long long *__restrict__ tab,
                             int n_tensors, float *__restrict__ dst) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    int t = 0;
    while (t + 1 < n_tensors && (long long)k >= tab[3 * (t + 1)]) ++t;
    dst[tab[3 * t + 1] + ((long long)k - tab[3 * t])] = (float)theta[k];
  }
}

__global__ void k_axpy(double *__restrict__ theta, const double *__restrict__ delta, double lr, size_t P,
                       const int *__restrict__ gate) {
  if (gate && !*gate) return;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x)
    theta[k] -= lr * delta[k];
}

// Adam (Kingma and Ba, Algorithm 1) on the SR direction delta, the optimiser's "gradient": with t the
// step count after this step, m = b1 m + (1 - b1) delta, v = b2 v + (1 - b2) delta^2,
// theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  FP64 throughout.
__global__ void k_adam(double *__restrict__ theta, const double *__restrict__ delta, double *__restrict__ m,
                       double *__restrict__ v, size_t P, double lr, double b1, double b2, double eps, double c1,
                       double c2, const int *__restrict__ gate, const double *__restrict__ dc) {
  if (gate && !*gate) return;
  if (dc) { c1 = dc[0]; c2 = dc[1]; }
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    const double d = delta[k];
    const double mk = b1 * m[k] + (1.0 - b1) * d;
    const double vk = b2 * v[k] + (1.0 - b2) * d * d;
    m[k] = mk;
    v[k] = vk;
    theta[k] -= lr * (mk / c1) / (sqrt(vk / c2) + eps);
  }
}

// Whether a replayed step may update the parameters: the CG solve ended without a breakdown or a non-finite
// value (outcome 0 or 1), L_loc was finite and no bounded wait gave up -- the conditions under which the
// step, run call by call, reaches its update.
__global__ void k_step_gate(const double *__restrict__ outcome, const int *__restrict__ nonfinite,
                            const int *__restrict__ err, int *__restrict__ ok) {
  const double o = *outcome;
  *ok = (o == 0.0 || o == 1.0) && *nonfinite == 0 && (err == nullptr || *err == 0);
}

// Ragged batches: counts of each chain length (shared-memory histogram per block, then global atomics).
__global__ void k_ragged_hist(const int32_t *__restrict__ n_sites, size_t B, unsigned long long *__restrict__ counts) {
  __shared__ unsigned int h[33];
  if (threadIdx.x < 33) h[threadIdx.x] = 0u;
  __syncthreads();
  for (size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x; b < B; b += gridDim.x * (size_t)blockDim.x) {
    const int n = n_sites[b];
    atomicAdd(&h[(n >= 1 && n <= 32) ? n : 0], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(counts + threadIdx.x, (unsigned long long)h[threadIdx.x]);
}

// Scatter into buckets: position cursor[N]++ (atomics; the order inside a bucket is arbitrary, the results
// go back through perm), perm = source index.  Entries outside 1..32 were rejected by the caller.
__global__ void k_ragged_scatter(const int32_t *__restrict__ n_sites, const uint32_t *__restrict__ sig,
                                 const uint32_t *__restrict__ sigp, size_t B, unsigned long long *__restrict__ cursor,
                                 uint32_t *__restrict__ ssig, uint32_t *__restrict__ ssigp, uint32_t *__restrict__ perm) {
  for (size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x; b < B; b += gridDim.x * (size_t)blockDim.x) {
    const unsigned long long pos = atomicAdd(cursor + n_sites[b], 1ull);
    ssig[pos] = sig[b];
    ssigp[pos] = sigp[b];
    perm[pos] = (uint32_t)b;
  }
}

__global__ void k_unpermute(const float2 *__restrict__ in, const uint32_t *__restrict__ perm, size_t B,
                            float2 *__restrict__ out) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < B; j += gridDim.x * (size_t)blockDim.x)
    out[perm[j]] = in[j];
}

}  // namespace tdo

static unsigned grid_for(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  if (g > 65535u * 8u) g = 65535u * 8u;
  return (unsigned)(g ? g : 1);
}

cudaError_t launch_connections(const ConnPattern *pat, int n_pat, const ConnContrib *con,
                               const uint32_t *sig, const uint32_t *sigp, size_t Ns, int32_t *count,
                               uint32_t *csig, uint32_t *csigp, float2 *ccoef, cudaStream_t st) {
  if (Ns == 0) return cudaSuccess;
  tdo::k_connections<<<grid_for(Ns * 32, 256), 256, 0, st>>>(pat, n_pat, con, sig, sigp, Ns, count, csig, csigp, ccoef);
  return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t *count, size_t Ns, int64_t *offs, cudaStream_t st) {
  tdo::k_scan<<<1, 1024, 0, st>>>(count, Ns, offs);
  return cudaGetLastError();
}

cudaError_t launch_compact(const int32_t *count, const int64_t *offs, size_t Ns, int M,
                           const uint32_t *csig, const uint32_t *csigp, const float2 *ccoef,
                           uint32_t *fsig, uint32_t *fsigp, float2 *fcoef, cudaStream_t st) {
  if (Ns == 0) return cudaSuccess;
  tdo::k_compact<<<grid_for(Ns * (size_t)M, 256), 256, 0, st>>>(count, offs, Ns, M, csig, csigp, ccoef, fsig, fsigp, fcoef);
  return cudaGetLastError();
}

cudaError_t launch_lloc(const int64_t *offs, size_t Ns, const float2 *fcoef, const float2 *flogrho,
                        double2 *lloc, double *l2, double *stats, int *nonfinite, cudaStream_t st) {
  if (Ns == 0) return cudaSuccess;
  tdo::k_lloc<<<grid_for(Ns * 32, 256), 256, 0, st>>>(offs, Ns, fcoef, flogrho, lloc, l2, nonfinite);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tdo::k_cost_stats<<<1, 1024, 0, st>>>(l2, Ns, stats);
  return cudaGetLastError();
}

cudaError_t launch_cotangent(const int64_t *offs, size_t Ns, const float2 *fcoef, const float2 *flogrho,
                             const double2 *lloc, const double *stats, float2 *cot, cudaStream_t st) {
  if (Ns == 0) return cudaSuccess;
  tdo::k_cotangent<<<grid_for(Ns * 32, 256), 256, 0, st>>>(offs, Ns, fcoef, flogrho, lloc, stats, cot);
  return cudaGetLastError();
}

cudaError_t launch_reduce_copies(const float *acc, int n_copies, size_t stride, size_t P, double *out,
                                 int accumulate, cudaStream_t st, const float *scale) {
  tdo::k_reduce_copies<<<grid_for(P, 256), 256, 0, st>>>(acc, n_copies, stride, P, out, accumulate, scale);
  return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const double *src, float *dst, size_t n, cudaStream_t st) {
  tdo::k_f64_to_f32<<<grid_for(n, 256), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_conv_table_k(int d, int c1, const float *Wc1, const float *bc1, const float *Wc2,
                                const float *bc2, float *table, cudaStream_t st) {
  tdo::k_conv_table<<<(64 * d + 255) / 256, 256, 0, st>>>(d, c1, Wc1, bc1, Wc2, bc2, table);
  return cudaGetLastError();
}

cudaError_t launch_params_f32(const double *theta, size_t P, const long long *tab, int n_tensors,
                              float *dst, cudaStream_t st) {
  tdo::k_params_f32<<<grid_for(P, 256), 256, 0, st>>>(theta, P, tab, n_tensors, dst);
  return cudaGetLastError();
}

cudaError_t launch_ragged_hist(const int32_t *n_sites, size_t B, unsigned long long *counts, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(counts, 0, 33 * sizeof(unsigned long long), st);
  if (e != cudaSuccess || B == 0) return e;
  tdo::k_ragged_hist<<<grid_for(B, 256), 256, 0, st>>>(n_sites, B, counts);
  return cudaGetLastError();
}

cudaError_t launch_ragged_scatter(const int32_t *n_sites, const uint32_t *sig, const uint32_t *sigp, size_t B,
                                  unsigned long long *cursor, uint32_t *ssig, uint32_t *ssigp, uint32_t *perm,
                                  cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  tdo::k_ragged_scatter<<<grid_for(B, 256), 256, 0, st>>>(n_sites, sig, sigp, B, cursor, ssig, ssigp, perm);
  return cudaGetLastError();
}

cudaError_t launch_unpermute(const float2 *in, const uint32_t *perm, size_t B, float2 *out, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  tdo::k_unpermute<<<grid_for(B, 256), 256, 0, st>>>(in, perm, B, out);
  return cudaGetLastError();
}

cudaError_t launch_axpy_update(double *theta, const double *delta, double lr, size_t P, cudaStream_t st,
                               const int *gate) {
  tdo::k_axpy<<<grid_for(P, 256), 256, 0, st>>>(theta, delta, lr, P, gate);
  return cudaGetLastError();
}

cudaError_t launch_adam_update(double *theta, const double *delta, double *m, double *v, size_t P, long long t,
                               double lr, double b1, double b2, double eps, cudaStream_t st, const int *gate,
                               const double *dc) {
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  tdo::k_adam<<<grid_for(P, 256), 256, 0, st>>>(theta, delta, m, v, P, lr, b1, b2, eps, c1, c2, gate, dc);
  return cudaGetLastError();
}

cudaError_t launch_step_gate(const double *outcome, const int *nonfinite, const int *err, int *ok, cudaStream_t st) {
  tdo::k_step_gate<<<1, 1, 0, st>>>(outcome, nonfinite, err, ok);
  return cudaGetLastError();
}
