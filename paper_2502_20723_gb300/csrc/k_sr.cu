// Stochastic reconfiguration solve (metric-tensor and regularisation sections):
//   (Re S + lambda I) x = rhs,  S_ij = <O_i^* O_j> - <O_i^*><O_j>  over Ns samples,
// by Jacobi-preconditioned conjugate gradients, matrix-free: with Obar = O - mean(O),
//   S v = (1/Ns) Re[Obar^H (Obar v)],
// O stored as FP32 (re, im) [Ns][P].  One iteration streams O twice from HBM (t = Obar v per sample,
// then w = Obar^H t per parameter) and is HBM-bound; both passes keep many independent loads in flight.
// Products are formed in FP32 over runs of 32 terms and accumulated in FP64 (GB300's FP64 rate is far
// below its FP32 rate); CG vectors and scalars are FP64 and stay on the device: a device flag ends the
// iteration, the host looks at it between groups of iterations only.
#include "tdo_internal.cuh"
#include "tdo_device.cuh"

namespace tdo {

constexpr int kSrBlock = 256;
constexpr int kRun = 32;     // FP32 products per FP64 accumulation

enum {
  S_RZ = 0, S_BN, S_AL, S_RN, S_DONE, S_IT, S_TOL, S_PAP, S_CR, S_CI, S_TR, S_TI, S_COUNT
};

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

// mean[k] = (1/Ns) sum_s O[s][k]   (thread per k, 4 independent loads in flight)
__global__ void k_sr_mean(const float2 *__restrict__ O, size_t Ns, size_t P, double2 *__restrict__ mean) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    double ar = 0.0, ai = 0.0;
    for (size_t s0 = 0; s0 < Ns; s0 += kRun) {
      const size_t s1 = s0 + kRun < Ns ? s0 + kRun : Ns;
      float fr[4] = {0, 0, 0, 0}, fi[4] = {0, 0, 0, 0};
      size_t s = s0;
      for (; s + 4 <= s1; s += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) { const float2 o = __ldg(O + (s + u) * P + k); fr[u] += o.x; fi[u] += o.y; }
      }
      for (; s < s1; ++s) { const float2 o = __ldg(O + s * P + k); fr[0] += o.x; fi[0] += o.y; }
      ar += (double)((fr[0] + fr[1]) + (fr[2] + fr[3]));
      ai += (double)((fi[0] + fi[1]) + (fi[2] + fi[3]));
    }
    mean[k] = make_double2(ar / (double)Ns, ai / (double)Ns);
  }
}

// diag[k] = (1/Ns) sum_s |O[s][k] - mean[k]|^2 + shift   (Jacobi preconditioner of S + shift I)
__global__ void k_sr_diag(const float2 *__restrict__ O, size_t Ns, size_t P, const double2 *__restrict__ mean,
                          double shift, double *__restrict__ diag) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    const float mr = (float)mean[k].x, mi = (float)mean[k].y;
    double a = 0.0;
    for (size_t s0 = 0; s0 < Ns; s0 += kRun) {
      const size_t s1 = s0 + kRun < Ns ? s0 + kRun : Ns;
      float f[4] = {0, 0, 0, 0};
      size_t s = s0;
      for (; s + 4 <= s1; s += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 o = __ldg(O + (s + u) * P + k);
          const float dr = o.x - mr, di = o.y - mi;
          f[u] = fmaf(dr, dr, fmaf(di, di, f[u]));
        }
      }
      for (; s < s1; ++s) {
        const float2 o = __ldg(O + s * P + k);
        const float dr = o.x - mr, di = o.y - mi;
        f[0] = fmaf(dr, dr, fmaf(di, di, f[0]));
      }
      a += (double)((f[0] + f[1]) + (f[2] + f[3]));
    }
    diag[k] = a / (double)Ns + shift;
  }
}

// vf = (float) v; block partials of mean . v (re, im)
__global__ void k_sr_vprep(size_t P, const double *__restrict__ v, const double2 *__restrict__ mean,
                           float *__restrict__ vf, double *__restrict__ part, double *__restrict__ part2,
                           const double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  double cr = 0.0, ci = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    const double x = v[k];
    vf[k] = (float)x;
    cr += mean[k].x * x;
    ci += mean[k].y * x;
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

// Partial dot products of the rows of O with v over one chunk of kChunk parameters: block (chunk, sg)
// streams the chunk of every sample row of sample group sg (8 KB contiguous per row), one warp per
// row at a time, with the chunk of v in shared memory.  part[chunk][s] = sum_{k in chunk} O[s][k] v[k].
constexpr int kChunk = 1024;
constexpr int kSampleGroups = 8;

__global__ void k_sr_tpart(const float2 *__restrict__ O, size_t Ns, size_t P, const float *__restrict__ vf,
                           double2 *__restrict__ part, const double *__restrict__ sc) {
  __shared__ float vs[kChunk];
  if (sc[S_DONE] != 0.0) return;
  const size_t k0 = (size_t)blockIdx.x * kChunk;
  const int kn = (int)((P - k0) < (size_t)kChunk ? (P - k0) : (size_t)kChunk);
  for (int i = threadIdx.x; i < kChunk; i += blockDim.x) vs[i] = i < kn ? vf[k0 + i] : 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const size_t per = (Ns + kSampleGroups - 1) / kSampleGroups;
  const size_t s_begin = (size_t)blockIdx.y * per;
  const size_t s_end = s_begin + per < Ns ? s_begin + per : Ns;
  for (size_t s = s_begin + warp; s < s_end; s += nw) {
    const float2 *row = O + s * P + k0;
    float ar = 0.f, ai = 0.f;
#pragma unroll 8
    for (int i = lane; i < kn; i += 32) {
      const float2 o = __ldg(row + i);
      const float x = vs[i];
      ar = fmaf(o.x, x, ar);
      ai = fmaf(o.y, x, ai);
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

// T = sum_s t[s]  (zero in exact arithmetic; subtracted explicitly below)
__global__ void k_sr_tsum(const float2 *__restrict__ t, size_t Ns, double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  double a = 0.0, b = 0.0;
  for (size_t s = threadIdx.x; s < Ns; s += blockDim.x) { a += t[s].x; b += t[s].y; }
  a = block_sum_d(a, sh);
  b = block_sum_d(b, sh);
  if (threadIdx.x == 0) { sc[S_TR] = a; sc[S_TI] = b; }
}

// Ap[k] = (1/Ns) [sum_s Re(conj(O[s][k]) t[s]) - Re(conj(mean[k]) T)] + shift p[k]; partials of p . Ap.
__global__ void k_sr_w(const float2 *__restrict__ O, size_t Ns, size_t P, const double2 *__restrict__ mean,
                       const float2 *__restrict__ t, const double *__restrict__ p, double shift,
                       double *__restrict__ Ap, double *__restrict__ part, const double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  const double Tr = sc[S_TR], Ti = sc[S_TI];
  double loc = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    double a = 0.0;
    for (size_t s0 = 0; s0 < Ns; s0 += kRun) {
      const size_t s1 = s0 + kRun < Ns ? s0 + kRun : Ns;
      float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      size_t s = s0;
      for (; s + 8 <= s1; s += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float2 o = __ldg(O + (s + u) * P + k);
          const float2 ts = t[s + u];
          f[u] = fmaf(o.x, ts.x, fmaf(o.y, ts.y, f[u]));
        }
      }
      for (; s < s1; ++s) {
        const float2 o = __ldg(O + s * P + k);
        const float2 ts = t[s];
        f[0] = fmaf(o.x, ts.x, fmaf(o.y, ts.y, f[0]));
      }
      a += (double)(((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])));
    }
    const double2 m = mean[k];
    const double v = (a - (m.x * Tr + m.y * Ti)) / (double)Ns + shift * p[k];
    Ap[k] = v;
    loc += v * p[k];
  }
  const double b = block_sum_d(loc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void k_sr_alpha(const double *__restrict__ part, int nb, double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  const double pap = sum_parts(part, nb, sh);
  if (threadIdx.x == 0) {
    sc[S_PAP] = pap;
    sc[S_AL] = (pap > 0.0) ? sc[S_RZ] / pap : 0.0;
    if (!(pap > 0.0)) sc[S_DONE] = 2.0;   // breakdown (S' must be positive definite)
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
    if (rr <= sc[S_TOL] * sc[S_BN]) sc[S_DONE] = 1.0;
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
                          double *__restrict__ part, double *__restrict__ part2, double *__restrict__ part3) {
  __shared__ double sh[32];
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
                                  const double *__restrict__ part3, int nb, double tol, double *__restrict__ sc) {
  __shared__ double sh[32];
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
    sc[S_DONE] = (rr <= tol * tol * bb) ? 1.0 : 0.0;
  }
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
  return q;
}

// S' v -> Ap (and the partials of v . Ap in q.part), all on the device.
static void matvec(const float2 *O, size_t Ns, size_t P, const double *v, double shift, SrPtrs &q, int nb,
                   int ngrid_t, cudaStream_t st) {
  (void)ngrid_t;
  const int nchunks = (int)((P + kChunk - 1) / kChunk);
  k_sr_vprep<<<nb, kSrBlock, 0, st>>>(P, v, q.mean, q.vf, q.part, q.part2, q.sc);
  k_sr_cfin<<<1, 1024, 0, st>>>(q.part, q.part2, nb, q.sc);
  k_sr_tpart<<<dim3(nchunks, kSampleGroups), kSrBlock, 0, st>>>(O, Ns, P, q.vf, q.tpart, q.sc);
  k_sr_tred<<<(unsigned)((Ns + 255) / 256), 256, 0, st>>>(q.tpart, nchunks, Ns, q.t, q.sc);
  k_sr_tsum<<<1, 1024, 0, st>>>(q.t, Ns, q.sc);
  k_sr_w<<<nb, kSrBlock, 0, st>>>(O, Ns, P, q.mean, q.t, v, shift, q.Ap, q.part, q.sc);
}

}  // namespace tdo

size_t sr_work_doubles(size_t Ns, size_t P) {
  // the regions carved by sr_carve, each rounded up to 16 bytes, plus slack
  const size_t nchunks = (P + tdo::kChunk - 1) / tdo::kChunk;
  const size_t bytes = 16 * P + 5 * (8 * P + 16) + 3 * 8 * 1024 + 8 * 32 + (4 * P + 16) + (8 * Ns + 16) +
                       16 * nchunks * Ns + 64;
  return (bytes + 7) / 8;
}

cudaError_t sr_cg_impl(const float *O, size_t Ns, size_t P, const double *rhs, const double *x0, double shift,
                       double tol, int max_iter, double *x, double *work, int n_sm, int *iters, double *resid,
                       long long *launches, cudaStream_t st) {
  using namespace tdo;
  SrPtrs q = sr_carve(work, Ns, P);
  const float2 *O2 = reinterpret_cast<const float2 *>(O);
  int nb = (int)((P + kSrBlock - 1) / kSrBlock);
  if (nb > 1024) nb = 1024;
  if (nb < 1) nb = 1;
  const int ngrid_t = n_sm;
  long long nl = 0;
  k_sr_mean<<<nb, kSrBlock, 0, st>>>(O2, Ns, P, q.mean);
  k_sr_diag<<<nb, kSrBlock, 0, st>>>(O2, Ns, P, q.mean, shift, q.diag);
  k_sr_clear<<<1, 32, 0, st>>>(q.sc);
  nl += 3;
  if (x0) { matvec(O2, Ns, P, x0, shift, q, nb, ngrid_t > 0 ? ngrid_t : 1, st); nl += 6; }
  k_sr_init<<<nb, kSrBlock, 0, st>>>(P, rhs, x0, q.Ap, x, q.r, q.z, q.p, q.diag, q.part, q.part2, q.part3);
  k_sr_init_scalars<<<1, 1024, 0, st>>>(q.part, q.part2, q.part3, nb, tol, q.sc);
  nl += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // Iterations are launched in groups; the done flag on the device makes the rest of a group a no-op,
  // and the host looks at it between groups only.
  const int group = 8;
  double h[S_COUNT];
  bool fetched = false;
  for (int it = 0; it < max_iter;) {
    const int end = it + group < max_iter ? it + group : max_iter;
    for (; it < end; ++it) {
      matvec(O2, Ns, P, q.p, shift, q, nb, ngrid_t > 0 ? ngrid_t : 1, st);
      k_sr_alpha<<<1, 1024, 0, st>>>(q.part, nb, q.sc);
      k_sr_xr<<<nb, kSrBlock, 0, st>>>(P, x, q.r, q.z, q.p, q.Ap, q.diag, q.part, q.part2, q.sc);
      k_sr_beta<<<1, 1024, 0, st>>>(q.part, q.part2, nb, q.sc);
      k_sr_p<<<nb, kSrBlock, 0, st>>>(P, q.p, q.z, q.sc);
      nl += 10;
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
  if (resid) *resid = h[S_BN] > 0 ? sqrt(h[S_RN] / h[S_BN]) : 0.0;
  if (launches) *launches = nl;
  if (h[S_DONE] == 2.0) return cudaErrorInvalidValue;   // not positive definite
  return cudaSuccess;
}
