// Stochastic reconfiguration solve (metric-tensor and regularisation sections):
//   (Re S + lambda I) x = rhs,  S_ij = <O_i^* O_j> - <O_i^*><O_j>  over Ns samples,
// by Jacobi-preconditioned conjugate gradients, matrix-free: S v = (1/Ns) Re[Obar^H (Obar v)] with
// Obar = O - mean(O), O stored as FP32 (re, im) [Ns][P].  Each iteration streams O twice from HBM
// (the bound of this solver).  Products are formed in FP32 over short runs and accumulated in FP64
// (GB300's FP64 rate is far below its FP32 rate); all CG vectors and scalars are FP64 and stay on the
// device (no host round trip per iteration; a device flag ends the iteration).
#include "tdo_internal.cuh"
#include "tdo_device.cuh"

namespace tdo {

constexpr int kSrBlock = 256;
constexpr int kRun = 32;   // FP32 products per FP64 accumulation

// scalars: [0] rz, [1] bnorm2, [2] alpha, [3] rnorm2, [4] done flag, [5] iterations, [6] tol2, [7] pAp
enum { S_RZ = 0, S_BN = 1, S_AL = 2, S_RN = 3, S_DONE = 4, S_IT = 5, S_TOL = 6, S_PAP = 7 };

// mean[k] = (1/Ns) sum_s O[s][k]; thread per k, coalesced over k.
__global__ void k_sr_mean(const float2 *__restrict__ O, size_t Ns, size_t P, double2 *__restrict__ mean) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    double ar = 0.0, ai = 0.0;
    for (size_t s0 = 0; s0 < Ns; s0 += kRun) {
      float fr = 0.f, fi = 0.f;
      const size_t s1 = s0 + kRun < Ns ? s0 + kRun : Ns;
      for (size_t s = s0; s < s1; ++s) { const float2 o = O[s * P + k]; fr += o.x; fi += o.y; }
      ar += fr;
      ai += fi;
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
      float f = 0.f;
      const size_t s1 = s0 + kRun < Ns ? s0 + kRun : Ns;
      for (size_t s = s0; s < s1; ++s) {
        const float2 o = O[s * P + k];
        const float dr = o.x - mr, di = o.y - mi;
        f = fmaf(dr, dr, fmaf(di, di, f));
      }
      a += f;
    }
    diag[k] = a / (double)Ns + shift;
  }
}

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

// t[s] = sum_k (O[s][k] - mean[k]) v[k]  (complex), one block per sample.
__global__ void k_sr_t(const float2 *__restrict__ O, size_t Ns, size_t P, const double2 *__restrict__ mean,
                       const double *__restrict__ v, double2 *__restrict__ t, const double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  for (size_t s = blockIdx.x; s < Ns; s += gridDim.x) {
    const float2 *row = O + s * P;
    double ar = 0.0, ai = 0.0;
    float fr = 0.f, fi = 0.f;
    int run = 0;
    for (size_t k = threadIdx.x; k < P; k += blockDim.x) {
      const float2 o = row[k];
      const double2 m = mean[k];
      const float vk = (float)v[k];
      fr = fmaf(o.x - (float)m.x, vk, fr);
      fi = fmaf(o.y - (float)m.y, vk, fi);
      if (++run == kRun) { ar += fr; ai += fi; fr = fi = 0.f; run = 0; }
    }
    ar += fr;
    ai += fi;
    const double r = block_sum_d(ar, sh);
    const double i = block_sum_d(ai, sh);
    if (threadIdx.x == 0) t[s] = make_double2(r, i);
  }
}

// Ap[k] = (1/Ns) sum_s Re(conj(O[s][k] - mean[k]) t[s]) + shift p[k]; block partials of p . Ap.
__global__ void k_sr_w(const float2 *__restrict__ O, size_t Ns, size_t P, const double2 *__restrict__ mean,
                       const double2 *__restrict__ t, const double *__restrict__ p, double shift,
                       double *__restrict__ Ap, double *__restrict__ part, const double *__restrict__ sc) {
  __shared__ double sh[32];
  if (sc[S_DONE] != 0.0) return;
  double loc = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    const float mr = (float)mean[k].x, mi = (float)mean[k].y;
    double a = 0.0;
    for (size_t s0 = 0; s0 < Ns; s0 += kRun) {
      float f = 0.f;
      const size_t s1 = s0 + kRun < Ns ? s0 + kRun : Ns;
      for (size_t s = s0; s < s1; ++s) {
        const float2 o = O[s * P + k];
        const double2 ts = t[s];
        f = fmaf(o.x - mr, (float)ts.x, fmaf(o.y - mi, (float)ts.y, f));
      }
      a += f;
    }
    const double v = a / (double)Ns + shift * p[k];
    Ap[k] = v;
    loc += v * p[k];
  }
  const double b = block_sum_d(loc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__device__ __forceinline__ double sum_parts(const double *part, int n, double *sh) {
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
  return block_sum_d(a, sh);
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

// initial state: x = 0, r = rhs, z = r/diag, p = z; partials of r.r and r.z
__global__ void k_sr_init(size_t P, const double *__restrict__ rhs, double *__restrict__ x, double *__restrict__ r,
                          double *__restrict__ z, double *__restrict__ p, const double *__restrict__ diag,
                          double *__restrict__ part, double *__restrict__ part2) {
  __shared__ double sh[32];
  double rr = 0.0, rz = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P; k += gridDim.x * (size_t)blockDim.x) {
    const double rk = rhs[k];
    x[k] = 0.0;
    r[k] = rk;
    const double zk = rk / diag[k];
    z[k] = zk;
    p[k] = zk;
    rr += rk * rk;
    rz += rk * zk;
  }
  const double a = block_sum_d(rr, sh);
  const double b = block_sum_d(rz, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = a; part2[blockIdx.x] = b; }
}

__global__ void k_sr_init_scalars(const double *__restrict__ part, const double *__restrict__ part2, int nb,
                                  double tol, double *__restrict__ sc) {
  __shared__ double sh[32];
  const double rr = sum_parts(part, nb, sh);
  const double rz = sum_parts(part2, nb, sh);
  if (threadIdx.x == 0) {
    sc[S_RZ] = rz;
    sc[S_BN] = rr;
    sc[S_RN] = rr;
    sc[S_AL] = 0.0;
    sc[S_IT] = 0.0;
    sc[S_TOL] = tol * tol;
    sc[S_PAP] = 0.0;
    sc[S_DONE] = (rr == 0.0) ? 1.0 : 0.0;
  }
}

}  // namespace tdo

size_t sr_work_doubles(size_t Ns, size_t P) {
  // mean 2P, diag, r, z, p, Ap (5P), t 2Ns, partials 2*1024, scalars 16
  return 2 * P + 5 * P + 2 * Ns + 2 * 1024 + 16;
}

cudaError_t sr_cg_impl(const float *O, size_t Ns, size_t P, const double *rhs, double shift, double tol,
                       int max_iter, double *x, double *work, int n_sm, int *iters, double *resid,
                       cudaStream_t st) {
  using namespace tdo;
  double2 *mean = reinterpret_cast<double2 *>(work);
  double *diag = work + 2 * P, *r = diag + P, *z = r + P, *p = z + P, *Ap = p + P;
  double2 *t = reinterpret_cast<double2 *>(Ap + P);
  double *part = reinterpret_cast<double *>(t + Ns), *part2 = part + 1024, *sc = part2 + 1024;
  const float2 *O2 = reinterpret_cast<const float2 *>(O);
  int nb = (int)((P + kSrBlock - 1) / kSrBlock);
  if (nb > 1024) nb = 1024;
  if (nb < 1) nb = 1;
  const int ngrid_t = (int)(Ns < (size_t)(8 * n_sm) ? Ns : (size_t)(8 * n_sm));
  k_sr_mean<<<nb, kSrBlock, 0, st>>>(O2, Ns, P, mean);
  k_sr_diag<<<nb, kSrBlock, 0, st>>>(O2, Ns, P, mean, shift, diag);
  k_sr_init<<<nb, kSrBlock, 0, st>>>(P, rhs, x, r, z, p, diag, part, part2);
  k_sr_init_scalars<<<1, 1024, 0, st>>>(part, part2, nb, tol, sc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // Iterations are launched in groups; the done flag on the device makes the rest of a group a no-op,
  // and the host looks at it between groups only.
  const int group = 16;
  double h[8];
  for (int it = 0; it < max_iter;) {
    const int end = it + group < max_iter ? it + group : max_iter;
    for (; it < end; ++it) {
      k_sr_t<<<ngrid_t > 0 ? ngrid_t : 1, kSrBlock, 0, st>>>(O2, Ns, P, mean, p, t, sc);
      k_sr_w<<<nb, kSrBlock, 0, st>>>(O2, Ns, P, mean, t, p, shift, Ap, part, sc);
      k_sr_alpha<<<1, 1024, 0, st>>>(part, nb, sc);
      k_sr_xr<<<nb, kSrBlock, 0, st>>>(P, x, r, z, p, Ap, diag, part, part2, sc);
      k_sr_beta<<<1, 1024, 0, st>>>(part, part2, nb, sc);
      k_sr_p<<<nb, kSrBlock, 0, st>>>(P, p, z, sc);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (h[S_DONE] != 0.0) break;
  }
  if (max_iter <= 0) {
    e = cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
  }
  if (iters) *iters = (int)h[S_IT];
  if (resid) *resid = h[S_BN] > 0 ? sqrt(h[S_RN] / h[S_BN]) : 0.0;
  if (h[S_DONE] == 2.0) return cudaErrorInvalidValue;   // not positive definite
  return cudaSuccess;
}
