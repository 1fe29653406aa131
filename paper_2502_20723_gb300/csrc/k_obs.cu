// Mixed-state observables and purity (supplement, "Mixed-State Observables"):
//   <A> = Tr(rho A) / Tr(rho) = E[s A~] / E[s] over alpha drawn from |rho(alpha, alpha)|, with the local
//   estimator A~(alpha) = sum_beta rho(alpha, beta) / rho(alpha, alpha) <beta|A|alpha> and
//   s = sign rho(alpha, alpha); for A = (1/N) sum_i sigma^a_i only beta = alpha and its N single flips
//   contribute: <alpha ^ e_i|sigma^x_i|alpha> = 1, <alpha ^ e_i|sigma^y_i|alpha> = i (1 - 2 alpha_i),
//   <alpha|sigma^z_i|alpha> = 1 - 2 alpha_i (bit 0 = |0>, sigma^z = +1).
//   Tr(rho)^2 / Tr(rho^2) = E[rho(sigma, sigma) rho(sigma', sigma') / |rho(sigma, sigma')|^2] over
//   (sigma, sigma') drawn from |rho|^2.
// The log rho values come from the forward over the row lists built here; the sums are FP64 block
// partials reduced in a fixed order (deterministic).
#include "tdo_internal.cuh"

namespace tdo {
namespace obs {

constexpr int kBlocks = 256, kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;   // valid in thread 0
}

__global__ void k_obs_rows(const uint32_t *__restrict__ alpha, size_t Ns, int n, uint32_t *__restrict__ rs,
                           uint32_t *__restrict__ rp) {
  const size_t total = Ns * (size_t)(n + 1);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += gridDim.x * (size_t)blockDim.x) {
    const size_t s = i / (size_t)(n + 1);
    const int j = (int)(i - s * (size_t)(n + 1));
    const uint32_t a = alpha[s];
    rs[i] = a;
    rp[i] = j == 0 ? a : a ^ (1u << (j - 1));
  }
}

// Thread per sample; part[q * gridDim.x + block] for the 6 sums: s, Re/Im s A~x, Re/Im s A~y, s A~z.
__global__ void k_obs_local(const uint32_t *__restrict__ alpha, size_t Ns, int n, const float2 *__restrict__ lr,
                            double *__restrict__ local, double *__restrict__ part) {
  __shared__ double sh[32];
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < Ns; s += gridDim.x * (size_t)blockDim.x) {
    const float2 *row = lr + s * (size_t)(n + 1);
    const double r0 = row[0].x, i0 = row[0].y;
    const double sg = cos(i0) < 0.0 ? -1.0 : 1.0;   // rho(alpha, alpha) is real: phase 0 or pi
    const uint32_t a = alpha[s];
    double xr = 0.0, xi = 0.0, yr = 0.0, yi = 0.0, z = 0.0;
    for (int i = 0; i < n; ++i) {
      const double m = exp((double)row[1 + i].x - r0), ph = (double)row[1 + i].y - i0;
      const double cr = m * cos(ph), ci = m * sin(ph);   // rho(alpha, alpha ^ e_i) / rho(alpha, alpha)
      const double zi = ((a >> i) & 1u) ? -1.0 : 1.0;
      xr += cr;
      xi += ci;
      yr -= zi * ci;   // i zi (cr + i ci) = -zi ci + i zi cr
      yi += zi * cr;
      z += zi;
    }
    const double inv = 1.0 / (double)n;
    xr *= inv; xi *= inv; yr *= inv; yi *= inv; z *= inv;
    if (local) {
      double *o = local + s * 8;
      o[0] = sg; o[1] = 0.0; o[2] = xr; o[3] = xi; o[4] = yr; o[5] = yi; o[6] = z; o[7] = 0.0;
    }
    acc[0] += sg;
    acc[1] += sg * xr; acc[2] += sg * xi;
    acc[3] += sg * yr; acc[4] += sg * yi;
    acc[5] += sg * z;
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const double t = block_sum(acc[q], sh);
    if (threadIdx.x == 0) part[q * gridDim.x + blockIdx.x] = t;
  }
}

// One block: out[q] = sum over the nb partials of q, in block order.
__global__ void k_sum_parts(const double *__restrict__ part, int nb, int nq, double *__restrict__ out) {
  __shared__ double sh[32];
  for (int q = 0; q < nq; ++q) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[q * nb + b];
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) out[q] = t;
  }
}

__global__ void k_pur_rows(const uint32_t *__restrict__ sig, const uint32_t *__restrict__ sigp, size_t Ns,
                           uint32_t *__restrict__ rs, uint32_t *__restrict__ rp) {
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < Ns; s += gridDim.x * (size_t)blockDim.x) {
    const uint32_t a = sig[s], b = sigp[s];
    rs[3 * s] = a; rp[3 * s] = b;
    rs[3 * s + 1] = a; rp[3 * s + 1] = a;
    rs[3 * s + 2] = b; rp[3 * s + 2] = b;
  }
}

__global__ void k_pur_local(const float2 *__restrict__ lr, size_t Ns, double *__restrict__ part) {
  __shared__ double sh[32];
  double f1 = 0.0, f2 = 0.0;
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < Ns; s += gridDim.x * (size_t)blockDim.x) {
    const float2 c = lr[3 * s], a = lr[3 * s + 1], b = lr[3 * s + 2];
    const double f = exp((double)a.x + (double)b.x - 2.0 * (double)c.x) * cos((double)a.y + (double)b.y);
    f1 += f;
    f2 += f * f;
  }
  const double t1 = block_sum(f1, sh), t2 = block_sum(f2, sh);
  if (threadIdx.x == 0) { part[blockIdx.x] = t1; part[gridDim.x + blockIdx.x] = t2; }
}

}  // namespace obs
}  // namespace tdo

static unsigned grid_for(size_t items) {
  const size_t g = (items + 255) / 256;
  return (unsigned)(g < 4096 ? (g ? g : 1) : 4096);
}

cudaError_t launch_obs_rows(const uint32_t *alpha, size_t Ns, int n, uint32_t *rs, uint32_t *rp, cudaStream_t st) {
  tdo::obs::k_obs_rows<<<grid_for(Ns * (size_t)(n + 1)), 256, 0, st>>>(alpha, Ns, n, rs, rp);
  return cudaGetLastError();
}

cudaError_t launch_obs_reduce(const uint32_t *alpha, size_t Ns, int n, const float2 *lr, double *local,
                              double *part, double *out, cudaStream_t st) {
  using namespace tdo::obs;
  k_obs_local<<<kBlocks, kThreads, 0, st>>>(alpha, Ns, n, lr, local, part);
  k_sum_parts<<<1, 256, 0, st>>>(part, kBlocks, 6, out);
  return cudaGetLastError();
}

cudaError_t launch_pur_rows(const uint32_t *sig, const uint32_t *sigp, size_t Ns, uint32_t *rs, uint32_t *rp,
                            cudaStream_t st) {
  tdo::obs::k_pur_rows<<<grid_for(Ns), 256, 0, st>>>(sig, sigp, Ns, rs, rp);
  return cudaGetLastError();
}

cudaError_t launch_pur_reduce(const float2 *lr, size_t Ns, double *part, double *out, cudaStream_t st) {
  using namespace tdo::obs;
  k_pur_local<<<kBlocks, kThreads, 0, st>>>(lr, Ns, part);
  k_sum_parts<<<1, 256, 0, st>>>(part, kBlocks, 2, out);
  return cudaGetLastError();
}
