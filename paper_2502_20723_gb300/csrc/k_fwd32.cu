// FP32 CUDA-core forward of the ansatz (architecture appendix) and the Metropolis sampler built on it
// (sampling section).  Persistent grids: one CTA of 256 threads per tile of <= 128 token rows.
#include "f32_tile.cuh"

namespace tdo {

template <int D>
__global__ void __launch_bounds__(kThreads) k_fwd32(DevModel m, const uint32_t *__restrict__ sig,
                                                     const uint32_t *__restrict__ sigp, size_t B,
                                                     float2 *__restrict__ out) {
  extern __shared__ float4 smem4[];
  float *sm = reinterpret_cast<float *>(smem4);
  using G = F32Geom<D>;
  uint32_t *csig = reinterpret_cast<uint32_t *>(sm + G::C_OFF);
  uint32_t *csigp = csig + kRows / 2;
  const float2 *res = reinterpret_cast<const float2 *>(sm + G::O_OFF);
  const int ts = seqs_per_tile(m.n_sites), tc = ts / 2;
  const size_t ntiles = (B + tc - 1) / tc;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (threadIdx.x < tc) {
      const size_t b = tile * tc + threadIdx.x;
      csig[threadIdx.x] = b < B ? sig[b] : 0u;
      csigp[threadIdx.x] = b < B ? sigp[b] : 0u;
    }
    __syncthreads();
    eval_tile_f32<D>(m, sm, ts);
    if (threadIdx.x < tc) {
      const size_t b = tile * tc + threadIdx.x;
      if (b < B) out[b] = res[threadIdx.x];
    }
    __syncthreads();
  }
}

// Each CTA owns tiles of ts/2 chains and runs every proposal of those chains: draw (bit, u), evaluate
// the proposed configurations as one tile, accept iff u < exp(min(0, 2 Re(log rho' - log rho))).
// diag: chains on |rho(alpha, alpha)| (sig = sigp = alpha): N proposals per sweep, each flipping one site
// in both entries, accepted iff u < exp(min(0, Re(log rho' - log rho))).
template <int D>
__global__ void __launch_bounds__(kThreads) k_sample32(DevModel m, size_t n_chains, size_t n_sweeps,
                                                        uint64_t seed, uint64_t counter,
                                                        uint32_t *__restrict__ sig,
                                                        uint32_t *__restrict__ sigp,
                                                        uint32_t *__restrict__ ssig,
                                                        uint32_t *__restrict__ ssigp,
                                                        unsigned long long *accepted, int diag) {
  extern __shared__ float4 smem4[];
  float *sm = reinterpret_cast<float *>(smem4);
  using G = F32Geom<D>;
  uint32_t *csig = reinterpret_cast<uint32_t *>(sm + G::C_OFF);
  uint32_t *csigp = csig + kRows / 2;
  const float2 *res = reinterpret_cast<const float2 *>(sm + G::O_OFF);
  const int n = m.n_sites;
  const int ts = seqs_per_tile(n), tc = ts / 2;
  const size_t ntiles = (n_chains + tc - 1) / tc;
  unsigned long long acc_count = 0;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t c = tile * tc + threadIdx.x;
    const bool mine = threadIdx.x < tc && c < n_chains;
    uint32_t cs = 0, cp = 0, ps = 0, pp = 0;
    float lcur = 0.f, u = 0.f;
    if (mine) { cs = sig[c]; cp = sigp[c]; }
    if (threadIdx.x < tc) { csig[threadIdx.x] = cs; csigp[threadIdx.x] = cp; }
    __syncthreads();
    eval_tile_f32<D>(m, sm, ts);
    if (threadIdx.x < tc) lcur = res[threadIdx.x].x;
    const int per = diag ? n : 2 * n;   // proposals per sweep
    for (size_t sw = 0; sw < n_sweeps; ++sw) {
      for (int j = 0; j < per; ++j) {
        const uint64_t t = counter + (uint64_t)sw * (uint64_t)per + (uint64_t)j;
        if (threadIdx.x < tc) {
          int bit;
          metropolis_draw(seed, (uint32_t)c, t, per, &bit, &u);
          ps = cs;
          pp = cp;
          if (diag) { ps ^= 1u << bit; pp ^= 1u << bit; }
          else if (bit < n) ps ^= 1u << bit;
          else pp ^= 1u << (bit - n);
          csig[threadIdx.x] = ps;
          csigp[threadIdx.x] = pp;
        }
        __syncthreads();
        eval_tile_f32<D>(m, sm, ts);
        if (threadIdx.x < tc) {
          const float lnew = res[threadIdx.x].x;
          const float d = (diag ? 1.0f : 2.0f) * (lnew - lcur);
          if (u < expf(fminf(0.0f, d))) {
            cs = ps; cp = pp; lcur = lnew;
            if (mine) ++acc_count;
          }
        }
      }
      if (mine && ssig) { ssig[sw * n_chains + c] = cs; ssigp[sw * n_chains + c] = cp; }
    }
    if (mine) { sig[c] = cs; sigp[c] = cp; }
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    unsigned long long v = acc_count;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0 && accepted) atomicAdd(accepted, v);
  }
}

template <int D>
static cudaError_t fwd_impl(const DevModel &m, const uint32_t *sig, const uint32_t *sigp, size_t B,
                            float2 *out, int n_sm, cudaStream_t st) {
  const size_t bytes = F32Geom<D>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_fwd32<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fwd32<D>, kThreads, bytes);
  if (e != cudaSuccess) return e;
  const int tc = seqs_per_tile(m.n_sites) / 2;
  const size_t ntiles = (B + tc - 1) / tc;
  size_t grid = (size_t)n_sm * (per_sm > 0 ? per_sm : 1);
  if (grid > ntiles) grid = ntiles;
  k_fwd32<D><<<(unsigned)grid, kThreads, bytes, st>>>(m, sig, sigp, B, out);
  return cudaGetLastError();
}

template <int D>
static cudaError_t sample_impl(const DevModel &m, size_t n_chains, size_t n_sweeps, uint64_t seed,
                               uint64_t counter, uint32_t *sig, uint32_t *sigp, uint32_t *ssig,
                               uint32_t *ssigp, unsigned long long *accepted, int diag, int n_sm,
                               cudaStream_t st) {
  const size_t bytes = F32Geom<D>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_sample32<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample32<D>, kThreads, bytes);
  if (e != cudaSuccess) return e;
  const int tc = seqs_per_tile(m.n_sites) / 2;
  const size_t ntiles = (n_chains + tc - 1) / tc;
  size_t grid = (size_t)n_sm * (per_sm > 0 ? per_sm : 1);
  if (grid > ntiles) grid = ntiles;
  k_sample32<D><<<(unsigned)grid, kThreads, bytes, st>>>(m, n_chains, n_sweeps, seed, counter, sig, sigp,
                                                         ssig, ssigp, accepted, diag);
  return cudaGetLastError();
}

}  // namespace tdo

cudaError_t launch_fwd32(const DevModel &m, const uint32_t *sig, const uint32_t *sigp, size_t B,
                         float2 *logrho, int n_sm, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  switch (m.d) {
    case 16: return tdo::fwd_impl<16>(m, sig, sigp, B, logrho, n_sm, st);
    case 32: return tdo::fwd_impl<32>(m, sig, sigp, B, logrho, n_sm, st);
    case 64: return tdo::fwd_impl<64>(m, sig, sigp, B, logrho, n_sm, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sample32(const DevModel &m, size_t n_chains, size_t n_sweeps, uint64_t seed,
                            uint64_t counter, uint32_t *sig, uint32_t *sigp, uint32_t *ssig,
                            uint32_t *ssigp, unsigned long long *accepted, int diag, int n_sm, cudaStream_t st) {
  if (n_chains == 0) return cudaSuccess;
  switch (m.d) {
    case 16: return tdo::sample_impl<16>(m, n_chains, n_sweeps, seed, counter, sig, sigp, ssig, ssigp, accepted, diag, n_sm, st);
    case 32: return tdo::sample_impl<32>(m, n_chains, n_sweeps, seed, counter, sig, sigp, ssig, ssigp, accepted, diag, n_sm, st);
    case 64: return tdo::sample_impl<64>(m, n_chains, n_sweeps, seed, counter, sig, sigp, ssig, ssigp, accepted, diag, n_sm, st);
    default: return cudaErrorInvalidValue;
  }
}
