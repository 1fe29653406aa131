// Test-only kernel: one tcgen05.mma chain D[128 x N] = A[128 x 128] . B[N x 128]^T on operands whose
// shared-memory byte images are prepared by the host, to pin the descriptor fields of K-major and
// MN-major operands: kind::f16 with BF16 operands (8 MMAs of K = 16), or, with f8 set, kind::f8f6f4
// with E4M3 operands in 8-bit K-major images (4 MMAs of K = 32).  All reads stay inside zero-filled 96 KB regions (any LBO/SBO reading of the
// fields keeps the MMA's addresses below 62 KB from the region start).
#include <stdint.h>

#include "../../paper_2502_20723_gb300/csrc/tcgen05.cuh"

using namespace tdo::tc;

constexpr int kRegion = 96 * 1024;

extern "C" __global__ void __launch_bounds__(128, 1)
    umma_probe(const uint8_t *a_img, int a_bytes, const uint8_t *b_img, int b_bytes, int N, int a_mn, int b_mn,
               uint32_t a_lbo, uint32_t a_sbo, uint32_t a_step, uint32_t b_lbo, uint32_t b_sbo, uint32_t b_step,
               int f8, float *D, int *err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t holder;
  for (int i = threadIdx.x; i < 2 * kRegion / 16; i += blockDim.x) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  for (int i = threadIdx.x; i < a_bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(sm)[i] = reinterpret_cast<const uint4 *>(a_img)[i];
  for (int i = threadIdx.x; i < b_bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(sm + kRegion)[i] = reinterpret_cast<const uint4 *>(b_img)[i];
  const uint32_t bar_a = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(bar_a, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&holder)), "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = holder;
  if (threadIdx.x == 0) {
    const uint32_t id = f8 ? idesc_e4m3(128, N) : idesc_bf16_major(128, N, a_mn, b_mn);
    const uint32_t a0 = smem_u32(sm), b0 = smem_u32(sm + kRegion);
    for (int kk = 0; kk < (f8 ? 4 : 8); ++kk) {
      const uint64_t ad = sdesc(a0 + kk * a_step, a_lbo, a_sbo);
      const uint64_t bd = sdesc(b0 + kk * b_step, b_lbo, b_sbo);
      if (f8) mma_e4m3(tmem, ad, bd, id, kk > 0 ? 1u : 0u);
      else mma_bf16(tmem, ad, bd, id, kk > 0 ? 1u : 0u);
    }
    mma_commit(bar_a);
  }
  const bool ok = mbar_wait(bar_a, 0);
  tc_fence_after();
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  const int warp = threadIdx.x >> 5;
  const uint32_t lane_addr = (uint32_t)(32 * warp) << 16;
  if (ok) {
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tmem_ld16(tmem + lane_addr + c, v);
      for (int e = 0; e < 16; ++e) D[threadIdx.x * N + c + e] = v[e];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
  }
}

// Host launcher (C ABI) for the test: device buffers in, D [128 x N] device out.
extern "C" int umma_probe_run(const uint8_t *a_img, int a_bytes, const uint8_t *b_img, int b_bytes, int N, int a_mn,
                              int b_mn, uint32_t a_lbo, uint32_t a_sbo, uint32_t a_step, uint32_t b_lbo,
                              uint32_t b_sbo, uint32_t b_step, int f8, float *D, int *err) {
  const int bytes = 2 * kRegion;
  cudaError_t e = cudaFuncSetAttribute(umma_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return (int)e;
  umma_probe<<<1, 128, bytes>>>(a_img, a_bytes, b_img, b_bytes, N, a_mn, b_mn, a_lbo, a_sbo, a_step, b_lbo, b_sbo,
                                b_step, f8, D, err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  return (int)cudaDeviceSynchronize();
}
