// tcgen05 / TMA / mbarrier PTX wrappers for sm_103a (inline PTX in our own kernels).
//
// Shared-memory operand layouts (no swizzle): a [rows][K] tile in the canonical K-major layout keeps
// element (row, k) at byte (row/8)*16K + (k/8)*128 + (row%8)*16 + (k%8)*2 — core matrices of 8 rows x
// 16 bytes.  The same bytes read with an MN-major descriptor describe the transposed operand (M or N =
// the K of the stored tile, K = its rows).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tdo {
namespace tc {

constexpr long long kSpinLimit = 1ll << 26;   // ~seconds of polling before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with parity `phase` to complete; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t phase, long long limit = kSpinLimit) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try(a, phase)) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

// Bulk (TMA engine) copy of `bytes` contiguous bytes global -> shared, completion on mbarrier `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major: start >> 4 at [0,14), LBO >> 4 at [16,30),
// SBO >> 4 at [32,46), fixed 0b001 at [46,49), layout type 0 (no swizzle) at [61,64).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 at [17,23), M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// The same with A = B = FP16 (format fields 0).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// kind::f8f6f4 with A = B = E4M3 (format fields 0, the same bit pattern as idesc_f16), D = F32; one
// instruction covers K = 32 (32 bytes of each operand row).
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) { return idesc_f16(M, N); }
__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (thread = lane).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16-byte global load issued where it stands: a volatile asm statement keeps its place among the other
// asm statements (barrier waits, MMA issue), so the compiler does not sink it towards its first use.
__device__ __forceinline__ float4 ld_pinned_f4(const float *p) {
  float4 v;
  asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}

// Two 16-column loads (addresses ta, tb) completed by one wait.
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, float (&va)[16], uint32_t tb, float (&vb)[16]) {
  uint32_t r[32];
  asm volatile(
      "{\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      "}"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    va[i] = __uint_as_float(r[i]);
    vb[i] = __uint_as_float(r[16 + i]);
  }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 2^x and tanh(x) on the SFU (PTX ex2.approx / tanh.approx); the BF16 path's error budget allows them.
__device__ __forceinline__ float ex2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_fast(float x) {   // PTX rcp.approx (softmax normalisation)
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float gelu_fast(float u) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  return 0.5f * u * (1.0f + tanh_fast(k0 * fmaf(k1 * u, u * u, u)));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %2, %1;" : "=r"(r) : "f"(a), "f"(b));
  return r;
}

// Byte offset of element (row, k) in a canonical K-major tile with K columns.
__host__ __device__ __forceinline__ uint32_t canon(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Byte offset of element (row, k) in a canonical K-major tile of 8-bit elements with K columns: core
// matrices of 8 rows x 16 bytes (16 elements), 128 B apart along K, 8-row groups K * 8 bytes apart.
__host__ __device__ __forceinline__ uint32_t canon8(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K * 8) + (k >> 4) * 128 + (row & 7) * 16 + (k & 15));
}

// Two E4M3 values (round to nearest even, saturating to +-448): a at the lower address.
__device__ __forceinline__ uint16_t pack_e4m3(float a, float b) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %2, %1;" : "=h"(r) : "f"(a), "f"(b));
  return r;
}

__device__ __forceinline__ uint32_t pack_f16(float a, float b) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %2, %1;" : "=r"(r) : "f"(a), "f"(b));
  return r;
}

// The 16-bit operand type of the tensor-core GEMM images: FP16 (F16) or BF16.  Both keep FP32
// accumulation; FP16 has three more mantissa bits, BF16 the FP32 exponent range.
template <bool F16>
__device__ __forceinline__ uint32_t pack16(float a, float b) {
  return F16 ? pack_f16(a, b) : pack_bf16(a, b);
}
template <bool F16>
__host__ __device__ constexpr uint32_t idesc16(int M, int N) {
  return F16 ? idesc_f16(M, N) : idesc_bf16(M, N);
}
template <bool F16>
constexpr uint32_t kOnePair = F16 ? 0x3C003C00u : 0x3F803F80u;   // two 1.0 values

// Store 8 consecutive k values (k0 % 8 == 0) of one row as 16-bit operands (one 16-byte store).
template <bool F16>
__device__ __forceinline__ void st_row8(uint8_t *base, int row, int k0, int K, const float *v) {
  uint4 q;
  q.x = pack16<F16>(v[0], v[1]);
  q.y = pack16<F16>(v[2], v[3]);
  q.z = pack16<F16>(v[4], v[5]);
  q.w = pack16<F16>(v[6], v[7]);
  *reinterpret_cast<uint4 *>(base + canon(row, k0, K)) = q;
}


// Instruction descriptor, kind::f16 with an explicit major-ness of A and B (bit 15: A MN-major,
// bit 16: B MN-major).
__host__ __device__ constexpr uint32_t idesc_bf16_major(int M, int N, int a_mn, int b_mn) {
  return idesc_bf16(M, N) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
}
template <bool F16>
__host__ __device__ constexpr uint32_t idesc16_major(int M, int N, int a_mn, int b_mn) {
  return idesc16<F16>(M, N) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
}

}  // namespace tc
}  // namespace tdo
