// Internal declarations shared by the CUDA translation units of libtdo.so (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#define TDO_MAX_LAYERS 8
#define TDO_MAX_N 32

// Device view of the FP32 parameter copy (the flat FP64 theta converted, same order and shapes).
struct DevLayer {
  const float *Wq, *Wk, *Wv, *Wo;   // [d][d], row = input feature
  const float *W1, *b1, *W2, *b2;   // [d][f], [f], [f][d], [d] (null when there is no MLP)
};

struct DevModel {
  int n_sites;     // N
  int d;           // model width
  int heads;       // h
  int dh;          // d / h
  int layers;
  int ffn;         // mlp_ratio * d (0 = no MLP)
  int embed;       // 0 token, 1 conv
  const float *etab;   // embedding table: 4 x d (token) or 64 x d (conv patterns of 3 sites)
  DevLayer L[TDO_MAX_LAYERS];
  const float *Wh, *bh;   // [d][2], [2]
};

// BF16 weights for the tensor-core forward: every matrix stored transposed ([out][in], K-major) in the
// canonical no-swizzle core-matrix layout expected by the tcgen05 shared-memory descriptors.
struct DevModelBF16 {
  const uint16_t *Wqkv[TDO_MAX_LAYERS];   // 3d x d
  const uint16_t *Wo[TDO_MAX_LAYERS];     // d x d
  const uint16_t *W1[TDO_MAX_LAYERS];     // f x d
  const uint16_t *W2[TDO_MAX_LAYERS];     // d x f
  const float *wscale;                    // E4M3 images only: [layers][6] inverse scales (q, k, v, o, w1, w2)
};

// One contribution to an element of a row of Lhat: for the row (s, s') and the connected configuration
// (s ^ lmask, s' ^ rmask) of its pattern, value = tab[2*bit(s, sel_l) + bit(s', sel_r)]
// * (-1)^(popc(s & m1) + popc(s' & m2)); a selector of -1 reads bit 0.
struct ConnContrib {
  double tab[4][2];
  uint32_t m1, m2;
  int sel_l, sel_r;
};
struct ConnPattern {
  uint32_t lmask, rmask;
  int c_begin, c_end;   // contributions [c_begin, c_end)
};

// ------------------------------------------------------------------ launchers (stream-ordered)
// FP32 forward over explicit configurations.
cudaError_t launch_fwd32(const DevModel &m, const uint32_t *sig, const uint32_t *sigp, size_t B,
                         float2 *logrho, int n_sm, cudaStream_t st);
// Metropolis on FP32 forward: n_chains chains in/out, samples optional, accepted counter (device u64);
// diag != 0: chains on |rho(alpha, alpha)| (sig = sigp = alpha, N proposals per sweep).
cudaError_t launch_sample32(const DevModel &m, size_t n_chains, size_t n_sweeps, uint64_t seed,
                            uint64_t counter, uint32_t *sig, uint32_t *sigp, uint32_t *ssig,
                            uint32_t *ssigp, unsigned long long *accepted, int diag, int n_sm, cudaStream_t st);
// A batch of configurations of chains of different lengths, sorted into buckets of equal N: bucket k
// (in tile order) holds count[k] configurations of N = n[k] from sorted position base[k], its tiles
// numbered from tile0[k] (tile0[nb] = all tiles).
struct RaggedTab {
  int nb;
  int n[32];
  long long tile0[33];
  long long base[32];
  long long count[32];
};

// Tensor-core forward and sampler, BF16 operands (the _f16 variants: FP16 operands).
cudaError_t launch_wait_probe(int *err_flag, long long spin, cudaStream_t st);
cudaError_t launch_fwd_bf16(const DevModel &m, const DevModelBF16 &mb, const uint32_t *sig,
                            const uint32_t *sigp, size_t B, float2 *logrho, int *err_flag, int n_sm,
                            cudaStream_t st);
cudaError_t launch_fwd_bf16_f16(const DevModel &m, const DevModelBF16 &mb, const uint32_t *sig,
                                const uint32_t *sigp, size_t B, float2 *logrho, int *err_flag, int n_sm,
                                cudaStream_t st);
bool bf16_supported(const DevModel &m);
// The ragged batch in one persistent launch (next: a device work counter, or null for a static schedule;
// ctas_per_sm_req: 1 or 2, capped by what fits).
cudaError_t launch_fwd_ragged(const DevModel &m, const DevModelBF16 &mb, const uint32_t *ssig, const uint32_t *ssigp,
                              const uint32_t *perm, const RaggedTab &tab, unsigned long long *next, float2 *out,
                              int *err_flag, int n_sm, int ctas_per_sm_req, cudaStream_t st);
cudaError_t launch_fwd_ragged_f16(const DevModel &m, const DevModelBF16 &mb, const uint32_t *ssig,
                                  const uint32_t *ssigp, const uint32_t *perm, const RaggedTab &tab,
                                  unsigned long long *next, float2 *out, int *err_flag, int n_sm, int ctas_per_sm_req,
                                  cudaStream_t st);
// Bucketing of a ragged batch: counts[N] for N in 1..32 (counts[0]: entries outside 1..32); then the
// scatter of sig, sigp into ssig, ssigp at cursor[N]++ (cursor preset to each bucket's base), perm = the
// source position; and out[perm[j]] = in[j] for the FP32 path's per-bucket results.
cudaError_t launch_ragged_hist(const int32_t *n_sites, size_t B, unsigned long long *counts, cudaStream_t st);
cudaError_t launch_ragged_scatter(const int32_t *n_sites, const uint32_t *sig, const uint32_t *sigp, size_t B,
                                  unsigned long long *cursor, uint32_t *ssig, uint32_t *ssigp, uint32_t *perm,
                                  cudaStream_t st);
cudaError_t launch_unpermute(const float2 *in, const uint32_t *perm, size_t B, float2 *out, cudaStream_t st);
cudaError_t launch_sample_bf16(const DevModel &m, const DevModelBF16 &mb, size_t n_chains,
                               size_t n_sweeps, uint64_t seed, uint64_t counter, uint32_t *sig,
                               uint32_t *sigp, uint32_t *ssig, uint32_t *ssigp,
                               unsigned long long *accepted, int *err_flag, int diag, int n_sm, cudaStream_t st,
                               const uint64_t *dcounter = nullptr);
cudaError_t launch_sample_bf16_f16(const DevModel &m, const DevModelBF16 &mb, size_t n_chains,
                                   size_t n_sweeps, uint64_t seed, uint64_t counter, uint32_t *sig,
                                   uint32_t *sigp, uint32_t *ssig, uint32_t *ssigp,
                                   unsigned long long *accepted, int *err_flag, int diag, int n_sm, cudaStream_t st,
                                   const uint64_t *dcounter = nullptr);

// Mixed-state observables.  Rows of the magnetisation estimator: sample s -> (alpha, alpha), then
// (alpha, alpha ^ e_i) for i < N, at rows s (N + 1) + j.
cudaError_t launch_obs_rows(const uint32_t *alpha, size_t Ns, int n, uint32_t *rs, uint32_t *rp, cudaStream_t st);
// From log rho of those rows: local[s] = (s, A~x, A~y, A~z) as complex pairs (may be NULL), and
// out[0..5] = sum s, Re/Im sum s A~x, Re/Im sum s A~y, sum s A~z (A~z is real; FP64, fixed order;
// part: 256 blocks x 6 doubles).
cudaError_t launch_obs_reduce(const uint32_t *alpha, size_t Ns, int n, const float2 *lr, double *local,
                              double *part, double *out, cudaStream_t st);
// Rows of the purity estimator: sample s -> (sigma, sigma'), (sigma, sigma), (sigma', sigma') at 3 s + j.
cudaError_t launch_pur_rows(const uint32_t *sig, const uint32_t *sigp, size_t Ns, uint32_t *rs, uint32_t *rp,
                            cudaStream_t st);
// out[0] = sum_s Re rho(s,s) rho(s',s') / |rho(s,s')|^2, out[1] = sum of squares (FP64, fixed order).
cudaError_t launch_pur_reduce(const float2 *lr, size_t Ns, double *part, double *out, cudaStream_t st);

// Connections: count[s], entries [s*M + j].
cudaError_t launch_connections(const ConnPattern *pat, int n_pat, const ConnContrib *con,
                               const uint32_t *sig, const uint32_t *sigp, size_t Ns, int32_t *count,
                               uint32_t *csig, uint32_t *csigp, float2 *ccoef, cudaStream_t st);
// Exclusive scan of count[Ns] -> offs[Ns+1] (single block, deterministic).
cudaError_t launch_scan(const int32_t *count, size_t Ns, int64_t *offs, cudaStream_t st);
// Compact [s*M + j] entries into flat rows at offs[s] + j.
cudaError_t launch_compact(const int32_t *count, const int64_t *offs, size_t Ns, int M,
                           const uint32_t *csig, const uint32_t *csigp, const float2 *ccoef,
                           uint32_t *fsig, uint32_t *fsigp, float2 *fcoef, cudaStream_t st);
// Gradient cotangents per flat row: c = scale * conj(L_loc) coef rho_y/rho_x, minus scale*cost on row 0.
cudaError_t launch_cotangent(const int64_t *offs, size_t Ns, const float2 *fcoef, const float2 *flogrho,
                             const double2 *lloc, const double *cost_stats, float2 *cot,
                             cudaStream_t st);
// FP64 reductions.
// scale (device pointer, may be NULL): every sum is multiplied by *scale (an exact power of two).
cudaError_t launch_reduce_copies(const float *acc, int n_copies, size_t stride, size_t P, double *out,
                                 int accumulate, cudaStream_t st, const float *scale = nullptr);
cudaError_t launch_f64_to_f32(const double *src, float *dst, size_t n, cudaStream_t st);
// 16-bit weight packing (BF16 operands; the _f16 variant packs FP16 operands).
cudaError_t launch_pack_bf16(const DevModel &m, uint16_t *dst, DevModelBF16 *views, cudaStream_t st);
cudaError_t launch_pack_bf16_f16(const DevModel &m, uint16_t *dst, DevModelBF16 *views, cudaStream_t st);

// E4M3 (FP8) forward for evaluation: the same kernels with 8-bit operand images, per-matrix weight scales and
// per-tile activation scales; dst of the packing holds f8_packed_bytes(m) bytes.
size_t f8_packed_bytes(const DevModel &m);
cudaError_t launch_pack_bf16_f8(const DevModel &m, uint16_t *dst, DevModelBF16 *views, cudaStream_t st);
cudaError_t launch_fwd_bf16_f8(const DevModel &m, const DevModelBF16 &mb, const uint32_t *sig, const uint32_t *sigp,
                               size_t B, float2 *logrho, int *err_flag, int n_sm, cudaStream_t st);
cudaError_t launch_fwd_ragged_f8(const DevModel &m, const DevModelBF16 &mb, const uint32_t *ssig,
                                 const uint32_t *ssigp, const uint32_t *perm, const RaggedTab &tab,
                                 unsigned long long *next, float2 *out, int *err_flag, int n_sm, int ctas_per_sm_req,
                                 cudaStream_t st);
cudaError_t launch_sample_bf16_f8(const DevModel &m, const DevModelBF16 &mb, size_t n_chains, size_t n_sweeps,
                                  uint64_t seed, uint64_t counter, uint32_t *sig, uint32_t *sigp, uint32_t *ssig,
                                  uint32_t *ssigp, unsigned long long *accepted, int *err_flag, int diag, int n_sm,
                                  cudaStream_t st, const uint64_t *dcounter = nullptr);

// gate (device int, may be NULL): the update is skipped when *gate is 0 (a replayed step whose solve failed).
cudaError_t launch_axpy_update(double *theta, const double *delta, double lr, size_t P, cudaStream_t st,
                               const int *gate = nullptr);
// Adam step t (>= 1) on the direction delta with first and second moments m, v (FP64 [P], updated).
// dc (device, may be NULL): the bias corrections 1 - b1^t, 1 - b2^t of the step, in place of t's.
cudaError_t launch_adam_update(double *theta, const double *delta, double *m, double *v, size_t P, long long t,
                               double lr, double b1, double b2, double eps, cudaStream_t st,
                               const int *gate = nullptr, const double *dc = nullptr);
// *ok = the solve's outcome slot is 0 or 1, *nonfinite is 0 and *err (may be NULL) is 0.
cudaError_t launch_step_gate(const double *outcome, const int *nonfinite, const int *err, int *ok, cudaStream_t st);

