// Host side of libtdo.so: the C ABI of include/tdo.h.  Owns the context (problem, parameters, device
// workspace), turns the problem statement into Lindbladian connection rules, stages host buffers and
// sequences the kernels of each call on the context's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <map>
#include <string>
#include <utility>
#include <vector>
#include <array>

#include "../../include/tdo.h"
#include "tdo_internal.cuh"

// launchers defined in the kernel translation units
cudaError_t launch_lloc(const int64_t *offs, size_t Ns, const float2 *fcoef, const float2 *flogrho,
                        double2 *lloc, double *l2, double *stats, int *nonfinite, cudaStream_t st);
cudaError_t launch_conv_table_k(int d, int c1, const float *Wc1, const float *bc1, const float *Wc2,
                                const float *bc2, float *table, cudaStream_t st);
size_t bwd32_scratch_floats(const DevModel &m, int grid);
int bwd32_grid(const DevModel &m, size_t B, int mode, int n_sm);
cudaError_t launch_bwd32_impl(const DevModel &m, int mode, const uint32_t *sig, const uint32_t *sigp,
                              size_t B, const float2 *cot, float *gacc, int n_copies, size_t g_stride,
                              float *O, uint16_t *O16, const float2 *oref, size_t P, size_t ldo,
                              const long long *flat_offsets, float *scratch, float *dtab, int grid, cudaStream_t st);
cudaError_t launch_oref(const float *O32, int n, size_t P, float *oref, cudaStream_t st);
cudaError_t launch_conv_vjp(int d, int c1, const float *Wc1, const float *bc1, const float *Wc2, const float *bc2,
                            const float *dT, int nsets, int ncopy, int mode, float *g, float *O, uint16_t *O16,
                            const float2 *oref, size_t ldo, long long o_wc1, long long o_bc1, long long o_wc2,
                            long long o_bc2, cudaStream_t st);
size_t sr_work_doubles(size_t Ns, size_t P);
cudaError_t sr_apply_impl(const uint32_t *O, size_t Ns, size_t P, size_t ldo, const double *v, double shift, double *Ap,
                          double *work, int product_mode, int *err, int *shape, cudaStream_t st);
cudaError_t measure_fma_peak(int fp64, int n_sm, cudaStream_t st, double *tflops);
cudaError_t sr_cg_impl(const void *O, int o_bf16, size_t Ns, size_t P, size_t ldo, const double *rhs, const double *x0,
                       double shift, double tol, int max_iter, double *x, double *work, int n_sm, int *iters,
                       double *resid, int *outcome, double *last_pap, long long *launches, cudaEvent_t *mv_ev,
                       int mv_cap, int *mv_used, int product_mode, int *err, int *shape, cudaStream_t st);
cudaError_t launch_params_f32(const double *theta, size_t P, const long long *tab, int n_tensors,
                              float *dst, cudaStream_t st);
cudaError_t sr_cg_capture(const void *O, int o_bf16, size_t Ns, size_t P, size_t ldo, const double *rhs, double *x,
                          double shift, double tol, int max_iter, double *work, int product_mode, const int *warm,
                          int *err, int *shape, cudaStream_t st);
cudaError_t sr_cg_result(double *work, size_t Ns, size_t P, int *iters, double *resid, int *outcome,
                         double *last_pap, int *restarted, cudaStream_t st);
const double *sr_outcome_slot(double *work, size_t Ns, size_t P);
size_t bf16_packed_bytes(const DevModel &m);
struct BwdTcLayer {
  const uint8_t *w1t[2], *w2r[2], *w1r[2];
  const uint8_t *wqkvT, *wor, *wqkvr;
};
struct BwdTcBuffers {
  uint8_t *x, *xmid, *dqkv;
  float *h, *f, *dF, *dxa, *dxb;
  size_t tiles;
  float *cscale;   // [2]: cotangent scale and its inverse (VJP mode)
};
size_t bwdtc_packed_bytes(const DevModel &m);
bool bwdtc_supported(const DevModel &m);
cudaError_t launch_pack_bwdtc(const DevModel &m, uint8_t *dst, BwdTcLayer *views, cudaStream_t st);
cudaError_t launch_pack_bwdtc_f16(const DevModel &m, uint8_t *dst, BwdTcLayer *views, cudaStream_t st);
struct BwdTcJac {
  float *o32;
  uint16_t *o16;
  const float2 *oref;
  size_t ldo, nvirt;
};
bool bwdtc_jac_supported(const DevModel &m);
cudaError_t launch_jac_virtual(const uint32_t *sig, const uint32_t *sigp, size_t Ns, uint32_t *vs, uint32_t *vp,
                               float2 *vc, cudaStream_t st);
cudaError_t launch_bwdtc(const DevModel &m, const DevModelBF16 &mb, const BwdTcLayer *views, const BwdTcBuffers &bf,
                         const uint32_t *sig, const uint32_t *sigp, size_t B, const float2 *cot, float *gacc,
                         size_t g_stride, const long long *fo, int *err, int n_sm, cudaStream_t st,
                         const BwdTcJac *jac = nullptr, const int64_t *dB = nullptr);
cudaError_t launch_bwdtc_f16(const DevModel &m, const DevModelBF16 &mb, const BwdTcLayer *views,
                             const BwdTcBuffers &bf, const uint32_t *sig, const uint32_t *sigp, size_t B,
                             const float2 *cot, float *gacc, size_t g_stride, const long long *fo, int *err, int n_sm,
                             cudaStream_t st, const BwdTcJac *jac = nullptr, const int64_t *dB = nullptr);
cudaError_t launch_fwd_bf16_store(const DevModel &m, const DevModelBF16 &mb, const uint32_t *sig,
                                  const uint32_t *sigp, size_t B, float2 *logrho, int *err_flag, int n_sm,
                                  cudaStream_t st, uint8_t *x_img, uint8_t *xmid_img, float *h, float *f,
                                  size_t tiles, const int64_t *dB = nullptr);
cudaError_t launch_fwd_bf16_store_f16(const DevModel &m, const DevModelBF16 &mb, const uint32_t *sig,
                                      const uint32_t *sigp, size_t B, float2 *logrho, int *err_flag, int n_sm,
                                      cudaStream_t st, uint8_t *x_img, uint8_t *xmid_img, float *h, float *f,
                                      size_t tiles, const int64_t *dB = nullptr);
// A tensor-core launcher of the context's operand type: fn (BF16) or fn_f16 (FP16).
#define TC_LAUNCH(c, fn, ...) ((c)->f16 ? fn##_f16(__VA_ARGS__) : fn(__VA_ARGS__))
// Evaluation-only launches (no parked activations): the E4M3 kernels and weights in FP8 contexts.
#define EVAL_LAUNCH(c, fn, ...) \
  ((c)->f8 ? fn##_f8((c)->dm, (c)->dmb8, __VA_ARGS__) : TC_LAUNCH(c, fn, (c)->dm, (c)->dmb, __VA_ARGS__))

namespace {

thread_local std::string g_create_error;

// Bumped by every (re)allocation or release of a device buffer: a recorded step graph holds buffer
// addresses, so it is recorded again when this has moved since.
unsigned long long g_buf_gen = 0;

struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    ++g_buf_gen;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    size_t want = need + need / 4 + 256;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) { p = nullptr; return e; }
    bytes = want;
    return cudaSuccess;
  }
  template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
  void release() { if (p) { cudaFree(p); ++g_buf_gen; } p = nullptr; bytes = 0; }
};

// Per-step values of a replayed step graph, read by its kernels from device memory: the sampler's counter,
// Adam's bias corrections, whether the solve starts from the previous solution (and may restart), and the
// update's gate (written by the graph).
struct StepDev {
  uint64_t counter;
  double c1, c2;
  int warm, ok;
};

struct TensorLoc { long long flat, pad, size; };

// G_SR_MV (the one-pass S' v kernel alone) is a subset of G_SR and is left out of "all".
enum Group { G_FWD = 0, G_SAMPLE, G_BWD_VJP, G_BWD_JAC, G_CONN, G_LLOC, G_SR, G_UPDATE, G_SR_MV, G_COUNT };
const char *kGroupNames[G_COUNT] = {"fwd", "sample", "bwd_vjp", "bwd_jac", "conn", "lloc", "sr", "update", "sr_mv"};

struct TimingRec { int group; cudaEvent_t a, b; long long launches; };

}  // namespace

struct tdo_ctx {
  int device = 0;
  int n_sm = 0;
  cudaStream_t stream = nullptr;
  tdo_model model{};
  int n = 0;
  size_t P = 0, P_pad = 0;
  std::vector<TensorLoc> tensors;          // in theta order
  long long flat_offsets[3 + 8 * TDO_MAX_LAYERS];   // FlatOffsets layout of the backward kernel
  // connection rules
  int n_pat = 0;
  DBuf d_pat, d_con;
  // parameters
  DBuf theta64, theta32, etab, tensor_tab, wbf16, errflag, wbwd, wf8;
  DBuf dtab;   // conv embedding: per-pattern table gradients
  DBuf oref, oref_scratch;   // BF16-stored O for SR: per-parameter shift and its FP32 sample
  DBuf jac_vs, jac_vp, jac_vc, jac_lr;   // tensor-core log-derivatives: virtual configurations
  DBuf obs_rs, obs_rp, obs_lr, obs_part, obs_out, obs_local;   // observables and purity
  DevModel dm{};
  DevModelBF16 dmb{};
  DevModelBF16 dmb8{};                 // views of the E4M3 weights (TDO_FP8)
  bool tc = false;                     // tensor-core path (TDO_BF16, TDO_FP16 or TDO_FP8 contexts)
  bool f16 = false;                    // its operands are FP16 (TDO_FP16; TDO_FP8's gradient) rather than BF16
  bool f8 = false;                     // TDO_FP8: evaluation on E4M3 operands (wf8, dmb8)
  bool tc_bwd = false;                 // tensor-core gradient (tensor-core contexts whose shape it supports)
  BwdTcLayer bwl[TDO_MAX_LAYERS];
  DBuf act_x, act_xmid, act_h, act_f, act_dF, act_dxa, act_dxb, act_dqkv;
  // workspace
  DBuf stage_in[4], stage_out;
  DBuf conn_cnt, conn_sig, conn_sigp, conn_coef, offs, fsig, fsigp, fcoef, flr, lloc, l2, stats,
      nonfinite, cot, gacc, scratch, grad, Obuf, srwork, delta, acc_u64, cscale;
  std::string err;
  double sr_tol = 1e-5;   // relative residual (the default of the CG that NetKet's SR preconditioner calls)
  int sr_max_iter = 100;
  // optimiser applied to the SR direction: TDO_OPT_SGD (theta -= lr delta) or TDO_OPT_ADAM
  int opt = TDO_OPT_SGD;
  double adam_b1 = 0.9, adam_b2 = 0.999, adam_eps = 1e-8;
  long long adam_t = 0;
  DBuf adam_m, adam_v;
  // ragged batches: bucket counts, cursors, sorted configurations, permutation, work counter, FP32 results
  DBuf rg_counts, rg_cursor, rg_ssig, rg_ssigp, rg_perm, rg_next, rg_tmp, rg_n;
  // autotuned launch shape of the ragged forward per mix of chain lengths (bit N-1 set for each N present):
  // (CTAs per SM, descending-N tile order, dynamic work counter)
  std::map<uint32_t, std::array<int, 3>> rg_tuned;
  bool have_delta = false;
  int last_sr_iters = 0;
  double last_sr_resid = 0;
  int last_sr_outcome = 0;      // 0 max_iter reached, 1 converged, 2 breakdown, 3 non-finite
  double last_sr_pap = 0;       // last p . S'p of the solve
  int last_sr_restarts = 0;     // 1 when the warm-started solve failed and was rerun from x = 0
  int sr_product = TDO_SR_PRODUCT_TWO_PASS;   // or TDO_SR_PRODUCT_ONE_PASS (where the storage allows it)
  int last_sr_shape[3] = {0, 0, 0};   // one pass used, cluster size, clusters (last solve)
  // whole-step CUDA graph (tdo_set_step_graph): the recorded step, the arguments and settings it was
  // recorded for, and its per-step values (uploaded from pinned host memory before each launch)
  bool step_graph = false;
  bool capturing = false;              // a recording is in progress: no timing events, no host reads
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t gstream = nullptr;      // the graph's own stream (a legacy or per-thread default stream cannot
  cudaEvent_t gevent = nullptr;        // be captured), ordered after and before the context's stream
  std::vector<uint64_t> gkey;
  DBuf gstep;                          // StepDev
  StepDev *gstep_host = nullptr;       // pinned
  long long graph_captures = 0, graph_replays = 0;
  // kernel timing (tdo_timing)
  bool timing = false;
  std::vector<TimingRec> trec;
  std::vector<cudaEvent_t> epool;
};

// Brackets the launches of one kernel group with CUDA events when timing is enabled.
struct Timed {
  tdo_ctx *c;
  int idx = -1;
  Timed(tdo_ctx *ctx, int group) : c(ctx) {
    if (!c->timing || c->capturing) return;
    cudaEvent_t a, b;
    if (c->epool.size() >= 2) { a = c->epool.back(); c->epool.pop_back(); b = c->epool.back(); c->epool.pop_back(); }
    else { cudaEventCreate(&a); cudaEventCreate(&b); }
    cudaEventRecord(a, c->stream);
    c->trec.push_back({group, a, b, 0});
    idx = (int)c->trec.size() - 1;
  }
  void done(long long launches) {
    if (idx < 0) return;
    cudaEventRecord(c->trec[idx].b, c->stream);
    c->trec[idx].launches = launches;
    idx = -1;
  }
  ~Timed() { done(1); }
};

static tdo_status fail(tdo_ctx *c, tdo_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_create_error = buf;
  return s;
}

#define CU(ctx, call)                                                                          \
  do {                                                                                         \
    cudaError_t _e = (call);                                                                   \
    if (_e != cudaSuccess)                                                                     \
      return fail(ctx, _e == cudaErrorMemoryAllocation ? TDO_ENOMEM : TDO_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(_e), __FILE__, __LINE__);                          \
  } while (0)

#define TRY(x)                       \
  do {                               \
    tdo_status _s = (x);             \
    if (_s != TDO_OK) return _s;     \
  } while (0)

// ----------------------------------------------------------------------------- parameter layout
static bool model_valid(const tdo_model *m, std::string *why) {
  if (!m) { *why = "model is NULL"; return false; }
  if (m->d_model != 16 && m->d_model != 32 && m->d_model != 64) { *why = "d_model must be 16, 32 or 64"; return false; }
  if (m->n_heads < 1 || m->d_model % m->n_heads) { *why = "n_heads must divide d_model"; return false; }
  const int dh = m->d_model / m->n_heads;
  if (dh > 16 || dh < 1) { *why = "head dimension must be <= 16"; return false; }
  if (m->n_layers < 1 || m->n_layers > TDO_MAX_LAYERS) { *why = "n_layers must be 1..8"; return false; }
  if (m->mlp_ratio < 0 || m->mlp_ratio > 4) { *why = "mlp_ratio must be 0..4"; return false; }
  if (m->embed != TDO_EMBED_TOKEN && m->embed != TDO_EMBED_CONV) { *why = "unknown embedding"; return false; }
  if (m->embed == TDO_EMBED_CONV && (m->conv_channels < 1 || m->conv_channels > 256)) { *why = "conv_channels must be 1..256"; return false; }
  if (m->precision != TDO_FP32 && m->precision != TDO_BF16 && m->precision != TDO_FP16 && m->precision != TDO_FP8) {
    *why = "unknown precision";
    return false;
  }
  return true;
}

static std::vector<long long> tensor_sizes(const tdo_model *m) {
  const long long d = m->d_model, f = (long long)m->mlp_ratio * d;
  std::vector<long long> s;
  if (m->embed == TDO_EMBED_TOKEN) s.push_back(4 * d);
  else { const long long c1 = m->conv_channels; s.push_back(4 * c1); s.push_back(c1); s.push_back(2 * c1 * d); s.push_back(d); }
  for (int l = 0; l < m->n_layers; ++l) {
    for (int i = 0; i < 4; ++i) s.push_back(d * d);
    if (f > 0) { s.push_back(d * f); s.push_back(f); s.push_back(f * d); s.push_back(d); }
  }
  s.push_back(2 * d);
  s.push_back(2);
  return s;
}

extern "C" size_t tdo_model_num_params(const tdo_model *model) {
  std::string why;
  if (!model_valid(model, &why)) return 0;
  size_t p = 0;
  for (long long v : tensor_sizes(model)) p += (size_t)v;
  return p;
}

// ----------------------------------------------------------------------------- connection rules
// Builds, for every distinct pair of flip masks (left, right), the contributions of Eq. VecLin:
//   -i H (x) I      : Pauli string P, coefficient c: <s|P|s^x> = (-i)^{#Y} (-1)^{popc(s & yz)}
//   +i I (x) H^T    : <s'^x|P|s'> = (+i)^{#Y} (-1)^{popc(s' & yz)}
//   g L (x) L^*     : g L[s_k][s_k^f] conj(L[s'_k][s'_k^f'])
//   -g/2 L^+L (x) I : -g/2 (L^+L)[s_k][s_k^f];   -g/2 I (x) L^T L^* : -g/2 (L^+L)[s'_k^f'][s'_k]
static tdo_status build_rules(tdo_ctx *c, const tdo_problem *p) {
  typedef std::complex<double> cd;
  const int n = p->n_sites;
  std::map<std::pair<uint32_t, uint32_t>, std::vector<ConnContrib>> groups;
  groups[{0u, 0u}];   // the diagonal is always present
  auto add = [&](uint32_t lm, uint32_t rm, const cd tab[4], uint32_t m1, uint32_t m2, int sl, int sr) {
    bool any = false;
    for (int i = 0; i < 4; ++i) any |= (tab[i] != cd(0, 0));
    if (!any) return;
    ConnContrib cc;
    for (int i = 0; i < 4; ++i) { cc.tab[i][0] = tab[i].real(); cc.tab[i][1] = tab[i].imag(); }
    cc.m1 = m1; cc.m2 = m2; cc.sel_l = sl; cc.sel_r = sr;
    groups[{lm, rm}].push_back(cc);
  };
  // Pauli product on one site: a * b = phase * r (X Y = i Z and cyclic, P P = I)
  auto pauli_index = [](char q) { return q == 'I' ? 0 : q == 'X' ? 1 : q == 'Y' ? 2 : q == 'Z' ? 3 : -1; };
  for (int t = 0; t < p->n_terms; ++t) {
    int site_op[2] = {-1, -1}, op_idx[2] = {0, 0};
    cd phase(1, 0);
    int nsites = 0;
    for (int j = 0; j < 2; ++j) {
      const int site = p->term_sites[2 * t + j];
      if (site < 0) continue;
      if (site >= n) return fail(c, TDO_EINVAL, "term %d: site %d out of range", t, site);
      const int q = pauli_index(p->term_paulis[2 * t + j]);
      if (q < 0) return fail(c, TDO_EUNSUPPORTED, "term %d: Pauli '%c' not in {I,X,Y,Z}", t, p->term_paulis[2 * t + j]);
      int k = 0;
      while (k < nsites && site_op[k] != site) ++k;
      if (k == nsites) { site_op[nsites] = site; op_idx[nsites] = q; ++nsites; continue; }
      const int a = op_idx[k], b = q;   // existing operator times the new one
      if (a == 0) op_idx[k] = b;
      else if (b == 0 || a == b) op_idx[k] = (a == b) ? 0 : a;
      else {
        const int r = 6 - a - b;   // the third Pauli
        const bool cyclic = (b == a % 3 + 1);   // X->Y, Y->Z, Z->X
        op_idx[k] = r;
        phase *= cyclic ? cd(0, 1) : cd(0, -1);
      }
    }
    uint32_t xm = 0, yzm = 0;
    int ny = 0;
    for (int k = 0; k < nsites; ++k) {
      const uint32_t bit = 1u << site_op[k];
      if (op_idx[k] == 1) xm |= bit;
      if (op_idx[k] == 2) { xm |= bit; yzm |= bit; ++ny; }
      if (op_idx[k] == 3) yzm |= bit;
    }
    const cd coef = p->term_coef[t] * phase;
    if (coef == cd(0, 0)) continue;
    cd ph_l(1, 0), ph_r(1, 0);
    for (int k = 0; k < ny; ++k) { ph_l *= cd(0, -1); ph_r *= cd(0, 1); }
    const cd vl = cd(0, -1) * coef * ph_l, vr = cd(0, 1) * coef * ph_r;
    const cd tl[4] = {vl, vl, vl, vl}, tr[4] = {vr, vr, vr, vr};
    add(xm, 0u, tl, yzm, 0u, -1, -1);
    add(0u, xm, tr, 0u, yzm, -1, -1);
  }
  for (int q = 0; q < p->n_jumps; ++q) {
    const int k = p->jump_site[q];
    if (k < 0 || k >= n) return fail(c, TDO_EINVAL, "jump %d: site %d out of range", q, k);
    const double g = p->jump_rate[q];
    if (!(g >= 0.0)) return fail(c, TDO_EINVAL, "jump %d: negative rate", q);
    cd L[2][2], LdL[2][2];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) L[a][b] = cd(p->jump_op[q * 8 + (a * 2 + b) * 2], p->jump_op[q * 8 + (a * 2 + b) * 2 + 1]);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) LdL[a][b] = std::conj(L[0][a]) * L[0][b] + std::conj(L[1][a]) * L[1][b];
    const uint32_t bit = 1u << k;
    for (int f = 0; f < 2; ++f)
      for (int fp = 0; fp < 2; ++fp) {
        cd tab[4];
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) tab[2 * a + b] = g * L[a][a ^ f] * std::conj(L[b][b ^ fp]);
        add(f ? bit : 0u, fp ? bit : 0u, tab, 0u, 0u, k, k);
      }
    for (int f = 0; f < 2; ++f) {
      cd tl[4], tr[4];
      for (int a = 0; a < 2; ++a) {
        tl[2 * a] = tl[2 * a + 1] = -0.5 * g * LdL[a][a ^ f];
        tr[a] = tr[2 + a] = -0.5 * g * LdL[a ^ f][a];
      }
      // left: selector on sigma_k only (b ignored, tab[2a+0] used); right: selector on sigma'_k only
      cd tl4[4] = {tl[0], tl[0], tl[2], tl[2]};
      cd tr4[4] = {tr[0], tr[1], tr[0], tr[1]};
      add(f ? bit : 0u, 0u, tl4, 0u, 0u, k, -1);
      add(0u, f ? bit : 0u, tr4, 0u, 0u, -1, k);
    }
  }
  std::vector<ConnPattern> pats;
  std::vector<ConnContrib> cons;
  // diagonal first, then the others in (left mask, right mask) order
  auto push = [&](const std::pair<uint32_t, uint32_t> &key, const std::vector<ConnContrib> &v) {
    ConnPattern P;
    P.lmask = key.first; P.rmask = key.second;
    P.c_begin = (int)cons.size();
    cons.insert(cons.end(), v.begin(), v.end());
    P.c_end = (int)cons.size();
    pats.push_back(P);
  };
  push({0u, 0u}, groups[{0u, 0u}]);
  for (auto &kv : groups)
    if (!(kv.first.first == 0u && kv.first.second == 0u)) push(kv.first, kv.second);
  c->n_pat = (int)pats.size();
  CU(c, c->d_pat.ensure(sizeof(ConnPattern) * pats.size()));
  CU(c, c->d_con.ensure(sizeof(ConnContrib) * std::max<size_t>(cons.size(), 1)));
  CU(c, cudaMemcpy(c->d_pat.p, pats.data(), sizeof(ConnPattern) * pats.size(), cudaMemcpyHostToDevice));
  if (!cons.empty())
    CU(c, cudaMemcpy(c->d_con.p, cons.data(), sizeof(ConnContrib) * cons.size(), cudaMemcpyHostToDevice));
  return TDO_OK;
}

// ----------------------------------------------------------------------------- parameters
static tdo_status layout_params(tdo_ctx *c) {
  const tdo_model *m = &c->model;
  std::vector<long long> sz = tensor_sizes(m);
  long long flat = 0, pad = 0;
  c->tensors.clear();
  for (long long s : sz) {
    c->tensors.push_back({flat, pad, s});
    flat += s;
    pad += (s + 15) / 16 * 16;
  }
  c->P = (size_t)flat;
  c->P_pad = (size_t)pad;
  // flat offsets in the backward kernel's FlatOffsets order
  for (auto &v : c->flat_offsets) v = 0;
  int t = 0;
  if (m->embed == TDO_EMBED_TOKEN) c->flat_offsets[0] = c->tensors[t++].flat;
  else { c->flat_offsets[0] = c->tensors[t].flat; t += 4; }
  long long *Wq = c->flat_offsets + 1, *Wk = Wq + TDO_MAX_LAYERS, *Wv = Wk + TDO_MAX_LAYERS, *Wo = Wv + TDO_MAX_LAYERS,
            *W1 = Wo + TDO_MAX_LAYERS, *b1 = W1 + TDO_MAX_LAYERS, *W2 = b1 + TDO_MAX_LAYERS, *b2 = W2 + TDO_MAX_LAYERS;
  for (int l = 0; l < m->n_layers; ++l) {
    Wq[l] = c->tensors[t++].flat; Wk[l] = c->tensors[t++].flat; Wv[l] = c->tensors[t++].flat; Wo[l] = c->tensors[t++].flat;
    if (m->mlp_ratio > 0) { W1[l] = c->tensors[t++].flat; b1[l] = c->tensors[t++].flat; W2[l] = c->tensors[t++].flat; b2[l] = c->tensors[t++].flat; }
  }
  c->flat_offsets[1 + 8 * TDO_MAX_LAYERS] = c->tensors[t++].flat;   // Wh
  c->flat_offsets[2 + 8 * TDO_MAX_LAYERS] = c->tensors[t++].flat;   // bh
  return TDO_OK;
}

static bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device copy of an input: the pointer itself if it is device memory, else a staged copy.
static tdo_status stage_in(tdo_ctx *c, int slot, const void *p, size_t bytes, const void **out, bool *host) {
  *host = false;
  if (!p || bytes == 0 || is_device_ptr(p)) { *out = p; return TDO_OK; }
  *host = true;
  CU(c, c->stage_in[slot].ensure(bytes));
  CU(c, cudaMemcpyAsync(c->stage_in[slot].p, p, bytes, cudaMemcpyHostToDevice, c->stream));
  *out = c->stage_in[slot].p;
  return TDO_OK;
}

// Refresh the FP32 parameter copy (and the conv embedding table) from the FP64 master.
static tdo_status refresh_params(tdo_ctx *c) {
  const tdo_model *m = &c->model;
  CU(c, launch_params_f32(c->theta64.as<double>(), c->P, c->tensor_tab.as<long long>(), (int)c->tensors.size(),
                          c->theta32.as<float>(), c->stream));
  if (m->embed == TDO_EMBED_CONV) {
    const float *b = c->theta32.as<float>();
    CU(c, launch_conv_table_k(m->d_model, m->conv_channels, b + c->tensors[0].pad, b + c->tensors[1].pad,
                              b + c->tensors[2].pad, b + c->tensors[3].pad, c->etab.as<float>(), c->stream));
  }
  if (c->tc) CU(c, TC_LAUNCH(c, launch_pack_bf16, c->dm, c->wbf16.as<uint16_t>(), &c->dmb, c->stream));
  if (c->f8) CU(c, launch_pack_bf16_f8(c->dm, c->wf8.as<uint16_t>(), &c->dmb8, c->stream));
  if (c->tc_bwd) CU(c, TC_LAUNCH(c, launch_pack_bwdtc, c->dm, c->wbwd.as<uint8_t>(), c->bwl, c->stream));
  return TDO_OK;
}

// Reports (and clears) a timeout flagged by a tensor-core kernel's bounded waits.
static tdo_status check_err_flag(tdo_ctx *c) {
  if (!c->tc || c->capturing) return TDO_OK;   // a recording step graph reads the flag after its launch
  int f = 0;
  CU(c, cudaMemcpyAsync(&f, c->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  if (f) {
    CU(c, cudaMemsetAsync(c->errflag.p, 0, sizeof(int), c->stream));
    return fail(c, TDO_ETIMEOUT, "a tensor-core kernel's bounded wait gave up (results of that launch are invalid)");
  }
  return TDO_OK;
}

static void build_devmodel(tdo_ctx *c) {
  const tdo_model *m = &c->model;
  const float *b = c->theta32.as<float>();
  DevModel &d = c->dm;
  memset(&d, 0, sizeof(d));
  d.n_sites = c->n;
  d.d = m->d_model;
  d.heads = m->n_heads;
  d.dh = m->d_model / m->n_heads;
  d.layers = m->n_layers;
  d.ffn = m->mlp_ratio * m->d_model;
  d.embed = m->embed;
  int t = 0;
  if (m->embed == TDO_EMBED_TOKEN) d.etab = b + c->tensors[t++].pad;
  else { d.etab = c->etab.as<float>(); t += 4; }
  for (int l = 0; l < m->n_layers; ++l) {
    d.L[l].Wq = b + c->tensors[t++].pad;
    d.L[l].Wk = b + c->tensors[t++].pad;
    d.L[l].Wv = b + c->tensors[t++].pad;
    d.L[l].Wo = b + c->tensors[t++].pad;
    if (m->mlp_ratio > 0) {
      d.L[l].W1 = b + c->tensors[t++].pad;
      d.L[l].b1 = b + c->tensors[t++].pad;
      d.L[l].W2 = b + c->tensors[t++].pad;
      d.L[l].b2 = b + c->tensors[t++].pad;
    }
  }
  d.Wh = b + c->tensors[t++].pad;
  d.bh = b + c->tensors[t++].pad;
}

// ----------------------------------------------------------------------------- ABI
extern "C" const char *tdo_last_error(const tdo_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

extern "C" tdo_status tdo_create(const tdo_problem *problem, const tdo_model *model, const double *theta,
                                 size_t n_theta, void *stream, tdo_ctx **out) {
  g_create_error.clear();
  if (!out) return fail(nullptr, TDO_EINVAL, "out is NULL");
  *out = nullptr;
  if (!problem) return fail(nullptr, TDO_EINVAL, "problem is NULL");
  std::string why;
  if (!model_valid(model, &why)) return fail(nullptr, TDO_EINVAL, "invalid model: %s", why.c_str());
  if (problem->n_sites < 1) return fail(nullptr, TDO_EINVAL, "n_sites must be >= 1");
  if (problem->n_sites > TDO_MAX_N) return fail(nullptr, TDO_EUNSUPPORTED, "n_sites %d > 32", problem->n_sites);
  if (problem->n_terms < 0 || problem->n_jumps < 0) return fail(nullptr, TDO_EINVAL, "negative term count");
  if ((problem->n_terms > 0 && (!problem->term_sites || !problem->term_paulis || !problem->term_coef)) ||
      (problem->n_jumps > 0 && (!problem->jump_site || !problem->jump_op || !problem->jump_rate)))
    return fail(nullptr, TDO_EINVAL, "problem arrays are NULL");
  if (model->precision != TDO_FP32 && model->embed != TDO_EMBED_TOKEN)
    return fail(nullptr, TDO_EUNSUPPORTED, "the tensor-core (BF16 / FP16) path supports the token embedding");
  const size_t P = tdo_model_num_params(model);
  if (!theta || n_theta != P) return fail(nullptr, TDO_EINVAL, "theta must hold %zu values (got %zu)", P, n_theta);

  tdo_ctx *c = new tdo_ctx();
  c->model = *model;
  c->tc = model->precision == TDO_BF16 || model->precision == TDO_FP16 || model->precision == TDO_FP8;
  c->f16 = model->precision == TDO_FP16 || model->precision == TDO_FP8;
  c->f8 = model->precision == TDO_FP8;
  c->n = problem->n_sites;
  c->stream = (cudaStream_t)stream;
  auto bail = [&](tdo_status s) {
    g_create_error = c->err;
    tdo_destroy(c);
    return s;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) { cudaGetLastError(); fail(c, TDO_ECUDA, "no CUDA device"); return bail(TDO_ECUDA); }
  cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
  if (c->n_sm <= 0) c->n_sm = 1;
  tdo_status s = layout_params(c);
  if (s == TDO_OK) s = build_rules(c, problem);
  if (s != TDO_OK) return bail(s);
  // tensor table for the FP64 -> FP32 padded conversion
  std::vector<long long> tab;
  for (auto &t : c->tensors) { tab.push_back(t.flat); tab.push_back(t.pad); tab.push_back(t.size); }
  cudaError_t e;
  if ((e = c->tensor_tab.ensure(sizeof(long long) * tab.size())) != cudaSuccess ||
      (e = c->theta64.ensure(sizeof(double) * P)) != cudaSuccess ||
      (e = c->theta32.ensure(sizeof(float) * c->P_pad)) != cudaSuccess ||
      (e = c->etab.ensure(sizeof(float) * 64 * model->d_model)) != cudaSuccess ||
      (e = c->nonfinite.ensure(sizeof(int) * 4)) != cudaSuccess) {
    fail(c, TDO_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    return bail(TDO_ENOMEM);
  }
  if ((e = cudaMemcpy(c->tensor_tab.p, tab.data(), sizeof(long long) * tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(c->theta32.p, 0, sizeof(float) * c->P_pad)) != cudaSuccess) {
    fail(c, TDO_ECUDA, "%s", cudaGetErrorString(e));
    return bail(TDO_ECUDA);
  }
  build_devmodel(c);
  if (c->tc) {
    if (!bf16_supported(c->dm)) {
      fail(c, TDO_EUNSUPPORTED, "tensor-core path: d_model 32 or 64, head dim a multiple of 8, an even head "
                                 "count, MLP width a multiple of min(4 d_model, 128)");
      return bail(TDO_EUNSUPPORTED);
    }
    if ((e = c->wbf16.ensure(bf16_packed_bytes(c->dm))) != cudaSuccess ||
        (c->f8 && (e = c->wf8.ensure(f8_packed_bytes(c->dm))) != cudaSuccess) ||
        (e = c->cscale.ensure(2 * sizeof(float))) != cudaSuccess ||
        (e = c->errflag.ensure(sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(c->errflag.p, 0, sizeof(int))) != cudaSuccess) {
      fail(c, TDO_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
      return bail(TDO_ENOMEM);
    }
    c->tc_bwd = bwdtc_supported(c->dm);
    if (c->tc_bwd && (e = c->wbwd.ensure(bwdtc_packed_bytes(c->dm))) != cudaSuccess) {
      fail(c, TDO_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
      return bail(TDO_ENOMEM);
    }
  }
  s = tdo_set_params(c, theta);
  if (s != TDO_OK) return bail(s);
  *out = c;
  return TDO_OK;
}

extern "C" tdo_status tdo_destroy(tdo_ctx *c) {
  if (!c) return TDO_OK;
  if (c->stream || true) cudaStreamSynchronize(c->stream);
  DBuf *bufs[] = {&c->d_pat, &c->d_con, &c->theta64, &c->theta32, &c->etab, &c->tensor_tab, &c->stage_in[0],
                  &c->stage_in[1], &c->stage_in[2], &c->stage_in[3], &c->stage_out, &c->conn_cnt, &c->conn_sig,
                  &c->conn_sigp, &c->conn_coef, &c->offs, &c->fsig, &c->fsigp, &c->fcoef, &c->flr, &c->lloc,
                  &c->l2, &c->stats, &c->nonfinite, &c->cot, &c->gacc, &c->scratch, &c->grad, &c->Obuf,
                  &c->srwork, &c->delta, &c->acc_u64, &c->wbf16, &c->wf8, &c->errflag, &c->wbwd, &c->act_x, &c->act_xmid,
                  &c->act_h, &c->act_f, &c->act_dF, &c->act_dxa, &c->act_dxb, &c->act_dqkv, &c->dtab,
                  &c->oref, &c->oref_scratch, &c->jac_vs, &c->jac_vp, &c->jac_vc, &c->jac_lr, &c->obs_rs,
                  &c->obs_rp, &c->obs_lr, &c->obs_part, &c->obs_out, &c->obs_local};
  for (DBuf *b : bufs) b->release();
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  if (c->gevent) cudaEventDestroy(c->gevent);
  c->gstep.release();
  if (c->gstep_host) cudaFreeHost(c->gstep_host);
  for (auto &r : c->trec) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : c->epool) cudaEventDestroy(e);
  delete c;
  return TDO_OK;
}

extern "C" size_t tdo_num_params(const tdo_ctx *c) { return c ? c->P : 0; }
extern "C" int tdo_max_connections(const tdo_ctx *c) { return c ? c->n_pat : 0; }

extern "C" tdo_status tdo_set_params(tdo_ctx *c, const double *theta) {
  if (!c) return TDO_EINVAL;
  c->have_delta = false;
  if (!theta) return fail(c, TDO_EINVAL, "theta is NULL");
  const cudaMemcpyKind kind = is_device_ptr(theta) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CU(c, cudaMemcpyAsync(c->theta64.p, theta, sizeof(double) * c->P, kind, c->stream));
  TRY(refresh_params(c));
  if (kind == cudaMemcpyHostToDevice) CU(c, cudaStreamSynchronize(c->stream));
  return TDO_OK;
}

extern "C" tdo_status tdo_get_params(tdo_ctx *c, double *theta) {
  if (!c) return TDO_EINVAL;
  if (!theta) return fail(c, TDO_EINVAL, "theta is NULL");
  const bool dev = is_device_ptr(theta);
  CU(c, cudaMemcpyAsync(theta, c->theta64.p, sizeof(double) * c->P, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (!dev) CU(c, cudaStreamSynchronize(c->stream));
  return TDO_OK;
}

// forward on device buffers
static tdo_status forward_dev(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t B, float2 *out) {
  if (B == 0) return TDO_OK;
  Timed tm(c, G_FWD);
  if (c->tc)
    CU(c, EVAL_LAUNCH(c, launch_fwd_bf16, sig, sigp, B, out, c->errflag.as<int>(), c->n_sm, c->stream));
  else
    CU(c, launch_fwd32(c->dm, sig, sigp, B, out, c->n_sm, c->stream));
  return TDO_OK;
}

// Copy a device result to a caller buffer (device or host); returns whether a sync is needed.
static tdo_status deliver(tdo_ctx *c, void *dst, const void *src, size_t bytes, bool *host) {
  *host = false;
  if (!dst || bytes == 0 || dst == src) return TDO_OK;
  const bool dev = is_device_ptr(dst);
  *host = !dev;
  CU(c, cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return TDO_OK;
}

extern "C" tdo_status tdo_log_rho(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t B, float *logrho) {
  if (!c) return TDO_EINVAL;
  if (B == 0) return TDO_OK;
  if (!sig || !sigp || !logrho) return fail(c, TDO_EINVAL, "NULL buffer");
  const void *ds, *dp;
  bool h1, h2, h3 = false;
  TRY(stage_in(c, 0, sig, 4 * B, &ds, &h1));
  TRY(stage_in(c, 1, sigp, 4 * B, &dp, &h2));
  float2 *dout = reinterpret_cast<float2 *>(logrho);
  if (!is_device_ptr(logrho)) {
    CU(c, c->stage_out.ensure(8 * B));
    dout = c->stage_out.as<float2>();
  }
  TRY(forward_dev(c, (const uint32_t *)ds, (const uint32_t *)dp, B, dout));
  TRY(deliver(c, logrho, dout, 8 * B, &h3));
  if (h1 || h2 || h3) {
    CU(c, cudaStreamSynchronize(c->stream));
    TRY(check_err_flag(c));
  }
  return TDO_OK;
}

// Ragged batch on the device: bucketing, then one persistent tensor-core launch (autotuned on the first call
// with a new mix of chain lengths), or one FP32 launch per bucket.
static tdo_status ragged_dev(tdo_ctx *c, const int32_t *dn, const uint32_t *ds, const uint32_t *dp, size_t B,
                             float2 *out) {
  CU(c, c->rg_counts.ensure(33 * sizeof(unsigned long long)));
  CU(c, c->rg_cursor.ensure(33 * sizeof(unsigned long long)));
  CU(c, c->rg_ssig.ensure(4 * B));
  CU(c, c->rg_ssigp.ensure(4 * B));
  CU(c, c->rg_perm.ensure(4 * B));
  CU(c, c->rg_next.ensure(sizeof(unsigned long long)));
  CU(c, launch_ragged_hist(dn, B, c->rg_counts.as<unsigned long long>(), c->stream));
  unsigned long long cnt[33];
  CU(c, cudaMemcpyAsync(cnt, c->rg_counts.p, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  if (cnt[0]) return fail(c, TDO_EUNSUPPORTED, "tdo_log_rho_ragged: %llu chain lengths outside 1..32", cnt[0]);
  unsigned long long base[33] = {0};
  uint32_t mix = 0;
  for (int n = 1; n <= 32; ++n) {
    base[n] = (n > 1 ? base[n - 1] + cnt[n - 1] : 0);
    if (cnt[n]) mix |= 1u << (n - 1);
  }
  CU(c, cudaMemcpyAsync(c->rg_cursor.p, base, sizeof(base), cudaMemcpyHostToDevice, c->stream));
  uint32_t *ss = c->rg_ssig.as<uint32_t>(), *sp = c->rg_ssigp.as<uint32_t>(), *perm = c->rg_perm.as<uint32_t>();
  CU(c, launch_ragged_scatter(dn, ds, dp, B, c->rg_cursor.as<unsigned long long>(), ss, sp, perm, c->stream));
  if (!c->tc) {   // FP32 path: one launch per bucket, the model's chain length set to the bucket's
    CU(c, c->rg_tmp.ensure(8 * B));
    Timed tm(c, G_FWD);
    int nl = 0;
    for (int n = 1; n <= 32; ++n) {
      if (!cnt[n]) continue;
      DevModel dm = c->dm;
      dm.n_sites = n;
      CU(c, launch_fwd32(dm, ss + base[n], sp + base[n], cnt[n], c->rg_tmp.as<float2>() + base[n], c->n_sm, c->stream));
      ++nl;
    }
    CU(c, launch_unpermute(c->rg_tmp.as<float2>(), perm, B, out, c->stream));
    tm.done(nl + 1);
    return TDO_OK;
  }
  auto table = [&](bool desc) {
    RaggedTab t{};
    long long tile = 0;
    for (int i = 0; i < 32; ++i) {
      const int n = desc ? 32 - i : 1 + i;
      if (!cnt[n]) continue;
      const int k = t.nb++;
      t.n[k] = n;
      t.base[k] = (long long)base[n];
      t.count[k] = (long long)cnt[n];
      t.tile0[k] = tile;
      const int ts = 2 * (128 / (2 * n)), tc = (ts < 2 ? 2 : ts) / 2;   // configurations per 128-row tile
      tile += ((long long)cnt[n] + tc - 1) / tc;
    }
    t.tile0[t.nb] = tile;
    return t;
  };
  auto launch = [&](const std::array<int, 3> &cfg) -> cudaError_t {
    const RaggedTab t = table(cfg[1] != 0);
    return EVAL_LAUNCH(c, launch_fwd_ragged, ss, sp, perm, t,
                     cfg[2] ? c->rg_next.as<unsigned long long>() : nullptr, out, c->errflag.as<int>(), c->n_sm,
                     cfg[0], c->stream);
  };
  auto it = c->rg_tuned.find(mix);
  if (it == c->rg_tuned.end()) {
    // autotune: time each candidate once on this batch (identical outputs), keep the fastest
    const std::array<int, 3> cand[4] = {{2, 1, 1}, {2, 0, 1}, {2, 0, 0}, {1, 1, 1}};
    cudaEvent_t e0, e1;
    CU(c, cudaEventCreate(&e0));
    CU(c, cudaEventCreate(&e1));
    float best = 0.f;
    int bi = 0;
    for (int i = 0; i < 4; ++i) {
      CU(c, cudaEventRecord(e0, c->stream));
      const cudaError_t e = launch(cand[i]);
      CU(c, cudaEventRecord(e1, c->stream));
      CU(c, e);
      CU(c, cudaEventSynchronize(e1));
      float ms = 0.f;
      CU(c, cudaEventElapsedTime(&ms, e0, e1));
      if (i == 0 || ms < best) { best = ms; bi = i; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    it = c->rg_tuned.emplace(mix, cand[bi]).first;
  }
  Timed tm(c, G_FWD);
  CU(c, launch(it->second));
  tm.done(1);
  return TDO_OK;
}

extern "C" tdo_status tdo_log_rho_ragged(tdo_ctx *c, const int32_t *n_sites, const uint32_t *sig, const uint32_t *sigp,
                                         size_t B, float *logrho) {
  if (!c) return TDO_EINVAL;
  if (B == 0) return TDO_OK;
  if (!n_sites || !sig || !sigp || !logrho) return fail(c, TDO_EINVAL, "NULL buffer");
  if (B > 0xFFFFFFFFull) return fail(c, TDO_EINVAL, "B must be below 2^32");
  const void *dn, *ds, *dp;
  bool h0, h1, h2, h3 = false;
  TRY(stage_in(c, 2, n_sites, 4 * B, &dn, &h0));
  TRY(stage_in(c, 0, sig, 4 * B, &ds, &h1));
  TRY(stage_in(c, 1, sigp, 4 * B, &dp, &h2));
  float2 *dout = reinterpret_cast<float2 *>(logrho);
  if (!is_device_ptr(logrho)) {
    CU(c, c->stage_out.ensure(8 * B));
    dout = c->stage_out.as<float2>();
  }
  TRY(ragged_dev(c, (const int32_t *)dn, (const uint32_t *)ds, (const uint32_t *)dp, B, dout));
  TRY(deliver(c, logrho, dout, 8 * B, &h3));
  CU(c, cudaStreamSynchronize(c->stream));
  TRY(check_err_flag(c));
  return TDO_OK;
}

extern "C" tdo_status tdo_ragged_tuning(const tdo_ctx *c, uint32_t mix, int *ctas_per_sm, int *descending,
                                        int *dynamic_schedule) {
  if (!c) return TDO_EINVAL;
  const auto it = c->rg_tuned.find(mix);
  if (it == c->rg_tuned.end()) return TDO_EINVAL;
  if (ctas_per_sm) *ctas_per_sm = it->second[0];
  if (descending) *descending = it->second[1];
  if (dynamic_schedule) *dynamic_schedule = it->second[2];
  return TDO_OK;
}

// Connections + compaction + forward over every row + L_loc and cost statistics (device buffers).
static tdo_status estimator_core(tdo_ctx *c, const uint32_t *ds, const uint32_t *dp, size_t Ns, int64_t *total,
                                 bool park = false);
static tdo_status forward_park(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t B, float2 *out);

static tdo_status estimator_core(tdo_ctx *c, const uint32_t *ds, const uint32_t *dp, size_t Ns, int64_t *total,
                                 bool park) {
  const int M = c->n_pat;
  CU(c, c->conn_cnt.ensure(sizeof(int32_t) * Ns));
  CU(c, c->conn_sig.ensure(sizeof(uint32_t) * Ns * M));
  CU(c, c->conn_sigp.ensure(sizeof(uint32_t) * Ns * M));
  CU(c, c->conn_coef.ensure(sizeof(float2) * Ns * M));
  CU(c, c->offs.ensure(sizeof(int64_t) * (Ns + 1)));
  {
    Timed tm(c, G_CONN);
    CU(c, launch_connections(c->d_pat.as<ConnPattern>(), M, c->d_con.as<ConnContrib>(), ds, dp, Ns,
                             c->conn_cnt.as<int32_t>(), c->conn_sig.as<uint32_t>(), c->conn_sigp.as<uint32_t>(),
                             c->conn_coef.as<float2>(), c->stream));
    CU(c, launch_scan(c->conn_cnt.as<int32_t>(), Ns, c->offs.as<int64_t>(), c->stream));
    tm.done(2);
  }
  int64_t tot = 0;
  CU(c, cudaMemcpyAsync(&tot, c->offs.as<int64_t>() + Ns, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  *total = tot;
  CU(c, c->fsig.ensure(sizeof(uint32_t) * tot));
  CU(c, c->fsigp.ensure(sizeof(uint32_t) * tot));
  CU(c, c->fcoef.ensure(sizeof(float2) * tot));
  CU(c, c->flr.ensure(sizeof(float2) * tot));
  {
    Timed tm(c, G_CONN);
    CU(c, launch_compact(c->conn_cnt.as<int32_t>(), c->offs.as<int64_t>(), Ns, M, c->conn_sig.as<uint32_t>(),
                         c->conn_sigp.as<uint32_t>(), c->conn_coef.as<float2>(), c->fsig.as<uint32_t>(),
                         c->fsigp.as<uint32_t>(), c->fcoef.as<float2>(), c->stream));
  }
  if (park) TRY(forward_park(c, c->fsig.as<uint32_t>(), c->fsigp.as<uint32_t>(), (size_t)tot, c->flr.as<float2>()));
  else TRY(forward_dev(c, c->fsig.as<uint32_t>(), c->fsigp.as<uint32_t>(), (size_t)tot, c->flr.as<float2>()));
  CU(c, c->lloc.ensure(sizeof(double2) * Ns));
  CU(c, c->l2.ensure(sizeof(double) * Ns));
  CU(c, c->stats.ensure(sizeof(double) * 4));
  CU(c, cudaMemsetAsync(c->nonfinite.p, 0, sizeof(int), c->stream));
  Timed tm(c, G_LLOC);
  CU(c, launch_lloc(c->offs.as<int64_t>(), Ns, c->fcoef.as<float2>(), c->flr.as<float2>(), c->lloc.as<double2>(),
                    c->l2.as<double>(), c->stats.as<double>(), c->nonfinite.as<int>(), c->stream));
  tm.done(2);
  return TDO_OK;
}

static tdo_status read_stats(tdo_ctx *c, size_t Ns, double *cost, double *se) {
  double st[2];
  int nf = 0;
  CU(c, cudaMemcpyAsync(st, c->stats.p, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaMemcpyAsync(&nf, c->nonfinite.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  TRY(check_err_flag(c));
  if (nf) return fail(c, TDO_ENUMERIC, "non-finite log rho or L_loc (rho = 0 exactly, or non-finite parameters)");
  const double mean = st[0] / (double)Ns;
  const double var = st[1] / (double)Ns - mean * mean;
  if (cost) *cost = mean;
  if (se) *se = var > 0 ? sqrt(var / (double)Ns) : 0.0;
  return TDO_OK;
}

extern "C" tdo_status tdo_connections(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t Ns,
                                      int32_t *count, uint32_t *conn_sig, uint32_t *conn_sigp, float *conn_coef) {
  if (!c) return TDO_EINVAL;
  if (Ns == 0) return TDO_OK;
  if (!sig || !sigp || !count || !conn_sig || !conn_sigp || !conn_coef) return fail(c, TDO_EINVAL, "NULL buffer");
  const int M = c->n_pat;
  const void *ds, *dp;
  bool h1, h2, h3 = false, h4 = false, h5 = false, h6 = false;
  TRY(stage_in(c, 0, sig, 4 * Ns, &ds, &h1));
  TRY(stage_in(c, 1, sigp, 4 * Ns, &dp, &h2));
  CU(c, c->conn_cnt.ensure(sizeof(int32_t) * Ns));
  CU(c, c->conn_sig.ensure(sizeof(uint32_t) * Ns * M));
  CU(c, c->conn_sigp.ensure(sizeof(uint32_t) * Ns * M));
  CU(c, c->conn_coef.ensure(sizeof(float2) * Ns * M));
  CU(c, launch_connections(c->d_pat.as<ConnPattern>(), M, c->d_con.as<ConnContrib>(), (const uint32_t *)ds,
                           (const uint32_t *)dp, Ns, c->conn_cnt.as<int32_t>(), c->conn_sig.as<uint32_t>(),
                           c->conn_sigp.as<uint32_t>(), c->conn_coef.as<float2>(), c->stream));
  TRY(deliver(c, count, c->conn_cnt.p, sizeof(int32_t) * Ns, &h3));
  TRY(deliver(c, conn_sig, c->conn_sig.p, sizeof(uint32_t) * Ns * M, &h4));
  TRY(deliver(c, conn_sigp, c->conn_sigp.p, sizeof(uint32_t) * Ns * M, &h5));
  TRY(deliver(c, conn_coef, c->conn_coef.p, sizeof(float2) * Ns * M, &h6));
  CU(c, cudaStreamSynchronize(c->stream));
  return TDO_OK;
}

extern "C" tdo_status tdo_local_estimator(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t Ns,
                                          double *lloc, double *cost, double *stderr_) {
  if (!c) return TDO_EINVAL;
  if (Ns == 0) return fail(c, TDO_EINVAL, "Ns must be > 0");
  if (!sig || !sigp) return fail(c, TDO_EINVAL, "NULL buffer");
  const void *ds, *dp;
  bool h1, h2, h3 = false;
  TRY(stage_in(c, 0, sig, 4 * Ns, &ds, &h1));
  TRY(stage_in(c, 1, sigp, 4 * Ns, &dp, &h2));
  int64_t total = 0;
  TRY(estimator_core(c, (const uint32_t *)ds, (const uint32_t *)dp, Ns, &total));
  if (lloc) TRY(deliver(c, lloc, c->lloc.p, sizeof(double2) * Ns, &h3));
  TRY(read_stats(c, Ns, cost, stderr_));
  return TDO_OK;
}


// Back-propagates the per-pattern table gradients the backward kernel left in c->dtab to the conv
// embedding parameters (mode 0: added into g; mode 1: written into O[b][k][seed]).
static tdo_status conv_vjp(tdo_ctx *c, int nsets, int ncopy, int mode, float *g, float *O, uint16_t *O16 = nullptr,
                           const float2 *oref = nullptr, size_t ldo = 0) {
  const float *b = c->theta32.as<float>();
  CU(c, launch_conv_vjp(c->model.d_model, c->model.conv_channels, b + c->tensors[0].pad, b + c->tensors[1].pad,
                        b + c->tensors[2].pad, b + c->tensors[3].pad, c->dtab.as<float>(), nsets, ncopy, mode, g, O,
                        O16, oref, ldo ? ldo : c->P,
                        c->tensors[0].flat, c->tensors[1].flat, c->tensors[2].flat, c->tensors[3].flat, c->stream));
  return TDO_OK;
}

// VJP over device rows: grad (FP64, device) = [accumulate ? grad : 0] + sum Re(cot * dlogrho).
static tdo_status vjp_dev(tdo_ctx *c, const uint32_t *ds, const uint32_t *dp, size_t B, const float2 *cot,
                          double *grad, int accumulate) {
  const bool conv = c->model.embed == TDO_EMBED_CONV;
  const int grid = bwd32_grid(c->dm, B, 0, c->n_sm);
  const int copies = grid < 16 ? grid : 16;   // 16 accumulator copies: L2-resident, low contention
  const size_t stride = (c->P + 3) / 4 * 4;   // 16-byte aligned copies (float4 atomics)
  const size_t tab = (size_t)64 * c->model.d_model;
  CU(c, c->gacc.ensure(sizeof(float) * copies * stride));
  CU(c, c->scratch.ensure(sizeof(float) * bwd32_scratch_floats(c->dm, grid)));
  CU(c, cudaMemsetAsync(c->gacc.p, 0, sizeof(float) * copies * stride, c->stream));
  if (conv) {   // one [64][d] table-gradient copy per accumulator copy
    CU(c, c->dtab.ensure(sizeof(float) * copies * tab));
    CU(c, cudaMemsetAsync(c->dtab.p, 0, sizeof(float) * copies * tab, c->stream));
  }
  Timed tm(c, G_BWD_VJP);
  CU(c, launch_bwd32_impl(c->dm, 0, ds, dp, B, cot, c->gacc.as<float>(), copies, stride, nullptr, nullptr, nullptr,
                          c->P, c->P, c->flat_offsets, c->scratch.as<float>(), conv ? c->dtab.as<float>() : nullptr, grid,
                          c->stream));
  if (conv) TRY(conv_vjp(c, 1, copies, 0, c->gacc.as<float>(), nullptr));
  CU(c, launch_reduce_copies(c->gacc.as<float>(), copies, stride, c->P, grad, accumulate, c->stream));
  tm.done(conv ? 3 : 2);
  return TDO_OK;
}

static tdo_status jacobian_tc(tdo_ctx *c, const uint32_t *ds, const uint32_t *dp, size_t Ns, float *O32,
                              uint16_t *O16, const float2 *oref, size_t ldo);

// Log-derivatives of B configurations: FP32 into O, or (O16 non-null) BF16 of O - oref; rows of ldo
// elements (0: P).  BF16 contexts whose tensor-core backward covers the model take the tensor-core
// path (per-configuration MMAs); the rest the FP32 backward.
static tdo_status jacobian_dev(tdo_ctx *c, const uint32_t *ds, const uint32_t *dp, size_t B, float *O,
                               uint16_t *O16 = nullptr, const float2 *oref = nullptr, size_t ldo = 0) {
  if (!ldo) ldo = c->P;
  if (c->tc_bwd && bwdtc_jac_supported(c->dm)) return jacobian_tc(c, ds, dp, B, O, O16, oref, ldo);
  const bool conv = c->model.embed == TDO_EMBED_CONV;
  const int grid = bwd32_grid(c->dm, B, 1, c->n_sm);
  CU(c, c->scratch.ensure(sizeof(float) * bwd32_scratch_floats(c->dm, grid)));
  if (conv) CU(c, c->dtab.ensure(sizeof(float) * 2 * B * 64 * c->model.d_model));
  Timed tm(c, G_BWD_JAC);
  CU(c, launch_bwd32_impl(c->dm, 1, ds, dp, B, nullptr, nullptr, 1, 0, O, O16, oref, c->P, ldo, c->flat_offsets,
                          c->scratch.as<float>(), conv ? c->dtab.as<float>() : nullptr, grid, c->stream));
  if (conv) TRY(conv_vjp(c, (int)(2 * B), 1, 1, nullptr, O, O16, oref, ldo));
  tm.done(conv ? 2 : 1);
  return TDO_OK;
}

// The SR matrix's log-derivatives in BF16 (BF16 contexts): the shift oref is the mean log-derivative of
// the first min(Ns, 64) samples (an FP32 Jacobian of those), so the stored values are spread-sized and
// their rounding does not scale with a parameter's mean (the centring of S removes the shift exactly).
static tdo_status jacobian_bf16_for_sr(tdo_ctx *c, const uint32_t *ds, const uint32_t *dp, size_t Ns, size_t ldo) {
  const int nref = Ns < 64 ? (int)Ns : 64;
  const size_t ref_bytes = sizeof(float) * 2 * c->P * (size_t)nref;
  float *O32 = nullptr;
  if (c->Obuf.bytes >= ref_bytes) {
    O32 = c->Obuf.as<float>();   // overwritten below by the BF16 log-derivatives
  } else {
    CU(c, c->oref_scratch.ensure(ref_bytes));
    O32 = c->oref_scratch.as<float>();
  }
  CU(c, c->oref.ensure(sizeof(float) * 2 * c->P));
  TRY(jacobian_dev(c, ds, dp, (size_t)nref, O32));
  {
    Timed tm(c, G_BWD_JAC);
    CU(c, launch_oref(O32, nref, c->P, c->oref.as<float>(), c->stream));
  }
  TRY(jacobian_dev(c, ds, dp, Ns, nullptr, c->Obuf.as<uint16_t>(), c->oref.as<float2>(), ldo));
  return TDO_OK;
}

extern "C" tdo_status tdo_log_rho_vjp(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t B,
                                      const float *cot, double *grad) {
  if (!c) return TDO_EINVAL;
  if (B == 0) return TDO_OK;
  if (!sig || !sigp || !cot || !grad) return fail(c, TDO_EINVAL, "NULL buffer");
  const void *ds, *dp, *dc;
  bool h1, h2, h3, h4 = false;
  TRY(stage_in(c, 0, sig, 4 * B, &ds, &h1));
  TRY(stage_in(c, 1, sigp, 4 * B, &dp, &h2));
  TRY(stage_in(c, 2, cot, 8 * B, &dc, &h3));
  double *dg = grad;
  if (!is_device_ptr(grad)) {
    CU(c, c->grad.ensure(sizeof(double) * c->P));
    CU(c, cudaMemcpyAsync(c->grad.p, grad, sizeof(double) * c->P, cudaMemcpyHostToDevice, c->stream));
    dg = c->grad.as<double>();
  }
  TRY(vjp_dev(c, (const uint32_t *)ds, (const uint32_t *)dp, B, (const float2 *)dc, dg, 1));
  TRY(deliver(c, grad, dg, sizeof(double) * c->P, &h4));
  if (h1 || h2 || h3 || h4) CU(c, cudaStreamSynchronize(c->stream));
  return TDO_OK;
}

extern "C" tdo_status tdo_jacobian(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t B, float *O) {
  if (!c) return TDO_EINVAL;
  if (B == 0) return TDO_OK;
  if (!sig || !sigp || !O) return fail(c, TDO_EINVAL, "NULL buffer");
  const void *ds, *dp;
  bool h1, h2, h3 = false;
  TRY(stage_in(c, 0, sig, 4 * B, &ds, &h1));
  TRY(stage_in(c, 1, sigp, 4 * B, &dp, &h2));
  float *dO = O;
  const size_t bytes = sizeof(float) * 2 * c->P * B;
  if (!is_device_ptr(O)) { CU(c, c->Obuf.ensure(bytes)); dO = c->Obuf.as<float>(); }
  TRY(jacobian_dev(c, (const uint32_t *)ds, (const uint32_t *)dp, B, dO));
  TRY(deliver(c, O, dO, bytes, &h3));
  if (h1 || h2 || h3) CU(c, cudaStreamSynchronize(c->stream));
  return TDO_OK;
}

// BF16 forward that also parks the activations the tensor-core backward needs.
static size_t tc_tiles(tdo_ctx *c, size_t B) {
  const int tc = (2 * (128 / (2 * c->n)) < 2 ? 2 : 2 * (128 / (2 * c->n))) / 2;
  return (B + tc - 1) / tc;
}
static tdo_status forward_park(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t B, float2 *out) {
  const size_t tiles = tc_tiles(c, B);
  const int ts = 2 * (128 / (2 * c->n)) < 2 ? 2 : 2 * (128 / (2 * c->n));
  const size_t img = (size_t)128 * c->dm.d * 2, L = c->dm.layers;
  CU(c, c->act_x.ensure(L * tiles * img));
  CU(c, c->act_xmid.ensure(c->dm.ffn > 0 ? L * tiles * img : 16));
  CU(c, c->act_h.ensure(sizeof(float) * tiles * ts * c->dm.d));
  CU(c, c->act_f.ensure(sizeof(float) * tiles * ts * 2));
  Timed tm(c, G_FWD);
  CU(c, TC_LAUNCH(c, launch_fwd_bf16_store, c->dm, c->dmb, sig, sigp, B, out, c->errflag.as<int>(), c->n_sm, c->stream,
                              c->act_x.as<uint8_t>(), c->dm.ffn > 0 ? c->act_xmid.as<uint8_t>() : nullptr,
                              c->act_h.as<float>(), c->act_f.as<float>(), tiles));
  return TDO_OK;
}

// Tensor-core VJP of the rows parked by forward_park (same rows, same order).
static tdo_status vjp_tc(tdo_ctx *c, const uint32_t *ds, const uint32_t *dp, size_t B, const float2 *cot,
                         double *grad) {
  const size_t tiles = tc_tiles(c, B);
  const int ts = 2 * (128 / (2 * c->n)) < 2 ? 2 : 2 * (128 / (2 * c->n));
  const size_t D = c->dm.d;
  const int copies = 16;
  const size_t stride = (c->P + 3) / 4 * 4;
  CU(c, c->act_dF.ensure(sizeof(float) * tiles * ts * 2));
  CU(c, c->act_dxa.ensure(sizeof(float) * tiles * 128 * D));
  CU(c, c->act_dxb.ensure(sizeof(float) * tiles * 128 * D));
  CU(c, c->act_dqkv.ensure(tiles * 128 * 3 * D * 2));
  CU(c, c->gacc.ensure(sizeof(float) * copies * stride));
  CU(c, cudaMemsetAsync(c->gacc.p, 0, sizeof(float) * copies * stride, c->stream));
  BwdTcBuffers bf{c->act_x.as<uint8_t>(), c->act_xmid.as<uint8_t>(), c->act_dqkv.as<uint8_t>(), c->act_h.as<float>(),
                  c->act_f.as<float>(), c->act_dF.as<float>(), c->act_dxa.as<float>(), c->act_dxb.as<float>(), tiles,
                  c->cscale.as<float>()};
  Timed tm(c, G_BWD_VJP);
  CU(c, TC_LAUNCH(c, launch_bwdtc, c->dm, c->dmb, c->bwl, bf, ds, dp, B, cot, c->gacc.as<float>(), stride, c->flat_offsets,
                     c->errflag.as<int>(), c->n_sm, c->stream));
  CU(c, launch_reduce_copies(c->gacc.as<float>(), copies, stride, c->P, grad, 0, c->stream, c->cscale.as<float>() + 1));
  tm.done(2 + (long long)c->dm.layers * (2 + (c->dm.ffn > 0 ? c->dm.ffn / 128 : 0)) + 2);
  return TDO_OK;
}

// Tensor-core log-derivatives: the Ns samples become 2 Ns virtual configurations (one per real cotangent
// seed), the BF16 forward parks their activations, and the backward writes each configuration's weight
// gradients (per-configuration MMAs over its 32 rows) to O[b][k] = (seed 0, seed 1).
static tdo_status jacobian_tc(tdo_ctx *c, const uint32_t *ds, const uint32_t *dp, size_t Ns, float *O32,
                              uint16_t *O16, const float2 *oref, size_t ldo) {
  const size_t nv = 2 * Ns;
  const size_t tiles = tc_tiles(c, nv);
  const int ts = 2 * (128 / (2 * c->n)) < 2 ? 2 : 2 * (128 / (2 * c->n));
  const size_t D = c->dm.d, img = (size_t)128 * D * 2, L = c->dm.layers;
  CU(c, c->jac_vs.ensure(4 * nv));
  CU(c, c->jac_vp.ensure(4 * nv));
  CU(c, c->jac_vc.ensure(sizeof(float2) * nv));
  CU(c, c->jac_lr.ensure(sizeof(float2) * nv));
  CU(c, c->act_x.ensure(L * tiles * img));
  CU(c, c->act_xmid.ensure(c->dm.ffn > 0 ? L * tiles * img : 16));
  CU(c, c->act_h.ensure(sizeof(float) * tiles * ts * D));
  CU(c, c->act_f.ensure(sizeof(float) * tiles * ts * 2));
  CU(c, c->act_dF.ensure(sizeof(float) * tiles * ts * 2));
  CU(c, c->act_dxa.ensure(sizeof(float) * tiles * 128 * D));
  CU(c, c->act_dxb.ensure(sizeof(float) * tiles * 128 * D));
  CU(c, c->act_dqkv.ensure(tiles * 128 * 3 * D * 2));
  uint32_t *vs = c->jac_vs.as<uint32_t>(), *vp = c->jac_vp.as<uint32_t>();
  Timed tm(c, G_BWD_JAC);
  CU(c, launch_jac_virtual(ds, dp, Ns, vs, vp, c->jac_vc.as<float2>(), c->stream));
  CU(c, TC_LAUNCH(c, launch_fwd_bf16_store, c->dm, c->dmb, vs, vp, nv, c->jac_lr.as<float2>(), c->errflag.as<int>(), c->n_sm,
                              c->stream, c->act_x.as<uint8_t>(), c->dm.ffn > 0 ? c->act_xmid.as<uint8_t>() : nullptr,
                              c->act_h.as<float>(), c->act_f.as<float>(), tiles));
  BwdTcBuffers bf{c->act_x.as<uint8_t>(), c->act_xmid.as<uint8_t>(), c->act_dqkv.as<uint8_t>(), c->act_h.as<float>(),
                  c->act_f.as<float>(), c->act_dF.as<float>(), c->act_dxa.as<float>(), c->act_dxb.as<float>(), tiles,
                  c->cscale.as<float>()};
  BwdTcJac jac{O32, O16, oref, ldo, nv};
  CU(c, TC_LAUNCH(c, launch_bwdtc, c->dm, c->dmb, c->bwl, bf, vs, vp, nv, c->jac_vc.as<float2>(), nullptr, 0, c->flat_offsets,
                     c->errflag.as<int>(), c->n_sm, c->stream, &jac));
  tm.done(4 + (long long)c->dm.layers * (2 + (c->dm.ffn > 0 ? c->dm.ffn / 128 : 0)));
  TRY(check_err_flag(c));
  return TDO_OK;
}

// gradient of the cost on device: grad (device FP64 [P])
static tdo_status grad_dev(tdo_ctx *c, const uint32_t *ds, const uint32_t *dp, size_t Ns, double *grad, double *cost) {
  int64_t total = 0;
  TRY(estimator_core(c, ds, dp, Ns, &total, c->tc_bwd));
  CU(c, c->cot.ensure(sizeof(float2) * total));
  {
    Timed tm(c, G_LLOC);
    CU(c, launch_cotangent(c->offs.as<int64_t>(), Ns, c->fcoef.as<float2>(), c->flr.as<float2>(), c->lloc.as<double2>(),
                           c->stats.as<double>(), c->cot.as<float2>(), c->stream));
  }
  if (c->tc_bwd)
    TRY(vjp_tc(c, c->fsig.as<uint32_t>(), c->fsigp.as<uint32_t>(), (size_t)total, c->cot.as<float2>(), grad));
  else
    TRY(vjp_dev(c, c->fsig.as<uint32_t>(), c->fsigp.as<uint32_t>(), (size_t)total, c->cot.as<float2>(), grad, 0));
  TRY(read_stats(c, Ns, cost, nullptr));
  return TDO_OK;
}

extern "C" tdo_status tdo_grad(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t Ns, double *grad,
                               double *cost, float *O) {
  if (!c) return TDO_EINVAL;
  if (Ns == 0) return fail(c, TDO_EINVAL, "Ns must be > 0");
  if (!sig || !sigp || !grad) return fail(c, TDO_EINVAL, "NULL buffer");
  const void *ds, *dp;
  bool h1, h2, h3 = false, h4 = false;
  TRY(stage_in(c, 0, sig, 4 * Ns, &ds, &h1));
  TRY(stage_in(c, 1, sigp, 4 * Ns, &dp, &h2));
  double *dg = grad;
  if (!is_device_ptr(grad)) { CU(c, c->grad.ensure(sizeof(double) * c->P)); dg = c->grad.as<double>(); }
  TRY(grad_dev(c, (const uint32_t *)ds, (const uint32_t *)dp, Ns, dg, cost));
  TRY(deliver(c, grad, dg, sizeof(double) * c->P, &h3));
  if (O) {
    float *dO = O;
    const size_t bytes = sizeof(float) * 2 * c->P * Ns;
    if (!is_device_ptr(O)) { CU(c, c->Obuf.ensure(bytes)); dO = c->Obuf.as<float>(); }
    TRY(jacobian_dev(c, (const uint32_t *)ds, (const uint32_t *)dp, Ns, dO));
    TRY(deliver(c, O, dO, bytes, &h4));
  }
  CU(c, cudaStreamSynchronize(c->stream));
  return TDO_OK;
}


// sr_cg_impl with, when timing is on, one event pair around every S' v launch (group "sr_mv").
static cudaError_t sr_cg_timed(tdo_ctx *c, const void *O, int o_bf16, size_t ldo, size_t Ns, const double *rhs,
                               const double *x0,
                               double shift, double tol, int max_iter, double *x, int *iters, double *resid,
                               int *outcome, double *last_pap, long long *launches) {
  std::vector<cudaEvent_t> ev;
  if (c->timing) {
    const int n = 2 * (max_iter + 1);
    while ((int)ev.size() < n) {
      cudaEvent_t e;
      if (!c->epool.empty()) { e = c->epool.back(); c->epool.pop_back(); }
      else if (cudaEventCreate(&e) != cudaSuccess) break;
      ev.push_back(e);
    }
  }
  int used = 0;
  const cudaError_t err = sr_cg_impl(O, o_bf16, Ns, c->P, ldo, rhs, x0, shift, tol, max_iter, x, c->srwork.as<double>(), c->n_sm,
                                     iters, resid, outcome, last_pap, launches, ev.empty() ? nullptr : ev.data(),
                                     (int)ev.size() / 2, &used, c->sr_product, c->tc ? c->errflag.as<int>() : nullptr,
                                     c->last_sr_shape, c->stream);
  for (int i = 0; i < (int)ev.size(); ++i) {
    if (i / 2 < used && i % 2 == 0) c->trec.push_back({G_SR_MV, ev[i], ev[i + 1], 1});
    else if (i / 2 >= used) c->epool.push_back(ev[i]);
  }
  return err;
}

// Status of a finished CG solve: a breakdown (p . S'p not positive before convergence, only possible
// for p = 0) or a non-finite value (gradient, log-derivatives, or a product) are TDO_ENUMERIC, each with
// its own message; stopping at max_iter is not an error (tdo_sr_info reports it).
static tdo_status sr_outcome_status(tdo_ctx *c, int outcome) {
  if (outcome == 3)
    return fail(c, TDO_ENUMERIC, "SR solve: non-finite value (NaN or Inf in the gradient, the log-derivatives or a product)");
  if (outcome == 2) return fail(c, TDO_ENUMERIC, "SR solve: CG breakdown (p . (S + shift I) p not positive)");
  return TDO_OK;
}

extern "C" tdo_status tdo_sr_solve(tdo_ctx *c, const float *O, size_t Ns, const double *rhs, double diag_shift,
                                   double tol, int max_iter, double *x, int *iters, double *resid) {
  if (!c) return TDO_EINVAL;
  if (Ns == 0) return fail(c, TDO_EINVAL, "Ns must be > 0");
  if (!O || !rhs || !x) return fail(c, TDO_EINVAL, "NULL buffer");
  if (!(diag_shift > 0.0)) return fail(c, TDO_EINVAL, "diag_shift must be > 0");
  const void *dO, *dr;
  bool h1, h2, h3 = false;
  TRY(stage_in(c, 0, O, sizeof(float) * 2 * c->P * Ns, &dO, &h1));
  TRY(stage_in(c, 1, rhs, sizeof(double) * c->P, &dr, &h2));
  double *dx = x;
  if (!is_device_ptr(x)) { CU(c, c->delta.ensure(sizeof(double) * c->P)); dx = c->delta.as<double>(); }
  CU(c, c->srwork.ensure(sizeof(double) * sr_work_doubles(Ns, c->P)));
  Timed tm(c, G_SR);
  int it_local = 0, outcome = 0;
  long long nl = 0;
  double pap = 0;
  cudaError_t e = sr_cg_timed(c, dO, 0, c->P, Ns, (const double *)dr, nullptr, diag_shift, tol, max_iter, dx,
                              &it_local, resid, &outcome, &pap, &nl);
  if (iters) *iters = it_local;
  tm.done(nl);
  CU(c, e);
  TRY(sr_outcome_status(c, outcome));
  TRY(deliver(c, x, dx, sizeof(double) * c->P, &h3));
  CU(c, cudaStreamSynchronize(c->stream));
  return TDO_OK;
}

extern "C" tdo_status tdo_sr_step(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t Ns, double lr,
                                  double diag_shift, double *cost) {
  if (!c) return TDO_EINVAL;
  if (Ns == 0) return fail(c, TDO_EINVAL, "Ns must be > 0");
  if (!sig || !sigp) return fail(c, TDO_EINVAL, "NULL buffer");
  if (!(diag_shift > 0.0)) return fail(c, TDO_EINVAL, "diag_shift must be > 0");
  const void *ds, *dp;
  bool h1, h2;
  TRY(stage_in(c, 0, sig, 4 * Ns, &ds, &h1));
  TRY(stage_in(c, 1, sigp, 4 * Ns, &dp, &h2));
  CU(c, c->grad.ensure(sizeof(double) * c->P));
  CU(c, c->delta.ensure(sizeof(double) * c->P));
  const int o_bf16 = c->tc ? 1 : 0;   // SR's O in BF16 for tensor-core contexts
  const size_t ldo = o_bf16 ? (c->P + 3) / 4 * 4 : (c->P + 1) / 2 * 2;   // rows on 16-byte boundaries
  CU(c, c->Obuf.ensure((o_bf16 ? sizeof(uint16_t) : sizeof(float)) * 2 * ldo * Ns));
  TRY(grad_dev(c, (const uint32_t *)ds, (const uint32_t *)dp, Ns, c->grad.as<double>(), cost));
  if (o_bf16) TRY(jacobian_bf16_for_sr(c, (const uint32_t *)ds, (const uint32_t *)dp, Ns, ldo));
  else TRY(jacobian_dev(c, (const uint32_t *)ds, (const uint32_t *)dp, Ns, c->Obuf.as<float>(), nullptr, nullptr, ldo));
  CU(c, c->srwork.ensure(sizeof(double) * sr_work_doubles(Ns, c->P)));
  int iters = 0, outcome = 0, restarts = 0;
  double resid = 0, pap = 0;
  cudaError_t e;
  {
    // warm start from the previous step's solution (same parameter layout); if that solve breaks down or
    // meets a non-finite value, solve once more from x = 0 before reporting the failure
    Timed tm(c, G_SR);
    long long nl = 0, nl2 = 0;
    const bool warm = c->have_delta;
    e = sr_cg_timed(c, c->Obuf.p, o_bf16, ldo, Ns, c->grad.as<double>(), warm ? c->delta.as<double>() : nullptr,
                    diag_shift, c->sr_tol, c->sr_max_iter, c->delta.as<double>(), &iters, &resid, &outcome, &pap, &nl);
    if (e == cudaSuccess && warm && (outcome == 2 || outcome == 3)) {
      restarts = 1;
      e = sr_cg_timed(c, c->Obuf.p, o_bf16, ldo, Ns, c->grad.as<double>(), nullptr, diag_shift, c->sr_tol,
                      c->sr_max_iter, c->delta.as<double>(), &iters, &resid, &outcome, &pap, &nl2);
    }
    tm.done(nl + nl2);
  }
  c->have_delta = (e == cudaSuccess && (outcome == 0 || outcome == 1));
  c->last_sr_iters = iters;
  c->last_sr_resid = resid;
  c->last_sr_outcome = outcome;
  c->last_sr_pap = pap;
  c->last_sr_restarts = restarts;
  CU(c, e);
  TRY(check_err_flag(c));
  TRY(sr_outcome_status(c, outcome));
  {
    Timed tm(c, G_UPDATE);
    if (c->opt == TDO_OPT_ADAM) {
      c->adam_t += 1;
      CU(c, launch_adam_update(c->theta64.as<double>(), c->delta.as<double>(), c->adam_m.as<double>(),
                               c->adam_v.as<double>(), c->P, c->adam_t, lr, c->adam_b1, c->adam_b2, c->adam_eps,
                               c->stream));
    } else {
      CU(c, launch_axpy_update(c->theta64.as<double>(), c->delta.as<double>(), lr, c->P, c->stream));
    }
    TRY(refresh_params(c));
    tm.done(c->model.embed == TDO_EMBED_CONV ? 3 : 2);
  }
  CU(c, cudaStreamSynchronize(c->stream));
  return TDO_OK;
}

static tdo_status sample_impl(tdo_ctx *c, size_t n_chains, size_t n_sweeps, uint64_t seed, uint64_t counter,
                              uint32_t *sig, uint32_t *sigp, uint32_t *samples_sig, uint32_t *samples_sigp,
                              uint64_t *accepted, int diag) {
  if (!c) return TDO_EINVAL;
  if (n_chains == 0) return TDO_OK;
  if (!sig || !sigp) return fail(c, TDO_EINVAL, "NULL buffer");
  if ((samples_sig == nullptr) != (samples_sigp == nullptr)) return fail(c, TDO_EINVAL, "give both sample buffers or neither");
  // chain state on device (staged both ways when host)
  const bool hs = !is_device_ptr(sig), hp = !is_device_ptr(sigp);
  uint32_t *dsig = sig, *dsigp = sigp;
  if (hs) { CU(c, c->stage_in[0].ensure(4 * n_chains)); dsig = c->stage_in[0].as<uint32_t>();
            CU(c, cudaMemcpyAsync(dsig, sig, 4 * n_chains, cudaMemcpyHostToDevice, c->stream)); }
  if (hp) { CU(c, c->stage_in[1].ensure(4 * n_chains)); dsigp = c->stage_in[1].as<uint32_t>();
            CU(c, cudaMemcpyAsync(dsigp, sigp, 4 * n_chains, cudaMemcpyHostToDevice, c->stream)); }
  uint32_t *dss = samples_sig, *dsp = samples_sigp;
  const size_t sbytes = 4 * n_chains * n_sweeps;
  const bool hss = samples_sig && !is_device_ptr(samples_sig), hsp = samples_sigp && !is_device_ptr(samples_sigp);
  if (hss) { CU(c, c->stage_in[2].ensure(sbytes)); dss = c->stage_in[2].as<uint32_t>(); }
  if (hsp) { CU(c, c->stage_in[3].ensure(sbytes)); dsp = c->stage_in[3].as<uint32_t>(); }
  CU(c, c->acc_u64.ensure(sizeof(unsigned long long)));
  CU(c, cudaMemsetAsync(c->acc_u64.p, 0, sizeof(unsigned long long), c->stream));
  Timed tm(c, G_SAMPLE);
  if (c->tc)
    CU(c, EVAL_LAUNCH(c, launch_sample_bf16, n_chains, n_sweeps, seed, counter, dsig, dsigp, dss, dsp,
                    c->acc_u64.as<unsigned long long>(), c->errflag.as<int>(), diag, c->n_sm, c->stream));
  else
    CU(c, launch_sample32(c->dm, n_chains, n_sweeps, seed, counter, dsig, dsigp, dss, dsp,
                          c->acc_u64.as<unsigned long long>(), diag, c->n_sm, c->stream));
  tm.done(1);
  if (hs) CU(c, cudaMemcpyAsync(sig, dsig, 4 * n_chains, cudaMemcpyDeviceToHost, c->stream));
  if (hp) CU(c, cudaMemcpyAsync(sigp, dsigp, 4 * n_chains, cudaMemcpyDeviceToHost, c->stream));
  if (hss) CU(c, cudaMemcpyAsync(samples_sig, dss, sbytes, cudaMemcpyDeviceToHost, c->stream));
  if (hsp) CU(c, cudaMemcpyAsync(samples_sigp, dsp, sbytes, cudaMemcpyDeviceToHost, c->stream));
  if (accepted) {
    if (is_device_ptr(accepted)) {
      CU(c, cudaMemcpyAsync(accepted, c->acc_u64.p, sizeof(uint64_t), cudaMemcpyDeviceToDevice, c->stream));
    } else {
      unsigned long long a = 0;
      CU(c, cudaMemcpyAsync(&a, c->acc_u64.p, sizeof(a), cudaMemcpyDeviceToHost, c->stream));
      CU(c, cudaStreamSynchronize(c->stream));
      *accepted = a;
    }
  }
  if (hs || hp || hss || hsp || accepted) {
    CU(c, cudaStreamSynchronize(c->stream));
    TRY(check_err_flag(c));
  }
  return TDO_OK;
}

extern "C" tdo_status tdo_sample(tdo_ctx *c, size_t n_chains, size_t n_sweeps, uint64_t seed, uint64_t counter,
                                 uint32_t *sig, uint32_t *sigp, uint32_t *samples_sig, uint32_t *samples_sigp,
                                 uint64_t *accepted) {
  return sample_impl(c, n_chains, n_sweeps, seed, counter, sig, sigp, samples_sig, samples_sigp, accepted, 0);
}

// The chain state alpha serves as both words of the pair (the kernels flip the same site in both).
extern "C" tdo_status tdo_sample_diag(tdo_ctx *c, size_t n_chains, size_t n_sweeps, uint64_t seed, uint64_t counter,
                                      uint32_t *alpha, uint32_t *samples, uint64_t *accepted) {
  return sample_impl(c, n_chains, n_sweeps, seed, counter, alpha, alpha, samples, samples, accepted, 1);
}

extern "C" tdo_status tdo_magnetisation(tdo_ctx *c, const uint32_t *alpha, size_t Ns, double *mag,
                                        double *sign_mean, double *local) {
  if (!c) return TDO_EINVAL;
  if (Ns == 0) return fail(c, TDO_EINVAL, "no samples");
  if (!alpha || !mag) return fail(c, TDO_EINVAL, "NULL buffer");
  const int n = c->n;
  const size_t rows = Ns * (size_t)(n + 1);
  const void *da;
  bool h1;
  TRY(stage_in(c, 0, alpha, 4 * Ns, &da, &h1));
  CU(c, c->obs_rs.ensure(4 * rows));
  CU(c, c->obs_rp.ensure(4 * rows));
  CU(c, c->obs_lr.ensure(8 * rows));
  CU(c, c->obs_part.ensure(8 * 7 * 256));
  CU(c, c->obs_out.ensure(8 * 8));
  double *dlocal = nullptr;
  if (local) {
    if (is_device_ptr(local)) dlocal = local;
    else { CU(c, c->obs_local.ensure(8 * 8 * Ns)); dlocal = c->obs_local.as<double>(); }
  }
  CU(c, launch_obs_rows((const uint32_t *)da, Ns, n, c->obs_rs.as<uint32_t>(), c->obs_rp.as<uint32_t>(), c->stream));
  TRY(forward_dev(c, c->obs_rs.as<uint32_t>(), c->obs_rp.as<uint32_t>(), rows, c->obs_lr.as<float2>()));
  CU(c, launch_obs_reduce((const uint32_t *)da, Ns, n, c->obs_lr.as<float2>(), dlocal, c->obs_part.as<double>(),
                          c->obs_out.as<double>(), c->stream));
  double h[6];
  CU(c, cudaMemcpyAsync(h, c->obs_out.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  if (local && dlocal != local) CU(c, cudaMemcpyAsync(local, dlocal, 8 * 8 * Ns, cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  TRY(check_err_flag(c));
  if (h[0] == 0.0) return fail(c, TDO_EINVAL, "the sample signs sum to zero");
  mag[0] = h[1] / h[0];
  mag[1] = h[3] / h[0];
  mag[2] = h[5] / h[0];
  if (sign_mean) *sign_mean = h[0] / (double)Ns;
  return TDO_OK;
}

extern "C" tdo_status tdo_purity(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t Ns, double *purity,
                                 double *stderr_) {
  if (!c) return TDO_EINVAL;
  if (Ns == 0) return fail(c, TDO_EINVAL, "no samples");
  if (!sig || !sigp || !purity) return fail(c, TDO_EINVAL, "NULL buffer");
  const void *ds, *dp;
  bool h1, h2;
  TRY(stage_in(c, 0, sig, 4 * Ns, &ds, &h1));
  TRY(stage_in(c, 1, sigp, 4 * Ns, &dp, &h2));
  CU(c, c->obs_rs.ensure(4 * 3 * Ns));
  CU(c, c->obs_rp.ensure(4 * 3 * Ns));
  CU(c, c->obs_lr.ensure(8 * 3 * Ns));
  CU(c, c->obs_part.ensure(8 * 7 * 256));
  CU(c, c->obs_out.ensure(8 * 8));
  CU(c, launch_pur_rows((const uint32_t *)ds, (const uint32_t *)dp, Ns, c->obs_rs.as<uint32_t>(),
                        c->obs_rp.as<uint32_t>(), c->stream));
  TRY(forward_dev(c, c->obs_rs.as<uint32_t>(), c->obs_rp.as<uint32_t>(), 3 * Ns, c->obs_lr.as<float2>()));
  CU(c, launch_pur_reduce(c->obs_lr.as<float2>(), Ns, c->obs_part.as<double>(), c->obs_out.as<double>(), c->stream));
  double h[2];
  CU(c, cudaMemcpyAsync(h, c->obs_out.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  TRY(check_err_flag(c));
  const double mean = h[0] / (double)Ns;
  if (!(mean > 0.0)) return fail(c, TDO_EINVAL, "non-positive estimate of Tr(rho)^2 / Tr(rho^2)");
  *purity = 1.0 / mean;
  if (stderr_) {   // delta method: se(1/m) = se(m) / m^2
    const double var = Ns > 1 ? (h[1] / (double)Ns - mean * mean) * (double)Ns / (double)(Ns - 1) : 0.0;
    *stderr_ = sqrt(var > 0.0 ? var / (double)Ns : 0.0) / (mean * mean);
  }
  return TDO_OK;
}

extern "C" tdo_status tdo_timing(tdo_ctx *c, int enable) {
  if (!c) return TDO_EINVAL;
  CU(c, cudaStreamSynchronize(c->stream));
  for (auto &r : c->trec) { c->epool.push_back(r.a); c->epool.push_back(r.b); }
  c->trec.clear();
  c->timing = enable != 0;
  return TDO_OK;
}

extern "C" tdo_status tdo_timing_read(tdo_ctx *c, const char *group, double *ms, long long *launches) {
  if (!c || !group) return TDO_EINVAL;
  int g = -1;
  const bool all = strcmp(group, "all") == 0;
  for (int i = 0; i < G_COUNT; ++i)
    if (strcmp(group, kGroupNames[i]) == 0) g = i;
  if (g < 0 && !all) return fail(c, TDO_EINVAL, "unknown timing group '%s'", group);
  CU(c, cudaStreamSynchronize(c->stream));
  double tot = 0;
  long long n = 0;
  for (auto &r : c->trec) {
    if (all ? r.group == G_SR_MV : r.group != g) continue;
    float e = 0;
    CU(c, cudaEventElapsedTime(&e, r.a, r.b));
    tot += e;
    n += r.launches;
  }
  if (ms) *ms = tot;
  if (launches) *launches = n;
  return TDO_OK;
}

extern "C" double tdo_schedule_value(long long step, double v0, long long i_switch, long long i_decay, double alpha) {
  if (step < i_switch) return v0;
  const double pi = 3.14159265358979323846;
  return v0 * (1.0 + cos(pi * (double)(step - i_switch) / (double)i_decay)) / 2.0 + alpha * v0;
}

// ----------------------------------------------------------------------------- whole-step graph
// One optimisation-workflow step (sweeps, connections, L_loc and cost, gradient, log-derivatives, SR solve,
// update) recorded once into a CUDA graph and replayed.  What the call-by-call step learns on the host
// in the middle of a step stays on the device: the connected-row count (every buffer and grid is sized for
// Ns x n_pat rows, and the kernels read the count from the scan's last offset), and the CG's iteration
// count (a conditional while node).  The sampler's counter and Adam's bias corrections come from device
// memory, uploaded before each launch; the update is skipped on the device when the solve fails or L_loc
// is not finite, and the host reports the failure after the launch, as the call-by-call step does.

// Tensor-core buffers of a forward store and its backward over `tiles` tiles.
static tdo_status graph_alloc_tiles(tdo_ctx *c, size_t tiles) {
  const int ts = 2 * (128 / (2 * c->n)) < 2 ? 2 : 2 * (128 / (2 * c->n));
  const size_t D = c->dm.d, img = (size_t)128 * D * 2, L = c->dm.layers;
  CU(c, c->act_x.ensure(L * tiles * img));
  CU(c, c->act_xmid.ensure(c->dm.ffn > 0 ? L * tiles * img : 16));
  CU(c, c->act_h.ensure(sizeof(float) * tiles * ts * D));
  CU(c, c->act_f.ensure(sizeof(float) * tiles * ts * 2));
  CU(c, c->act_dF.ensure(sizeof(float) * tiles * ts * 2));
  CU(c, c->act_dxa.ensure(sizeof(float) * tiles * 128 * D));
  CU(c, c->act_dxb.ensure(sizeof(float) * tiles * 128 * D));
  CU(c, c->act_dqkv.ensure(tiles * 128 * 3 * D * 2));
  return TDO_OK;
}

// Log-derivative buffers of B samples (jacobian_dev's).
static tdo_status graph_alloc_jac(tdo_ctx *c, size_t B) {
  if (bwdtc_jac_supported(c->dm)) {
    const size_t nv = 2 * B;
    CU(c, c->jac_vs.ensure(4 * nv));
    CU(c, c->jac_vp.ensure(4 * nv));
    CU(c, c->jac_vc.ensure(sizeof(float2) * nv));
    CU(c, c->jac_lr.ensure(sizeof(float2) * nv));
    return graph_alloc_tiles(c, tc_tiles(c, nv));
  }
  CU(c, c->scratch.ensure(sizeof(float) * bwd32_scratch_floats(c->dm, bwd32_grid(c->dm, B, 1, c->n_sm))));
  return TDO_OK;
}

// Every allocation of a recorded step, made before the recording (a recording may not allocate).
static tdo_status graph_alloc(tdo_ctx *c, size_t Ns, size_t ldo) {
  const size_t M = (size_t)c->n_pat, R = Ns * M, P = c->P;
  CU(c, c->conn_cnt.ensure(sizeof(int32_t) * Ns));
  CU(c, c->conn_sig.ensure(sizeof(uint32_t) * Ns * M));
  CU(c, c->conn_sigp.ensure(sizeof(uint32_t) * Ns * M));
  CU(c, c->conn_coef.ensure(sizeof(float2) * Ns * M));
  CU(c, c->offs.ensure(sizeof(int64_t) * (Ns + 1)));
  CU(c, c->fsig.ensure(sizeof(uint32_t) * R));
  CU(c, c->fsigp.ensure(sizeof(uint32_t) * R));
  CU(c, c->fcoef.ensure(sizeof(float2) * R));
  CU(c, c->flr.ensure(sizeof(float2) * R));
  CU(c, c->cot.ensure(sizeof(float2) * R));
  CU(c, c->lloc.ensure(sizeof(double2) * Ns));
  CU(c, c->l2.ensure(sizeof(double) * Ns));
  CU(c, c->stats.ensure(sizeof(double) * 4));
  TRY(graph_alloc_tiles(c, tc_tiles(c, R)));
  CU(c, c->gacc.ensure(sizeof(float) * 16 * ((P + 3) / 4 * 4)));
  CU(c, c->grad.ensure(sizeof(double) * P));
  CU(c, c->delta.ensure(sizeof(double) * P));
  CU(c, c->Obuf.ensure(sizeof(uint16_t) * 2 * ldo * Ns));
  const size_t nref = Ns < 64 ? Ns : 64;
  if (c->Obuf.bytes < sizeof(float) * 2 * P * nref) CU(c, c->oref_scratch.ensure(sizeof(float) * 2 * P * nref));
  CU(c, c->oref.ensure(sizeof(float) * 2 * P));
  TRY(graph_alloc_jac(c, nref));
  TRY(graph_alloc_jac(c, Ns));
  CU(c, c->srwork.ensure(sizeof(double) * sr_work_doubles(Ns, P)));
  CU(c, c->gstep.ensure(sizeof(StepDev)));
  if (!c->gstep_host) {
    void *h = nullptr;
    CU(c, cudaHostAlloc(&h, sizeof(StepDev), cudaHostAllocDefault));
    c->gstep_host = static_cast<StepDev *>(h);
  }
  return TDO_OK;
}

// The launches of one step, recorded on c->stream (capture in progress; graph_alloc done).
static tdo_status graph_record(tdo_ctx *c, uint32_t *ds, uint32_t *dp, size_t Ns, size_t n_sweeps, uint64_t seed,
                               double lr, double shift, size_t ldo) {
  StepDev *gs = c->gstep.as<StepDev>();
  const int M = c->n_pat;
  const size_t R = Ns * (size_t)M, tiles = tc_tiles(c, R), P = c->P;
  int *err = c->errflag.as<int>();
  if (n_sweeps > 0)
    CU(c, EVAL_LAUNCH(c, launch_sample_bf16, Ns, n_sweeps, seed, 0, ds, dp, nullptr, nullptr, nullptr, err, 0, c->n_sm,
                      c->stream, &gs->counter));
  CU(c, launch_connections(c->d_pat.as<ConnPattern>(), M, c->d_con.as<ConnContrib>(), ds, dp, Ns,
                           c->conn_cnt.as<int32_t>(), c->conn_sig.as<uint32_t>(), c->conn_sigp.as<uint32_t>(),
                           c->conn_coef.as<float2>(), c->stream));
  CU(c, launch_scan(c->conn_cnt.as<int32_t>(), Ns, c->offs.as<int64_t>(), c->stream));
  const int64_t *dtot = c->offs.as<int64_t>() + Ns;   // this step's connected rows
  CU(c, launch_compact(c->conn_cnt.as<int32_t>(), c->offs.as<int64_t>(), Ns, M, c->conn_sig.as<uint32_t>(),
                       c->conn_sigp.as<uint32_t>(), c->conn_coef.as<float2>(), c->fsig.as<uint32_t>(),
                       c->fsigp.as<uint32_t>(), c->fcoef.as<float2>(), c->stream));
  CU(c, TC_LAUNCH(c, launch_fwd_bf16_store, c->dm, c->dmb, c->fsig.as<uint32_t>(), c->fsigp.as<uint32_t>(), R,
                  c->flr.as<float2>(), err, c->n_sm, c->stream, c->act_x.as<uint8_t>(),
                  c->dm.ffn > 0 ? c->act_xmid.as<uint8_t>() : nullptr, c->act_h.as<float>(), c->act_f.as<float>(),
                  tiles, dtot));
  CU(c, cudaMemsetAsync(c->nonfinite.p, 0, sizeof(int), c->stream));
  CU(c, launch_lloc(c->offs.as<int64_t>(), Ns, c->fcoef.as<float2>(), c->flr.as<float2>(), c->lloc.as<double2>(),
                    c->l2.as<double>(), c->stats.as<double>(), c->nonfinite.as<int>(), c->stream));
  CU(c, launch_cotangent(c->offs.as<int64_t>(), Ns, c->fcoef.as<float2>(), c->flr.as<float2>(), c->lloc.as<double2>(),
                         c->stats.as<double>(), c->cot.as<float2>(), c->stream));
  const int copies = 16;
  const size_t stride = (P + 3) / 4 * 4;
  CU(c, cudaMemsetAsync(c->gacc.p, 0, sizeof(float) * copies * stride, c->stream));
  BwdTcBuffers bf{c->act_x.as<uint8_t>(), c->act_xmid.as<uint8_t>(), c->act_dqkv.as<uint8_t>(), c->act_h.as<float>(),
                  c->act_f.as<float>(), c->act_dF.as<float>(), c->act_dxa.as<float>(), c->act_dxb.as<float>(), tiles,
                  c->cscale.as<float>()};
  CU(c, TC_LAUNCH(c, launch_bwdtc, c->dm, c->dmb, c->bwl, bf, c->fsig.as<uint32_t>(), c->fsigp.as<uint32_t>(), R,
                  c->cot.as<float2>(), c->gacc.as<float>(), stride, c->flat_offsets, err, c->n_sm, c->stream, nullptr,
                  dtot));
  CU(c, launch_reduce_copies(c->gacc.as<float>(), copies, stride, P, c->grad.as<double>(), 0, c->stream,
                             c->cscale.as<float>() + 1));
  TRY(jacobian_bf16_for_sr(c, ds, dp, Ns, ldo));
  CU(c, sr_cg_capture(c->Obuf.p, 1, Ns, P, ldo, c->grad.as<double>(), c->delta.as<double>(), shift, c->sr_tol,
                      c->sr_max_iter, c->srwork.as<double>(), c->sr_product, &gs->warm, err, c->last_sr_shape,
                      c->stream));
  CU(c, launch_step_gate(sr_outcome_slot(c->srwork.as<double>(), Ns, P), c->nonfinite.as<int>(), err, &gs->ok,
                         c->stream));
  if (c->opt == TDO_OPT_ADAM)
    CU(c, launch_adam_update(c->theta64.as<double>(), c->delta.as<double>(), c->adam_m.as<double>(),
                             c->adam_v.as<double>(), P, 1, lr, c->adam_b1, c->adam_b2, c->adam_eps, c->stream, &gs->ok,
                             &gs->c1));
  else
    CU(c, launch_axpy_update(c->theta64.as<double>(), c->delta.as<double>(), lr, P, c->stream, &gs->ok));
  TRY(refresh_params(c));
  return TDO_OK;
}

static uint64_t bits_of(double v) {
  uint64_t u;
  memcpy(&u, &v, sizeof(u));
  return u;
}

// While a graph-mode step runs, the context's work goes to its graph stream, which starts after what
// was queued on the context's stream and ends before anything queued there later.
struct GraphStream {
  tdo_ctx *c;
  cudaStream_t saved;
  explicit GraphStream(tdo_ctx *ctx) : c(ctx), saved(ctx->stream) {
    cudaEventRecord(c->gevent, saved);
    cudaStreamWaitEvent(c->gstream, c->gevent, 0);
    c->stream = c->gstream;
  }
  ~GraphStream() {
    cudaEventRecord(c->gevent, c->gstream);
    cudaStreamWaitEvent(saved, c->gevent, 0);
    c->stream = saved;
  }
};

// tdo_vmc_step in graph mode: record the step when anything it was recorded for has changed, upload the
// step's values, launch, then read the outcome (one synchronisation).
static tdo_status vmc_step_graph(tdo_ctx *c, uint32_t *sig, uint32_t *sigp, size_t Ns, size_t n_sweeps,
                                 uint64_t seed, uint64_t *counter, double lr, double shift, double *cost) {
  if (Ns == 0) return fail(c, TDO_EINVAL, "Ns must be > 0");
  if (!sig || !sigp) return fail(c, TDO_EINVAL, "NULL buffer");
  if (!(shift > 0.0)) return fail(c, TDO_EINVAL, "diag_shift must be > 0");
  if (!c->gstream) CU(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
  if (!c->gevent) CU(c, cudaEventCreateWithFlags(&c->gevent, cudaEventDisableTiming));
  GraphStream on_graph_stream(c);
  const bool hs = !is_device_ptr(sig), hp = !is_device_ptr(sigp);
  uint32_t *ds = sig, *dp = sigp;
  if (hs) { CU(c, c->stage_in[0].ensure(4 * Ns)); ds = c->stage_in[0].as<uint32_t>(); }
  if (hp) { CU(c, c->stage_in[1].ensure(4 * Ns)); dp = c->stage_in[1].as<uint32_t>(); }
  const size_t P = c->P, ldo = (P + 3) / 4 * 4;
  TRY(graph_alloc(c, Ns, ldo));
  const std::vector<uint64_t> key = {Ns, n_sweeps, seed, bits_of(lr), bits_of(shift), bits_of(c->sr_tol),
                                     (uint64_t)c->sr_max_iter, (uint64_t)c->opt, bits_of(c->adam_b1),
                                     bits_of(c->adam_b2), bits_of(c->adam_eps), (uint64_t)c->sr_product,
                                     (uint64_t)(uintptr_t)ds, (uint64_t)(uintptr_t)dp, g_buf_gen};
  if (!c->gexec || key != c->gkey) {
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    CU(c, cudaStreamSynchronize(c->stream));
    CU(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
    c->capturing = true;
    const unsigned long long gen = g_buf_gen;
    const tdo_status rs = graph_record(c, ds, dp, Ns, n_sweeps, seed, lr, shift, ldo);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    c->capturing = false;
    if (rs != TDO_OK) { if (g) cudaGraphDestroy(g); return rs; }
    if (ee != cudaSuccess) { if (g) cudaGraphDestroy(g); CU(c, ee); }
    if (g_buf_gen != gen) {
      cudaGraphDestroy(g);
      return fail(c, TDO_ECUDA, "step graph: a buffer was allocated while the step was recorded");
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) { c->gexec = nullptr; CU(c, ei); }
    c->gkey = key;
    ++c->graph_captures;
  }
  // this step's values
  StepDev *h = c->gstep_host;
  h->counter = *counter;
  const long long t = c->adam_t + 1;
  h->c1 = 1.0 - pow(c->adam_b1, (double)t);
  h->c2 = 1.0 - pow(c->adam_b2, (double)t);
  h->warm = c->have_delta ? 1 : 0;
  h->ok = 0;
  if (!c->have_delta) CU(c, cudaMemsetAsync(c->delta.p, 0, sizeof(double) * P, c->stream));
  CU(c, cudaMemcpyAsync(c->gstep.p, h, sizeof(StepDev), cudaMemcpyHostToDevice, c->stream));
  if (hs) CU(c, cudaMemcpyAsync(ds, sig, 4 * Ns, cudaMemcpyHostToDevice, c->stream));
  if (hp) CU(c, cudaMemcpyAsync(dp, sigp, 4 * Ns, cudaMemcpyHostToDevice, c->stream));
  CU(c, cudaGraphLaunch(c->gexec, c->stream));
  ++c->graph_replays;
  *counter += (uint64_t)n_sweeps * (uint64_t)(2 * c->n);
  if (hs) CU(c, cudaMemcpyAsync(sig, ds, 4 * Ns, cudaMemcpyDeviceToHost, c->stream));
  if (hp) CU(c, cudaMemcpyAsync(sigp, dp, 4 * Ns, cudaMemcpyDeviceToHost, c->stream));
  double st[2];
  int nf = 0, ef = 0, ok = 0, iters = 0, outcome = 0, restarted = 0;
  double resid = 0, pap = 0;
  CU(c, cudaMemcpyAsync(st, c->stats.p, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaMemcpyAsync(&nf, c->nonfinite.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaMemcpyAsync(&ef, c->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaMemcpyAsync(&ok, &c->gstep.as<StepDev>()->ok, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(c, sr_cg_result(c->srwork.as<double>(), Ns, P, &iters, &resid, &outcome, &pap, &restarted, c->stream));
  c->last_sr_iters = iters;
  c->last_sr_resid = resid;
  c->last_sr_outcome = outcome;
  c->last_sr_pap = pap;
  c->last_sr_restarts = restarted;
  c->have_delta = ok != 0;
  if (ef) {
    CU(c, cudaMemsetAsync(c->errflag.p, 0, sizeof(int), c->stream));
    return fail(c, TDO_ETIMEOUT, "a tensor-core kernel's bounded wait gave up (results of that launch are invalid)");
  }
  if (nf) return fail(c, TDO_ENUMERIC, "non-finite log rho or L_loc (rho = 0 exactly, or non-finite parameters)");
  TRY(sr_outcome_status(c, outcome));
  if (c->opt == TDO_OPT_ADAM) c->adam_t = t;
  if (cost) *cost = st[0] / (double)Ns;
  return TDO_OK;
}

extern "C" tdo_status tdo_set_step_graph(tdo_ctx *c, int enable) {
  if (!c) return TDO_EINVAL;
  if (enable && !(c->tc && c->tc_bwd))
    return fail(c, TDO_EUNSUPPORTED, "the step graph needs a tensor-core context whose gradient runs on the tensor cores");
  c->step_graph = enable != 0;
  if (!c->step_graph && c->gexec) {
    cudaStreamSynchronize(c->gstream);
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gkey.clear();
  }
  return TDO_OK;
}

extern "C" tdo_status tdo_step_graph_stats(const tdo_ctx *c, long long *recordings, long long *launches) {
  if (!c) return TDO_EINVAL;
  if (recordings) *recordings = c->graph_captures;
  if (launches) *launches = c->graph_replays;
  return TDO_OK;
}

extern "C" tdo_status tdo_vmc_step(tdo_ctx *c, uint32_t *sig, uint32_t *sigp, size_t n_chains, size_t n_sweeps,
                                   uint64_t seed, uint64_t *counter, long long step, const tdo_schedule *sched,
                                   double *cost) {
  if (!c) return TDO_EINVAL;
  if (!counter) return fail(c, TDO_EINVAL, "NULL counter");
  const tdo_schedule paper = {0.0061, 30000, 40000, 0.001, 0.004, 30000, 40000, 0.01};
  const tdo_schedule &sc = sched ? *sched : paper;
  if (sc.i_decay <= 0 || sc.i_decay_sr <= 0) return fail(c, TDO_EINVAL, "decay periods must be > 0");
  if (c->step_graph) {
    const double lr = tdo_schedule_value(step, sc.eta0, sc.i_switch, sc.i_decay, sc.alpha);
    const double shift = tdo_schedule_value(step, sc.lambda0, sc.i_switch_sr, sc.i_decay_sr, sc.alpha_sr);
    return vmc_step_graph(c, sig, sigp, n_chains, n_sweeps, seed, counter, lr, shift, cost);
  }
  if (n_sweeps > 0) {
    TRY(tdo_sample(c, n_chains, n_sweeps, seed, *counter, sig, sigp, nullptr, nullptr, nullptr));
    *counter += (uint64_t)n_sweeps * (uint64_t)(2 * c->n);
  }
  const double lr = tdo_schedule_value(step, sc.eta0, sc.i_switch, sc.i_decay, sc.alpha);
  const double shift = tdo_schedule_value(step, sc.lambda0, sc.i_switch_sr, sc.i_decay_sr, sc.alpha_sr);
  return tdo_sr_step(c, sig, sigp, n_chains, lr, shift, cost);
}

extern "C" tdo_status tdo_set_optimizer(tdo_ctx *c, int kind, double beta1, double beta2, double eps) {
  if (!c) return TDO_EINVAL;
  if (kind != TDO_OPT_SGD && kind != TDO_OPT_ADAM) return fail(c, TDO_EINVAL, "unknown optimiser %d", kind);
  if (kind == TDO_OPT_ADAM) {
    if (!(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
      return fail(c, TDO_EINVAL, "Adam needs 0 <= beta1, beta2 < 1 and eps > 0");
    CU(c, c->adam_m.ensure(sizeof(double) * c->P));
    CU(c, c->adam_v.ensure(sizeof(double) * c->P));
    CU(c, cudaMemsetAsync(c->adam_m.p, 0, sizeof(double) * c->P, c->stream));
    CU(c, cudaMemsetAsync(c->adam_v.p, 0, sizeof(double) * c->P, c->stream));
    c->adam_b1 = beta1;
    c->adam_b2 = beta2;
    c->adam_eps = eps;
  }
  c->adam_t = 0;
  c->opt = kind;
  return TDO_OK;
}

extern "C" tdo_status tdo_set_sr_options(tdo_ctx *c, double tol, int max_iter) {
  if (!c) return TDO_EINVAL;
  if (!(tol >= 0.0) || max_iter < 0) return fail(c, TDO_EINVAL, "tol must be >= 0 and max_iter >= 0");
  c->sr_tol = tol;
  c->sr_max_iter = max_iter;
  return TDO_OK;
}

extern "C" tdo_status tdo_sr_info(const tdo_ctx *c, int *iters, double *resid) {
  if (!c) return TDO_EINVAL;
  if (iters) *iters = c->last_sr_iters;
  if (resid) *resid = c->last_sr_resid;
  return TDO_OK;
}

extern "C" tdo_status tdo_measure_peak(int kind, void *stream, double *tflops) {
  if ((kind != 0 && kind != 1) || !tflops) return TDO_EINVAL;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return TDO_ECUDA;
  }
  const cudaError_t e = measure_fma_peak(kind, n_sm, static_cast<cudaStream_t>(stream), tflops);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TDO_ECUDA;
  }
  return TDO_OK;
}

extern "C" tdo_status tdo_wait_selftest(tdo_ctx *c, long long spin_limit) {
  if (!c) return TDO_EINVAL;
  if (!c->tc) return fail(c, TDO_EUNSUPPORTED, "tdo_wait_selftest needs a tensor-core (BF16 / FP16) context");
  if (spin_limit < 1 || spin_limit > (1ll << 20))
    return fail(c, TDO_EINVAL, "tdo_wait_selftest: spin_limit must be in [1, 2^20]");
  CU(c, cudaMemsetAsync(c->errflag.p, 0, sizeof(int), c->stream));
  CU(c, launch_wait_probe(c->errflag.as<int>(), spin_limit, c->stream));
  return check_err_flag(c);
}

extern "C" tdo_status tdo_set_sr_product(tdo_ctx *c, int mode) {
  if (!c) return TDO_EINVAL;
  if (mode != TDO_SR_PRODUCT_TWO_PASS && mode != TDO_SR_PRODUCT_ONE_PASS && mode != TDO_SR_PRODUCT_GRID)
    return fail(c, TDO_EINVAL,
                "tdo_set_sr_product: mode must be TDO_SR_PRODUCT_TWO_PASS, TDO_SR_PRODUCT_ONE_PASS or TDO_SR_PRODUCT_GRID");
  c->sr_product = mode;
  return TDO_OK;
}

extern "C" tdo_status tdo_sr_apply(tdo_ctx *c, const uint32_t *O, size_t Ns, size_t ldo, const double *v, double shift,
                                   double *Ap) {
  if (!c) return TDO_EINVAL;
  if (Ns == 0) return fail(c, TDO_EINVAL, "Ns must be > 0");
  if (!O || !v || !Ap) return fail(c, TDO_EINVAL, "NULL buffer");
  if (ldo < c->P) return fail(c, TDO_EINVAL, "tdo_sr_apply: ldo must be >= the parameter count");
  if (!is_device_ptr(O) || !is_device_ptr(v) || !is_device_ptr(Ap))
    return fail(c, TDO_EINVAL, "tdo_sr_apply: O, v and Ap must be device memory");
  CU(c, c->srwork.ensure(sizeof(double) * sr_work_doubles(Ns, c->P)));
  CU(c, sr_apply_impl(O, Ns, c->P, ldo, v, shift, Ap, c->srwork.as<double>(), c->tc ? c->sr_product : TDO_SR_PRODUCT_TWO_PASS,
                      c->tc ? c->errflag.as<int>() : nullptr, c->last_sr_shape, c->stream));
  TRY(check_err_flag(c));
  CU(c, cudaStreamSynchronize(c->stream));
  return TDO_OK;
}

extern "C" tdo_status tdo_sr_product_shape(const tdo_ctx *c, int *one_pass, int *cluster, int *clusters) {
  if (!c) return TDO_EINVAL;
  if (one_pass) *one_pass = c->last_sr_shape[0];
  if (cluster) *cluster = c->last_sr_shape[1];
  if (clusters) *clusters = c->last_sr_shape[2];
  return TDO_OK;
}

extern "C" tdo_status tdo_sr_report(const tdo_ctx *c, int *outcome, double *last_pap, int *restarts) {
  if (!c) return TDO_EINVAL;
  if (outcome) *outcome = c->last_sr_outcome;
  if (last_pap) *last_pap = c->last_sr_pap;
  if (restarts) *restarts = c->last_sr_restarts;
  return TDO_OK;
}

// ----------------------------------------------------------------------------- no-allocation estimator
// A variant of tdo_local_estimator for callers that must not allocate device memory once they are
// running: e.g. a host application whose device memory is entirely owned by another allocator (a
// framework's caching pool that has reserved the free memory), or a latency-critical loop where the
// device-wide synchronisation that cudaMalloc / cudaFree can imply is not acceptable.  Its scratch is
// one file-scope device array of fixed size, present on every GPU that loads the library until the
// process exits.
#define TDO_NOALLOC_MAX_SAMPLES (1 << 14)   // samples per call
#define TDO_NOALLOC_MAX_ENTRIES (1 << 18)   // samples x tdo_max_connections() per call

namespace {
constexpr size_t kNaCnt = 0;                                                  // int32 [MAX_SAMPLES]
constexpr size_t kNaOffs = kNaCnt + 4ull * TDO_NOALLOC_MAX_SAMPLES;           // int64 [MAX_SAMPLES + 1]
constexpr size_t kNaLl2 = kNaOffs + 8ull * (TDO_NOALLOC_MAX_SAMPLES + 32);    // double [MAX_SAMPLES]
constexpr size_t kNaStats = kNaLl2 + 8ull * TDO_NOALLOC_MAX_SAMPLES;          // double [4]
constexpr size_t kNaFlag = kNaStats + 32;                                     // int (starts at zero)
constexpr size_t kNaCsig = kNaFlag + 256 - 32;                                // u32 [MAX_ENTRIES]
constexpr size_t kNaCsigp = kNaCsig + 4ull * TDO_NOALLOC_MAX_ENTRIES;
constexpr size_t kNaCcoef = kNaCsigp + 4ull * TDO_NOALLOC_MAX_ENTRIES;        // float2
constexpr size_t kNaFsig = kNaCcoef + 8ull * TDO_NOALLOC_MAX_ENTRIES;
constexpr size_t kNaFsigp = kNaFsig + 4ull * TDO_NOALLOC_MAX_ENTRIES;
constexpr size_t kNaFcoef = kNaFsigp + 4ull * TDO_NOALLOC_MAX_ENTRIES;        // float2
constexpr size_t kNaFlr = kNaFcoef + 8ull * TDO_NOALLOC_MAX_ENTRIES;          // float2
constexpr size_t kNaBytes = kNaFlr + 8ull * TDO_NOALLOC_MAX_ENTRIES;          // 10,813,952 bytes (about 10.8 MB)
static_assert(kNaCsig % 256 == 0 && kNaFlr % 16 == 0, "scratch alignment");
static_assert(kNaBytes == 10813952ull, "the documented size of the fixed scratch array");

void *g_noalloc_ptr[64];   // device address of g_noalloc_scratch per device (set up on first use)
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

extern "C" tdo_status tdo_local_estimator_noalloc(tdo_ctx *c, const uint32_t *sig, const uint32_t *sigp, size_t Ns,
                                                  double *lloc, double *cost, double *stderr_) {
  if (!c) return TDO_EINVAL;
  if (Ns == 0) return fail(c, TDO_EINVAL, "Ns must be > 0");
  if (!sig || !sigp || !lloc) return fail(c, TDO_EINVAL, "NULL buffer");
  if (!is_device_ptr(sig) || !is_device_ptr(sigp) || !is_device_ptr(lloc))
    return fail(c, TDO_EINVAL, "tdo_local_estimator_noalloc takes device pointers for sig, sigp and lloc");
  if (reinterpret_cast<uintptr_t>(lloc) % 16 != 0)
    return fail(c, TDO_EINVAL, "tdo_local_estimator_noalloc: lloc must be 16-byte aligned");
  const int M = c->n_pat;
  if (Ns > (size_t)TDO_NOALLOC_MAX_SAMPLES || Ns * (size_t)M > (size_t)TDO_NOALLOC_MAX_ENTRIES)
    return fail(c, TDO_EINVAL,
                "tdo_local_estimator_noalloc: Ns = %zu with %d connections per sample exceeds its fixed scratch "
                "(at most %d samples and %d samples x connections); split the call or use tdo_local_estimator",
                Ns, M, TDO_NOALLOC_MAX_SAMPLES, TDO_NOALLOC_MAX_ENTRIES);
  int dev = 0;
  CU(c, cudaGetDevice(&dev));
  if (dev != c->device)
    return fail(c, TDO_EINVAL, "tdo_local_estimator_noalloc: the current device (%d) is not the context's device (%d)",
                dev, c->device);
  if (dev < 0 || dev >= 64) return fail(c, TDO_EUNSUPPORTED, "device index %d out of range", dev);
  if (!g_noalloc_ptr[dev]) {   // one-time set-up on the context's device (current, checked above)
    void *p = nullptr;
    CU(c, cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  unsigned char *base = static_cast<unsigned char *>(g_noalloc_ptr[dev]);
  int32_t *cnt = reinterpret_cast<int32_t *>(base + kNaCnt);
  int64_t *offs = reinterpret_cast<int64_t *>(base + kNaOffs);
  double *l2 = reinterpret_cast<double *>(base + kNaLl2);
  double *stats = reinterpret_cast<double *>(base + kNaStats);
  int *flag = reinterpret_cast<int *>(base + kNaFlag);
  uint32_t *csig = reinterpret_cast<uint32_t *>(base + kNaCsig), *csigp = reinterpret_cast<uint32_t *>(base + kNaCsigp);
  float2 *ccoef = reinterpret_cast<float2 *>(base + kNaCcoef);
  uint32_t *fsig = reinterpret_cast<uint32_t *>(base + kNaFsig), *fsigp = reinterpret_cast<uint32_t *>(base + kNaFsigp);
  float2 *fcoef = reinterpret_cast<float2 *>(base + kNaFcoef), *flr = reinterpret_cast<float2 *>(base + kNaFlr);

  CU(c, cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  CU(c, launch_connections(c->d_pat.as<ConnPattern>(), M, c->d_con.as<ConnContrib>(), sig, sigp, Ns, cnt, csig, csigp,
                           ccoef, c->stream));
  CU(c, launch_scan(cnt, Ns, offs, c->stream));
  int64_t total = 0;
  CU(c, cudaMemcpyAsync(&total, offs + Ns, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  CU(c, launch_compact(cnt, offs, Ns, M, csig, csigp, ccoef, fsig, fsigp, fcoef, c->stream));
  if (c->tc)
    CU(c, EVAL_LAUNCH(c, launch_fwd_bf16, fsig, fsigp, (size_t)total, flr, c->errflag.as<int>(), c->n_sm,
                    c->stream));
  else
    CU(c, launch_fwd32(c->dm, fsig, fsigp, (size_t)total, flr, c->n_sm, c->stream));
  CU(c, launch_lloc(offs, Ns, fcoef, flr, reinterpret_cast<double2 *>(lloc), l2, stats, flag, c->stream));
  double st[2];
  int nf = 0;
  CU(c, cudaMemcpyAsync(st, stats, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaMemcpyAsync(&nf, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  TRY(check_err_flag(c));
  if (nf) return fail(c, TDO_ENUMERIC, "non-finite log rho or L_loc (rho = 0 exactly, or non-finite parameters)");
  const double mean = st[0] / (double)Ns;
  const double var = st[1] / (double)Ns - mean * mean;
  if (cost) *cost = mean;
  if (stderr_) *stderr_ = var > 0 ? sqrt(var / (double)Ns) : 0.0;
  return TDO_OK;
}
