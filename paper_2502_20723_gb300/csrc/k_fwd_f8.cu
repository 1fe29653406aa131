// The tensor-core forward and sampler with E4M3 (FP8) GEMM operands (tcgen05.mma kind::f8f6f4, FP32
// accumulation): the same kernels as k_fwd_bf16.cu, compiled with TDO_F8 = 1 into their own namespace
// (launchers named *_f8).  Weights carry one power-of-two scale per matrix and every activation image one
// per tile, so that E4M3's 3 mantissa bits cover each tensor's own range; the attention, softmax, GELU,
// residual stream and head stay as in the 16-bit builds.  Evaluation only (log rho, the local estimator's
// rows, the sampler): the gradient and the log-derivatives use the FP16 kernels.
#define TDO_F8 1
#include "k_fwd_bf16.cu"
