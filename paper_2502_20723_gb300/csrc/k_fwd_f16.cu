// The tensor-core forward, sampler and weight packing with FP16 operands (FP32 accumulation): the same
// kernels as k_fwd_bf16.cu, compiled with TDO_F16 = 1 into their own namespace (launchers named *_f16).
// FP16 keeps 11 significant bits against BF16's 8, which the log-derivatives and the cost gradient fed to
// the SR solve need (a BF16 rounding error in them is amplified by 1 / diag_shift).
#define TDO_F16 1
#include "k_fwd_bf16.cu"
