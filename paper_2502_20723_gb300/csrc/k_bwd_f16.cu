// The tensor-core backward (cost-gradient VJP and per-configuration log-derivatives) with FP16 operands
// (FP32 accumulation): the same kernels as k_bwd_bf16.cu, compiled with TDO_F16 = 1 into their own
// namespace (launchers named *_f16).
#define TDO_F16 1
#include "k_bwd_bf16.cu"
