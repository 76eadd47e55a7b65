// The Wilson solver, apply and stencil benchmark instantiated for FP32 iteration.
#include "hp_wilson_impl.cuh"

HP_WILSON_INSTANTIATE(PR32, fp32)
