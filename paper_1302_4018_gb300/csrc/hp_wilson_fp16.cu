// The Wilson solver, apply and stencil benchmark instantiated for FP16 (per-site norm) iteration.
#include "hp_wilson_impl.cuh"

HP_WILSON_INSTANTIATE(PR16, fp16)
