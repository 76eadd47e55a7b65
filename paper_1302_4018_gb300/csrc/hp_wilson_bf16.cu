// The Wilson solver, apply and stencil benchmark instantiated for BF16 (per-site norm) iteration.
#include "hp_wilson_impl.cuh"

HP_WILSON_INSTANTIATE(PRB16, bf16)
