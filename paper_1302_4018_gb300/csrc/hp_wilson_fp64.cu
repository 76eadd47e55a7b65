// The Wilson solver, apply and stencil benchmark instantiated for FP64 iteration.
#include "hp_wilson_impl.cuh"

HP_WILSON_INSTANTIATE(PR64, fp64)
