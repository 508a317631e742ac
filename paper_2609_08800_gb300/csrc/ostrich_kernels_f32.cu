// Step and adjoint kernels and their launchers, FP32 instantiation.
#define OST_REAL float
#include "ostrich_kernels.cuh"
