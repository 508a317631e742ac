// Step and adjoint kernels and their launchers, FP64 instantiation.
#define OST_REAL double
#include "ostrich_kernels.cuh"
