// Kernels and launchers of expansion order 1 (see fmm_order.cuh).
#define DAFMM_P 1
#include "fmm_order.cuh"
