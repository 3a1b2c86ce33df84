// Kernels and launchers of expansion order 3 (see fmm_order.cuh).
#define DAFMM_P 3
#include "fmm_order.cuh"
