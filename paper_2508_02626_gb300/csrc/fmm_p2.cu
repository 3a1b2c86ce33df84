// Kernels and launchers of expansion order 2 (see fmm_order.cuh).
#define DAFMM_P 2
#include "fmm_order.cuh"
