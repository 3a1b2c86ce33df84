// Kernels and launchers of expansion order 0 (see fmm_order.cuh).
#define DAFMM_P 0
#include "fmm_order.cuh"
