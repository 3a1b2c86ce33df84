// Kernels and launchers of expansion order 8 (see fmm_order.cuh).
#define DAFMM_P 8
#include "fmm_order.cuh"
