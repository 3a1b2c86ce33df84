// Kernels and launchers of expansion order 7 (see fmm_order.cuh).
#define DAFMM_P 7
#include "fmm_order.cuh"
