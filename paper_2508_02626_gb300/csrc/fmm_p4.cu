// Kernels and launchers of expansion order 4 (see fmm_order.cuh).
#define DAFMM_P 4
#include "fmm_order.cuh"
