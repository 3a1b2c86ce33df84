// Kernels and launchers of expansion order 5 (see fmm_order.cuh).
#define DAFMM_P 5
#include "fmm_order.cuh"
