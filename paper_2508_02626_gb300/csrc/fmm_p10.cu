// Kernels and launchers of expansion order 10 (see fmm_order.cuh).
#define DAFMM_P 10
#include "fmm_order.cuh"
