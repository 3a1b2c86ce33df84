// Kernels and launchers of expansion order 6 (see fmm_order.cuh).
#define DAFMM_P 6
#include "fmm_order.cuh"
