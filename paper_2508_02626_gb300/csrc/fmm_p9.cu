// Kernels and launchers of expansion order 9 (see fmm_order.cuh).
#define DAFMM_P 9
#include "fmm_order.cuh"
