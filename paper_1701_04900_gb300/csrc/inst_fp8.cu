// Kernel and launcher instantiation for A stored as __nv_fp8_e4m3.
#include "launch.cuh"

ASYFLEXA_INSTANTIATE(__nv_fp8_e4m3)
