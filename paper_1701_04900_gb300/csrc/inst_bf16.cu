// Kernel and launcher instantiation for A stored as __nv_bfloat16.
#include "launch.cuh"

ASYFLEXA_INSTANTIATE(__nv_bfloat16)
