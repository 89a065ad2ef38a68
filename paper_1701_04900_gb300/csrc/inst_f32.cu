// Kernel and launcher instantiation for A stored as float.
#include "launch.cuh"

ASYFLEXA_INSTANTIATE(float)
