// Kernel and launcher instantiation for A stored as double.
#include "launch.cuh"

ASYFLEXA_INSTANTIATE(double)
