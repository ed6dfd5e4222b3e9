// WZ2 kernels at rate 24 (bits per value): instantiation unit.
#include "wz2_dispatch.cuh"
WHFF_INSTANTIATE_WZ2(24)
