// Chain and scoring kernels for map format 3 (see map_fmt in device_common.cuh).
#include "dock_kernels.cuh"
DSDP_INSTANTIATE_FMT(3)
