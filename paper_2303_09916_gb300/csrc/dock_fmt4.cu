// Chain and scoring kernels for map format 4 (see map_fmt in device_common.cuh).
#include "dock_kernels.cuh"
DSDP_INSTANTIATE_FMT(4)
