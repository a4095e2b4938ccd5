// Kernels and launchers of the map i64 i32 container kind.
#include "hc_kernels.cuh"

HC_INSTANTIATE_KIND(hc::KIND_MAP_I64_I32, map_i64_i32)
