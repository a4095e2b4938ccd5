// Kernels and launchers of the map u64 u64 container kind.
#include "hc_kernels.cuh"

HC_INSTANTIATE_KIND(hc::KIND_MAP_U64_U64, map_u64_u64)
