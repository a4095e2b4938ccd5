// Kernels and launchers of the set u64 container kind.
#include "hc_kernels.cuh"

HC_INSTANTIATE_KIND(hc::KIND_SET_U64, set_u64)
