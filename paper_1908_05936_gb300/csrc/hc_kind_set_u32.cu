// Kernels and launchers of the set u32 container kind.
#include "hc_kernels.cuh"

HC_INSTANTIATE_KIND(hc::KIND_SET_U32, set_u32)
