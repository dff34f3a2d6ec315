// temporal_w16.cu -- k_temporal launchers at depth 1 for 16-bit planes read
// 8 values (16 bytes) per lane: the single step of bf16 / half handles.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(rdk::Wide16<__nv_bfloat16>, 1)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide16<__half>, 1)
