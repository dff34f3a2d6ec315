// temporal_bf16c.cu -- k_temporal launchers, __nv_bfloat16 storage, depths 7-8.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 7)
RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 8)
