// temporal_bf16b.cu -- k_temporal launchers, __nv_bfloat16 storage, depths 5-6.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 5)
RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 6)
