// temporal_bf16b.cu -- k_temporal launchers, __nv_bfloat16 storage (FP32 arithmetic), depths 5-8.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 5)
RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 6)
RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 7)
RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 8)
