// temporal_bf16a.cu -- k_temporal launchers, __nv_bfloat16 storage (FP32 arithmetic), depths 1-4.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 1)
RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 2)
RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 3)
RDK_INSTANTIATE_TEMPORAL(__nv_bfloat16, 4)
