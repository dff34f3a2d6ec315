// batch_bf16c.cu -- batched temporal launchers, bf16 planes (FP32
// arithmetic): two halo lanes, depths 6-8.
#include "batch_kernels.cuh"

RDK_INSTANTIATE_BATCH(__nv_bfloat16, 6, 2)
RDK_INSTANTIATE_BATCH(__nv_bfloat16, 7, 2)
RDK_INSTANTIATE_BATCH(__nv_bfloat16, 8, 2)
