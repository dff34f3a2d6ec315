// batch_bf16b.cu -- batched temporal launchers, bf16 planes (FP32
// arithmetic): two halo lanes, depths 3-5.
#include "batch_kernels.cuh"

RDK_INSTANTIATE_BATCH(__nv_bfloat16, 3, 2)
RDK_INSTANTIATE_BATCH(__nv_bfloat16, 4, 2)
RDK_INSTANTIATE_BATCH(__nv_bfloat16, 5, 2)
