// batch_bf16a.cu -- batched temporal launchers, bf16 planes (FP32
// arithmetic): one halo lane (depths 1-4) and two halo lanes, depths 1-2.
#include "batch_kernels.cuh"

RDK_INSTANTIATE_BATCH(__nv_bfloat16, 1, 1)
RDK_INSTANTIATE_BATCH(__nv_bfloat16, 2, 1)
RDK_INSTANTIATE_BATCH(__nv_bfloat16, 3, 1)
RDK_INSTANTIATE_BATCH(__nv_bfloat16, 4, 1)
RDK_INSTANTIATE_BATCH(__nv_bfloat16, 1, 2)
RDK_INSTANTIATE_BATCH(__nv_bfloat16, 2, 2)
