// batch_f16c.cu -- batched temporal launchers, IEEE half planes (FP32
// arithmetic): two halo lanes, depths 6-8.
#include "batch_kernels.cuh"

RDK_INSTANTIATE_BATCH(__half, 6, 2)
RDK_INSTANTIATE_BATCH(__half, 7, 2)
RDK_INSTANTIATE_BATCH(__half, 8, 2)
