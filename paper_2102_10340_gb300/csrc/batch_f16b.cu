// batch_f16b.cu -- batched temporal launchers, IEEE half planes (FP32
// arithmetic): two halo lanes, depths 3-5.
#include "batch_kernels.cuh"

RDK_INSTANTIATE_BATCH(__half, 3, 2)
RDK_INSTANTIATE_BATCH(__half, 4, 2)
RDK_INSTANTIATE_BATCH(__half, 5, 2)
