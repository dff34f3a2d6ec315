// batch_f16a.cu -- batched temporal launchers, IEEE half planes (FP32
// arithmetic): one halo lane (depths 1-4) and two halo lanes, depths 1-2.
#include "batch_kernels.cuh"

RDK_INSTANTIATE_BATCH(__half, 1, 1)
RDK_INSTANTIATE_BATCH(__half, 2, 1)
RDK_INSTANTIATE_BATCH(__half, 3, 1)
RDK_INSTANTIATE_BATCH(__half, 4, 1)
RDK_INSTANTIATE_BATCH(__half, 1, 2)
RDK_INSTANTIATE_BATCH(__half, 2, 2)
