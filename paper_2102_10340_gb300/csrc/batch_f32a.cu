// batch_f32a.cu -- batched temporal launchers, FP32: one halo lane (depths 1-4)
// and two halo lanes, depths 1-2.
#include "batch_kernels.cuh"

RDK_INSTANTIATE_BATCH(float, 1, 1)
RDK_INSTANTIATE_BATCH(float, 2, 1)
RDK_INSTANTIATE_BATCH(float, 3, 1)
RDK_INSTANTIATE_BATCH(float, 4, 1)
RDK_INSTANTIATE_BATCH(float, 1, 2)
RDK_INSTANTIATE_BATCH(float, 2, 2)
