// batch_f32c.cu -- batched temporal launchers, FP32, two halo lanes, depths 6-8.
#include "batch_kernels.cuh"

RDK_INSTANTIATE_BATCH(float, 6, 2)
RDK_INSTANTIATE_BATCH(float, 7, 2)
RDK_INSTANTIATE_BATCH(float, 8, 2)
