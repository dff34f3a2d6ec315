// batch_f32b.cu -- batched temporal launchers, FP32, two halo lanes, depths 3-5.
#include "batch_kernels.cuh"

RDK_INSTANTIATE_BATCH(float, 3, 2)
RDK_INSTANTIATE_BATCH(float, 4, 2)
RDK_INSTANTIATE_BATCH(float, 5, 2)
