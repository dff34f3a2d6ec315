// batch_f64.cu -- batched temporal launchers, FP64 (depths 1-2 with one halo
// lane, 1-4 with two).
#include "batch_kernels.cuh"

RDK_INSTANTIATE_BATCH(double, 1, 1)
RDK_INSTANTIATE_BATCH(double, 2, 1)
RDK_INSTANTIATE_BATCH(double, 1, 2)
RDK_INSTANTIATE_BATCH(double, 2, 2)
RDK_INSTANTIATE_BATCH(double, 3, 2)
RDK_INSTANTIATE_BATCH(double, 4, 2)
