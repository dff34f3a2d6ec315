// adjoint_f32a.cu -- the adjoint's recompute / reverse launchers, FP32, one halo lane, depths 1-4.
#include "adjoint_kernels.cuh"

RDK_INSTANTIATE_ADJ(float, 1, 1)
RDK_INSTANTIATE_ADJ(float, 2, 1)
RDK_INSTANTIATE_ADJ(float, 3, 1)
RDK_INSTANTIATE_ADJ(float, 4, 1)
