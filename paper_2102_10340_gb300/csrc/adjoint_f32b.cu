// adjoint_f32b.cu -- the adjoint's recompute / reverse launchers, FP32, two halo lanes, depths 1-4.
#include "adjoint_kernels.cuh"

RDK_INSTANTIATE_ADJ(float, 1, 2)
RDK_INSTANTIATE_ADJ(float, 2, 2)
RDK_INSTANTIATE_ADJ(float, 3, 2)
RDK_INSTANTIATE_ADJ(float, 4, 2)
