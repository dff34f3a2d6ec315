// adjoint_f32c.cu -- the adjoint's recompute / reverse launchers, FP32, two halo lanes, depths 5-6.
#include "adjoint_kernels.cuh"

RDK_INSTANTIATE_ADJ(float, 5, 2)
RDK_INSTANTIATE_ADJ(float, 6, 2)
