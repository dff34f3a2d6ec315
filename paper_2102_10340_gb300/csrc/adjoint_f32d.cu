// adjoint_f32d.cu -- the adjoint's recompute / reverse launchers, FP32, two halo lanes, depth 7.
#include "adjoint_kernels.cuh"

RDK_INSTANTIATE_ADJ(float, 7, 2)
