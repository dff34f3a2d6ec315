// adjoint_f32e.cu -- the adjoint's recompute / reverse launchers, FP32, two halo lanes, depth 8.
#include "adjoint_kernels.cuh"

RDK_INSTANTIATE_ADJ(float, 8, 2)
