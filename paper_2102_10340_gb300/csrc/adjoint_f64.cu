// adjoint_f64.cu -- the adjoint's recompute / reverse launchers, FP64, one halo lane (depths 1-2) and two
// (depths 1-4).
#include "adjoint_kernels.cuh"

RDK_INSTANTIATE_ADJ(double, 1, 1)
RDK_INSTANTIATE_ADJ(double, 2, 1)
RDK_INSTANTIATE_ADJ(double, 1, 2)
RDK_INSTANTIATE_ADJ(double, 2, 2)
RDK_INSTANTIATE_ADJ(double, 3, 2)
RDK_INSTANTIATE_ADJ(double, 4, 2)
