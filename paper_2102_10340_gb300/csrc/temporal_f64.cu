// temporal_f64.cu -- k_temporal launchers, FP64, depths 1-4.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(double, 1)
RDK_INSTANTIATE_TEMPORAL(double, 2)
RDK_INSTANTIATE_TEMPORAL(double, 3)
RDK_INSTANTIATE_TEMPORAL(double, 4)
