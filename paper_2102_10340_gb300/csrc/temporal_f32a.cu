// temporal_f32a.cu -- k_temporal launchers, FP32, depths 1-4.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(float, 1)
RDK_INSTANTIATE_TEMPORAL(float, 2)
RDK_INSTANTIATE_TEMPORAL(float, 3)
RDK_INSTANTIATE_TEMPORAL(float, 4)
