// temporal_f32b.cu -- k_temporal launchers, FP32, depths 5-8.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(float, 5)
RDK_INSTANTIATE_TEMPORAL(float, 6)
RDK_INSTANTIATE_TEMPORAL(float, 7)
RDK_INSTANTIATE_TEMPORAL(float, 8)
