// temporal_f32c.cu -- k_temporal launchers, float storage, depths 7-8.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(float, 7)
RDK_INSTANTIATE_TEMPORAL(float, 8)
