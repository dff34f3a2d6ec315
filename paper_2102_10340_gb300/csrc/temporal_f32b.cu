// temporal_f32b.cu -- k_temporal launchers, float storage, depths 5-6.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(float, 5)
RDK_INSTANTIATE_TEMPORAL(float, 6)
