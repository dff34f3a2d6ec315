// temporal_f16c.cu -- k_temporal launchers, __half storage, depths 7-8.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(__half, 7)
RDK_INSTANTIATE_TEMPORAL(__half, 8)
