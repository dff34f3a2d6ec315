// temporal_f16b.cu -- k_temporal launchers, __half storage, depths 5-6.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(__half, 5)
RDK_INSTANTIATE_TEMPORAL(__half, 6)
