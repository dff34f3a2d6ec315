// temporal_f16b.cu -- k_temporal launchers, __half storage (FP32 arithmetic), depths 5-8.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(__half, 5)
RDK_INSTANTIATE_TEMPORAL(__half, 6)
RDK_INSTANTIATE_TEMPORAL(__half, 7)
RDK_INSTANTIATE_TEMPORAL(__half, 8)
