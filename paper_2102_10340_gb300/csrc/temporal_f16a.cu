// temporal_f16a.cu -- k_temporal launchers, __half storage (FP32 arithmetic), depths 1-4.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(__half, 1)
RDK_INSTANTIATE_TEMPORAL(__half, 2)
RDK_INSTANTIATE_TEMPORAL(__half, 3)
RDK_INSTANTIATE_TEMPORAL(__half, 4)
