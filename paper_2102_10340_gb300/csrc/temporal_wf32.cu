// temporal_wf32.cu -- k_temporal launchers for FP32 planes read 8 values
// (32 bytes) per lane (RDCNN_VARIANT_TEMPORAL_WIDE): one halo lane per side.
// Deeper pipelines spill at this lane width.
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(rdk::Wide<float>, 1)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide<float>, 2)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide<float>, 3)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide<float>, 4)
