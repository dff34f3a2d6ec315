// temporal_w16.cu -- k_temporal launchers for 16-bit planes read 8 values
// (16 bytes) per lane: the single step of bf16 / half handles (depth 1) and
// RDCNN_VARIANT_TEMPORAL_WIDE (depths 1-4).
#include "temporal_launch.cuh"

RDK_INSTANTIATE_TEMPORAL(rdk::Wide<__nv_bfloat16>, 1)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide<__nv_bfloat16>, 2)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide<__nv_bfloat16>, 3)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide<__nv_bfloat16>, 4)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide<__half>, 1)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide<__half>, 2)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide<__half>, 3)
RDK_INSTANTIATE_TEMPORAL(rdk::Wide<__half>, 4)
