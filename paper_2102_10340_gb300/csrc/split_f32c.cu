// split_f32c.cu -- warp-pair temporal launchers, FP32, depths 7-8.
#include "split_launch.cuh"

RDK_INSTANTIATE_SPLIT(float, 7)
RDK_INSTANTIATE_SPLIT(float, 8)
