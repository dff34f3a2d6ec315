// split_f32b.cu -- warp-pair temporal launchers, FP32, depths 5-6.
#include "split_launch.cuh"

RDK_INSTANTIATE_SPLIT(float, 5)
RDK_INSTANTIATE_SPLIT(float, 6)
