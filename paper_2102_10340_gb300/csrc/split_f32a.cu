// split_f32a.cu -- warp-pair temporal launchers, FP32, depths 2-4.
#include "split_launch.cuh"

RDK_INSTANTIATE_SPLIT(float, 2)
RDK_INSTANTIATE_SPLIT(float, 3)
RDK_INSTANTIATE_SPLIT(float, 4)
