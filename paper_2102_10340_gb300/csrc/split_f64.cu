// split_f64.cu -- warp-pair temporal launchers, FP64, depths 2-4.
#include "split_launch.cuh"

RDK_INSTANTIATE_SPLIT(double, 2)
RDK_INSTANTIATE_SPLIT(double, 3)
RDK_INSTANTIATE_SPLIT(double, 4)
