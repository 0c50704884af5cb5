// kernels_p1.cu -- kernels of precision 1 (mixed, FP64 phase).
#include "kernels_impl.cuh"

namespace gwns {

template cudaError_t launch_likelihood_p<1>(int, int, const EventDev*, const double*, int, double*, int32_t*,
                                             cudaStream_t);
template cudaError_t launch_unit_likelihood_p<1>(int, int, const EventDev*, const double*, int, double*,
                                                  cudaStream_t);
template cudaError_t launch_walk_p<1>(int, int, const EventDev*, WalkTask*, const int32_t*, const int32_t*, int,
                                       cudaStream_t, bool);
template cudaError_t launch_hrss_p<1>(int, int, const EventDev*, WalkTask*, const int32_t*, const int32_t*, int,
                                       cudaStream_t);

}  // namespace gwns
