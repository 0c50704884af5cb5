// kernels_p2.cu -- kernels of precision 2 (mixed, float-float phase).
#include "kernels_impl.cuh"

namespace gwns {

template cudaError_t launch_likelihood_p<2>(int, int, const EventDev*, const double*, int, double*, int32_t*,
                                             cudaStream_t);
template cudaError_t launch_unit_likelihood_p<2>(int, int, const EventDev*, const double*, int, double*,
                                                  cudaStream_t);
template cudaError_t launch_walk_p<2>(int, int, const EventDev*, WalkTask*, const int32_t*, const int32_t*, int,
                                       cudaStream_t, bool);
template cudaError_t launch_hrss_p<2>(int, int, const EventDev*, WalkTask*, const int32_t*, const int32_t*, int,
                                       cudaStream_t);

}  // namespace gwns
