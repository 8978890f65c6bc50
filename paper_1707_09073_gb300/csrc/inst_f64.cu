// double instantiations of the particle kernels (parity build)
#include "kernels.cuh"

namespace emc {
template void launch_flight<double>(const DevParams&, bool, int, int, int, int, cudaStream_t);
template void launch_init<double>(const DevParams&, bool, cudaStream_t);
template void launch_rescale<double>(const DevParams&, int, int64_t, const double*, cudaStream_t);
template void launch_inject<double>(const DevParams&, cudaStream_t);
template cudaError_t pair_prepare<double>(const DevParams&, bool, const DevParams&, bool, int, size_t*, int*);
template void launch_flight_pair<double>(const DevParams&, bool, int, int, const DevParams&, bool, int, int, int, int, size_t,
                                    cudaStream_t);
template void launch_free_counts<double>(const DevParams&, long long*, cudaStream_t);
template cudaError_t flight_set_smem<double>(size_t);
template size_t flight_smem_bytes<double>(int, int);
template int flight_blocks_per_sm<double>(bool, int, size_t);
template void launch_sort<double>(const DevParams&, const DevParams&, bool, uint32_t*, unsigned int*, const unsigned int*,
                                unsigned int*, int, cudaStream_t);
}  // namespace emc
