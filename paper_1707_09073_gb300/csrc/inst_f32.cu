// float instantiations of the particle kernels (production build)
#include "kernels.cuh"

namespace emc {
template void launch_flight<float>(const DevParams&, bool, int, int, int, int, cudaStream_t);
template void launch_init<float>(const DevParams&, bool, cudaStream_t);
template void launch_rescale<float>(const DevParams&, int, int64_t, const double*, cudaStream_t);
template void launch_inject<float>(const DevParams&, cudaStream_t);
template cudaError_t pair_prepare<float>(const DevParams&, bool, const DevParams&, bool, int, size_t*, int*);
template void launch_flight_pair<float>(const DevParams&, bool, int, int, const DevParams&, bool, int, int, int, int, size_t,
                                    cudaStream_t);
template void launch_free_counts<float>(const DevParams&, long long*, cudaStream_t);
template cudaError_t flight_set_smem<float>(size_t);
template size_t flight_smem_bytes<float>(int, int);
template int flight_blocks_per_sm<float>(bool, int, size_t);
template void launch_sort<float>(const DevParams&, const DevParams&, bool, uint32_t*, unsigned int*, const unsigned int*,
                                unsigned int*, int, cudaStream_t);
}  // namespace emc
