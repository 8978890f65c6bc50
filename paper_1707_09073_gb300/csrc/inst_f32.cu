// float (production) instantiations of the particle kernels
#include "kernels.cuh"

namespace emc {
template void launch_flight<float>(const DevParams&, bool, int, int, int, cudaStream_t);
template void launch_init<float>(const DevParams&, bool, cudaStream_t);
template void launch_inject<float>(const DevParams&, cudaStream_t);
template cudaError_t flight_set_smem<float>(size_t);
template size_t flight_smem_bytes<float>(int);
}  // namespace emc
