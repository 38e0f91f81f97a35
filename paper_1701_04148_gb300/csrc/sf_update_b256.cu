// sf_update_b256.cu -- the chunked insert/delete kernels instantiated for 256-thread blocks (one of the
// launch shapes the batch autotuner chooses from; the kernels are in sf_update_kernels.cuh).
#include "sf_update_kernels.cuh"

namespace sfk {

template cudaError_t launch_batch_block<256>(const BatchArgs&, uint32_t, int, cudaStream_t);
template int blocks_per_sm_block<256>(uint32_t);

}  // namespace sfk
