// sf_update_b128.cu -- the chunked insert/delete kernels instantiated for 128-thread blocks (one of the
// launch shapes the batch autotuner chooses from; the kernels are in sf_update_kernels.cuh).
#include "sf_update_kernels.cuh"

namespace sfk {

template cudaError_t launch_batch_block<128>(const BatchArgs&, uint32_t, int, cudaStream_t);
template int blocks_per_sm_block<128>(uint32_t);

}  // namespace sfk
