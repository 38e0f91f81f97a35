// sf_update.cu -- the chunked insert/delete kernels for 512-thread blocks, and the host dispatch over
// block sizes (the kernels themselves are in sf_update_kernels.cuh).
#include "sf_update_kernels.cuh"

namespace sfk {

template cudaError_t launch_batch_block<512>(const BatchArgs&, uint32_t, int, cudaStream_t);
template int blocks_per_sm_block<512>(uint32_t);
// instantiated in sf_update_b256.cu and sf_update_b128.cu
extern template cudaError_t launch_batch_block<256>(const BatchArgs&, uint32_t, int, cudaStream_t);
extern template int blocks_per_sm_block<256>(uint32_t);
extern template cudaError_t launch_batch_block<128>(const BatchArgs&, uint32_t, int, cudaStream_t);
extern template int blocks_per_sm_block<128>(uint32_t);

int chunk_update_blocks_per_sm(uint32_t d, int block) {
    switch (block) {
        case 512: return blocks_per_sm_block<512>(d);
        case 256: return blocks_per_sm_block<256>(d);
        case 128: return blocks_per_sm_block<128>(d);
        default: return 0;
    }
}

uint32_t chunk_claims_cap(uint64_t flat_len, int grid, int block) {
    // a block claims at most one slot per update it handles: iterations per round x block size
    const uint64_t per_iter = (uint64_t)grid * (uint64_t)block;
    const uint64_t iters = (flat_len + per_iter - 1) / per_iter;
    return (uint32_t)(iters * (uint64_t)block);
}

cudaError_t launch_batch_update(const BatchArgs& a, uint32_t d, int grid, int block, cudaStream_t st) {
    if (!a.claims_global && (uint64_t)a.claims_cap * sizeof(uint2) > (uint64_t)claim_smem_max(block))
        return cudaErrorInvalidValue;
    switch (block) {
        case 512: return launch_batch_block<512>(a, d, grid, st);
        case 256: return launch_batch_block<256>(a, d, grid, st);
        case 128: return launch_batch_block<128>(a, d, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_chunk_update(const SketchRun& one, uint32_t* ctrl, uint64_t bar_base, uint32_t claims_cap,
                                int grid, cudaStream_t st, bool keys_in_host) {
    BatchArgs a{};
    a.runs = nullptr;
    a.one = one;
    a.one.flat_base = 0;
    a.n_runs = 1;
    a.claims_cap = claims_cap;
    a.flat_len = round_up32(one.S);
    a.n_rounds = (one.n + one.S - 1) / one.S;
    a.ctrl = ctrl;
    a.bar_base = bar_base;
    a.timeout_ns = kBarrierTimeoutNs;
    a.may_ins = one.ops != nullptr || one.op_const > 0;
    a.may_del = one.ops != nullptr || one.op_const < 0;
    a.max_chunk = one.S;
    a.keys_in_host = keys_in_host ? 1 : 0;
    return launch_batch_update(a, one.s.d, grid, kChunkBlock, st);
}

}  // namespace sfk
