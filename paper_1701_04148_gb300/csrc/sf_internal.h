// sf_internal.h -- launchers shared by the host runtime and the kernel translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sf_device.cuh"

namespace sfk {

struct ChunkArgs {
    SketchDesc s;
    const uint8_t* keys;
    const int8_t* ops;    // nullptr: every update is op_const
    int32_t op_const;
    uint64_t n;
    uint32_t S;
    uint32_t cap_mask;    // dictionary capacity - 1 (power of two)
    DictEntry* dict;
    uint32_t* ctrl;
    uint64_t bar_base;    // grid barriers this scratch buffer has passed before this launch
    uint32_t claims_cap;  // dictionary claims one block can make per chunk (shared-memory list)
    uint64_t timeout_ns;
};

struct SeqArgs {
    SketchDesc s;
    const uint8_t* keys;
    const int8_t* ops;
    int32_t op_const;
    uint64_t n;
    uint32_t* ctrl;
    int slim_in_smem;
};

struct QueryArgs {
    SketchDesc s;         // A = the Slim counters, B unused
    const uint8_t* keys;
    uint64_t n;
    uint32_t* out;
};

constexpr int kChunkBlock = 512;
constexpr int kSeqBlock = 256;
constexpr int kQueryBlock = 256;
constexpr uint64_t kBarrierTimeoutNs = 2000000000ull;  // 2 s per wait

// Chunked update: one cooperative persistent launch for the whole call; 2 grid barriers per chunk.
cudaError_t launch_chunk_update(const ChunkArgs& a, int grid, cudaStream_t st);
int chunk_update_blocks_per_sm(uint32_t d);
uint32_t chunk_claims_cap(uint32_t S, int grid);
// One-at-a-time update (S = 1).
cudaError_t launch_seq_update(const SeqArgs& a, cudaStream_t st, int smem_limit);
// Point queries.
cudaError_t launch_query(const QueryArgs& a, int num_sms, cudaStream_t st);

// Dictionary capacity: a power of two >= 4 S (load factor <= 1/4 keeps probe chains short).
inline uint32_t dict_capacity(uint32_t S) {
    uint64_t need = 4ull * (uint64_t)S;
    uint64_t cap = 64;
    while (cap < need) cap <<= 1;
    return (uint32_t)cap;
}

}  // namespace sfk
