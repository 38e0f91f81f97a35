// sf_internal.h -- launchers shared by the host runtime and the kernel translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sf_device.cuh"

namespace sfk {

// One sketch's share of a chunked-update launch.  A launch walks its sketches in lockstep
// rounds: round r processes chunk r (updates [r*S, min((r+1)*S, n))) of every sketch.
struct SketchRun {
    SketchDesc s;
    const uint8_t* keys;
    const int8_t* ops;     // nullptr: every update is op_const
    int32_t op_const;
    uint32_t S;            // chunk size (semantic)
    uint64_t n;            // updates of this call
    uint64_t flat_base;    // first slot of this sketch in every round's flat slot range (multiple of 32)
    DictEntry* dict;       // this sketch's chunk dictionary
    uint32_t cap_mask;     // its capacity - 1 (power of two)
    uint32_t claim_mask;   // entries - 1 of each half of the same bytes as 8-byte claim entries (single-iteration launches)
};

struct BatchArgs {
    const SketchRun* runs;  // device table of n_runs sketches, sorted by flat_base; nullptr: `one`
    SketchRun one;
    uint32_t n_runs;
    uint32_t claims_cap;    // dictionary claims one block can make per round (shared-memory list)
    uint64_t flat_len;      // slots per round: sum of S rounded up to a multiple of 32
    uint64_t n_rounds;      // max over sketches of ceil(n / S)
    uint32_t* ctrl;         // error word + barrier counter
    uint64_t bar_base;      // grid barriers the counter has passed before this launch
    uint64_t timeout_ns;
    int32_t may_ins;        // some update of the launch may be an insertion
    int32_t may_del;        // ... a deletion
    uint2* claims_global;   // per-block claim lists in global memory (claims_cap each), or nullptr: shared memory
    uint32_t max_chunk;     // largest S of the launch's sketches
    int32_t keys_in_host;   // some sketch's keys (or operations) live in host memory, read over the host link
};

inline uint64_t round_up32(uint64_t x) { return (x + 31) & ~31ull; }

// Row seeds of a sketch (the hash reading of sf.h): the first d outputs of SplitMix64 started at
// `seed` (Steele, Lea, Flood, OOPSLA 2014) -- the state advances by the golden gamma and each
// output is the state passed through the generator's finaliser.  Entries d..kMaxD-1 are 0.
// Every host path that hands row seeds to a kernel (sketch handles, queries on an exported Slim,
// collector uploads, the allocation-free update) derives them here, so they cannot drift apart.
inline void row_seeds(uint64_t seed, uint32_t d, uint64_t* rs) {
    uint64_t st = seed;
    for (uint32_t i = 0; i < (uint32_t)kMaxD; ++i) {
        if (i >= d) {
            rs[i] = 0;
            continue;
        }
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        rs[i] = z ^ (z >> 31);
    }
}

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

// One request of a multi-request query launch (the collector's batches): its keys are
// key_bytes-wide at keys + key_off, its answers go to out[out_off .. out_off + n).
struct QueryReq {
    const uint32_t* A;     // Slim counters of the sketch version the request is bound to
    uint32_t d, w, key_bytes, n;
    uint64_t rs[kMaxD];
    uint64_t key_off;      // byte offset of the request's keys in the batch key buffer
    uint64_t out_off;      // first answer slot (prefix of the n of earlier requests)
};

struct MultiQueryArgs {
    const QueryReq* reqs;  // device, sorted by out_off
    uint32_t n_reqs;
    uint64_t total;        // sum of n
    const uint8_t* keys;
    uint32_t* out;
};

constexpr int kChunkBlock = 512;  // default block of the chunked-update kernels (also built for 256 and 128)
constexpr int kSeqBlock = 256;
constexpr int kQueryBlock = 256;
constexpr uint64_t kBarrierTimeoutNs = 2000000000ull;  // 2 s per wait
constexpr int kMaxClaimSmem = 96 * 1024;               // dynamic shared memory for the claim list

// Chunked update: one cooperative persistent launch per call (one sketch or a batch of sketches
// sharing d) of `grid` blocks of `block` threads (512, 256 or 128); 2 grid barriers per round.
cudaError_t launch_batch_update(const BatchArgs& a, uint32_t d, int grid, int block, cudaStream_t st);
// Per-block dispatch over d, instantiated for each block size in its own translation unit.
template <int B>
cudaError_t launch_batch_block(const BatchArgs& a, uint32_t d, int grid, cudaStream_t st);
template <int B>
int blocks_per_sm_block(uint32_t d);
// Dynamic shared memory a block may use for its claim list: 96 KiB at 512 threads, in proportion
// below, so that 512 / block blocks of a launch fit one SM.
inline int claim_smem_max(int block) { return kMaxClaimSmem * block / kChunkBlock; }
// Global claim-list bytes a launch over rounds of up to max_round_slots slots may need (any grid <= 1024 blocks).
inline uint64_t claims_global_bytes(uint64_t max_round_slots) {
    return (max_round_slots + 1024ull * kChunkBlock) * 8ull;
}
int chunk_update_blocks_per_sm(uint32_t d, int block = kChunkBlock);
// A launch whose rounds give every worker lane at most one update, with chunks of at most
// kClaimMaxChunk updates, runs the single-iteration kernel, which builds each chunk's dictionary one round ahead
// (8-byte claim entries with 16-bit positions and counts).  Both kernels pass two grid barriers per
// round.
constexpr uint32_t kClaimMaxChunk = 65536;
// Keys in host memory go to the multi-iteration kernel: the single-iteration kernel reads each
// chunk's keys inside a barrier window and re-reads a claimer's key to confirm a fingerprint match,
// so host-link latency would sit on its critical path (measured: 1.39x the multi-iteration kernel's
// time at Zipf 1 with pinned 13-byte keys, although 1.18x faster with device-resident ones).
inline bool chunk_rounds_single(uint64_t flat_len, uint32_t max_chunk, int grid, bool keys_in_host = false,
                                int block = kChunkBlock) {
    // warp 0 of each block only passes the grid barriers, so the workers hold block - 32 slots
    return !keys_in_host && flat_len <= (uint64_t)grid * (uint64_t)(block - 32) && max_chunk <= kClaimMaxChunk;
}
// Entries per half of the claim dictionary: a power of two >= load x S.  Two halves of 8-byte entries
// take 16 x that many bytes.  Sketches use load 16 (factor <= 1/16: short probe chains, measured
// faster than 1/8 and 1/4), which fits their DictEntry dictionary bytes (32 B x pow2 >= 16 S); the
// allocation-free entry point uses 8, which fits its fixed array (32 B x pow2 >= 4 S).
constexpr uint32_t kClaimLoad = 16;
constexpr uint32_t kClaimLoadNoAlloc = 8;
inline uint32_t claim_capacity(uint32_t S, uint32_t load = kClaimLoad) {
    uint64_t need = (uint64_t)load * (uint64_t)S;
    uint64_t cap = 64;
    while (cap < need) cap <<= 1;
    return (uint32_t)cap;
}
uint32_t chunk_claims_cap(uint64_t flat_len, int grid, int block = kChunkBlock);
// Single sketch: a batch of one.
cudaError_t launch_chunk_update(const SketchRun& one, uint32_t* ctrl, uint64_t bar_base, uint32_t claims_cap,
                                int grid, cudaStream_t st, bool keys_in_host = false);
// One-at-a-time update (S = 1).
cudaError_t launch_seq_update(const SeqArgs& a, cudaStream_t st, int smem_limit);
// One-at-a-time insertions as a dependency graph over pieces of up to kDagN updates (sf_seqdag.cu):
// for insertion-only calls on sketches of width >= kDagMinW, with a workspace of
// dag_workspace_bytes(d) bytes (4-byte aligned) owned by the sketch.
constexpr uint32_t kDagN = 131072;
constexpr uint32_t kDagMinW = 1024;
uint64_t dag_workspace_bytes(uint32_t d);
cudaError_t launch_seq_dag(const SketchDesc& s, const uint8_t* keys, uint64_t n, void* ws_base, uint32_t* ctrl,
                           int smem_limit, cudaStream_t st);
// Point queries.
cudaError_t launch_query(const QueryArgs& a, int num_sms, cudaStream_t st);
cudaError_t launch_multi_query(const MultiQueryArgs& a, int num_sms, cudaStream_t st);

// Dictionary capacity: a power of two >= 16 S for chunks of up to 65,536 updates, >= 8 S above.
// Each probe of the open-addressing table is one 128-bit CAS round trip and a chunk waits for its
// slowest key, so the longest probe chain matters: at load 1/4 it reaches ~11 slots over 65,536
// keys, at load 1/16 ~5.  Larger chunks run many warp-iterations per round, which hide a longer
// chain: there load 1/8 measured as fast as 1/16 (batches of 1,024 sketches at 16 and 32 rounds,
// a 2^28-update stream in chunks of 2^20) with half the bytes, and 1/4 1-2 % slower.  Chunks of
// up to 65,536 updates keep 16 S: the single-iteration kernel's two claim halves live in these bytes.
inline uint32_t dict_capacity(uint32_t S) {
    uint64_t need = (S > kClaimMaxChunk ? 8ull : 16ull) * (uint64_t)S;
    uint64_t cap = 64;
    while (cap < need) cap <<= 1;
    return (uint32_t)cap;
}

}  // namespace sfk
