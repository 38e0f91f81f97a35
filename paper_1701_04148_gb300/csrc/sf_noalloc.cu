// sf_noalloc.cu -- an update entry point that needs no scratch buffer from the caller.
//
// Some callers cannot allocate device memory when they update a sketch: a packet-processing or
// serving loop that reserved all of its device memory up front and must not call cudaMalloc
// (which can block and synchronise the whole device), or a plugin that runs inside another
// framework's memory pool and has no allocator of its own.  sf_update_batch_noalloc serves them:
// the caller passes only the sketch counters and the update batch, and the per-chunk key
// dictionary and control words live in the fixed device array below, which every GPU that loads
// this library keeps until the process exits.
#include <mutex>

#include "sf.h"
#include "sf_handle.h"
#include "sf_internal.h"

namespace {

constexpr uint64_t kNoAllocCtrlBytes = 256;
constexpr uint64_t kNoAllocScratchBytes =
    kNoAllocCtrlBytes + (uint64_t)(4u * SF_NOALLOC_MAX_CHUNK) * sizeof(sfk::DictEntry);  // 2 MiB + 256 B

// Dictionary capacity inside the fixed array: a power of two >= 4 S (load factor <= 1/4).
constexpr uint32_t noalloc_capacity(uint32_t S) {
    uint32_t cap = 64;
    while (cap < 4u * S) cap <<= 1;
    return cap;
}
static_assert(kNoAllocCtrlBytes + (uint64_t)noalloc_capacity(SF_NOALLOC_MAX_CHUNK) * sizeof(sfk::DictEntry) <=
                  kNoAllocScratchBytes,
              "the largest dictionary must fit the fixed scratch array");
static_assert(sfk::kClaimLoadNoAlloc <= 8, "two halves of claim entries must fit the dictionary bytes of 4 S DictEntry slots");
static_assert(sfk::kClaimLoad <= 32, "two halves of claim entries must fit a sketch's dictionary bytes of 16 S DictEntry slots");

// The shared scratch: control words (error bits, barrier counter) then the key dictionary.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device.  Host code cannot pass the symbol
// itself to a kernel: on the host it names a host-side stand-in, not device memory.
sf_status scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return SF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SF_ERR_CUDA;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return SF_OK;
}

}  // namespace

extern "C" sf_status sf_update_batch_noalloc(const sf_params* p, uint32_t* fat_dev, uint32_t* slim_dev,
                                             const void* keys_dev, const int8_t* ops_dev, uint64_t n,
                                             uint32_t* err_dev, void* cuda_stream) {
    if (!fat_dev || !slim_dev) return SF_ERR_INVALID;
    // the same parameter range as sf_create, minus the explicit-index mode, and chunks that fit the array
    if (!sf_params_ok(p) || (p->flags & SF_FLAG_EXPLICIT_INDEX)) return SF_ERR_INVALID;
    if (p->chunk < 2 || p->chunk > SF_NOALLOC_MAX_CHUNK) return SF_ERR_INVALID;  // beyond the fixed scratch
    if (((uintptr_t)fat_dev & 15u) || ((uintptr_t)slim_dev & 15u)) return SF_ERR_INVALID;
    if (n == 0) return SF_OK;
    if (!keys_dev) return SF_ERR_INVALID;
    const void *keys_acc = nullptr, *ops_acc = nullptr;
    bool keys_host = false, ops_host = false;
    if (sf_device_access(keys_dev, &keys_acc, &keys_host) != SF_OK ||
        sf_device_access(ops_dev, &ops_acc, &ops_host) != SF_OK)
        return SF_ERR_INVALID;
    keys_dev = keys_acc;
    ops_dev = static_cast<const int8_t*>(ops_acc);
    if ((p->key_bytes == 4 || p->key_bytes == 8) && ((uintptr_t)keys_dev % p->key_bytes) != 0) return SF_ERR_INVALID;

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SF_ERR_CUDA;
    void* scratch = nullptr;
    const sf_status st = scratch_address(dev, &scratch);
    if (st != SF_OK) return st;
    const int bps = sfk::chunk_update_blocks_per_sm(p->d);
    if (bps <= 0) return SF_ERR_CUDA;
    const int grid = sms * (bps < 2 ? bps : 2);
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // The array keeps whatever the previous call left: zero the control words and the dictionary
    // (a call that stopped early may leave claimed entries behind).
    const uint32_t cap = noalloc_capacity(p->chunk);
    if (cudaMemsetAsync(scratch, 0, kNoAllocCtrlBytes + (uint64_t)cap * sizeof(sfk::DictEntry), stream) != cudaSuccess)
        return SF_ERR_CUDA;

    sfk::SketchRun one{};
    one.s.A = slim_dev;
    one.s.B = fat_dev;
    one.s.d = p->d;
    one.s.w = p->w;
    one.s.z = p->z;
    one.s.key_bytes = p->key_bytes;
    sfk::row_seeds(p->seed, p->d, one.s.rs);
    one.s.idx_table = nullptr;
    one.s.n_ids = 0;
    one.s.sf4_delete = (p->flags & SF_FLAG_SF4_DELETE) ? 1u : 0u;
    one.keys = (const uint8_t*)keys_dev;
    one.ops = ops_dev;
    one.op_const = 1;
    one.S = p->chunk;
    one.n = n;
    one.dict = (sfk::DictEntry*)((uint8_t*)scratch + kNoAllocCtrlBytes);
    one.cap_mask = cap - 1u;
    one.claim_mask = sfk::claim_capacity(p->chunk, sfk::kClaimLoadNoAlloc) - 1u;
    // the barrier counter was just zeroed, so this launch starts from barrier 0
    if (sfk::launch_chunk_update(one, (uint32_t*)scratch, 0, sfk::chunk_claims_cap(sfk::round_up32(p->chunk), grid),
                                 grid, stream, keys_host || ops_host) != cudaSuccess)
        return SF_ERR_CUDA;
    if (err_dev && cudaMemcpyAsync(err_dev, scratch, sizeof(uint32_t), cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
        return SF_ERR_CUDA;
    return SF_OK;
}
