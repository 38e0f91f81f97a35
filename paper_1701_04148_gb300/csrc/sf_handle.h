// sf_handle.h -- the host-side sketch handle shared by the runtime translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sf.h"
#include "sf_internal.h"

// Device-usable address of a caller buffer that a kernel reads or writes (keys, operations, query
// answers): device or managed memory as it is; page-locked host memory (cudaHostAlloc,
// cudaHostRegister) through its mapping into the device's address space, so the kernel itself
// moves those bytes over the host link and no staging copy is needed.  Pageable host memory and
// unknown pointers are refused with SF_ERR_INVALID before anything is launched.  NULL maps to NULL.
// *host (if given) tells whether the bytes live in host memory.
inline sf_status sf_device_access(const void* p, const void** out, bool* host = nullptr) {
    *out = nullptr;
    if (host) *host = false;
    if (!p) return SF_OK;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return SF_ERR_INVALID;
    }
    switch (at.type) {
        case cudaMemoryTypeDevice:
        case cudaMemoryTypeManaged:
            *out = p;
            return SF_OK;
        case cudaMemoryTypeHost:
            if (!at.devicePointer) return SF_ERR_INVALID;
            *out = at.devicePointer;
            if (host) *host = true;
            return SF_OK;
        default:
            return SF_ERR_INVALID;
    }
}

// Range checks of sf_params shared by every entry point that takes one (sf_required_bytes,
// sf_create, sf_update_batch_noalloc), so they accept the same parameters.
inline bool sf_params_ok(const sf_params* p) {
    if (!p) return false;
    if (p->d < 1 || p->d > SF_MAX_D) return false;
    if (p->w < 1 || p->w > 0x7FFFFFFFu) return false;
    if (p->z < 1 || p->z > SF_MAX_Z) return false;
    if (p->key_bytes < 1 || p->key_bytes > SF_MAX_KEY_BYTES) return false;
    if (p->chunk < 1 || p->chunk > SF_MAX_CHUNK) return false;
    if ((p->flags & ~(SF_FLAG_EXPLICIT_INDEX | SF_FLAG_SF4_DELETE | SF_FLAG_SHARED_DICT)) != 0) return false;
    if ((p->flags & SF_FLAG_EXPLICIT_INDEX) && p->key_bytes != 4) return false;
    if ((uint64_t)p->d * p->w * p->z > (1ull << 40)) return false;
    return true;
}

// Makes `dev` the current device for the scope of a call and restores the caller's device on
// every return path.
struct DeviceGuard {
    int prev = -1;
    bool switched = false, ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        if (prev != dev) {
            if (cudaSetDevice(dev) != cudaSuccess) return;
            switched = true;
        }
        ok = true;
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

struct sf_sketch {
    sf_params p;
    uint32_t* A;
    uint32_t* B;
    uint8_t* scratch;
    cudaStream_t stream;
    int device;
    int num_sms;
    int chunk_grid;
    int smem_optin;
    uint64_t rs[SF_MAX_D];
    uint32_t* ctrl;
    sfk::DictEntry* dict;   // in the scratch, or (SF_FLAG_SHARED_DICT) from sf_set_dictionary, or null
    uint32_t cap;
    const uint32_t* idx_table;
    uint32_t n_ids;
    uint64_t bar_epoch;     // grid barriers passed on this scratch buffer (monotonic counter)
    uint32_t claims_cap;    // per-block claim list length of the chunk kernel
    void* dag_ws;           // S = 1 sketches of width >= kDagMinW: workspace of the graph path, else nullptr
    // Update calls with page-locked host keys stage them through the upper half of the dictionary
    // region (unused by the single-iteration kernel) on a copy stream of their own, created at the
    // first such call.  stage_dirty: that half holds staged bytes, so it is zeroed before a launch
    // that reads the whole region as a dictionary; stage_foreign: such a launch ran since the last
    // staged call, so the next one waits for the sketch's stream before its first copy.
    sf_pipeline* stage_pipe;
    cudaStream_t stage_cs;
    bool stage_dirty, stage_foreign;
};

// Zeroes the staged half of a sketch's dictionary region on `st` before a launch that reads the
// whole region (the multi-iteration kernel, a batch), and marks the region as used by it.
inline sf_status sf_stage_release(sf_sketch* s, cudaStream_t st) {
    if (s->stage_dirty) {
        if (cudaMemsetAsync(reinterpret_cast<uint8_t*>(s->dict) + (uint64_t)s->cap * 16ull, 0,
                            (uint64_t)s->cap * 16ull, st) != cudaSuccess)
            return SF_ERR_CUDA;
        s->stage_dirty = false;
    }
    s->stage_foreign = true;
    return SF_OK;
}

