// sf_handle.h -- the host-side sketch handle shared by the runtime translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sf.h"
#include "sf_internal.h"

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
    sfk::DictEntry* dict;
    uint32_t cap;
    const uint32_t* idx_table;
    uint32_t n_ids;
    uint64_t bar_epoch;     // grid barriers passed on this scratch buffer (monotonic counter)
    uint32_t claims_cap;    // per-block claim list length of the chunk kernel
};

