// sf_api.cu -- host runtime behind the C ABI of include/sf.h.
//
// A handle binds caller-owned device buffers (Fat, Slim, scratch) to one CUDA stream.  No call
// allocates device memory.  Device-side errors are latched in the control words at the start
// of the scratch buffer and collected by sf_sync.
#include <cstdint>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "sf.h"
#include "sf_internal.h"
#include "sf_seqdag.h"

#include "sf_handle.h"

namespace {

constexpr uint64_t kCtrlBytes = 256;

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// defined with the pipeline below
sf_status run_staged(sf_sketch* s, const void* keys_host, const int8_t* ops_host, int op_const, uint64_t n,
                     bool* staged);
void pipeline_release(sf_pipeline* p);

sfk::SketchDesc desc_of(const sf_sketch* s) {
    sfk::SketchDesc d{};
    d.A = s->A;
    d.B = s->B;
    d.d = s->p.d;
    d.w = s->p.w;
    d.z = s->p.z;
    d.key_bytes = s->p.key_bytes;
    for (int i = 0; i < SF_MAX_D; ++i) d.rs[i] = s->rs[i];
    d.idx_table = s->idx_table;
    d.n_ids = s->n_ids;
    d.sf4_delete = (s->p.flags & SF_FLAG_SF4_DELETE) ? 1u : 0u;
    return d;
}

sf_status run_update(sf_sketch* s, const void* keys_in, const int8_t* ops_in, int op_const, uint64_t n) {
    if (!s) return SF_ERR_INVALID;
    if (n == 0) return SF_OK;
    if (!keys_in) return SF_ERR_INVALID;
    const void *keys = nullptr, *ops_v = nullptr;
    bool keys_host = false, ops_host = false;
    if (sf_device_access(keys_in, &keys, &keys_host) != SF_OK || sf_device_access(ops_in, &ops_v, &ops_host) != SF_OK)
        return SF_ERR_INVALID;
    const int8_t* ops = static_cast<const int8_t*>(ops_v);
    const uint32_t kb = s->p.key_bytes;
    if ((kb == 4 || kb == 8) && ((uintptr_t)keys % kb) != 0) return SF_ERR_INVALID;
    if ((s->p.flags & SF_FLAG_EXPLICIT_INDEX) && !s->idx_table) return SF_ERR_INVALID;
    DeviceGuard guard(s->device);
    if (!guard.ok) return SF_ERR_CUDA;
    // page-locked host keys (and operations) of a sketch whose chunk rounds run the single-iteration
    // kernel: staged through the idle half of its dictionary region, so that kernel reads them from
    // device memory (the one that reads host keys itself waits on the host link every round)
    const bool single = s->p.chunk > 1 && sfk::chunk_rounds_single(sfk::round_up32(s->p.chunk), s->p.chunk,
                                                                   s->chunk_grid, keys_host || ops_host);
    if (keys_host && (!ops || ops_host) && s->p.chunk > 1 && !(s->p.flags & SF_FLAG_SHARED_DICT) && s->dict &&
        sfk::chunk_rounds_single(sfk::round_up32(s->p.chunk), s->p.chunk, s->chunk_grid)) {
        bool staged = false;
        const sf_status st = run_staged(s, keys_in, ops_in, op_const, n, &staged);
        if (staged || st != SF_OK) return st;
    }
    cudaError_t e;
    if (s->p.chunk == 1 && s->dag_ws && !ops && op_const > 0) {
        // insertions only: the dependency-graph path (sf_seqdag.cu)
        e = sfk::launch_seq_dag(desc_of(s), (const uint8_t*)keys, n, s->dag_ws, s->ctrl, s->smem_optin, s->stream);
    } else if (s->p.chunk == 1) {
        sfk::SeqArgs a{};
        a.s = desc_of(s);
        a.keys = (const uint8_t*)keys;
        a.ops = ops;
        a.op_const = op_const;
        a.n = n;
        a.ctrl = s->ctrl;
        e = sfk::launch_seq_update(a, s->stream, s->smem_optin);
    } else {
        if (!s->dict) return SF_ERR_INVALID;  // SF_FLAG_SHARED_DICT without sf_set_dictionary
        // the multi-iteration kernel reads the whole dictionary region
        if (!single && !(s->p.flags & SF_FLAG_SHARED_DICT) && sf_stage_release(s, s->stream) != SF_OK)
            return SF_ERR_CUDA;
        sfk::SketchRun one{};
        one.s = desc_of(s);
        one.keys = (const uint8_t*)keys;
        one.ops = ops;
        one.op_const = op_const;
        one.S = s->p.chunk;
        one.n = n;
        one.flat_base = 0;
        one.dict = s->dict;
        one.cap_mask = s->cap - 1u;
        one.claim_mask = sfk::claim_capacity(s->p.chunk) - 1u;
        e = sfk::launch_chunk_update(one, s->ctrl, s->bar_epoch, s->claims_cap, s->chunk_grid, s->stream,
                                     keys_host || ops_host);
        if (e == cudaSuccess) s->bar_epoch += 2ull * ((n + s->p.chunk - 1) / s->p.chunk);
    }
    return e == cudaSuccess ? SF_OK : SF_ERR_CUDA;
}

}  // namespace

extern "C" {

const char* sf_status_str(sf_status s) {
    switch (s) {
        case SF_OK: return "ok";
        case SF_ERR_INVALID: return "invalid argument";
        case SF_ERR_OOM: return "buffer too small";
        case SF_ERR_CUDA: return "CUDA runtime error";
        case SF_ERR_TIMEOUT: return "device wait timed out";
        case SF_ERR_UNDERFLOW: return "delete of an item that was not inserted (Fat counter underflow)";
        case SF_ERR_BUDGET: return "not admissible under the memory budget";
        case SF_ERR_VERSION: return "Slim header mismatch";
        case SF_PENDING: return "pending";
        default: return "unknown status";
    }
}

sf_status sf_required_bytes(const sf_params* p, uint64_t* fat_bytes, uint64_t* slim_bytes,
                            uint64_t* scratch_bytes) {
    if (!sf_params_ok(p)) return SF_ERR_INVALID;
    if (fat_bytes) *fat_bytes = (uint64_t)p->d * p->w * p->z * 4ull;
    if (slim_bytes) *slim_bytes = (uint64_t)p->d * p->w * 4ull;
    if (scratch_bytes) {
        const uint64_t cap = (p->chunk > 1 && !(p->flags & SF_FLAG_SHARED_DICT)) ? sfk::dict_capacity(p->chunk) : 0;
        // S = 1 sketches wide enough for the dependency-graph path also hold its workspace
        const uint64_t dag = (p->chunk == 1 && sfk::dag_eligible(p->w, p->z)) ? sfk::dag_workspace_bytes(p->d) : 0;
        *scratch_bytes = kCtrlBytes + cap * sizeof(sfk::DictEntry) + dag;
    }
    return SF_OK;
}

sf_status sf_dictionary_bytes(const sf_params* p, uint64_t* dict_bytes) {
    if (!sf_params_ok(p) || !dict_bytes) return SF_ERR_INVALID;
    *dict_bytes = p->chunk > 1 ? (uint64_t)sfk::dict_capacity(p->chunk) * sizeof(sfk::DictEntry) : 0;
    return SF_OK;
}

sf_status sf_set_dictionary(sf_sketch* s, void* dict_dev, uint64_t bytes) {
    if (!s || !(s->p.flags & SF_FLAG_SHARED_DICT) || s->p.chunk < 2 || !dict_dev || !aligned16(dict_dev))
        return SF_ERR_INVALID;
    const uint64_t need = (uint64_t)s->cap * sizeof(sfk::DictEntry);
    if (bytes < need) return SF_ERR_INVALID;
    DeviceGuard guard(s->device);
    if (!guard.ok) return SF_ERR_CUDA;
    if (cudaMemsetAsync(dict_dev, 0, need, s->stream) != cudaSuccess) return SF_ERR_CUDA;
    s->dict = (sfk::DictEntry*)dict_dev;
    return SF_OK;
}

sf_status sf_create(const sf_params* p, void* fat_dev, void* slim_dev, void* scratch_dev,
                    void* cuda_stream, sf_sketch** out) {
    if (!out) return SF_ERR_INVALID;
    *out = nullptr;
    if (!sf_params_ok(p)) return SF_ERR_INVALID;
    if (!fat_dev || !slim_dev || !scratch_dev) return SF_ERR_INVALID;
    if (!aligned16(fat_dev) || !aligned16(slim_dev) || !aligned16(scratch_dev)) return SF_ERR_INVALID;
    sf_sketch* s = new (std::nothrow) sf_sketch();
    if (!s) return SF_ERR_OOM;
    s->p = *p;
    s->A = (uint32_t*)slim_dev;
    s->B = (uint32_t*)fat_dev;
    s->scratch = (uint8_t*)scratch_dev;
    s->stream = (cudaStream_t)cuda_stream;
    s->ctrl = (uint32_t*)scratch_dev;
    s->dict = (p->flags & SF_FLAG_SHARED_DICT) ? nullptr : (sfk::DictEntry*)((uint8_t*)scratch_dev + kCtrlBytes);
    s->cap = p->chunk > 1 ? sfk::dict_capacity(p->chunk) : 0;
    s->dag_ws = (p->chunk == 1 && sfk::dag_eligible(p->w, p->z)) ? (uint8_t*)scratch_dev + kCtrlBytes : nullptr;
    sfk::row_seeds(p->seed, p->d, s->rs);
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device) != cudaSuccess) {
        delete s;
        return SF_ERR_CUDA;
    }
    const int bps = sfk::chunk_update_blocks_per_sm(p->d);
    if (bps <= 0) {
        delete s;
        return SF_ERR_CUDA;
    }
    s->chunk_grid = s->num_sms * (bps < 2 ? bps : 2);
    s->stage_foreign = true;  // the first staged call waits for the sketch's earlier work
    s->claims_cap = sfk::chunk_claims_cap(sfk::round_up32(p->chunk), s->chunk_grid);
    s->bar_epoch = 0;
    uint64_t fb, sb, xb;
    sf_required_bytes(p, &fb, &sb, &xb);
    if (cudaMemsetAsync(fat_dev, 0, fb, s->stream) != cudaSuccess ||
        cudaMemsetAsync(slim_dev, 0, sb, s->stream) != cudaSuccess ||
        cudaMemsetAsync(scratch_dev, 0, xb, s->stream) != cudaSuccess) {
        delete s;
        return SF_ERR_CUDA;
    }
    *out = s;
    return SF_OK;
}

sf_status sf_destroy(sf_sketch* s) {
    if (!s) return SF_ERR_INVALID;
    {
        DeviceGuard guard(s->device);
        if (s->stage_pipe) pipeline_release(s->stage_pipe);  // its events go once their work completed
        if (s->stage_cs) cudaStreamDestroy(s->stage_cs);
    }
    delete s;
    return SF_OK;
}

sf_status sf_reset(sf_sketch* s) {
    if (!s) return SF_ERR_INVALID;
    DeviceGuard guard(s->device);
    if (!guard.ok) return SF_ERR_CUDA;
    uint64_t fb = 0, sb = 0, xb = 0;
    if (sf_required_bytes(&s->p, &fb, &sb, &xb) != SF_OK) return SF_ERR_INVALID;
    // chunked sketches: control words only (the dictionary is zero between calls); chunk-1: all
    const uint64_t scratch_bytes = s->p.chunk > 1 ? kCtrlBytes : xb;
    if (cudaMemsetAsync(s->B, 0, fb, s->stream) != cudaSuccess || cudaMemsetAsync(s->A, 0, sb, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->scratch, 0, scratch_bytes, s->stream) != cudaSuccess)
        return SF_ERR_CUDA;
    s->bar_epoch = 0;
    return SF_OK;
}

sf_status sf_set_index_table(sf_sketch* s, const uint32_t* table_dev, uint32_t n_keys) {
    if (!s || !(s->p.flags & SF_FLAG_EXPLICIT_INDEX) || !table_dev) return SF_ERR_INVALID;
    s->idx_table = table_dev;
    s->n_ids = n_keys;
    return SF_OK;
}

sf_status sf_insert_batch(sf_sketch* s, const void* keys_dev, uint64_t n) {
    return run_update(s, keys_dev, nullptr, +1, n);
}

sf_status sf_delete_batch(sf_sketch* s, const void* keys_dev, uint64_t n) {
    return run_update(s, keys_dev, nullptr, -1, n);
}

sf_status sf_update_batch(sf_sketch* s, const void* keys_dev, const int8_t* ops_dev, uint64_t n) {
    if (n && !ops_dev) return SF_ERR_INVALID;
    return run_update(s, keys_dev, ops_dev, 0, n);
}

sf_status sf_export_slim(const sf_sketch* s, uint32_t* dst_dev, uint64_t cap_elems, sf_slim_header* hdr) {
    if (!s || !dst_dev) return SF_ERR_INVALID;
    const uint64_t nelem = (uint64_t)s->p.d * s->p.w;
    if (cap_elems < nelem) return SF_ERR_OOM;
    if (cudaMemcpyAsync(dst_dev, s->A, nelem * 4ull, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
        return SF_ERR_CUDA;
    if (hdr) {
        hdr->magic = SF_SLIM_MAGIC;
        hdr->version = SF_SLIM_VERSION;
        hdr->d = s->p.d;
        hdr->w = s->p.w;
        hdr->key_bytes = s->p.key_bytes;
        hdr->hash_id = (s->p.flags & SF_FLAG_EXPLICIT_INDEX) ? SF_HASH_EXPLICIT : SF_HASH_SPLITMIX_LEMIRE;
        hdr->seed = s->p.seed;
    }
    return SF_OK;
}

sf_status sf_query_batch(const sf_slim_view* v, const void* keys_dev, uint64_t n, uint32_t* out_dev,
                         void* cuda_stream) {
    if (!v) return SF_ERR_INVALID;
    const sf_slim_header& h = v->hdr;
    if (h.magic != SF_SLIM_MAGIC || h.version != SF_SLIM_VERSION) return SF_ERR_VERSION;
    if (h.hash_id != SF_HASH_SPLITMIX_LEMIRE && h.hash_id != SF_HASH_EXPLICIT) return SF_ERR_VERSION;
    if (h.d < 1 || h.d > SF_MAX_D || h.w < 1 || h.key_bytes < 1 || h.key_bytes > SF_MAX_KEY_BYTES)
        return SF_ERR_INVALID;
    if (h.hash_id == SF_HASH_EXPLICIT && (!v->index_table || h.key_bytes != 4)) return SF_ERR_INVALID;
    if (n == 0) return SF_OK;
    if (!v->counters || !keys_dev || !out_dev) return SF_ERR_INVALID;
    const void *keys_acc = nullptr, *out_acc = nullptr;
    if (sf_device_access(keys_dev, &keys_acc) != SF_OK || sf_device_access(out_dev, &out_acc) != SF_OK)
        return SF_ERR_INVALID;
    keys_dev = keys_acc;
    out_dev = (uint32_t*)out_acc;
    if ((h.key_bytes == 4 || h.key_bytes == 8) && ((uintptr_t)keys_dev % h.key_bytes) != 0) return SF_ERR_INVALID;
    sfk::QueryArgs q{};
    q.s.A = (uint32_t*)v->counters;
    q.s.B = nullptr;
    q.s.d = h.d;
    q.s.w = h.w;
    q.s.z = 0xFFFFFFFFu;  // a query never reads the Fat: f_i is not bounded by any z here
    q.s.key_bytes = h.key_bytes;
    sfk::row_seeds(h.seed, h.d, q.s.rs);
    q.s.idx_table = h.hash_id == SF_HASH_EXPLICIT ? v->index_table : nullptr;
    q.s.n_ids = v->n_index_keys;
    q.keys = (const uint8_t*)keys_dev;
    q.n = n;
    q.out = out_dev;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SF_ERR_CUDA;
    return sfk::launch_query(q, sms, (cudaStream_t)cuda_stream) == cudaSuccess ? SF_OK : SF_ERR_CUDA;
}

sf_status sf_query_pipelined(const sf_slim_view* v, const void* keys_host, uint64_t n, uint32_t* out_host,
                             void* keys_dev, uint32_t* out_dev, uint32_t n_streams, void* const* streams) {
    if (!v || n_streams == 0 || !streams) return SF_ERR_INVALID;
    if (n == 0) return SF_OK;
    if (!keys_host || !out_host || !keys_dev || !out_dev) return SF_ERR_INVALID;
    const uint64_t kb = v->hdr.key_bytes;
    const uint64_t base = n / n_streams, extra = n % n_streams;
    uint64_t off = 0;
    for (uint32_t q = 0; q < n_streams; ++q) {
        const uint64_t len = base + (q < extra ? 1 : 0);  // the first n % n_streams parts take one more
        if (len == 0) continue;
        cudaStream_t st = (cudaStream_t)streams[q];
        const uint8_t* kh = (const uint8_t*)keys_host + off * kb;
        uint8_t* kd = (uint8_t*)keys_dev + off * kb;
        if (cudaMemcpyAsync(kd, kh, len * kb, cudaMemcpyHostToDevice, st) != cudaSuccess) return SF_ERR_CUDA;
        const sf_status qs = sf_query_batch(v, kd, len, out_dev + off, st);
        if (qs != SF_OK) return qs;
        if (cudaMemcpyAsync(out_host + off, out_dev + off, len * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SF_ERR_CUDA;
        off += len;
    }
    return SF_OK;
}

}  // extern "C"

// Two alternating halves of a staging buffer with, per half, the event of its last copy and of the
// last update that read it.
struct sf_pipeline {
    uint8_t* staging = nullptr;
    uint64_t half_bytes = 0;  // 16-byte multiple
    cudaStream_t cs = nullptr;
    int device = 0;
    cudaEvent_t copied[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};
    bool used_recorded[2] = {false, false};
    int next = 0;  // the half the next piece goes to
};

namespace {

void pipeline_release(sf_pipeline* p) {
    for (cudaEvent_t e : {p->copied[0], p->copied[1], p->used[0], p->used[1]})
        if (e) cudaEventDestroy(e);  // released once the work recorded on it has completed
    delete p;
}

sf_status pipeline_init(sf_pipeline* p, void* staging_dev, uint64_t staging_bytes, void* copy_stream) {
    p->staging = (uint8_t*)staging_dev;
    p->half_bytes = (staging_bytes / 2) & ~15ull;
    p->cs = (cudaStream_t)copy_stream;
    if (cudaGetDevice(&p->device) != cudaSuccess) return SF_ERR_CUDA;
    for (int h = 0; h < 2; ++h)
        if (cudaEventCreateWithFlags(&p->copied[h], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->used[h], cudaEventDisableTiming) != cudaSuccess)
            return SF_ERR_CUDA;
    return SF_OK;
}

// Updates per piece: the largest whole number of chunks whose keys (padded to a 16-byte multiple)
// and operations fit a half of half_bytes; 0 when not even one chunk does.
uint64_t pipeline_piece(uint64_t half_bytes, uint64_t S, uint64_t kb, bool with_ops) {
    const uint64_t per = kb + (with_ops ? 1u : 0u);
    uint64_t c = half_bytes / (S * per);
    while (c > 0 && ((c * S * kb + 15) & ~15ull) + (with_ops ? c * S : 0) > half_bytes) --c;
    return c * S;
}

// The pieces of one call: whole chunks that fit a half (keys, then the operations 16-byte aligned),
// each copied on the pipeline's copy stream once the last update that read its half is done, and
// applied on the sketch's stream once it has landed.
sf_status pipeline_run(sf_sketch* s, sf_pipeline* p, const void* keys_host, const int8_t* ops_host, int32_t op_const,
                       uint64_t n) {
    const uint64_t kb = s->p.key_bytes;
    const uint64_t piece = pipeline_piece(p->half_bytes, s->p.chunk, kb, ops_host != nullptr);
    if (piece == 0) return SF_ERR_OOM;
    const uint64_t keys_half = (piece * kb + 15) & ~15ull;  // the operations of a half follow its keys
    for (uint64_t off = 0; off < n;) {
        const uint64_t len = n - off < piece ? n - off : piece;
        const int h = p->next;
        uint8_t* kd = p->staging + (uint64_t)h * p->half_bytes;
        int8_t* od = ops_host ? (int8_t*)(kd + keys_half) : nullptr;
        if ((p->used_recorded[h] && cudaStreamWaitEvent(p->cs, p->used[h], 0) != cudaSuccess) ||
            cudaMemcpyAsync(kd, (const uint8_t*)keys_host + off * kb, len * kb, cudaMemcpyHostToDevice, p->cs) !=
                cudaSuccess ||
            (od && cudaMemcpyAsync(od, ops_host + off, len, cudaMemcpyHostToDevice, p->cs) != cudaSuccess) ||
            cudaEventRecord(p->copied[h], p->cs) != cudaSuccess ||
            cudaStreamWaitEvent(s->stream, p->copied[h], 0) != cudaSuccess)
            return SF_ERR_CUDA;
        const sf_status st = run_update(s, kd, od, ops_host ? 0 : op_const, len);
        if (st != SF_OK) return st;
        if (cudaEventRecord(p->used[h], s->stream) != cudaSuccess) return SF_ERR_CUDA;
        p->used_recorded[h] = true;
        p->next = h ^ 1;
        off += len;
    }
    return SF_OK;
}

bool pipeline_args_ok(const void* keys_host, const int8_t* ops_host, int32_t op_const) {
    return keys_host && (ops_host || op_const == 1 || op_const == -1);
}

// A staged call whose pieces would be smaller than this many updates reads the host keys in the
// kernel instead (many short launches would cost more than the link's latency).
constexpr uint64_t kStageMinPiece = 1ull << 18;

// The update calls' own pipeline: the upper half of the sketch's dictionary region (cap x 16 bytes;
// the single-iteration kernel's two halves of 8-byte claim entries fill the lower half) and a copy
// stream of the sketch's own.  *staged is false when the call should read the keys in the kernel.
sf_status run_staged(sf_sketch* s, const void* keys_host, const int8_t* ops_host, int op_const, uint64_t n,
                     bool* staged) {
    *staged = false;
    const uint64_t region = (uint64_t)s->cap * 16ull;
    const uint64_t piece = pipeline_piece((region / 2) & ~15ull, s->p.chunk, s->p.key_bytes, ops_host != nullptr);
    if (piece == 0 || (n > piece && piece < kStageMinPiece)) return SF_OK;
    if (!s->stage_pipe) {
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return SF_ERR_CUDA;
        sf_pipeline* p = new (std::nothrow) sf_pipeline();
        if (!p) {
            cudaStreamDestroy(cs);
            return SF_ERR_OOM;
        }
        if (pipeline_init(p, reinterpret_cast<uint8_t*>(s->dict) + region, region, cs) != SF_OK) {
            pipeline_release(p);
            cudaStreamDestroy(cs);
            return SF_ERR_CUDA;
        }
        s->stage_pipe = p;
        s->stage_cs = cs;
    }
    sf_pipeline* p = s->stage_pipe;
    if (s->stage_foreign) {
        // a launch that read the whole region (or the sketch's creation) came since the last staged
        // call: the first copies wait for the sketch's stream
        if (cudaEventRecord(p->used[0], s->stream) != cudaSuccess || cudaEventRecord(p->used[1], s->stream) != cudaSuccess)
            return SF_ERR_CUDA;
        p->used_recorded[0] = p->used_recorded[1] = true;
        s->stage_foreign = false;
    }
    *staged = true;
    s->stage_dirty = true;
    return pipeline_run(s, p, keys_host, ops_host, op_const, n);
}

}  // namespace

extern "C" {

sf_status sf_update_pipelined(sf_sketch* s, const void* keys_host, const int8_t* ops_host, int32_t op_const,
                              uint64_t n, void* staging_dev, uint64_t staging_bytes, void* copy_stream) {
    if (!s) return SF_ERR_INVALID;
    if (n == 0) return SF_OK;
    if (!staging_dev || !aligned16(staging_dev) || !pipeline_args_ok(keys_host, ops_host, op_const))
        return SF_ERR_INVALID;
    DeviceGuard guard(s->device);
    if (!guard.ok) return SF_ERR_CUDA;
    sf_pipeline* p = new (std::nothrow) sf_pipeline();
    if (!p) return SF_ERR_OOM;
    sf_status st = pipeline_init(p, staging_dev, staging_bytes, copy_stream);
    // the staging may still be read by the sketch's earlier work: the first copy waits for all of it
    if (st == SF_OK && (cudaEventRecord(p->used[1], s->stream) != cudaSuccess ||
                        cudaStreamWaitEvent(p->cs, p->used[1], 0) != cudaSuccess))
        st = SF_ERR_CUDA;
    if (st == SF_OK) st = pipeline_run(s, p, keys_host, ops_host, op_const, n);
    pipeline_release(p);
    return st;
}

sf_status sf_pipeline_create(void* staging_dev, uint64_t staging_bytes, void* copy_stream, sf_pipeline** out) {
    if (!out) return SF_ERR_INVALID;
    *out = nullptr;
    if (!staging_dev || !aligned16(staging_dev) || staging_bytes < 64) return SF_ERR_INVALID;
    sf_pipeline* p = new (std::nothrow) sf_pipeline();
    if (!p) return SF_ERR_OOM;
    const sf_status st = pipeline_init(p, staging_dev, staging_bytes, copy_stream);
    if (st != SF_OK) {
        pipeline_release(p);
        return st;
    }
    *out = p;
    return SF_OK;
}

sf_status sf_pipeline_destroy(sf_pipeline* p) {
    if (!p) return SF_ERR_INVALID;
    DeviceGuard guard(p->device);
    pipeline_release(p);
    return SF_OK;
}

sf_status sf_update_pipeline(sf_sketch* s, sf_pipeline* p, const void* keys_host, const int8_t* ops_host,
                             int32_t op_const, uint64_t n) {
    if (!s || !p) return SF_ERR_INVALID;
    if (n == 0) return SF_OK;
    if (!pipeline_args_ok(keys_host, ops_host, op_const) || p->device != s->device) return SF_ERR_INVALID;
    DeviceGuard guard(s->device);
    if (!guard.ok) return SF_ERR_CUDA;
    return pipeline_run(s, p, keys_host, ops_host, op_const, n);
}

sf_status sf_sync(sf_sketch* s) {
    if (!s) return SF_ERR_INVALID;
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, s->ctrl + sfk::kCtrlErr, 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
        return SF_ERR_CUDA;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return SF_ERR_CUDA;
    if (err == 0) return SF_OK;
    cudaError_t e;
    if (err & sfk::kErrTimeout) {
        // a grid wait gave up: barrier words and dictionary may be inconsistent; reset them (a
        // dictionary set by sf_set_dictionary too)
        uint64_t xb = 0;
        sf_required_bytes(&s->p, nullptr, nullptr, &xb);
        e = cudaMemsetAsync(s->scratch, 0, xb, s->stream);
        if (e == cudaSuccess && (s->p.flags & SF_FLAG_SHARED_DICT) && s->dict)
            e = cudaMemsetAsync(s->dict, 0, (uint64_t)s->cap * sizeof(sfk::DictEntry), s->stream);
        s->bar_epoch = 0;
        s->stage_dirty = false;   // the staged half went with the scratch
        s->stage_foreign = true;
    } else {
        e = cudaMemsetAsync(s->ctrl + sfk::kCtrlErr, 0, 4, s->stream);
    }
    if (e != cudaSuccess || cudaStreamSynchronize(s->stream) != cudaSuccess) return SF_ERR_CUDA;
    if (err & sfk::kErrTimeout) return SF_ERR_TIMEOUT;
    if (err & (sfk::kErrBadKey | sfk::kErrDictFull)) return SF_ERR_INVALID;
    if (err & sfk::kErrUnderflow) return SF_ERR_UNDERFLOW;
    return SF_ERR_INVALID;
}

}  // extern "C"
