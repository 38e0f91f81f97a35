// sf_batch.cu -- batched many-sketch update: one persistent cooperative launch per call,
// captured in a CUDA graph and replayed while the batch shape repeats.
//
// The launch walks all sketches of the call in lockstep rounds (round r = chunk r of every
// sketch, each with its own chunk size), with two grid barriers per round; see sf_update.cu for
// the per-chunk phases.  Sketches are independent, so the lockstep changes nothing in any
// sketch's result: it only spreads every stream over the whole GPU.
#include <cstring>
#include <new>
#include <vector>

#include "sf_handle.h"

struct sf_batch {
    uint32_t max_sketches;
    uint64_t max_round_slots;
    uint2* claims_dev;
    uint8_t* scratch;
    uint32_t* ctrl;
    sfk::SketchRun* table_dev;
    sfk::SketchRun* staging;  // pinned host copy of the run table
    cudaStream_t stream;
    cudaStream_t cap_stream;  // private stream used only for graph capture
    cudaEvent_t staged;
    bool staging_busy;
    uint32_t flags;
    int device;
    int num_sms;
    // graph of the last launch plan
    bool have_exec;
    cudaGraphExec_t exec;
    std::vector<sfk::BatchArgs> exec_plan;
    uint32_t exec_d;
    int exec_grid;
    int exec_block;
    int block;  // threads per block of the launches (sf_batch_set_block_threads)
    uint32_t graph_launches, graph_captures;
    uint64_t rounds_last;
    uint64_t group_bytes;                        // counter footprint per launch group (0: one launch)
    uint32_t groups_last;
    std::vector<const void*> keys_acc, ops_acc;  // device-usable item pointers of the current call
    std::vector<uint8_t> in_host;                // the item's keys or operations live in host memory
    std::vector<uint32_t> order;                 // item of each table row (group by group)
    std::vector<sfk::BatchArgs> plan;            // one cooperative launch per group
    uint8_t* arena = nullptr;                    // dictionary arena of SF_FLAG_SHARED_DICT sketches
    uint64_t arena_bytes = 0;
};

namespace {

constexpr uint64_t kBatchCtrlBytes = 256;

bool same_shape(const sfk::BatchArgs& x, const sfk::BatchArgs& y) {
    return x.n_runs == y.n_runs && x.claims_cap == y.claims_cap && x.flat_len == y.flat_len &&
           x.n_rounds == y.n_rounds && x.may_ins == y.may_ins && x.may_del == y.may_del && x.runs == y.runs &&
           x.claims_global == y.claims_global && x.max_chunk == y.max_chunk && x.keys_in_host == y.keys_in_host;
}

bool same_plan(const std::vector<sfk::BatchArgs>& x, const std::vector<sfk::BatchArgs>& y) {
    if (x.size() != y.size()) return false;
    for (size_t g = 0; g < x.size(); ++g)
        if (!same_shape(x[g], y[g])) return false;
    return true;
}

// One table upload, then per launch group: barrier-counter reset and the cooperative launch.
cudaError_t enqueue(sf_batch* b, const std::vector<sfk::BatchArgs>& plan, uint32_t d, int grid, int block,
                    size_t table_bytes, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(b->table_dev, b->staging, table_bytes, cudaMemcpyHostToDevice, st);
    for (size_t g = 0; e == cudaSuccess && g < plan.size(); ++g) {
        e = cudaMemsetAsync(b->ctrl + sfk::kCtrlBarrier64, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = sfk::launch_batch_update(plan[g], d, grid, block, st);
    }
    return e;
}

bool shared_dict(const sf_sketch* s) { return (s->p.flags & SF_FLAG_SHARED_DICT) != 0; }
uint64_t dict_bytes_of(const sf_sketch* s) { return (uint64_t)s->cap * sizeof(sfk::DictEntry); }

// Counter footprint of one sketch in a round: Fat + Slim + the dictionary entries a chunk can touch.
uint64_t item_footprint(const sf_sketch* s) {
    const uint64_t dw = (uint64_t)s->p.d * s->p.w;
    return dw * s->p.z * 4ull + dw * 4ull + (uint64_t)s->p.chunk * sizeof(sfk::DictEntry);
}

}  // namespace

extern "C" {

static uint64_t table_bytes_of(uint32_t max_sketches) {
    return ((uint64_t)max_sketches * sizeof(sfk::SketchRun) + 255) / 256 * 256;
}

sf_status sf_batch_required_bytes(uint32_t max_sketches, uint64_t max_round_slots, uint64_t* scratch_bytes) {
    if (max_sketches == 0 || max_round_slots == 0 || !scratch_bytes) return SF_ERR_INVALID;
    *scratch_bytes = kBatchCtrlBytes + table_bytes_of(max_sketches) + sfk::claims_global_bytes(max_round_slots);
    return SF_OK;
}

sf_status sf_batch_create(uint32_t max_sketches, uint64_t max_round_slots, void* scratch_dev, void* cuda_stream,
                          uint32_t flags, sf_batch** out) {
    if (!out || !scratch_dev || max_sketches == 0 || max_round_slots == 0 || ((uintptr_t)scratch_dev & 15u) ||
        (flags & ~SF_BATCH_GRAPH))
        return SF_ERR_INVALID;
    *out = nullptr;
    sf_batch* b = new (std::nothrow) sf_batch();
    if (!b) return SF_ERR_OOM;
    b->max_sketches = max_sketches;
    b->max_round_slots = max_round_slots;
    try {
        b->keys_acc.assign(max_sketches, nullptr);
        b->ops_acc.assign(max_sketches, nullptr);
        b->in_host.assign(max_sketches, 0);
        b->order.reserve(max_sketches);
    } catch (...) {
        delete b;
        return SF_ERR_OOM;
    }
    b->claims_dev = (uint2*)((uint8_t*)scratch_dev + kBatchCtrlBytes + table_bytes_of(max_sketches));
    b->scratch = (uint8_t*)scratch_dev;
    b->ctrl = (uint32_t*)scratch_dev;
    b->table_dev = (sfk::SketchRun*)((uint8_t*)scratch_dev + kBatchCtrlBytes);
    b->stream = (cudaStream_t)cuda_stream;
    b->flags = flags;
    b->block = sfk::kChunkBlock;
    uint64_t xb = kBatchCtrlBytes + table_bytes_of(max_sketches);  // claim lists need no zeroing
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
        cudaHostAlloc((void**)&b->staging, (size_t)max_sketches * sizeof(sfk::SketchRun), cudaHostAllocDefault) !=
            cudaSuccess) {
        delete b;
        return SF_ERR_CUDA;
    }
    // default launch groups: counters of up to 3/4 of L2 per group (GB300: 126 MiB -> ~95 MiB)
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->device) != cudaSuccess) l2 = 0;
    b->group_bytes = (uint64_t)l2 * 3u / 4u;
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) != cudaSuccess ||
        cudaMemsetAsync(scratch_dev, 0, xb, b->stream) != cudaSuccess) {
        cudaFreeHost(b->staging);
        delete b;
        return SF_ERR_CUDA;
    }
    *out = b;
    return SF_OK;
}

sf_status sf_batch_update(sf_batch* b, uint32_t n_items, const sf_batch_item* items) {
    if (!b || (n_items && !items) || n_items > b->max_sketches) return SF_ERR_INVALID;
    if (n_items == 0) return SF_OK;
    const uint32_t d = items[0].sketch ? items[0].sketch->p.d : 0;
    for (uint32_t i = 0; i < n_items; ++i) {
        const sf_sketch* s = items[i].sketch;
        if (!s || s->p.d != d || s->p.chunk < 2 || s->device != b->device || (s->p.flags & SF_FLAG_EXPLICIT_INDEX))
            return SF_ERR_INVALID;
        if (items[i].n && !items[i].keys_dev) return SF_ERR_INVALID;
        bool kh = false, oh = false;
        if (sf_device_access(items[i].keys_dev, &b->keys_acc[i], &kh) != SF_OK ||
            sf_device_access(items[i].ops_dev, &b->ops_acc[i], &oh) != SF_OK)
            return SF_ERR_INVALID;
        b->in_host[i] = (kh || oh) ? 1 : 0;
        const uint32_t kb = s->p.key_bytes;
        if ((kb == 4 || kb == 8) && ((uintptr_t)b->keys_acc[i] % kb) != 0) return SF_ERR_INVALID;
        if (shared_dict(s)) {
            if (b->arena && dict_bytes_of(s) > b->arena_bytes) return SF_ERR_OOM;
            if (!b->arena && !s->dict) return SF_ERR_INVALID;
        }
    }
    DeviceGuard guard(b->device);
    if (!guard.ok) return SF_ERR_CUDA;
    if (b->staging_busy && cudaEventSynchronize(b->staged) != cudaSuccess) return SF_ERR_CUDA;
    // a sketch's own dictionary region must read as empty: zero what its staged calls left there
    // (only sketches that own their dictionary stage anything)
    for (uint32_t i = 0; i < n_items; ++i)
        if (sf_stage_release(items[i].sketch, b->stream) != SF_OK) return SF_ERR_CUDA;

    // every launch shape keeps 512 threads per SM: 512 / block co-resident blocks of `block` threads
    const int block = b->block;
    const int bps = sfk::chunk_update_blocks_per_sm(d, block);
    if (bps <= 0) return SF_ERR_CUDA;
    const int per_sm = sfk::kChunkBlock / block;
    const int grid = b->num_sms * (bps < per_sm ? bps : per_sm);

    // Launch groups.  Sketches are independent, so they may run in any grouping.  Sketches whose
    // counters fit the group budget are packed, in input order, into groups whose counters fit it
    // together, so each launch works out of L2.  A group whose rounds would not give every thread
    // of the grid a slot gains nothing from running alone, so it joins the shared launch, as do
    // the sketches larger than the budget: batching those at least fills the GPU.  A zero budget
    // puts every sketch in one launch.
    b->order.clear();
    std::vector<std::pair<uint32_t, uint32_t>> groups;  // [first, last) rows of the table
    {
        const uint64_t budget = b->group_bytes;
        const uint64_t min_slots = (uint64_t)grid * (uint64_t)block;
        std::vector<uint32_t> shared, cur_g;
        uint64_t gb = 0, gs = 0;
        auto close = [&]() {
            if (cur_g.empty()) return;
            if (gs >= min_slots) {
                groups.emplace_back((uint32_t)b->order.size(), (uint32_t)(b->order.size() + cur_g.size()));
                b->order.insert(b->order.end(), cur_g.begin(), cur_g.end());
            } else {
                shared.insert(shared.end(), cur_g.begin(), cur_g.end());
            }
            cur_g.clear();
            gb = gs = 0;
        };
        for (uint32_t i = 0; i < n_items; ++i) {
            const uint64_t fb = item_footprint(items[i].sketch);
            if (budget == 0 || fb > budget) {
                shared.push_back(i);
                continue;
            }
            if (gb > 0 && gb + fb > budget) close();
            cur_g.push_back(i);
            gb += fb;
            gs += sfk::round_up32(items[i].sketch->p.chunk);
        }
        close();
        if (!shared.empty()) {
            groups.emplace_back((uint32_t)b->order.size(), (uint32_t)(b->order.size() + shared.size()));
            b->order.insert(b->order.end(), shared.begin(), shared.end());
        }
    }

    // With a dictionary arena, the flagged sketches of a launch take their dictionaries from its
    // start (launches run one after another); a group whose dictionaries do not fit together is
    // split into launches that fit, in order.
    if (b->arena) {
        std::vector<std::pair<uint32_t, uint32_t>> split;
        for (const auto& gr : groups) {
            uint32_t first = gr.first;
            uint64_t used = 0;
            for (uint32_t row = gr.first; row < gr.second; ++row) {
                const sf_sketch* s = items[b->order[row]].sketch;
                const uint64_t need = shared_dict(s) ? dict_bytes_of(s) : 0;
                if (row > first && used + need > b->arena_bytes) {
                    split.emplace_back(first, row);
                    first = row;
                    used = 0;
                }
                used += need;
            }
            split.emplace_back(first, gr.second);
        }
        groups.swap(split);
    }

    b->plan.clear();
    uint64_t rounds_all = 0;
    for (const auto& gr : groups) {
        uint64_t flat = 0, rounds = 0, arena_off = 0;
        uint32_t max_chunk = 0;
        bool may_ins = false, may_del = false, in_host = false;
        for (uint32_t row = gr.first; row < gr.second; ++row) {
            const uint32_t i = b->order[row];
            const sf_sketch* s = items[i].sketch;
            sfk::SketchRun& R = b->staging[row];
            std::memset(&R, 0, sizeof(R));
            R.s.A = s->A;
            R.s.B = s->B;
            R.s.d = s->p.d;
            R.s.w = s->p.w;
            R.s.z = s->p.z;
            R.s.key_bytes = s->p.key_bytes;
            for (int r = 0; r < SF_MAX_D; ++r) R.s.rs[r] = s->rs[r];
            R.s.sf4_delete = (s->p.flags & SF_FLAG_SF4_DELETE) ? 1u : 0u;
            R.keys = (const uint8_t*)b->keys_acc[i];
            R.ops = (const int8_t*)b->ops_acc[i];
            R.op_const = 1;
            R.S = s->p.chunk;
            R.n = items[i].n;
            R.flat_base = flat;  // slots are numbered per launch group
            if (shared_dict(s) && b->arena) {
                R.dict = reinterpret_cast<sfk::DictEntry*>(b->arena + arena_off);
                arena_off += dict_bytes_of(s);
            } else {
                R.dict = s->dict;
            }
            R.cap_mask = s->cap - 1u;
            R.claim_mask = sfk::claim_capacity(R.S) - 1u;
            flat += sfk::round_up32(R.S);
            max_chunk = R.S > max_chunk ? R.S : max_chunk;
            in_host |= b->in_host[i] != 0;
            const uint64_t nr = (R.n + R.S - 1) / R.S;
            rounds = nr > rounds ? nr : rounds;
            if (R.n) {
                may_ins |= R.ops != nullptr;
                may_del |= R.ops != nullptr;
                may_ins |= R.ops == nullptr;
            }
        }
        if (flat > b->max_round_slots) return SF_ERR_INVALID;
        if (rounds == 0) continue;  // nothing to update in this group
        sfk::BatchArgs a{};
        a.runs = b->table_dev + gr.first;
        a.n_runs = gr.second - gr.first;
        a.flat_len = flat;
        a.n_rounds = rounds;
        a.claims_cap = sfk::chunk_claims_cap(flat, grid, block);
        a.ctrl = b->ctrl;
        a.bar_base = 0;  // each launch zeroes the barrier counter first
        a.timeout_ns = sfk::kBarrierTimeoutNs;
        a.may_ins = may_ins;
        a.may_del = may_del;
        a.max_chunk = max_chunk;
        a.keys_in_host = in_host ? 1 : 0;
        // claim lists in shared memory when they fit, else in the batch scratch (launches run in order)
        a.claims_global =
            ((uint64_t)a.claims_cap * sizeof(uint2) > (uint64_t)sfk::claim_smem_max(block)) ? b->claims_dev : nullptr;
        b->plan.push_back(a);
        rounds_all = rounds > rounds_all ? rounds : rounds_all;
    }
    const size_t table_bytes = (size_t)n_items * sizeof(sfk::SketchRun);
    b->rounds_last = rounds_all;
    b->groups_last = (uint32_t)b->plan.size();

    cudaError_t e = cudaSuccess;
    bool launched = false;
    if (b->flags & SF_BATCH_GRAPH) {
        if (!b->have_exec || !same_plan(b->exec_plan, b->plan) || b->exec_d != d || b->exec_grid != grid ||
            b->exec_block != block) {
            if (b->have_exec) {
                cudaGraphExecDestroy(b->exec);
                b->have_exec = false;
            }
            cudaGraph_t g = nullptr;
            bool ok = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const cudaError_t ce = enqueue(b, b->plan, d, grid, block, table_bytes, b->cap_stream);
                ok = cudaStreamEndCapture(b->cap_stream, &g) == cudaSuccess && ce == cudaSuccess && g;
            }
            if (ok) ok = cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            if (ok) {
                b->have_exec = true;
                b->exec_plan = b->plan;
                b->exec_d = d;
                b->exec_grid = grid;
                b->exec_block = block;
                b->graph_captures++;
            } else {
                cudaGetLastError();           // capture not supported here: launch directly from now on
                b->flags &= ~SF_BATCH_GRAPH;
            }
        }
        if (b->have_exec) {
            e = cudaGraphLaunch(b->exec, b->stream);
            launched = true;
            if (e == cudaSuccess) b->graph_launches++;
        }
    }
    if (!launched) e = enqueue(b, b->plan, d, grid, block, table_bytes, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->staged, b->stream);
    b->staging_busy = true;
    return e == cudaSuccess ? SF_OK : SF_ERR_CUDA;
}

sf_status sf_batch_sync(sf_batch* b) {
    if (!b) return SF_ERR_INVALID;
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, b->ctrl + sfk::kCtrlErr, 4, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return SF_ERR_CUDA;
    if (err == 0) return SF_OK;
    // a grid wait that gave up may leave dictionary entries claimed: the arena is zeroed again
    if ((err & sfk::kErrTimeout) && b->arena && cudaMemsetAsync(b->arena, 0, b->arena_bytes, b->stream) != cudaSuccess)
        return SF_ERR_CUDA;
    if (cudaMemsetAsync(b->ctrl, 0, kBatchCtrlBytes, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return SF_ERR_CUDA;
    if (err & sfk::kErrTimeout) return SF_ERR_TIMEOUT;
    if (err & (sfk::kErrBadKey | sfk::kErrDictFull)) return SF_ERR_INVALID;
    if (err & sfk::kErrUnderflow) return SF_ERR_UNDERFLOW;
    return SF_ERR_INVALID;
}

sf_status sf_batch_set_group_bytes(sf_batch* b, uint64_t bytes) {
    if (!b) return SF_ERR_INVALID;
    b->group_bytes = bytes;
    return SF_OK;
}

sf_status sf_batch_set_dictionary_arena(sf_batch* b, void* arena_dev, uint64_t bytes) {
    if (!b || (arena_dev && ((uintptr_t)arena_dev & 15u))) return SF_ERR_INVALID;
    if (!arena_dev || bytes == 0) {
        b->arena = nullptr;
        b->arena_bytes = 0;
        return SF_OK;
    }
    DeviceGuard guard(b->device);
    if (!guard.ok) return SF_ERR_CUDA;
    if (cudaMemsetAsync(arena_dev, 0, bytes, b->stream) != cudaSuccess) return SF_ERR_CUDA;
    b->arena = (uint8_t*)arena_dev;
    b->arena_bytes = bytes & ~15ull;
    return SF_OK;
}

sf_status sf_batch_set_block_threads(sf_batch* b, uint32_t threads) {
    if (!b || (threads != 512 && threads != 256 && threads != 128)) return SF_ERR_INVALID;
    b->block = (int)threads;
    return SF_OK;
}

sf_status sf_batch_groups(const sf_batch* b, uint32_t* groups_last, uint64_t* group_bytes) {
    if (!b) return SF_ERR_INVALID;
    if (groups_last) *groups_last = b->groups_last;
    if (group_bytes) *group_bytes = b->group_bytes;
    return SF_OK;
}

sf_status sf_batch_info(const sf_batch* b, uint32_t* graph_launches, uint32_t* graph_captures, uint64_t* rounds_last) {
    if (!b) return SF_ERR_INVALID;
    if (graph_launches) *graph_launches = b->graph_launches;
    if (graph_captures) *graph_captures = b->graph_captures;
    if (rounds_last) *rounds_last = b->rounds_last;
    return SF_OK;
}

sf_status sf_batch_destroy(sf_batch* b) {
    if (!b) return SF_ERR_INVALID;
    if (b->staging_busy) cudaEventSynchronize(b->staged);
    if (b->have_exec) cudaGraphExecDestroy(b->exec);
    cudaEventDestroy(b->staged);
    cudaStreamDestroy(b->cap_stream);
    cudaFreeHost(b->staging);
    delete b;
    return SF_OK;
}

}  // extern "C"
