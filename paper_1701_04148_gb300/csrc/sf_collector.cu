// sf_collector.cu -- the collector's serving loop: resident Slims, budget admission,
// continuous batching of point queries over several CUDA streams.
//
// Paper context: monitoring nodes periodically send their Slim-subsketch to a remote collector that
// answers queries (Abstract, Sec. 1.1); the paper's GPU query path batches queries and overlaps
// copies and kernels over several streams (Sec. 4.2).  Here a worker thread forms batches from
// whatever requests have arrived, up to n_streams batches run at once, and a request that arrives
// while batches are in flight joins the next batch as soon as a stream slot frees.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sf.h"
#include "sf_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr uint64_t kAlign = 256;

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// First-fit allocator over the arena (offsets), coalescing on free.
class Arena {
   public:
    void init(uint64_t bytes) {
        free_.clear();
        free_[0] = bytes;
        used_ = 0;
    }
    bool alloc(uint64_t bytes, uint64_t* off) {
        bytes = align_up(bytes, kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const uint64_t rest = it->second - bytes;
                const uint64_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = align_up(bytes, kAlign);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    uint64_t used() const { return used_; }

   private:
    std::map<uint64_t, uint64_t> free_;
    uint64_t used_ = 0;
};

struct Version {
    uint64_t off = 0, bytes = 0;
    sf_slim_header hdr{};
    uint64_t rs[SF_MAX_D] = {};
    int refs = 0;  // the table's reference + queries bound to it
};

struct Request {
    uint64_t ticket = 0;
    Version* v = nullptr;
    const uint8_t* keys = nullptr;
    uint64_t n = 0;
    uint32_t* out = nullptr;
    Clock::time_point t_submit;
    std::atomic<int> done{0};
    sf_status status = SF_OK;
};

struct Slot {  // one in-flight batch
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    sfk::QueryReq* reqs_dev = nullptr;
    uint8_t* keys_host = nullptr;  // pinned, mapped: the query kernel reads the keys from here
    uint32_t* out_host = nullptr;  // pinned, mapped: the query kernel writes the answers here
    sfk::QueryReq* reqs_host = nullptr;  // pinned
    const uint8_t* keys_map = nullptr;   // device addresses of keys_host / out_host
    uint32_t* out_map = nullptr;
    std::vector<std::shared_ptr<Request>> members;
};

struct Layout {
    uint64_t keys_bytes, out_bytes, reqs_bytes, slot_bytes;
};

Layout layout_of(const sfc_config* c) {
    Layout L;
    L.keys_bytes = align_up((uint64_t)c->max_batch_keys * SF_MAX_KEY_BYTES + (uint64_t)c->max_batch_reqs * 16, kAlign);
    L.out_bytes = align_up((uint64_t)c->max_batch_keys * 4, kAlign);
    L.reqs_bytes = align_up((uint64_t)c->max_batch_reqs * sizeof(sfk::QueryReq), kAlign);
    L.slot_bytes = L.reqs_bytes;  // device staging holds only the request tables: keys and answers
                                  // stay in mapped pinned host memory
    return L;
}

bool config_ok(const sfc_config* c) {
    return c && c->arena_dev && c->arena_bytes && c->staging_dev && c->max_sketches && c->n_streams >= 1 &&
           c->n_streams <= 16 && c->max_batch_keys >= 1 && c->max_batch_reqs >= 1 &&
           ((uintptr_t)c->arena_dev % kAlign) == 0 && ((uintptr_t)c->staging_dev % kAlign) == 0;
}

}  // namespace

struct sfc {
    sfc_config cfg{};
    int device = 0, num_sms = 0;
    uint8_t* arena_dev = nullptr;
    Arena arena;
    std::vector<Version*> table;  // current version per sketch id (nullptr: none)
    std::vector<Slot> slots;
    cudaStream_t upload_stream = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    uint64_t pending_keys = 0;  // keys of the pending requests (kept with the queue, under mu)
    std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    // stats
    std::vector<double> lat_us;
    uint64_t st_requests = 0, st_keys = 0, st_batches = 0, st_uploads = 0, st_rejected = 0, st_evictions = 0;
    Clock::time_point window_start;
    bool window_started = false;
    Clock::time_point last_done;

    void unref(Version* v) {  // caller holds mu
        if (v && --v->refs == 0) {
            arena.release(v->off, v->bytes);
            delete v;
        }
    }

    void complete(Slot& s) {  // caller holds mu; the slot's event has fired
        const auto now = Clock::now();
        for (auto& r : s.members) {
            lat_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
            unref(r->v);
            r->v = nullptr;
            r->done.store(1);
        }
        last_done = now;
        s.members.clear();
        s.busy = false;
        cv_done.notify_all();
    }

    // The worker loop.  The lock guards the queue, the tickets, the version table and the stats;
    // the slots belong to this thread alone, so the host copies of keys and answers (megabytes per
    // batch) run unlocked, and submitting threads are not held up by them.
    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            // finished batches: copy their answers out of pinned staging (unlocked), then complete; a
            // batch whose event reports an error (not just "not ready") completes with SF_ERR_CUDA, so
            // no request waits on it forever
            bool any_busy = false;
            Slot* fin[16];
            bool failed[16];
            uint32_t nfin = 0;
            lk.unlock();
            for (auto& s : slots) {
                if (!s.busy) continue;
                const cudaError_t q = cudaEventQuery(s.ev);
                if (q == cudaErrorNotReady) {
                    any_busy = true;
                    continue;
                }
                if (q == cudaSuccess) {
                    uint64_t off = 0;
                    for (auto& r : s.members) {
                        if (r->n) std::memcpy(r->out, s.out_host + off, r->n * sizeof(uint32_t));
                        off += r->n;
                    }
                }
                failed[nfin] = q != cudaSuccess;
                fin[nfin++] = &s;
            }
            lk.lock();
            for (uint32_t f = 0; f < nfin; ++f) {
                if (failed[f])
                    for (auto& r : fin[f]->members) r->status = SF_ERR_CUDA;
                complete(*fin[f]);
            }
            if (stop && pending.empty() && !any_busy) break;
            // launch as many batches as free slots and pending work allow
            bool launched = false;
            for (auto& s : slots) {
                if (s.busy || pending.empty()) continue;
                const auto waited = std::chrono::duration<double, std::micro>(Clock::now() - pending.front()->t_submit).count();
                const bool full = pending_keys >= cfg.max_batch_keys || pending.size() >= cfg.max_batch_reqs;
                if (!full && any_busy && waited < (double)cfg.max_wait_us && !stop) break;
                take(s);
                lk.unlock();
                const bool ok = pack_and_launch(s);
                lk.lock();
                if (!ok) {
                    for (auto& r : s.members) r->status = SF_ERR_CUDA;
                    complete(s);
                    continue;
                }
                launched = true;
                any_busy = true;
            }
            if (launched) continue;
            if (any_busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(5));
                lk.lock();
            } else if (pending.empty()) {
                cv_work.wait(lk, [&] { return stop || !pending.empty(); });
            } else {
                cv_work.wait_for(lk, std::chrono::microseconds(cfg.max_wait_us ? cfg.max_wait_us : 1));
            }
        }
    }

    // Moves pending requests into slot s, up to the batch limits (holds mu).
    void take(Slot& s) {
        uint64_t nkeys = 0;
        uint32_t nreq = 0;
        while (!pending.empty() && nreq < cfg.max_batch_reqs) {
            auto& r = pending.front();
            if (nkeys + r->n > cfg.max_batch_keys && nreq > 0) break;
            nkeys += r->n;
            pending_keys -= r->n;
            s.members.push_back(r);
            pending.pop_front();
            ++nreq;
        }
        s.busy = true;
        st_batches++;
    }

    // Packs the slot's requests into its pinned staging and enqueues the request-table copy and the
    // kernel, which reads the keys from the slot's pinned host buffer and writes the answers to
    // another one over the host link (no key or answer copies on the batch's critical path).  Runs
    // unlocked: the requests' versions are pinned by their references and never change.
    bool pack_and_launch(Slot& s) {
        uint64_t nkeys = 0, koff = 0;
        uint32_t nreq = 0;
        for (auto& r : s.members) {
            const Version* v = r->v;
            sfk::QueryReq& q = s.reqs_host[nreq];
            q.A = (const uint32_t*)(arena_dev + v->off);
            q.d = v->hdr.d;
            q.w = v->hdr.w;
            q.key_bytes = v->hdr.key_bytes;
            q.n = (uint32_t)r->n;
            for (int i = 0; i < SF_MAX_D; ++i) q.rs[i] = v->rs[i];
            koff = align_up(koff, 16);
            q.key_off = koff;
            q.out_off = nkeys;
            if (r->n) std::memcpy(s.keys_host + koff, r->keys, r->n * v->hdr.key_bytes);
            koff += r->n * v->hdr.key_bytes;
            nkeys += r->n;
            ++nreq;
        }
        sfk::MultiQueryArgs a{};
        a.reqs = s.reqs_dev;
        a.n_reqs = nreq;
        a.total = nkeys;
        a.keys = s.keys_map;
        a.out = s.out_map;
        cudaError_t e =
            cudaMemcpyAsync(s.reqs_dev, s.reqs_host, nreq * sizeof(sfk::QueryReq), cudaMemcpyHostToDevice, s.stream);
        if (e == cudaSuccess) e = sfk::launch_multi_query(a, num_sms, s.stream);
        if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.stream);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(s.stream);
            return false;
        }
        return true;
    }
};

extern "C" {

sf_status sfc_required_staging_bytes(const sfc_config* c, uint64_t* bytes) {
    if (!c || !bytes || c->n_streams < 1 || c->n_streams > 16 || !c->max_batch_keys || !c->max_batch_reqs)
        return SF_ERR_INVALID;
    *bytes = layout_of(c).slot_bytes * c->n_streams;
    return SF_OK;
}

sf_status sfc_create(const sfc_config* c, sfc** out) {
    if (!out || !config_ok(c)) return SF_ERR_INVALID;
    *out = nullptr;
    uint64_t need = 0;
    sfc_required_staging_bytes(c, &need);
    if (c->staging_bytes < need) return SF_ERR_OOM;
    sfc* x = new (std::nothrow) sfc();
    if (!x) return SF_ERR_OOM;
    x->cfg = *c;
    x->arena_dev = (uint8_t*)c->arena_dev;
    x->arena.init(c->arena_bytes);
    x->table.assign(c->max_sketches, nullptr);
    if (cudaGetDevice(&x->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&x->num_sms, cudaDevAttrMultiProcessorCount, x->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&x->upload_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete x;
        return SF_ERR_CUDA;
    }
    const Layout L = layout_of(c);
    x->slots.resize(c->n_streams);
    for (uint32_t i = 0; i < c->n_streams; ++i) {
        Slot& s = x->slots[i];
        uint8_t* base = (uint8_t*)c->staging_dev + i * L.slot_bytes;
        s.reqs_dev = (sfk::QueryReq*)base;
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc((void**)&s.keys_host, L.keys_bytes, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostAlloc((void**)&s.out_host, L.out_bytes, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostAlloc((void**)&s.reqs_host, L.reqs_bytes, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostGetDevicePointer((void**)&s.keys_map, s.keys_host, 0) != cudaSuccess ||
            cudaHostGetDevicePointer((void**)&s.out_map, s.out_host, 0) != cudaSuccess) {
            sfc_destroy(x);
            return SF_ERR_CUDA;
        }
    }
    x->worker = std::thread([x] { x->run(); });
    *out = x;
    return SF_OK;
}

sf_status sfc_upload(sfc* c, uint32_t sketch_id, const uint32_t* counters, const sf_slim_header* hdr) {
    if (!c || !counters || !hdr || sketch_id >= c->cfg.max_sketches) return SF_ERR_INVALID;
    if (hdr->magic != SF_SLIM_MAGIC || hdr->version != SF_SLIM_VERSION || hdr->hash_id != SF_HASH_SPLITMIX_LEMIRE)
        return SF_ERR_VERSION;
    if (hdr->d < 1 || hdr->d > SF_MAX_D || hdr->w < 1 || hdr->key_bytes < 1 || hdr->key_bytes > SF_MAX_KEY_BYTES)
        return SF_ERR_INVALID;
    const uint64_t bytes = (uint64_t)hdr->d * hdr->w * 4ull;
    Version* v = new (std::nothrow) Version();
    if (!v) return SF_ERR_OOM;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->arena.alloc(bytes, &v->off)) {
            delete v;
            c->st_rejected++;
            return SF_ERR_BUDGET;
        }
    }
    v->bytes = bytes;
    v->hdr = *hdr;
    sfk::row_seeds(hdr->seed, hdr->d, v->rs);
    v->refs = 1;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != c->device) cudaSetDevice(c->device);
    const bool ok = cudaMemcpyAsync(c->arena_dev + v->off, counters, bytes, cudaMemcpyDefault, c->upload_stream) ==
                        cudaSuccess &&
                    cudaStreamSynchronize(c->upload_stream) == cudaSuccess;
    if (cur != c->device) cudaSetDevice(cur);
    std::lock_guard<std::mutex> lk(c->mu);
    if (!ok) {
        c->arena.release(v->off, v->bytes);
        delete v;
        return SF_ERR_CUDA;
    }
    Version* old = c->table[sketch_id];
    c->table[sketch_id] = v;
    c->unref(old);
    c->st_uploads++;
    return SF_OK;
}

sf_status sfc_evict(sfc* c, uint32_t sketch_id) {
    if (!c || sketch_id >= c->cfg.max_sketches) return SF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    Version* old = c->table[sketch_id];
    if (!old) return SF_ERR_INVALID;
    c->table[sketch_id] = nullptr;
    c->unref(old);
    c->st_evictions++;
    return SF_OK;
}

sf_status sfc_query_submit(sfc* c, uint32_t sketch_id, const void* keys_host, uint64_t n, uint32_t* out_host,
                           uint64_t* ticket) {
    if (!c || !ticket || sketch_id >= c->cfg.max_sketches || n > c->cfg.max_batch_keys) return SF_ERR_INVALID;
    if (n && (!keys_host || !out_host)) return SF_ERR_INVALID;
    auto r = std::make_shared<Request>();
    r->keys = (const uint8_t*)keys_host;
    r->n = n;
    r->out = out_host;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(c->mu);
        Version* v = c->table[sketch_id];
        if (!v) return SF_ERR_INVALID;
        v->refs++;
        r->v = v;
        r->ticket = c->next_ticket++;
        *ticket = r->ticket;
        c->tickets[r->ticket] = r;
        c->pending.push_back(r);
        c->pending_keys += n;
        c->st_requests++;
        c->st_keys += n;
        if (!c->window_started) {
            c->window_started = true;
            c->window_start = r->t_submit;
        }
    }
    c->cv_work.notify_one();
    return SF_OK;
}

static sf_status finish_ticket(sfc* c, uint64_t ticket, bool block) {
    std::unique_lock<std::mutex> lk(c->mu);
    auto it = c->tickets.find(ticket);
    if (it == c->tickets.end()) return SF_ERR_INVALID;
    std::shared_ptr<Request> r = it->second;
    if (block) c->cv_done.wait(lk, [&] { return r->done.load() != 0; });
    if (!r->done.load()) return SF_PENDING;
    c->tickets.erase(it);
    return r->status;
}

sf_status sfc_poll(sfc* c, uint64_t ticket) { return c ? finish_ticket(c, ticket, false) : SF_ERR_INVALID; }

sf_status sfc_wait(sfc* c, uint64_t ticket) { return c ? finish_ticket(c, ticket, true) : SF_ERR_INVALID; }

sf_status sfc_stats_get(sfc* c, sfc_stats* out, int reset) {
    if (!c || !out) return SF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    std::memset(out, 0, sizeof(*out));
    out->requests = c->st_requests;
    out->keys = c->st_keys;
    out->batches = c->st_batches;
    out->uploads = c->st_uploads;
    out->rejected_uploads = c->st_rejected;
    out->evictions = c->st_evictions;
    out->arena_used_bytes = c->arena.used();
    if (!c->lat_us.empty()) {
        std::vector<double> v = c->lat_us;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->max_us = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_us = sum / v.size();
        const double secs = std::chrono::duration<double>(c->last_done - c->window_start).count();
        out->qps = secs > 0 ? (double)c->st_keys / secs : 0.0;
    }
    if (reset) {
        c->lat_us.clear();
        c->st_requests = c->st_keys = c->st_batches = 0;
        c->window_started = false;
    }
    return SF_OK;
}

sf_status sfc_destroy(sfc* c) {
    if (!c) return SF_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop = true;
    }
    c->cv_work.notify_all();
    if (c->worker.joinable()) c->worker.join();
    for (auto& s : c->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.ev) cudaEventDestroy(s.ev);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.keys_host) cudaFreeHost(s.keys_host);
        if (s.out_host) cudaFreeHost(s.out_host);
        if (s.reqs_host) cudaFreeHost(s.reqs_host);
    }
    if (c->upload_stream) cudaStreamDestroy(c->upload_stream);
    for (Version* v : c->table) delete v;
    delete c;
    return SF_OK;
}

}  // extern "C"
