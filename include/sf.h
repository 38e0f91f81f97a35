/*
 * sf.h -- C ABI of the GB300 (sm_103a) SF-sketch library.
 *
 * The SF-sketch (Yang et al., "SF-sketch: A Two-stage Sketch for Data Streams") keeps two
 * subsketches at a monitoring node:
 *   - the Slim-subsketch A: d arrays of w uint32 counters A_i[j]            (Sec. 3.1, Table 1)
 *   - the Fat-subsketch  B: d arrays of w buckets of z uint32 counters B_i[j][k]; the bucket of
 *     item e in row i is h_i(e) (shared with the Slim), the counter inside it is f_i(e)
 *                                                                           (Sec. 3.4, SF_4/SF_F)
 * Insertions and deletions update the Fat, read it back, and then raise or lower the item's
 * Slim counters (Sec. 3.4 "Insertion", Sec. 3.5 "Deletion").  Only the Slim is sent to the
 * remote collector (Abstract; Sec. 1.1), which answers point queries as the minimum of the
 * item's d Slim counters (Sec. 3.1 "Query").
 *
 * Batched semantics.  The paper updates one item at a time.  A call here processes its stream
 * in chunks of params.chunk = S updates (a call always starts a new chunk; the last chunk may
 * be short).  With A0, B0 the state at chunk start: the Fat receives every +1/-1 of the chunk;
 * each distinct key e inserted c_e times in the chunk raises its Slim counters to
 *     T_e = min( min_i A0_i[h_i(e)] + c_e ,  min_i B_i[h_i(e)][f_i(e)] after the chunk );
 * each delete lowers A_i[h_i(e)] to max_k B_i[h_i(e)][k] after the chunk when it is larger;
 * per counter these operations apply in stream order.  S = 1 is exactly the paper's
 * one-at-a-time rule.  The result is a deterministic function of the input: every counter
 * is an exact integer, independent of thread scheduling.
 *
 * Hashing (the paper asks only for independent uniform h_i, f_i): row seeds are the first d
 * outputs of SplitMix64 from params.seed; H_i = mix64(x0 ^ s_i) for keys of at most 8 bytes,
 * mix64(mix64(x0 ^ s_i) ^ x1) for longer keys (x0, x1 = key bytes 0..7 and 8..14 read
 * little-endian, zero-padded); h_i = (hi32(H_i) * w) >> 32, f_i = (lo32(H_i) * z) >> 32.
 *
 * Memory ownership.  The caller allocates every device buffer (Fat, Slim, scratch, keys,
 * outputs) and keeps it alive while the handle uses it; sf_required_bytes gives the sizes.
 * The library allocates no device memory.  Every call is asynchronous on the handle's
 * CUDA stream; sf_sync waits and reports errors raised on the device.  A handle is used
 * by one host thread at a time.
 *
 * Where the key, operation and answer buffers may live.  The arguments named *_dev that carry
 * keys (sf_insert_batch, sf_delete_batch, sf_update_batch, sf_batch_item, sf_query_batch,
 * sf_update_batch_noalloc), operations, and query answers (sf_query_batch out_dev) may be device
 * or managed memory, or page-locked host memory (cudaHostAlloc / cudaHostRegister): the kernels
 * then read the keys and write the answers over the host link themselves, with no staging
 * copy -- except the update calls of a sketch that owns its dictionary and whose chunks (2 to
 * 65,536 updates) fit one round of the grid, given page-locked keys and page-locked (or no)
 * operations: those copy them, in pieces of whole chunks, into the half of the sketch's dictionary
 * region that such rounds leave unused, on a copy stream the sketch creates at its first such call,
 * each piece applied while the next is copied (pieces under 262,144 updates, unless one piece holds
 * the whole call, read over the link instead).  Either way the host buffers stay in use until
 * sf_sync returns.  Each pointer is checked with cudaPointerGetAttributes before any launch;
 * pageable host memory returns SF_ERR_INVALID.  Fat, Slim and scratch buffers are device memory.
 *
 * Errors.  No exception crosses the ABI.  Argument errors return immediately; errors found
 * on the device are latched in the scratch buffer and returned by the next sf_sync.
 */
#ifndef SF_H_
#define SF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sf_status;

#define SF_OK              0
#define SF_ERR_INVALID    -1  /* bad argument, handle, alignment or key id                  */
#define SF_ERR_OOM        -2  /* a caller buffer is smaller than required                   */
#define SF_ERR_CUDA       -3  /* a CUDA runtime call failed                                 */
#define SF_ERR_TIMEOUT    -4  /* a device-side wait gave up; the sketch contents are lost   */
#define SF_ERR_UNDERFLOW  -5  /* a delete removed an occurrence that was never inserted     */
#define SF_ERR_BUDGET     -6  /* collector: upload not admissible under the memory budget   */
#define SF_ERR_VERSION    -7  /* Slim header magic/version/hash id mismatch                 */
#define SF_PENDING         1  /* collector: ticket not finished yet                         */

#define SF_MAX_D 8
#define SF_MAX_Z 64
#define SF_MAX_KEY_BYTES 15
#define SF_MAX_CHUNK (1u << 20)

#define SF_SLIM_MAGIC   0x4D494C53u  /* "SLIM" */
#define SF_SLIM_VERSION 1u
#define SF_HASH_SPLITMIX_LEMIRE 1u   /* the hash described above                           */
#define SF_HASH_EXPLICIT        2u   /* indices from a caller table (explicit-index mode)  */

/* params.flags */
#define SF_FLAG_EXPLICIT_INDEX 1u    /* keys are uint32 ids into a table of (h_i, f_i)    */
#define SF_FLAG_SF4_DELETE     2u    /* deletions follow the SF_4 rule (Sec. 3.4): A_i[h_i] is
                                        decremented by 1 when above the bucket SUM
                                        sum_k B_i[h_i][k] after the Fat decrement, instead of
                                        SF_F's clamp to the bucket maximum (Sec. 3.5).  Kept for
                                        the ablation against SF_F; insertions and queries are
                                        the same.  Chunked updates apply it as a clamp to the
                                        chunk-end bucket sum (equal, since A <= sum holds)   */
#define SF_FLAG_SHARED_DICT    4u    /* the chunk dictionary is not in the sketch's scratch:
                                        a batch with a dictionary arena places it there per
                                        launch group, and standalone updates use the memory
                                        given by sf_set_dictionary (see below)                */

typedef struct sf_params {
    uint32_t d;          /* rows, 1..SF_MAX_D                                   (Table 1: d) */
    uint32_t w;          /* Slim counters per row = Fat buckets per row, >= 1   (Table 1: w) */
    uint32_t z;          /* Fat counters per bucket, 1..SF_MAX_Z                (Table 1: z) */
    uint32_t key_bytes;  /* packed key width, 1..SF_MAX_KEY_BYTES (4 in explicit mode)       */
    uint64_t seed;       /* hash seed                                                        */
    uint32_t chunk;      /* S updates per chunk, 1..SF_MAX_CHUNK (semantic: see above)       */
    uint32_t flags;      /* SF_FLAG_*                                                        */
} sf_params;

typedef struct sf_slim_header {
    uint32_t magic;      /* SF_SLIM_MAGIC   */
    uint32_t version;    /* SF_SLIM_VERSION */
    uint32_t d, w, key_bytes, hash_id;
    uint64_t seed;
} sf_slim_header;

/* A Slim-subsketch as the collector sees it: d*w uint32 counters, row-major A[i*w + j]. */
typedef struct sf_slim_view {
    const uint32_t *counters;       /* device */
    sf_slim_header hdr;
    const uint32_t *index_table;    /* device, explicit-index mode only, else NULL */
    uint32_t n_index_keys;
} sf_slim_view;

typedef struct sf_sketch sf_sketch;

/* Human-readable name of a status code (static string). */
const char *sf_status_str(sf_status s);

/*
 * Device bytes the caller must provide for a sketch with these parameters
 * (Sec. 3.4: the Fat is d*w*z counters, the Slim d*w counters).
 *   fat_bytes     = d*w*z*4, layout B[((i*w + j)*z + k]  (bucket-contiguous, Sec. 3.4: all z
 *                   counters of a bucket sit together so one access reads them)
 *   slim_bytes    = d*w*4,   layout A[i*w + j]
 *   scratch_bytes = control words + the per-chunk key dictionary: 32 B x a power of two
 *                   >= 16*chunk slots for chunks up to 65,536, >= 8*chunk above (no
 *                   dictionary with SF_FLAG_SHARED_DICT: see sf_set_dictionary);
 *                   sketches with chunk == 1 and w >= 1024 also hold the one-at-a-time
 *                   dependency-graph workspace (about (16 + 8d) * 512 KiB)
 * Any output pointer may be NULL.  Returns SF_ERR_INVALID for parameters out of range.
 */
sf_status sf_required_bytes(const sf_params *p, uint64_t *fat_bytes, uint64_t *slim_bytes,
                            uint64_t *scratch_bytes);

/*
 * Initialisation (Sec. 3.1: all counters set to zero): zeroes the Fat, the Slim and the
 * scratch on `cuda_stream` (a cudaStream_t; NULL = the legacy default stream) and returns a
 * host handle in *out.  Buffers: device memory of at least sf_required_bytes, 16-byte aligned,
 * owned by the caller and not freed before sf_destroy.  The handle captures the current device.
 */
sf_status sf_create(const sf_params *p, void *fat_dev, void *slim_dev, void *scratch_dev,
                    void *cuda_stream, sf_sketch **out);

/* Releases the host handle (not the caller's device buffers).  Does not synchronise. */
sf_status sf_destroy(sf_sketch *s);

/*
 * Initialisation again on the same buffers (Sec. 3.1: all counters zero): zeroes the Fat, the Slim
 * and the control words on the handle's stream, after its queued work.  The chunk dictionary is left
 * as it is, because every update call leaves it zeroed (and sf_sync re-zeroes the whole scratch after
 * SF_ERR_TIMEOUT); chunk-1 sketches also re-zero their one-at-a-time workspace.  Cheaper than a new
 * handle when the dictionary is large (it reserves 256 to 1,024 B per chunk slot).
 */
sf_status sf_reset(sf_sketch *s);

/*
 * Explicit-index mode (params.flags & SF_FLAG_EXPLICIT_INDEX): keys are uint32 ids and the
 * device table holds, for id q and row i, h_i = table[(q*d + i)*2], f_i = table[(q*d + i)*2 + 1]
 * (h_i < w, f_i < z).  Used to replay worked examples with hand-chosen indices (Sec. 3.2).
 * Ids >= n_keys are rejected on the device (SF_ERR_INVALID at the next sf_sync): such an update
 * changes no counter, and the others apply as they would with its operation removed from its
 * chunk (its stream position still counts towards the chunk boundaries).
 */
sf_status sf_set_index_table(sf_sketch *s, const uint32_t *table_dev, uint32_t n_keys);

/*
 * The per-chunk key dictionary outside the sketch's scratch (params.flags & SF_FLAG_SHARED_DICT).
 * A chunked update keys a dictionary by the distinct keys of each chunk (its entries are zero
 * between launches: every launch clears the entries it claimed); a sketch owns one in its scratch
 * unless it was created with SF_FLAG_SHARED_DICT, and then scratch_bytes holds the control words
 * only.  The dictionary is live only while one of the sketch's updates runs, so sketches whose
 * updates never run at the same time -- calls on one stream, or the launch groups of one batch --
 * can share one.
 *   sf_dictionary_bytes: the dictionary a sketch with these parameters needs (0 for chunk 1).
 *   sf_set_dictionary: dict_dev, 16-byte aligned device memory of at least that many bytes, is the
 *     dictionary of the sketch's standalone updates (sf_update_batch and the calls built on it);
 *     the call zeroes it on the sketch's stream.  The caller keeps it alive, and lets no two
 *     updates that use it run at the same time.  The sf_sync that returns SF_ERR_TIMEOUT re-zeroes
 *     it with the scratch.  SF_ERR_INVALID for a sketch without the flag or too small a buffer.
 *     A flagged sketch with chunk > 1 and no dictionary refuses standalone updates
 *     (SF_ERR_INVALID).
 */
sf_status sf_dictionary_bytes(const sf_params *p, uint64_t *dict_bytes);
sf_status sf_set_dictionary(sf_sketch *s, void *dict_dev, uint64_t bytes);

/*
 * Insertion of n items (Sec. 3.4 "Insertion", used unchanged by SF_F, Sec. 3.5), under the
 * chunked semantics above.  keys_dev: n*key_bytes packed bytes on the device (4- or 8-byte
 * keys must be aligned to their width).  n = 0 is a no-op.  Asynchronous.
 */
sf_status sf_insert_batch(sf_sketch *s, const void *keys_dev, uint64_t n);

/*
 * Deletion of n items (Sec. 3.5 "Deletion").  Precondition: every deleted occurrence was
 * inserted before (the paper's proofs assume it).  A Fat counter seen negative at the end
 * of a chunk is reported as SF_ERR_UNDERFLOW by sf_sync; counters are then unspecified.
 */
sf_status sf_delete_batch(sf_sketch *s, const void *keys_dev, uint64_t n);

/*
 * Mixed stream: ops_dev[t] = +1 (insert) or -1 (delete) for key t, stream order preserved
 * inside each chunk; 0 skips the update.  Same rules as the two calls above.
 */
sf_status sf_update_batch(sf_sketch *s, const void *keys_dev, const int8_t *ops_dev, uint64_t n);

/*
 * Slim transfer (Abstract, Sec. 1.1: only the Slim goes to the collector): copies the d*w
 * Slim counters to dst_dev (device, cap_elems >= d*w) after all queued updates, on the
 * handle's stream, and fills *hdr (may be NULL).  SF_ERR_OOM if cap_elems is too small.
 */
sf_status sf_export_slim(const sf_sketch *s, uint32_t *dst_dev, uint64_t cap_elems,
                         sf_slim_header *hdr);

/*
 * Point queries (Sec. 3.1 "Query"): out_dev[t] = min_i A_i[h_i(key_t)] on an exported Slim.
 * keys_dev: n packed keys of slim->hdr.key_bytes bytes (device); out_dev: n uint32 (device).
 * Runs on cuda_stream.  SF_ERR_VERSION if the header is not a Slim of this library.
 */
sf_status sf_query_batch(const sf_slim_view *slim, const void *keys_dev, uint64_t n,
                         uint32_t *out_dev, void *cuda_stream);

/* Waits for the handle's stream and returns (then clears) errors latched on the device. */
sf_status sf_sync(sf_sketch *s);

/*
 * Multi-stream query pipeline (Sec. 4.2.2): a batch of n host keys is split over n_streams CUDA
 * streams in parts of nearly equal size (the first n % n_streams parts take one key more); on each
 * stream its part is copied to the device, queried (Sec. 3.1) and its answers copied back, so the
 * copies of one part overlap the kernels of another.  keys_host / out_host: host buffers (pinned
 * for the copies to overlap); keys_dev / out_dev: device staging of n keys / n answers;
 * streams: n_streams cudaStream_t.  Asynchronous: synchronise the streams before reading out_host.
 */
sf_status sf_query_pipelined(const sf_slim_view *slim, const void *keys_host, uint64_t n, uint32_t *out_host,
                             void *keys_dev, uint32_t *out_dev, uint32_t n_streams, void *const *streams);

/*
 * Update from host memory, copies overlapped with the kernels (the multi-stream pipeline of Sec.
 * 4.2.2, applied to insertions and deletions).  The n keys (and operations) at keys_host / ops_host
 * -- page-locked host memory for the copies to overlap -- are copied in pieces of a whole number of
 * chunks (params.chunk updates each) into two alternating halves of staging_dev, on copy_stream
 * (a cudaStream_t other than the sketch's), and each piece is applied on the sketch's stream as soon
 * as it has landed, while the next piece is copied.  Pieces end on chunk boundaries, so the counters
 * equal one sf_update_batch call over all n updates.  ops_host NULL: every update is op_const
 * (+1 insert or -1 delete).  staging_dev: 16-byte aligned device memory (else SF_ERR_INVALID) of
 * staging_bytes >= 2 * (chunk * (key_bytes + (ops_host ? 1 : 0)) + 32) bytes, enough for a piece of
 * one chunk (each half holds a piece's keys padded to a 16-byte multiple, then its operations), else
 * SF_ERR_OOM.  Asynchronous: the host buffers and the staging stay in use until sf_sync on the
 * sketch returns.
 */
sf_status sf_update_pipelined(sf_sketch *s, const void *keys_host, const int8_t *ops_host, int32_t op_const,
                              uint64_t n, void *staging_dev, uint64_t staging_bytes, void *copy_stream);

/*
 * The same pipeline kept across calls (Sec. 4.2.2's overlap of copies and kernels, carried from
 * one call to the next).  A pipeline owns a staging buffer's two halves and, per half, the event of
 * the last update that read it.  A call's first piece then goes into the half the previous call did
 * not end on and waits only for the last update that read that half -- not for all of the sketch's
 * earlier work, as sf_update_pipelined does -- so successive calls, on one sketch or on several
 * sketches sharing the pipeline, overlap each call's first copy with the previous call's last
 * update.
 *   sf_pipeline_create: staging_dev: 16-byte aligned device memory of staging_bytes (>= 64) that the
 *     pipeline uses alone until every update through it has completed (sf_sync of each sketch);
 *     copy_stream: a cudaStream_t on which no sketch using the pipeline updates.  The pipeline
 *     belongs to the current device.  SF_ERR_INVALID for a bad argument, SF_ERR_CUDA if its events
 *     cannot be created.
 *   sf_update_pipeline: the pieces and results of sf_update_pipelined (equal to one
 *     sf_update_batch call over the n updates); a piece is the whole number of the sketch's chunks
 *     that fits half the staging, SF_ERR_OOM when not even one chunk does.  Asynchronous like
 *     sf_update_pipelined.  One host thread at a time may use a pipeline.
 *   sf_pipeline_destroy: releases the pipeline (its events go once their work has completed); the
 *     staging stays the caller's.
 */
typedef struct sf_pipeline sf_pipeline;
sf_status sf_pipeline_create(void *staging_dev, uint64_t staging_bytes, void *copy_stream, sf_pipeline **out);
sf_status sf_update_pipeline(sf_sketch *s, sf_pipeline *p, const void *keys_host, const int8_t *ops_host,
                             int32_t op_const, uint64_t n);
sf_status sf_pipeline_destroy(sf_pipeline *p);

/*
 * ---- Batched many-sketch update --------------------------------------------------------------
 * Monitoring nodes each fill their own sketch (Sec. 1.1); a collector-side or node-side host may
 * hold thousands of them.  The paper updates one sketch at a time; a batch applies one call's
 * stream to each of many sketches in ONE persistent cooperative launch (captured in a CUDA graph
 * and replayed when the batch shape repeats).  Every sketch gets exactly the chunked semantics of
 * sf_update_batch with its own params.chunk: round r of the launch processes chunk r of every
 * sketch, so the result equals one sf_update_batch call per sketch, bit for bit.
 */
typedef struct sf_batch sf_batch;

typedef struct sf_batch_item {
    sf_sketch *sketch;        /* distinct sketches, all with the same d, on the batch's device   */
    const void *keys_dev;     /* n packed keys of the sketch's key_bytes (device)                */
    const int8_t *ops_dev;    /* +1 insert / -1 delete / 0 skip per key, or NULL (all inserts)  */
    uint64_t n;
} sf_batch_item;

#define SF_BATCH_GRAPH 1u     /* capture the launch in a CUDA graph and replay it               */

/*
 * Device scratch of a batch of up to max_sketches items whose chunk sizes, each rounded up to a
 * multiple of 32, sum to at most max_round_slots: control words, the run table and the per-block
 * lists of dictionary claims of one round.
 */
sf_status sf_batch_required_bytes(uint32_t max_sketches, uint64_t max_round_slots, uint64_t *scratch_bytes);

/*
 * Creates a batch bound to cuda_stream and to caller-owned scratch_dev (sf_batch_required_bytes,
 * 16-byte aligned; zeroed here).  The batch allocates a pinned host staging table and a private
 * capture stream, no device memory.  flags: SF_BATCH_GRAPH or 0 (direct launches).
 */
sf_status sf_batch_create(uint32_t max_sketches, uint64_t max_round_slots, void *scratch_dev, void *cuda_stream,
                          uint32_t flags, sf_batch **out);

/*
 * Enqueues items[0..n_items) as one launch on the batch's stream.  The sketches' own pending work
 * must be ordered before it (same stream, or synchronised).  A call whose chunk sizes (rounded up
 * to multiples of 32) sum above max_round_slots returns SF_ERR_INVALID.  Device errors: sf_batch_sync.
 */
sf_status sf_batch_update(sf_batch *b, uint32_t n_items, const sf_batch_item *items);

/* Waits for the batch's stream; returns (then clears) device errors of the batch's launches.
 * After SF_ERR_TIMEOUT the sketches of the last call must be re-created. */
sf_status sf_batch_sync(sf_batch *b);

/*
 * Launch grouping of sf_batch_update (no counterpart in the paper).  Sketches are independent, so a
 * call may update them in any grouping: sketches whose counters (Fat + Slim + the dictionary entries
 * one chunk can touch, 32 B per chunk slot) fit `bytes` are packed, in input order, into groups
 * whose counters fit it together, one cooperative launch per group, so each launch works out of L2;
 * sketches larger than `bytes` share one launch.  bytes = 0 puts every sketch of a call in one
 * launch.  The default is 3/4 of the device's L2 (about 95 MiB on a GB300).  Results do not depend
 * on the grouping (each sketch's updates are the same); only the speed does.
 */
sf_status sf_batch_set_group_bytes(sf_batch *b, uint64_t bytes);

/*
 * Dictionary arena of a batch, for its SF_FLAG_SHARED_DICT sketches: launch groups run one after
 * another on the batch's stream, so each group's flagged sketches take their dictionaries
 * (sf_dictionary_bytes each) from the start of the arena, and a group whose flagged sketches'
 * dictionaries do not fit together is split into launches that fit.  arena_dev: 16-byte aligned
 * device memory of `bytes` that the batch uses alone while it lives; the call zeroes it on the
 * batch's stream (sf_batch_sync zeroes it again after SF_ERR_TIMEOUT).  NULL / 0 removes the
 * arena; flagged sketches then use the dictionary given by sf_set_dictionary (SF_ERR_INVALID
 * without one).  A flagged sketch whose dictionary alone exceeds the arena is SF_ERR_OOM.
 */
sf_status sf_batch_set_dictionary_arena(sf_batch *b, void *arena_dev, uint64_t bytes);
/*
 * Launch shape of sf_batch_update (no counterpart in the paper): `threads` per block, 512 (the
 * default), 256 or 128, with 512 / threads co-resident blocks per SM, so each shape runs the same
 * number of threads; smaller blocks mean finer-grained block merges and grid-barrier arrivals.
 * Results do not depend on the shape, only the speed does (the batch autotuner picks it).
 * SF_ERR_INVALID for another value.
 */
sf_status sf_batch_set_block_threads(sf_batch *b, uint32_t threads);

/* The group budget and the number of launches the last sf_batch_update used. */
sf_status sf_batch_groups(const sf_batch *b, uint32_t *groups_last, uint64_t *group_bytes);

/* Counters: graph launches, graph captures, and the round count of the last call. */
sf_status sf_batch_info(const sf_batch *b, uint32_t *graph_launches, uint32_t *graph_captures,
                        uint64_t *rounds_last);

sf_status sf_batch_destroy(sf_batch *b);

/*
 * ---- Collector serving loop --------------------------------------------------------------------
 * The remote collector receives Slim-subsketches from many monitoring nodes and answers point
 * queries from them (Abstract; Sec. 1.1; GPU batching and multi-stream pipelining, Sec. 4.2).
 * sfc_* keeps uploaded Slims resident in a caller-provided device arena -- the memory budget --
 * and serves queries with continuous batching: a worker thread packs the requests that have
 * arrived into one multi-request query launch per batch, keeps up to n_streams batches in flight
 * on separate CUDA streams, and admits new requests into the next batch as soon as a stream frees,
 * while earlier batches still run.  Each query binds to the sketch version current at submit
 * (uploads replace in place; an old version's memory returns to the arena when its last query
 * finishes).  Answers equal sf_query_batch on the same Slim.
 */
typedef struct sfc sfc;

typedef struct sfc_config {
    void *arena_dev;          /* device memory holding resident Slims: the admission budget      */
    uint64_t arena_bytes;
    void *staging_dev;        /* device memory for the request tables of in-flight batches
                                 (sfc_required_staging_bytes); their keys and answers live in
                                 mapped pinned host memory that the query kernel reads and writes */
    uint64_t staging_bytes;
    uint32_t max_sketches;    /* sketch ids are 0 .. max_sketches-1                              */
    uint32_t n_streams;       /* batches in flight at once, 1..16                                */
    uint32_t max_batch_keys;  /* keys per launched batch; one request may not exceed it          */
    uint32_t max_batch_reqs;  /* requests per launched batch                                     */
    uint32_t max_wait_us;     /* a partly filled batch waits at most this long for more requests */
} sfc_config;

typedef struct sfc_stats {
    uint64_t requests, keys, batches, uploads, rejected_uploads, evictions;
    double p50_us, p99_us, mean_us, max_us;  /* submit -> answers in the caller's host buffer   */
    double qps;                               /* keys answered per second over the stats window  */
    uint64_t arena_used_bytes;
} sfc_stats;

/* Device staging bytes for a configuration (the request tables of n_streams batches). */
sf_status sfc_required_staging_bytes(const sfc_config *c, uint64_t *bytes);

/* Starts a collector (and its worker thread) on the current device.  Host staging is pinned
 * memory allocated here; device memory is only the caller's arena and staging. */
sf_status sfc_create(const sfc_config *c, sfc **out);

/*
 * Upload (or replace) the Slim of sketch_id: d*w counters at `counters` (device or host pointer,
 * e.g. from sf_export_slim) with its header.  Returns after the copy; queries submitted afterwards
 * see the new version.  SF_ERR_BUDGET: the arena cannot hold it now (nothing changes);
 * SF_ERR_VERSION: not a Slim header of this library.
 */
sf_status sfc_upload(sfc *c, uint32_t sketch_id, const uint32_t *counters, const sf_slim_header *hdr);

/* Drops sketch_id; its memory returns to the arena once queries bound to it finish. */
sf_status sfc_evict(sfc *c, uint32_t sketch_id);

/*
 * Submits n point queries (host keys of the sketch's key_bytes) against the current version of
 * sketch_id; answers are written to out_host (n uint32) before the ticket completes.  Both
 * buffers must stay valid until then.  n <= max_batch_keys.
 */
sf_status sfc_query_submit(sfc *c, uint32_t sketch_id, const void *keys_host, uint64_t n, uint32_t *out_host,
                           uint64_t *ticket);

/* The ticket's status once it finished (the ticket is then released): SF_OK, or SF_ERR_CUDA when
 * its batch could not be launched or its completion event reported a device error (out_host is
 * then not written); SF_PENDING while it runs. */
sf_status sfc_poll(sfc *c, uint64_t ticket);

/* Blocks until the ticket finished; then like sfc_poll. */
sf_status sfc_wait(sfc *c, uint64_t ticket);

/* Statistics since creation or the last reset (reset != 0 clears them after reading). */
sf_status sfc_stats_get(sfc *c, sfc_stats *out, int reset);

/* Stops the worker after finishing submitted requests; frees host resources. */
sf_status sfc_destroy(sfc *c);

/*
 * Update without any caller scratch -- the paper has no counterpart; this is a deployment aid.
 *
 * For callers that cannot allocate device memory at update time: a serving or packet loop that
 * reserved all of its memory at start-up and must not call cudaMalloc (it can block and
 * synchronise the device), or a plugin living inside another framework's memory pool.  It applies
 * the same chunked insert/delete rules as sf_update_batch to the caller's Fat (fat_dev) and Slim
 * (slim_dev) -- laid out as sf_required_bytes describes and zeroed by the caller before the first
 * update -- but takes no scratch buffer and no handle.  ops_dev may be NULL (all insertions).
 *
 * The per-chunk dictionary and control words live in one fixed device array of this library
 * (2 MiB + 256 B), which every GPU that loads the library keeps until the process exits.  Hence:
 *   - params->chunk must be 2..SF_NOALLOC_MAX_CHUNK; larger chunks return SF_ERR_INVALID (the
 *     array is sized for that maximum), as do explicit-index flags (SF_FLAG_SF4_DELETE is
 *     accepted; SF_FLAG_SHARED_DICT changes nothing here, the dictionary being the fixed array);
 *   - all calls share the array, so calls that may overlap on the GPU (different streams,
 *     different threads) race and corrupt each other's result: serialise them;
 *   - the call zeroes the array's control words and dictionary itself before its kernel runs;
 *   - the first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 *     that device current) and keeps it for the life of the process; make that first call before
 *     capturing any CUDA stream.  The kept address does not survive cudaDeviceReset (which reloads
 *     the library's device code): do not call this entry point on a device after resetting it.
 * No device memory is allocated: no cudaMalloc/cudaFree, no allocating library call.  If err_dev
 * (device, 4 bytes) is not NULL it receives the device-side error bits of this call: 0 = none;
 * bit 0 (1) = a Fat counter went negative, i.e. a delete of an item never inserted; bit 1 (2) = a
 * device wait timed out; bit 3 (8) = the per-chunk dictionary overflowed (cannot happen within
 * the chunk limit above, since the dictionary holds four slots per update of a chunk); bit 2 (4)
 * is the explicit-index key-id check, which this entry point never runs.  Any non-zero value
 * means the counters are unspecified.  Asynchronous on cuda_stream.
 */
#define SF_NOALLOC_MAX_CHUNK 16384u
sf_status sf_update_batch_noalloc(const sf_params *p, uint32_t *fat_dev, uint32_t *slim_dev,
                                  const void *keys_dev, const int8_t *ops_dev, uint64_t n,
                                  uint32_t *err_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SF_H_ */
