// sf_seqdag.cu -- the S = 1 insertion path as a dependency graph over the whole stream (sm_103a).
//
// The paper's one-at-a-time insertion (Sec. 3.4, kept by SF_F in Sec. 3.5) makes an update
// depend on an earlier one only when the two share a bucket (i, h_i) in some row: every counter
// either touches -- Slim A_i[h_i], Fat B_i[h_i][.] -- lies in its d buckets.  So any order that
// keeps, in every bucket, the stream order of the updates hashed to it gives the stream-order
// result.  For a call of insertions only, taken in pieces of up to kDagN updates:
//   1. hash every update (parallel);
//   2. per row, a stable radix sort of (bucket, position) gives every update its predecessor and
//      successor in each of its buckets (the neighbouring entries of the sorted row); the same
//      launches sort every row a second time, by Fat counter (bucket x z + slot), for step 4;
//   3. runs (Lemma 2): an update whose predecessor in every row is the same earlier update with
//      the same Fat slots continues that update's run; a run is a block of consecutive entries
//      of row 0's sorted order, so a prefix maximum over that order finds each run's first
//      update (its head), which counts the run's length r and records its last member;
//   4. the Fat only grows under insertions, so the value a Fat counter holds right after an
//      update is its value at the start of the piece plus the number of the piece's updates on
//      that counter up to and including this one, in stream order.  The rows sorted by counter
//      give those counts, and with them each run's Fat estimate F (the minimum over rows, after
//      its last member) before anything runs; the whole piece's Fat increments are then added
//      in parallel;
//   5. a run can go once, in every row, the run before it in that bucket has gone: heads count
//      their pending predecessors, and one block walks the graph frontier by frontier, with the
//      pending counts (four bits per update) and, where it fits, the Slim in shared memory.  A
//      run's Slim counters rise to T = min(m + r, F) where lower, m being their minimum when the
//      run goes and r its length.  Runs of one frontier share no bucket, so they touch disjoint
//      counters.
// A piece's graph is only as deep as its longest chain of runs through shared buckets.
#include "sf_internal.h"
#include "sf_seqdag.h"

namespace sfk {

namespace {

constexpr uint32_t kDagNone = 0xFFFFFFFFu;

// The graph path is a chain of short launches over one piece (15 for two radix passes).  Each goes
// with programmatic stream serialization, so it is launched while the kernel before it drains, and
// starts by waiting (griddepcontrol.wait) until that kernel has completed and its writes are
// visible: every read of an earlier kernel's output and every overwrite of a buffer an earlier
// kernel reads comes after that wait.  Measured on the one-at-a-time u32 workload (100,000 updates,
// bit-exact): 0.412 -> 0.376 ms; three pieces (300,000): 1.216 -> 1.110 ms.  Triggering the next
// launch explicitly at kernel entry instead of at block exit measured the same.
__device__ __forceinline__ void wait_prior_kernel() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static cudaError_t dag_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}
constexpr int kDagTile = 1024;           // elements per radix tile (one block)
constexpr int kDagTiles = kDagN / kDagTile;
constexpr int kDagRadixBits = 8;
constexpr int kDagBins = 1 << kDagRadixBits;

// Workspace arrays of one piece (kDagN updates, d rows), carved out of the sketch scratch.
struct DagWs {
    uint4* rec;                   // [N][4G] walk record of every run head (dag_npred_kernel)
    uint32_t* cnt;                // [d][N] the Fat counter of each update, counted up to it
    uint32_t *hb, *fb;            // [d][N] bucket and slot of every update
    uint32_t *sk0, *sv0, *sk1, *sv1;  // [2d][N] radix sort keys and values (positions): rows 0..d-1
                                      // keyed by bucket, rows d..2d-1 by Fat counter
    uint32_t *pred, *succ;        // [d][N] previous / next update in the same bucket
    uint32_t *par0, *par1;        // [N] run parent links, then every update's run head
    uint32_t *rlen, *lastm;       // [N] run length and last member, at heads
    uint32_t *npred;              // [N / 8] pending predecessors of the heads, four bits each
    uint32_t *bad;                // [N] the key had no valid index (explicit-index mode)
    uint32_t *q0, *q1;            // [N] frontier queues
    uint32_t *qcount;             // [4] queue counters
    uint32_t *hist;               // [2d][bins][tiles] digit counts, then offsets
};

// A walk record holds one uint4 per row i, {bucket h_i, successor head in that bucket, run
// length, Fat estimate}, so the lane of row i reads its part in one load; records sit 4G uint4
// apart, G = ceil(d / 4) (64 bytes for d <= 4, 128 for d <= 8).
__host__ __device__ inline uint32_t dag_groups(uint32_t d) { return d <= 4 ? 1u : 2u; }

__host__ __device__ inline uint64_t dag_bytes_for(uint32_t d) {
    const uint64_t N = kDagN;
    return (16ull * dag_groups(d) * N + 13ull * d * N + 8ull * N + 64ull + 2ull * d * kDagBins * kDagTiles) * 4ull;
}

DagWs dag_carve(void* base, uint32_t d) {
    uint32_t* p = static_cast<uint32_t*>(base);
    const uint64_t N = kDagN;
    DagWs w;
    w.rec = reinterpret_cast<uint4*>(p);
    p += 16 * dag_groups(d) * N;
    w.cnt = p;
    p += d * N;
    w.hb = p;
    p += d * N;
    w.fb = p;
    p += d * N;
    w.sk0 = p;
    p += 2 * d * N;
    w.sv0 = p;
    p += 2 * d * N;
    w.sk1 = p;
    p += 2 * d * N;
    w.sv1 = p;
    p += 2 * d * N;
    w.pred = p;
    p += d * N;
    w.succ = p;
    p += d * N;
    w.par0 = p;
    p += N;
    w.par1 = p;
    p += N;
    w.rlen = p;
    p += N;
    w.lastm = p;
    p += N;
    w.npred = p;
    p += N;
    w.bad = p;
    p += N;
    w.q0 = p;
    p += N;
    w.q1 = p;
    p += N;
    w.qcount = p;
    p += 64;
    w.hist = p;
    return w;
}

// 1. hash every update of the piece; initialise the per-update arrays
__global__ void __launch_bounds__(256) dag_hash_kernel(SketchDesc s, const uint8_t* keys, uint32_t n, DagWs w,
                                                       uint32_t* ctrl) {
    wait_prior_kernel();
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const Key k = load_key(keys, j, s.key_bytes);
    uint32_t h[kMaxD], f[kMaxD];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
        h[i] = f[i] = 0u;
        if (i < (int)s.d) ok &= row_index(s, k, (uint32_t)i, &h[i], &f[i]);
    }
    if (!ok) {
        atomicOr(ctrl + kCtrlErr, kErrBadKey);
#pragma unroll
        for (int i = 0; i < kMaxD; ++i) h[i] = f[i] = 0u;  // a placeholder bucket; the update does nothing
    }
    // sort keys: the bucket (rows 0..d-1) and the Fat counter, bucket x z + slot (rows d..2d-1);
    // an update without a valid index counts on no counter and takes the spare key w x z
    const uint32_t wz = s.w * s.z;
    for (uint32_t i = 0; i < s.d; ++i) {
        w.hb[i * kDagN + j] = h[i];
        w.fb[i * kDagN + j] = f[i];
        w.sk0[i * kDagN + j] = h[i];
        w.sv0[i * kDagN + j] = j;
        w.sk0[(s.d + i) * kDagN + j] = ok ? h[i] * s.z + f[i] : wz;
        w.sv0[(s.d + i) * kDagN + j] = j;
        w.pred[i * kDagN + j] = kDagNone;
        w.succ[i * kDagN + j] = kDagNone;
    }
    if (j < 4) w.qcount[j] = 0u;
    w.rlen[j] = 0u;
    w.lastm[j] = 0u;
    if ((j & 7u) == 0u) w.npred[j >> 3] = 0u;
    w.bad[j] = ok ? 0u : 1u;
}

// 2a. digit counts of one tile of one row
__global__ void __launch_bounds__(256) dag_hist_kernel(const uint32_t* __restrict__ keys, uint32_t n, uint32_t shift,
                                                       uint32_t* __restrict__ hist) {
    wait_prior_kernel();
    __shared__ uint32_t bins[kDagBins];
    const uint32_t tile = blockIdx.x, row = blockIdx.y;
    for (uint32_t b = threadIdx.x; b < kDagBins; b += blockDim.x) bins[b] = 0u;
    __syncthreads();
    const uint32_t e0 = tile * kDagTile;
    for (uint32_t e = e0 + threadIdx.x; e < e0 + kDagTile && e < n; e += blockDim.x)
        atomicAdd(&bins[(keys[row * kDagN + e] >> shift) & (kDagBins - 1)], 1u);
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < kDagBins; b += blockDim.x)
        hist[((uint64_t)row * kDagBins + b) * kDagTiles + tile] = bins[b];
    if (tile == gridDim.x - 1) {  // zero the entries of the tiles past the piece's end (the scan reads all)
        const uint32_t spare = kDagTiles - gridDim.x;
        for (uint32_t i = threadIdx.x; i < kDagBins * spare; i += blockDim.x)
            hist[((uint64_t)row * kDagBins + i / spare) * kDagTiles + gridDim.x + i % spare] = 0u;
    }
}

// 2b. per row, exclusive scan of the counts in (digit, tile) order: the first output index of
//     each tile's elements of each digit.  Warp q scans the q-th 1,024 counts 32 at a time with
//     coalesced loads and shuffles; the 32 warp totals are scanned last.
__global__ void __launch_bounds__(1024) dag_scan_kernel(uint32_t* __restrict__ hist) {
    wait_prior_kernel();
    constexpr uint32_t kLen = kDagBins * kDagTiles;
    constexpr uint32_t kPerWarp = kLen / 32;
    static_assert(kPerWarp == 32 * 32, "one warp scans 32 steps of 32 counts");
    __shared__ uint32_t s_tot[32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t* hw = hist + (uint64_t)blockIdx.x * kLen + warp * kPerWarp;
    uint32_t x[32];
#pragma unroll
    for (uint32_t q = 0; q < 32; ++q) x[q] = hw[q * 32 + lane];
    uint32_t carry = 0;
#pragma unroll
    for (uint32_t q = 0; q < 32; ++q) {
        uint32_t incl = x[q];
#pragma unroll
        for (uint32_t off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off) incl += y;
        }
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        x[q] = carry + incl - x[q];
        carry += tot;
    }
    if (lane == 0) s_tot[warp] = carry;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = s_tot[lane];
        uint32_t incl = v;
#pragma unroll
        for (uint32_t off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off) incl += y;
        }
        s_tot[lane] = incl - v;
    }
    __syncthreads();
    const uint32_t base = s_tot[warp];
#pragma unroll
    for (uint32_t q = 0; q < 32; ++q) hw[q * 32 + lane] = base + x[q];
}

// 2c. stable scatter of one tile of one row.  Every warp ranks its elements among equal digits
//     (by lane) and counts its digits; the counts of each digit are then scanned over the warps
//     in order, on top of the tile's offset for that digit, so equal digits keep their order.
__global__ void __launch_bounds__(kDagTile) dag_scatter_kernel(const uint32_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint32_t* __restrict__ kout,
                                                               uint32_t* __restrict__ vout, uint32_t n,
                                                               uint32_t shift, const uint32_t* __restrict__ hist) {
    wait_prior_kernel();
    constexpr uint32_t kWarps = kDagTile / 32;
    __shared__ uint32_t s_cnt[kWarps][kDagBins];  // per warp and digit: count, then first output index
    const uint32_t tile = blockIdx.x, row = blockIdx.y;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (uint32_t b = lane; b < kDagBins; b += 32) s_cnt[warp][b] = 0u;
    const uint32_t e = tile * kDagTile + threadIdx.x;
    const bool valid = e < n;
    const uint32_t key = valid ? kin[row * kDagN + e] : 0u;
    const uint32_t val = valid ? vin[row * kDagN + e] : 0u;
    const uint32_t dig = (key >> shift) & (kDagBins - 1);
    const unsigned act = __ballot_sync(0xFFFFFFFFu, valid);
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, valid ? dig : 0x80000000u | lane) & act;
    const uint32_t rank = (uint32_t)__popc(peers & ((1u << lane) - 1u));
    __syncwarp();
    if (valid && rank == 0u) s_cnt[warp][dig] = (uint32_t)__popc(peers);
    __syncthreads();
    if (threadIdx.x < kDagBins) {
        const uint32_t b = threadIdx.x;
        uint32_t run = hist[((uint64_t)row * kDagBins + b) * kDagTiles + tile];
        for (uint32_t wv = 0; wv < kWarps; ++wv) {
            const uint32_t c = s_cnt[wv][b];
            s_cnt[wv][b] = run;
            run += c;
        }
    }
    __syncthreads();
    if (valid) {
        const uint32_t dst = s_cnt[warp][dig] + rank;
        kout[row * kDagN + dst] = key;
        vout[row * kDagN + dst] = val;
    }
}

// 3a. neighbours in bucket order: sorted entries k-1 and k of a row with the same bucket
__global__ void __launch_bounds__(256) dag_adj_kernel(DagWs w, uint32_t n) {
    wait_prior_kernel();
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y;
    if (k == 0 || k >= n) return;
    const uint32_t* sk = w.sk0 + row * kDagN;
    const uint32_t* sv = w.sv0 + row * kDagN;
    if (sk[k - 1] == sk[k]) {
        const uint32_t prev = sv[k - 1], pos = sv[k];
        w.pred[row * kDagN + pos] = prev;
        w.succ[row * kDagN + prev] = pos;
    }
}

// 3b. run links: j continues p's run when p precedes j in every row and has the same Fat slots
__global__ void __launch_bounds__(256) dag_run_kernel(DagWs w, uint32_t n, uint32_t d) {
    wait_prior_kernel();
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t p = w.pred[j];
    bool cont = p != kDagNone && !w.bad[j] && !w.bad[p];
    for (uint32_t i = 0; cont && i < d; ++i)
        cont = w.pred[i * kDagN + j] == p && w.fb[i * kDagN + j] == w.fb[i * kDagN + p];
    w.par0[j] = cont ? p : j;
}

// 3c. run heads.  A run occupies consecutive entries of row 0's bucket order (each member's
//     row-0 predecessor is the member before it), so an update's head is the last entry, at or
//     before it in that order, that starts a run: a prefix maximum of the starting entries'
//     indices, per tile (dag_headtile_kernel) and then with the maximum of the earlier tiles
//     (dag_head_kernel), which also counts every run's length and records its last member.
__device__ __forceinline__ uint32_t block_max_scan(uint32_t v, uint32_t* s_w) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (uint32_t off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, v, off);
        if (lane >= off) v = max(v, y);
    }
    if (lane == 31) s_w[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t x = s_w[lane];
#pragma unroll
        for (uint32_t off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x = max(x, y);
        }
        s_w[lane] = x;
    }
    __syncthreads();
    return warp > 0 ? max(v, s_w[warp - 1]) : v;
}

// 1 + the sorted index of the entry, if it starts a run, else 0
__device__ __forceinline__ uint32_t run_start_mark(const uint32_t* __restrict__ sv0, const uint32_t* __restrict__ par,
                                                   uint32_t q, uint32_t n) {
    if (q >= n) return 0u;
    const uint32_t pos = sv0[q];
    return par[pos] == pos ? q + 1u : 0u;
}

__global__ void __launch_bounds__(kDagTile) dag_headtile_kernel(const uint32_t* __restrict__ sv0,
                                                                const uint32_t* __restrict__ par, uint32_t n,
                                                                uint32_t* __restrict__ agg) {
    wait_prior_kernel();
    __shared__ uint32_t s_w[32];
    const uint32_t v = block_max_scan(run_start_mark(sv0, par, blockIdx.x * kDagTile + threadIdx.x, n), s_w);
    if (threadIdx.x == kDagTile - 1) agg[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kDagTile) dag_head_kernel(const uint32_t* __restrict__ sv0,
                                                            const uint32_t* __restrict__ par, uint32_t n,
                                                            const uint32_t* __restrict__ agg,
                                                            uint32_t* __restrict__ head, uint32_t* __restrict__ rlen,
                                                            uint32_t* __restrict__ lastm) {
    wait_prior_kernel();
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_carry;
    if (threadIdx.x < 32) {
        uint32_t c = 0;
        for (uint32_t t = threadIdx.x; t < blockIdx.x; t += 32) c = max(c, agg[t]);
#pragma unroll
        for (uint32_t off = 16; off > 0; off >>= 1) c = max(c, __shfl_xor_sync(0xFFFFFFFFu, c, off));
        if (threadIdx.x == 0) s_carry = c;
    }
    const uint32_t q = blockIdx.x * kDagTile + threadIdx.x;
    uint32_t v = block_max_scan(run_start_mark(sv0, par, q, n), s_w);  // its barriers also publish s_carry
    v = max(v, s_carry);
    if (q < n) {
        const uint32_t pos = sv0[q], hd = sv0[v - 1u];  // v >= 1: entry 0 of a row always starts a run
        head[pos] = hd;
        // the run's length and last member, at its head
        atomicAdd(&rlen[hd], 1u);
        atomicMax(&lastm[hd], pos);
    }
}

// 4a. counts: in a row sorted by counter (stable, so stream order within a counter), the update at
//     sorted index q is the (q - first + 1)-th of the piece on its counter, where first is the
//     counter's first sorted index (a binary search over the sorted keys)
__global__ void __launch_bounds__(256) dag_rank_kernel(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv,
                                                       uint32_t* __restrict__ cnt, uint32_t n) {
    wait_prior_kernel();
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y;
    if (q >= n) return;
    const uint32_t* k = sk + row * kDagN;
    const uint32_t key = k[q];
    uint32_t lo = 0, hi = q;  // the first index in [lo, hi] whose key equals key
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (k[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    cnt[row * kDagN + sv[row * kDagN + q]] = q - lo + 1u;
}

// 4b. the piece's Fat increments, one atomic per counter: the last update of a counter in sorted
//     order adds the counter's count
__global__ void __launch_bounds__(256) dag_fatadd_kernel(SketchDesc s, const uint32_t* __restrict__ sk,
                                                         const uint32_t* __restrict__ sv,
                                                         const uint32_t* __restrict__ cnt, uint32_t n, uint32_t wz) {
    wait_prior_kernel();
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x, row = blockIdx.y;
    if (q >= n) return;
    const uint32_t* k = sk + row * kDagN;
    const uint32_t key = k[q];
    if (key >= wz || (q + 1 < n && k[q + 1] == key)) return;
    atomicAdd(s.B + (uint64_t)row * wz + key, cnt[row * kDagN + sv[row * kDagN + q]]);
}

// 4c. pending predecessors of every head (one per row that has one), and its successors: the
//     next update, in each row's bucket, after the run's last member -- always another run's
//     head, since a run member's predecessors are all inside its run.  Everything the walk needs
//     of a head goes into its record: buckets, successor heads, the run length (0 for an update
//     that does nothing) and the Fat estimate after the run, min_i (B_i + count_i of the last
//     member) with B the Fat at the start of the piece (read before dag_fatadd_kernel runs).
//     Heads without any predecessor start the walk.
__global__ void __launch_bounds__(256) dag_npred_kernel(SketchDesc s, DagWs w, const uint32_t* __restrict__ head,
                                                        uint32_t n) {
    wait_prior_kernel();
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || head[j] != j) return;
    const uint32_t d = s.d;
    const uint32_t l = w.lastm[j];
    const bool ok = !w.bad[j];
    uint32_t c = 0, F = 0xFFFFFFFFu, hb[kMaxD], sx[kMaxD];
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
        hb[i] = 0u;
        sx[i] = kDagNone;
        if (i < (int)d) {
            c += w.pred[i * kDagN + j] != kDagNone ? 1u : 0u;
            hb[i] = w.hb[i * kDagN + j];
            sx[i] = w.succ[i * kDagN + l];
            if (ok) {
                const uint32_t b0 = __ldcg(s.B + ((uint64_t)i * s.w + hb[i]) * s.z + w.fb[i * kDagN + j]);
                F = min(F, b0 + w.cnt[i * kDagN + l]);
            }
        }
    }
    const uint32_t G = dag_groups(d), rl = ok ? w.rlen[j] : 0u;
    uint4* r = w.rec + 4ull * G * j;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i)
        if (i < (int)d) r[i] = make_uint4(hb[i], sx[i], rl, F);
    if (c != 0) atomicOr(&w.npred[j >> 3], c << (4u * (j & 7u)));
    else w.q0[atomicAdd(&w.qcount[0], 1u)] = j;
}

// 5. the graph walk, one block, level by level.  A head is taken by P = 1, 2, 4 or 8 lanes
//    (the power of two >= d), lane i for row i: it reads its row's 16 bytes of the head's
//    record, its Slim counter and its successor's pending count, and the lanes of a head
//    combine their Slim minimum with shuffles, so a head costs a few instructions per lane and
//    a warp's record loads touch one cache line per head.  Shared memory holds the
//    pending counts (four bits per update of the piece: at most d <= 8 each), the frontier
//    queues up to qcap heads (the rest in the global queues) and, with kSmemSlim, the Slim;
//    it stays small enough to leave the L1 room for the successors' record chunks, which each
//    lane copies towards the L1 while their predecessors run.
constexpr int kDagWalkThreads = 1024;

// Words of the pending-count nibbles of n updates, rounded to whole uint4 (the Slim after them
// stays 16-byte aligned).
__host__ __device__ inline uint32_t walk_np_words(uint32_t n) { return ((n + 7u) / 8u + 3u) & ~3u; }
static_assert(kMaxD <= 15, "a pending count fits four bits");

// Warms the L1 with the 16-byte chunk at p: an asynchronous copy into this thread's scratch
// slot in shared memory, cached at every level on the way (cp.async.ca).  Nothing reads the
// slot; the L1 line is what the next level's load of the chunk hits.  (prefetch.global.L1 and
// ld.global.ca loads measured no faster than no prefetch at all; this copy took C1 from 0.449 to
// 0.414 ms.)  The kernel waits for its copies before it returns.
__device__ __forceinline__ void warm_l1(uint4* slot, const uint4* p) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(slot)), "l"(p)
                 : "memory");
}

template <int D>
struct WalkLanes {
    static constexpr int P = D <= 1 ? 1 : D <= 2 ? 2 : D <= 4 ? 4 : 8;
    static constexpr int G = D <= 4 ? 1 : 2;  // uint4 groups of buckets (and of successors)
};

template <int D, bool kSmemSlim>
__global__ void __launch_bounds__(kDagWalkThreads, 1) dag_walk_kernel(SketchDesc s, DagWs w, uint32_t n,
                                                                      uint32_t qcap, uint32_t* ctrl) {
    wait_prior_kernel();
    constexpr int P = WalkLanes<D>::P, G = WalkLanes<D>::G;
    constexpr uint32_t kHeadsPerIter = kDagWalkThreads / P;
    extern __shared__ __align__(16) uint32_t s_dyn[];  // read and written as uint4 as well
    __shared__ uint32_t s_next[3];
    __shared__ uint4 s_warm[kDagWalkThreads];  // destinations of the L1-warming copies
    // dynamic shared memory: queues [2][qcap], pending-count nibbles, then the Slim (both copied
    // in with 16-byte loads)
    uint32_t* s_q = s_dyn;
    uint32_t* s_np = s_q + 2ull * qcap;
    const uint32_t np_words = walk_np_words(n);
    uint32_t* sA = s_np + np_words;
    const uint64_t slim_n = (uint64_t)D * s.w;
    {
        const uint4* src = reinterpret_cast<const uint4*>(w.npred);
        uint4* dst = reinterpret_cast<uint4*>(s_np);
        for (uint32_t t = threadIdx.x; t < np_words / 4u; t += blockDim.x) dst[t] = __ldcg(src + t);
    }
    if (kSmemSlim) {
        const uint4* src = reinterpret_cast<const uint4*>(s.A);
        uint4* dst = reinterpret_cast<uint4*>(sA);
        for (uint64_t t = threadIdx.x; t < slim_n / 4u; t += blockDim.x) dst[t] = __ldcg(src + t);
        for (uint64_t i = (slim_n & ~3ull) + threadIdx.x; i < slim_n; i += blockDim.x) sA[i] = __ldcg(s.A + i);
    }
    uint32_t* A = kSmemSlim ? sA : s.A;
    const uint32_t row = threadIdx.x % P;            // this lane's row (idle when >= D)
    const uint32_t slot = threadIdx.x / P;           // this lane's head within an iteration
    const bool live_row = row < (uint32_t)D;
    uint32_t ncur = __ldcg(&w.qcount[0]);
    for (uint32_t q = threadIdx.x; q < ncur && q < qcap; q += blockDim.x) s_q[q] = __ldcg(w.q0 + q);
    // Queue counters rotate over three words, so one barrier per level suffices: level L pushes
    // into s_next[L % 3], every thread reads it after the level's barrier, and thread 0 clears
    // s_next[(L + 1) % 3] during level L -- last read at the end of level L - 2, before the
    // barrier of level L - 1.
    if (threadIdx.x == 0) {
        s_next[0] = 0u;
        s_next[1] = 0u;
    }
    uint32_t cb = 0;  // which queue holds the current frontier
    __syncthreads();
    for (uint32_t step = 0; ncur > 0; ++step) {
        if (step > n) {  // a graph of n updates has at most n levels
            if (threadIdx.x == 0) atomicOr(ctrl + kCtrlErr, kErrTimeout);
            break;
        }
        const uint32_t c_now = step % 3u;
        if (threadIdx.x == 0) s_next[(step + 1u) % 3u] = 0u;
        const uint32_t nb = cb ^ 1u;
        uint32_t* gcur = cb ? w.q1 : w.q0;
        uint32_t* gnext = cb ? w.q0 : w.q1;
        // the lanes of a warp run the same iterations (the shuffles need the whole warp); a warp
        // whose first head slot is past the frontier has nothing left to do in this level
        const uint32_t warp_first_slot = (threadIdx.x & ~31u) / P;
        for (uint32_t base = 0; base + warp_first_slot < ncur; base += kHeadsPerIter) {
            const uint32_t hq = base + slot;
            const bool live = hq < ncur;
            uint32_t j = 0;
            if (live) j = hq < qcap ? s_q[(uint64_t)cb * qcap + hq] : __ldcg(gcur + hq);
            uint32_t hb = 0, sx = kDagNone, r = 0, F = 0, a = 0xFFFFFFFFu;
            if (live && live_row) {
                const uint4 c = __ldg(w.rec + 4ull * G * j + row);  // {h_i, successor, r, F}
                hb = c.x;
                sx = c.y;
                r = c.z;
                F = c.w;
            }
            if (sx != kDagNone) warm_l1(&s_warm[threadIdx.x], w.rec + 4ull * G * sx + row);
            if (live && live_row) a = A[(uint64_t)row * s.w + hb];
            uint32_t m = a;
#pragma unroll
            for (int off = 1; off < P; off <<= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
            if (live_row && r != 0u) {
                const uint64_t mr = (uint64_t)m + r;
                const uint32_t T = mr < (uint64_t)F ? (uint32_t)mr : F;
                if (a < T) A[(uint64_t)row * s.w + hb] = T;
            }
            // one pending predecessor less for this row's successor; the last one queues it, in a
            // slot reserved once per warp
            bool rel = false;
            if (sx != kDagNone) {
                const uint32_t sh = 4u * (sx & 7u);
                const uint32_t old = atomicSub(&s_np[sx >> 3], 1u << sh);
                rel = ((old >> sh) & 0xFu) == 1u;
            }
            const unsigned relb = __ballot_sync(0xFFFFFFFFu, rel);
            if (relb) {
                const uint32_t lane = threadIdx.x & 31u, leader = (uint32_t)(__ffs(relb) - 1);
                uint32_t first = 0;
                if (lane == leader) first = atomicAdd(&s_next[c_now], (uint32_t)__popc(relb));
                first = __shfl_sync(0xFFFFFFFFu, first, leader);
                if (rel) {
                    const uint32_t idx = first + (uint32_t)__popc(relb & ((1u << lane) - 1u));
                    if (idx < qcap) s_q[(uint64_t)nb * qcap + idx] = sx;
                    else gnext[idx] = sx;
                }
            }
        }
        __syncthreads();
        ncur = s_next[c_now];
        cb = nb;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (kSmemSlim) {
        __syncthreads();
        const uint4* src = reinterpret_cast<const uint4*>(sA);
        uint4* dst = reinterpret_cast<uint4*>(s.A);
        for (uint64_t t = threadIdx.x; t < slim_n / 4u; t += blockDim.x) dst[t] = src[t];
        for (uint64_t i = (slim_n & ~3ull) + threadIdx.x; i < slim_n; i += blockDim.x) s.A[i] = sA[i];
    }
}

template <int D>
static cudaError_t launch_walk_d(const SketchDesc& s, const DagWs& w, uint32_t nc, int smem_limit, uint32_t* ctrl,
                                 cudaStream_t st) {
    // dynamic shared memory: the pending-count nibbles of a full piece, queues of qcap heads per
    // frontier (up to 2,048, at least 256) and the Slim when it fits beside them
    const uint64_t np_bytes = walk_np_words(kDagN) * 4ull;
    const uint64_t slim_bytes = (uint64_t)D * s.w * 4ull;
    const uint64_t budget = (uint64_t)smem_limit - 1024ull - 16ull * kDagWalkThreads;  // static arrays, slack
    if (budget < np_bytes + 2ull * 256ull * 4ull) return cudaErrorInvalidValue;
    const bool slim_in_smem = np_bytes + slim_bytes + 2ull * 256ull * 4ull <= budget;
    uint64_t qcap = (budget - np_bytes - (slim_in_smem ? slim_bytes : 0ull)) / 8ull;
    if (qcap > 2048) qcap = 2048;
    qcap &= ~31ull;
    const size_t dyn_max = (size_t)(2ull * qcap * 4ull + np_bytes + (slim_in_smem ? slim_bytes : 0ull));
    const size_t dyn = (size_t)(2ull * qcap * 4ull + walk_np_words(nc) * 4ull + (slim_in_smem ? slim_bytes : 0ull));
    cudaError_t e;
    if (slim_in_smem) {
        e = cudaFuncSetAttribute(dag_walk_kernel<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
        if (e != cudaSuccess) return e;
        return dag_launch(dag_walk_kernel<D, true>, dim3(1), dim3(kDagWalkThreads), dyn, st, s, w, nc,
                          (uint32_t)qcap, ctrl);
    } else {
        e = cudaFuncSetAttribute(dag_walk_kernel<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
        if (e != cudaSuccess) return e;
        return dag_launch(dag_walk_kernel<D, false>, dim3(1), dim3(kDagWalkThreads), dyn, st, s, w, nc,
                          (uint32_t)qcap, ctrl);
    }
}

static cudaError_t launch_walk(const SketchDesc& s, const DagWs& w, uint32_t nc, int smem_limit, uint32_t* ctrl,
                               cudaStream_t st) {
    switch (s.d) {
        case 1: return launch_walk_d<1>(s, w, nc, smem_limit, ctrl, st);
        case 2: return launch_walk_d<2>(s, w, nc, smem_limit, ctrl, st);
        case 3: return launch_walk_d<3>(s, w, nc, smem_limit, ctrl, st);
        case 4: return launch_walk_d<4>(s, w, nc, smem_limit, ctrl, st);
        case 5: return launch_walk_d<5>(s, w, nc, smem_limit, ctrl, st);
        case 6: return launch_walk_d<6>(s, w, nc, smem_limit, ctrl, st);
        case 7: return launch_walk_d<7>(s, w, nc, smem_limit, ctrl, st);
        case 8: return launch_walk_d<8>(s, w, nc, smem_limit, ctrl, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

uint64_t dag_workspace_bytes(uint32_t d) { return dag_bytes_for(d); }

// One stable LSD radix sort of `rows` rows: keys ki, values vi (both [rows][N]), by every bit up
// to the highest of key_limit; ko, vo are the other buffers.  Returns the buffers holding the
// sorted rows.
static cudaError_t dag_sort_rows(const DagWs& w, uint32_t rows, uint32_t nc, uint64_t key_limit, uint32_t*& ki,
                                 uint32_t*& vi, uint32_t*& ko, uint32_t*& vo, cudaStream_t st) {
    const uint32_t tiles = (nc + kDagTile - 1) / kDagTile;
    for (uint32_t shift = 0; shift < 32 && (shift == 0 || (key_limit >> shift) != 0); shift += kDagRadixBits) {
        cudaError_t e = dag_launch(dag_hist_kernel, dim3(tiles, rows), dim3(256), 0, st, ki, nc, shift, w.hist);
        if (e == cudaSuccess) e = dag_launch(dag_scan_kernel, dim3(rows), dim3(1024), 0, st, w.hist);
        if (e == cudaSuccess)
            e = dag_launch(dag_scatter_kernel, dim3(tiles, rows), dim3(kDagTile), 0, st, ki, vi, ko, vo, nc, shift,
                           w.hist);
        if (e != cudaSuccess) return e;
        uint32_t* t = ki;
        ki = ko;
        ko = t;
        t = vi;
        vi = vo;
        vo = t;
    }
    return cudaSuccess;
}

cudaError_t launch_seq_dag(const SketchDesc& s, const uint8_t* keys, uint64_t n, void* ws_base, uint32_t* ctrl,
                           int smem_limit, cudaStream_t st) {
    const DagWs w = dag_carve(ws_base, s.d);
    const uint64_t wz64 = (uint64_t)s.w * s.z;
    if (s.w < kDagMinW || wz64 >= (1ull << 32)) return cudaErrorInvalidValue;
    const uint32_t wz = (uint32_t)wz64;
    cudaError_t e = cudaSuccess;
    for (uint64_t base = 0; base < n; base += kDagN) {
        const uint32_t nc = (uint32_t)(n - base < (uint64_t)kDagN ? n - base : (uint64_t)kDagN);
        const uint32_t blocks = (nc + 255) / 256;
        e = dag_launch(dag_hash_kernel, dim3(blocks), dim3(256), 0, st, s, keys + base * s.key_bytes, nc, w, ctrl);
        if (e != cudaSuccess) return e;
        // one stable sort of 2d rows: by bucket (each update's neighbours in its buckets) and by
        // Fat counter (each update's count on its counters); the spare counter key wz exists
        // only with explicit indices
        uint32_t *ki = w.sk0, *vi = w.sv0, *ko = w.sk1, *vo = w.sv1;
        e = dag_sort_rows(w, 2u * s.d, nc, s.idx_table ? (uint64_t)wz : (uint64_t)wz - 1u, ki, vi, ko, vo, st);
        if (e != cudaSuccess) return e;
        DagWs ws = w;
        ws.sk0 = ki;  // the sorted rows are in whichever buffers the last pass wrote
        ws.sv0 = vi;
        const uint32_t* kc = ki + (uint64_t)s.d * kDagN;  // rows sorted by Fat counter
        const uint32_t* vc = vi + (uint64_t)s.d * kDagN;
        const uint32_t tiles = (nc + kDagTile - 1) / kDagTile;
        const uint32_t* pa = w.par1;  // the head of every update
        e = dag_launch(dag_adj_kernel, dim3(blocks, s.d), dim3(256), 0, st, ws, nc);
        if (e == cudaSuccess) e = dag_launch(dag_run_kernel, dim3(blocks), dim3(256), 0, st, ws, nc, s.d);
        if (e == cudaSuccess)
            e = dag_launch(dag_headtile_kernel, dim3(tiles), dim3(kDagTile), 0, st, ws.sv0, w.par0, nc, w.hist);
        if (e == cudaSuccess)
            e = dag_launch(dag_head_kernel, dim3(tiles), dim3(kDagTile), 0, st, ws.sv0, w.par0, nc, w.hist, w.par1,
                           w.rlen, w.lastm);
        if (e == cudaSuccess) e = dag_launch(dag_rank_kernel, dim3(blocks, s.d), dim3(256), 0, st, kc, vc, w.cnt, nc);
        if (e == cudaSuccess) e = dag_launch(dag_npred_kernel, dim3(blocks), dim3(256), 0, st, s, ws, pa, nc);
        if (e == cudaSuccess)
            e = dag_launch(dag_fatadd_kernel, dim3(blocks, s.d), dim3(256), 0, st, s, kc, vc, w.cnt, nc, wz);
        if (e != cudaSuccess) return e;
        e = launch_walk(s, ws, nc, smem_limit, ctrl, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sfk
