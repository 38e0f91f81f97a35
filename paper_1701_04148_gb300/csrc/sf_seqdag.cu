// sf_seqdag.cu -- the S = 1 insertion path as a dependency graph over the whole stream (sm_103a).
//
// The paper's one-at-a-time insertion (Sec. 3.4, kept by SF_F in Sec. 3.5) makes an update
// depend on an earlier one only when the two share a bucket (i, h_i) in some row: every counter
// either touches -- Slim A_i[h_i], Fat B_i[h_i][.] -- lies in its d buckets.  So any order that
// keeps, in every bucket, the stream order of the updates hashed to it gives the stream-order
// result.  For a call of insertions only, taken in pieces of up to kDagN updates:
//   1. hash every update (parallel);
//   2. per row, a stable radix sort of (bucket, position) gives every update its predecessor and
//      successor in each of its buckets (the neighbouring entries of the sorted row);
//   3. runs (Lemma 2): an update whose predecessor in every row is the same earlier update with
//      the same Fat slots continues that update's run; pointer jumping finds each run's first
//      update (its head), which counts the run's length r and records its last member;
//   4. a run can go once, in every row, the run before it in that bucket has gone: heads count
//      their pending predecessors, and one block walks the graph frontier by frontier.  A run
//      adds r to its d Fat counters with returning atomics: every earlier update on those
//      counters has run and no later one can have, so the returned value plus r is the counter
//      after the run, and F is their minimum; T = min(m + r, F) with m the minimum of its Slim
//      counters, which rise to T where lower.  Runs of one frontier share no bucket, so they
//      touch disjoint counters.
// A piece's graph is only as deep as its longest chain of runs through shared buckets.
#include "sf_internal.h"

namespace sfk {

namespace {

constexpr uint32_t kDagNone = 0xFFFFFFFFu;
constexpr int kDagTile = 1024;           // elements per radix tile (one block)
constexpr int kDagTiles = kDagN / kDagTile;
constexpr int kDagRadixBits = 8;
constexpr int kDagBins = 1 << kDagRadixBits;
constexpr int kDagExecThreads = 1024;

// Workspace arrays of one piece (kDagN updates, d rows), carved out of the sketch scratch.
struct DagWs {
    uint4* rec;                   // [N][4G] walk record of every run head (dag_npred_kernel)
    uint32_t *hb, *fb;            // [d][N] bucket and slot of every update
    uint32_t *sk0, *sv0, *sk1, *sv1;  // [d][N] radix sort keys (buckets) and values (positions)
    uint32_t *pred, *succ;        // [d][N] previous / next update in the same bucket
    uint32_t *par0, *par1;        // [N] run parent links (pointer jumping)
    uint32_t *rlen, *lastm;       // [N] run length and last member, at heads
    uint32_t *npred;              // [N] pending predecessors, at heads
    uint32_t *bad;                // [N] the key had no valid index (explicit-index mode)
    uint32_t *q0, *q1;            // [N] frontier queues
    uint32_t *qcount;             // [4] queue counters
    uint32_t *hist;               // [d][bins][tiles] digit counts, then offsets
};

// A walk record holds G = ceil(d / 4) uint4 groups each of buckets, Fat slots and successor
// heads, then the run length: 4G uint4 (64 bytes for d <= 4, 128 for d <= 8).
__host__ __device__ inline uint32_t dag_groups(uint32_t d) { return d <= 4 ? 1u : 2u; }

__host__ __device__ inline uint64_t dag_bytes_for(uint32_t d) {
    const uint64_t N = kDagN;
    return (16ull * dag_groups(d) * N + 8ull * d * N + 8ull * N + 64ull + (uint64_t)d * kDagBins * kDagTiles) * 4ull;
}

DagWs dag_carve(void* base, uint32_t d) {
    uint32_t* p = static_cast<uint32_t*>(base);
    const uint64_t N = kDagN;
    DagWs w;
    w.rec = reinterpret_cast<uint4*>(p);
    p += 16 * dag_groups(d) * N;
    w.hb = p;
    p += d * N;
    w.fb = p;
    p += d * N;
    w.sk0 = p;
    p += d * N;
    w.sv0 = p;
    p += d * N;
    w.sk1 = p;
    p += d * N;
    w.sv1 = p;
    p += d * N;
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
    for (uint32_t i = 0; i < s.d; ++i) {
        w.hb[i * kDagN + j] = h[i];
        w.fb[i * kDagN + j] = f[i];
        w.sk0[i * kDagN + j] = h[i];
        w.sv0[i * kDagN + j] = j;
        w.pred[i * kDagN + j] = kDagNone;
        w.succ[i * kDagN + j] = kDagNone;
    }
    w.rlen[j] = 0u;
    w.lastm[j] = 0u;
    w.npred[j] = 0u;
    w.bad[j] = ok ? 0u : 1u;
}

// 2a. digit counts of one tile of one row
__global__ void __launch_bounds__(256) dag_hist_kernel(const uint32_t* __restrict__ keys, uint32_t n, uint32_t shift,
                                                       uint32_t* __restrict__ hist) {
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
}

// 2b. per row, exclusive scan of the counts in (digit, tile) order: the first output index of
//     each tile's elements of each digit
__global__ void __launch_bounds__(1024) dag_scan_kernel(uint32_t* __restrict__ hist) {
    constexpr uint32_t kLen = kDagBins * kDagTiles;
    constexpr uint32_t kPer = kLen / 1024;
    __shared__ uint32_t part[1024];
    uint32_t* h = hist + (uint64_t)blockIdx.x * kLen;
    const uint32_t t = threadIdx.x;
    uint32_t sum = 0;
    for (uint32_t q = 0; q < kPer; ++q) sum += h[t * kPer + q];
    part[t] = sum;
    __syncthreads();
    for (uint32_t off = 1; off < 1024; off <<= 1) {  // inclusive scan of the parts
        const uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - sum;  // exclusive prefix of this thread's part
    for (uint32_t q = 0; q < kPer; ++q) {
        const uint32_t c = h[t * kPer + q];
        h[t * kPer + q] = run;
        run += c;
    }
}

// 2c. stable scatter of one tile of one row: warps in order, equal digits ranked by lane
__global__ void __launch_bounds__(kDagTile) dag_scatter_kernel(const uint32_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint32_t* __restrict__ kout,
                                                               uint32_t* __restrict__ vout, uint32_t n,
                                                               uint32_t shift, const uint32_t* __restrict__ hist) {
    __shared__ uint32_t next[kDagBins];
    const uint32_t tile = blockIdx.x, row = blockIdx.y;
    for (uint32_t b = threadIdx.x; b < kDagBins; b += blockDim.x)
        next[b] = hist[((uint64_t)row * kDagBins + b) * kDagTiles + tile];
    const uint32_t e = tile * kDagTile + threadIdx.x;
    const bool valid = e < n;
    const uint32_t key = valid ? kin[row * kDagN + e] : 0u;
    const uint32_t val = valid ? vin[row * kDagN + e] : 0u;
    const uint32_t dig = (key >> shift) & (kDagBins - 1);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    __syncthreads();
    for (uint32_t wv = 0; wv < kDagTile / 32; ++wv) {
        if (warp == wv) {
            const unsigned act = __ballot_sync(0xFFFFFFFFu, valid);
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, valid ? dig : 0x80000000u | lane) & act;
            if (valid) {
                const uint32_t rank = (uint32_t)__popc(peers & ((1u << lane) - 1u));
                const uint32_t dst = next[dig] + rank;
                kout[row * kDagN + dst] = key;
                vout[row * kDagN + dst] = val;
            }
            __syncwarp();
            if (valid && lane == (uint32_t)(31 - __clz(peers))) next[dig] += (uint32_t)__popc(peers);
        }
        __syncthreads();
    }
}

// 3a. neighbours in bucket order: sorted entries k-1 and k of a row with the same bucket
__global__ void __launch_bounds__(256) dag_adj_kernel(DagWs w, uint32_t n) {
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
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t p = w.pred[j];
    bool cont = p != kDagNone && !w.bad[j] && !w.bad[p];
    for (uint32_t i = 0; cont && i < d; ++i)
        cont = w.pred[i * kDagN + j] == p && w.fb[i * kDagN + j] == w.fb[i * kDagN + p];
    w.par0[j] = cont ? p : j;
}

__global__ void __launch_bounds__(256) dag_jump_kernel(const uint32_t* __restrict__ a, uint32_t* __restrict__ b,
                                                       uint32_t n) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) b[j] = a[a[j]];
}

// 3c. run lengths and last members, at heads
__global__ void __launch_bounds__(256) dag_count_kernel(DagWs w, const uint32_t* __restrict__ head, uint32_t n) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t hd = head[j];
    atomicAdd(&w.rlen[hd], 1u);
    atomicMax(&w.lastm[hd], j);
}

// 3d. pending predecessors of every head (one per row that has one), and its successors: the
//     next update, in each row's bucket, after the run's last member -- always another run's
//     head, since a run member's predecessors are all inside its run.  Everything the walk needs
//     of a head goes into its 64-byte record: buckets, Fat slots, successor heads, and the run
//     length (0 for an update that does nothing).  Heads without any predecessor start the walk.
__global__ void __launch_bounds__(256) dag_npred_kernel(DagWs w, const uint32_t* __restrict__ head, uint32_t n,
                                                        uint32_t d) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || head[j] != j) return;
    const uint32_t l = w.lastm[j];
    uint32_t c = 0, hb[kMaxD], fb[kMaxD], sx[kMaxD];
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
        hb[i] = fb[i] = 0u;
        sx[i] = kDagNone;
        if (i < (int)d) {
            c += w.pred[i * kDagN + j] != kDagNone ? 1u : 0u;
            hb[i] = w.hb[i * kDagN + j];
            fb[i] = w.fb[i * kDagN + j];
            sx[i] = w.succ[i * kDagN + l];
        }
    }
    const uint32_t G = dag_groups(d);
    uint4* r = w.rec + 4ull * G * j;
#pragma unroll
    for (uint32_t g = 0; g < 2; ++g) {
        if (g < G) {
            r[g] = make_uint4(hb[4 * g], hb[4 * g + 1], hb[4 * g + 2], hb[4 * g + 3]);
            r[G + g] = make_uint4(fb[4 * g], fb[4 * g + 1], fb[4 * g + 2], fb[4 * g + 3]);
            r[2 * G + g] = make_uint4(sx[4 * g], sx[4 * g + 1], sx[4 * g + 2], sx[4 * g + 3]);
        }
    }
    r[3 * G] = make_uint4(w.bad[j] ? 0u : w.rlen[j], 0u, 0u, 0u);
    w.npred[j] = c;
    if (c == 0) w.q0[atomicAdd(&w.qcount[0], 1u)] = j;
}

// 4. the graph walk, one block; the Slim in shared memory (kSmemSlim) or in place.  The frontier
//    queues live in shared memory up to kDagQCap entries, the rest in the global queues.  A
//    level's cost is its longest chain of dependent memory round trips, so each head's record
//    comes in four vector loads, and while a head's atomics are in flight the records of its
//    successors are prefetched into L1 for the next level.
constexpr uint32_t kDagQCap = 4096;

__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

template <bool kSmemSlim>
__global__ void __launch_bounds__(kDagExecThreads, 1) dag_exec_kernel(SketchDesc s, DagWs w, uint32_t n,
                                                                      uint32_t* ctrl) {
    extern __shared__ uint32_t sA[];
    __shared__ uint32_t s_q[2][kDagQCap];
    __shared__ uint32_t s_next;
    const uint64_t slim_n = (uint64_t)s.d * s.w;
    if (kSmemSlim) {
        for (uint64_t i = threadIdx.x; i < slim_n; i += blockDim.x) sA[i] = __ldcg(s.A + i);
    }
    uint32_t* A = kSmemSlim ? sA : s.A;
    const uint32_t G = dag_groups(s.d);
    uint32_t ncur = __ldcg(&w.qcount[0]);
    for (uint32_t q = threadIdx.x; q < ncur && q < kDagQCap; q += blockDim.x) s_q[0][q] = __ldcg(w.q0 + q);
    uint32_t cb = 0;  // which queue holds the current frontier
    __syncthreads();
    for (uint32_t step = 0; ncur > 0; ++step) {
        if (step > n) {  // a graph of n updates has at most n levels
            if (threadIdx.x == 0) atomicOr(ctrl + kCtrlErr, kErrTimeout);
            break;
        }
        if (threadIdx.x == 0) s_next = 0u;
        __syncthreads();
        const uint32_t nb = cb ^ 1u;
        uint32_t* gcur = cb ? w.q1 : w.q0;
        uint32_t* gnext = cb ? w.q0 : w.q1;
        for (uint32_t q = threadIdx.x; q < ncur; q += blockDim.x) {
            const uint32_t j = q < kDagQCap ? s_q[cb][q] : __ldcg(gcur + q);
            const uint4* rj = w.rec + 4ull * G * j;
            uint32_t hb[kMaxD], fb[kMaxD], sx[kMaxD];
#pragma unroll
            for (uint32_t g = 0; g < 2; ++g) {
                uint4 h4 = make_uint4(0u, 0u, 0u, 0u), f4 = h4, x4 = make_uint4(kDagNone, kDagNone, kDagNone, kDagNone);
                if (g < G) {
                    h4 = __ldg(rj + g);
                    f4 = __ldg(rj + G + g);
                    x4 = __ldg(rj + 2 * G + g);
                }
                hb[4 * g] = h4.x, hb[4 * g + 1] = h4.y, hb[4 * g + 2] = h4.z, hb[4 * g + 3] = h4.w;
                fb[4 * g] = f4.x, fb[4 * g + 1] = f4.y, fb[4 * g + 2] = f4.z, fb[4 * g + 3] = f4.w;
                sx[4 * g] = x4.x, sx[4 * g + 1] = x4.y, sx[4 * g + 2] = x4.z, sx[4 * g + 3] = x4.w;
            }
            const uint32_t r = __ldg(&rj[3 * G].x);
            // the run's Fat increments and its successors' pending counts, all in flight together
            // (every return value is collected before any is used)
            uint32_t old_v[kMaxD], left[kMaxD];
#pragma unroll
            for (int i = 0; i < kMaxD; ++i) {
                old_v[i] = 0u;
                left[i] = 0xFFFFFFFFu;
                if (i < (int)s.d) {
                    if (r != 0u) old_v[i] = atomicAdd(s.B + ((uint64_t)i * s.w + hb[i]) * s.z + fb[i], r);
                    if (sx[i] != kDagNone) left[i] = atomicSub(&w.npred[sx[i]], 1u);
                }
            }
#pragma unroll
            for (int i = 0; i < kMaxD; ++i)
                if (i < (int)s.d && sx[i] != kDagNone) prefetch_l1(w.rec + 4ull * G * sx[i]);
            if (r != 0u) {
                uint32_t F = 0xFFFFFFFFu, m = 0xFFFFFFFFu, a[kMaxD];
#pragma unroll
                for (int i = 0; i < kMaxD; ++i) {
                    a[i] = 0u;
                    if (i < (int)s.d) {
                        a[i] = A[(uint64_t)i * s.w + hb[i]];
                        m = min(m, a[i]);
                    }
                }
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d) F = min(F, old_v[i] + r);
                const uint64_t mr = (uint64_t)m + r;
                const uint32_t T = mr < (uint64_t)F ? (uint32_t)mr : F;
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d && a[i] < T) A[(uint64_t)i * s.w + hb[i]] = T;
            }
#pragma unroll
            for (int i = 0; i < kMaxD; ++i) {
                if (i < (int)s.d && left[i] == 1u) {  // the last pending predecessor of that head
                    const uint32_t idx = atomicAdd(&s_next, 1u);
                    if (idx < kDagQCap) s_q[nb][idx] = sx[i];
                    else gnext[idx] = sx[i];
                }
            }
        }
        __syncthreads();
        ncur = s_next;
        cb = nb;
        __syncthreads();
    }
    if (kSmemSlim) {
        __syncthreads();
        for (uint64_t i = threadIdx.x; i < slim_n; i += blockDim.x) s.A[i] = sA[i];
    }
}

}  // namespace

uint64_t dag_workspace_bytes(uint32_t d) { return dag_bytes_for(d); }

cudaError_t launch_seq_dag(const SketchDesc& s, const uint8_t* keys, uint64_t n, void* ws_base, uint32_t* ctrl,
                           int smem_limit, cudaStream_t st) {
    const DagWs w = dag_carve(ws_base, s.d);
    const uint64_t slim_bytes = (uint64_t)s.d * s.w * 4ull;
    const bool slim_in_smem = slim_bytes + 2 * kDagQCap * 4 + 1024 <= (uint64_t)smem_limit;
    if (slim_in_smem) {
        cudaError_t e = cudaFuncSetAttribute(dag_exec_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)slim_bytes);
        if (e != cudaSuccess) return e;
    }
    for (uint64_t base = 0; base < n; base += kDagN) {
        const uint32_t nc = (uint32_t)(n - base < (uint64_t)kDagN ? n - base : (uint64_t)kDagN);
        const uint32_t blocks = (nc + 255) / 256;
        const uint32_t tiles = (nc + kDagTile - 1) / kDagTile;
        dag_hash_kernel<<<blocks, 256, 0, st>>>(s, keys + base * s.key_bytes, nc, w, ctrl);
        // stable LSD radix sort of every row by bucket
        uint32_t *ki = w.sk0, *vi = w.sv0, *ko = w.sk1, *vo = w.sv1;
        for (uint32_t shift = 0; shift < 32 && (shift == 0 || ((s.w - 1) >> shift) != 0); shift += kDagRadixBits) {
            cudaError_t e = cudaMemsetAsync(w.hist, 0, (uint64_t)s.d * kDagBins * kDagTiles * 4ull, st);
            if (e != cudaSuccess) return e;
            dag_hist_kernel<<<dim3(tiles, s.d), 256, 0, st>>>(ki, nc, shift, w.hist);
            dag_scan_kernel<<<s.d, 1024, 0, st>>>(w.hist);
            dag_scatter_kernel<<<dim3(tiles, s.d), kDagTile, 0, st>>>(ki, vi, ko, vo, nc, shift, w.hist);
            uint32_t* t = ki;
            ki = ko;
            ko = t;
            t = vi;
            vi = vo;
            vo = t;
        }
        DagWs ws = w;
        ws.sk0 = ki;  // the sorted row is in whichever buffer the last pass wrote
        ws.sv0 = vi;
        dag_adj_kernel<<<dim3(blocks, s.d), 256, 0, st>>>(ws, nc);
        dag_run_kernel<<<blocks, 256, 0, st>>>(ws, nc, s.d);
        uint32_t *pa = w.par0, *pb = w.par1;
        for (uint32_t span = 1; span < nc; span <<= 1) {
            dag_jump_kernel<<<blocks, 256, 0, st>>>(pa, pb, nc);
            uint32_t* t = pa;
            pa = pb;
            pb = t;
        }
        dag_count_kernel<<<blocks, 256, 0, st>>>(ws, pa, nc);
        cudaError_t e = cudaMemsetAsync(w.qcount, 0, 16, st);
        if (e != cudaSuccess) return e;
        dag_npred_kernel<<<blocks, 256, 0, st>>>(ws, pa, nc, s.d);
        if (slim_in_smem)
            dag_exec_kernel<true><<<1, kDagExecThreads, (size_t)slim_bytes, st>>>(s, ws, nc, ctrl);
        else
            dag_exec_kernel<false><<<1, kDagExecThreads, 0, st>>>(s, ws, nc, ctrl);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sfk
