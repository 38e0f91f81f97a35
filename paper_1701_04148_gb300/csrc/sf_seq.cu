// sf_seq.cu -- the S = 1 update kernel (sm_103a): the paper's one-at-a-time rule.
//
// Paper rules (Yang et al., SF-sketch):
//   insertion (Sec. 3.4, kept by SF_F in Sec. 3.5): B_i[h_i][f_i] += 1 for every row; with
//     Bmin the minimum of those d counters after the increment and m = min_i A_i[h_i], every
//     A_l[h_l] equal to m is incremented when m < Bmin.
//   deletion (Sec. 3.5): B_i[h_i][f_i] -= 1; A_i[h_i] is lowered to max_k B_i[h_i][k] when
//     larger.
#include "sf_internal.h"

namespace sfk {

namespace {

// S = 1: the paper's one-at-a-time rule, exactly.  One warp takes 32 consecutive updates per
// window; an update depends on an earlier one only if they share a bucket (i, h_i) in some row
// (Slim counter (i, j) and Fat bucket (i, j) go together).  In each step every pending update with
// no pending earlier dependency runs in parallel -- updates on disjoint counters commute, so the
// result equals stream order.
//
// A window without deletions needs no Fat access inside its steps: the Fat counters only grow, so
// the value lane j's insertion leaves in B_i[h_i][f_i] is the counter's value before the window
// plus the number of insertions of lanes <= j on that counter.  One increment per distinct counter
// (by its lowest lane, with the group's count) returns the value before the window, match_any
// gives each lane its rank, and the steps touch only the Slim.  The next window's increments are
// issued once the current window's have returned and run while the current window's steps do;
// keys are fetched two windows ahead.
//
// A window holding a deletion runs its Fat updates inside its steps.  There, inserts run as r
// copies of one key at once: an insert of a key e with r >= 1 copies makes the Fat counters
// B_i[h_i][f_i] += r, and then raises every Slim counter of e to T = min(m0 + r, F), where m0 is
// the smallest of e's Slim counters before and F the smallest of its Fat counters after.  For
// r = 1 this is the paper's rule (the minimal counters rise by one when below F).  For r > 1 it is
// the paper's rule applied r times in a row: the minimal counters rise by one per insertion, in
// lockstep, while they stay below the Fat estimate, which itself grows by one per insertion.  So a
// run of same-key insertions with no other update of its buckets in between collapses into one.

// Key and operation of one lane of a window.
struct SeqRaw {
    int op;
    Key k;
};

// Ring of windows whose keys and operation bytes are being copied into shared memory ahead of use
// (cp.async, so no register waits on the copy): 32 keys of up to 15 bytes span at most 31
// 16-byte granules, 32 operation bytes at most 3.
constexpr int kSeqRing = 4;
constexpr int kSeqKeyGran = 32;
constexpr int kSeqOpGran = 3;

__device__ __forceinline__ void cp_async_bytes(void* dst_smem, const void* src, int bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
    if (bytes == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Copies bytes [off, off + len) of buffer base[0 .. total) into dst as whole 16-byte granules
// (dst[0] holds the byte at the granule boundary at or below base + off).  A granule that reaches
// past either end of the buffer is copied byte by byte, so nothing outside the buffer is read.
__device__ __forceinline__ void stage_granules(const uint8_t* base, uint64_t total, uint64_t off, uint64_t len,
                                               uint32_t lane, uint8_t* dst) {
    const uintptr_t addr = reinterpret_cast<uintptr_t>(base);
    const uint8_t* al = reinterpret_cast<const uint8_t*>(addr & ~(uintptr_t)15);
    const uint64_t lo = addr & 15u, hi = lo + total;  // valid bytes, relative to al
    const uint64_t b0 = lo + off, g0 = b0 & ~15ull;
    const uint32_t ngran = (uint32_t)((b0 + len - g0 + 15) >> 4);
    if (lane < ngran) {
        const uint64_t gb = g0 + 16ull * lane;
        if (gb >= lo && gb + 16 <= hi) {
            cp_async_bytes(dst + 16 * lane, al + gb, 16);
        } else {
            for (uint32_t q = 0; q < 16; ++q)
                if (gb + q >= lo && gb + q < hi) dst[16 * lane + q] = __ldg(al + gb + q);
        }
    }
}

// Starts copying window t0's keys and operation bytes into one ring slot; always commits one
// copy group (possibly empty), so the consumer can count groups.
__device__ __forceinline__ void seq_stage(const SeqArgs& a, uint64_t t0, uint32_t lane, uint8_t* kslot,
                                          uint8_t* oslot) {
    if (t0 < a.n) {
        const uint32_t nvalid = a.n - t0 < 32 ? (uint32_t)(a.n - t0) : 32u;
        const uint32_t kb = a.s.key_bytes;
        if (kb == 4 || kb == 8) {  // keys aligned to their width
            if (lane < nvalid) cp_async_bytes(kslot + lane * kb, a.keys + (t0 + lane) * kb, (int)kb);
        } else {
            stage_granules(a.keys, a.n * kb, t0 * kb, (uint64_t)nvalid * kb, lane, kslot);
        }
        if (a.ops) stage_granules(reinterpret_cast<const uint8_t*>(a.ops), a.n, t0, nvalid, lane, oslot);
    }
    cp_async_commit();
}

// Key and operation of this lane of window t0 from its (completed) ring slot.
__device__ __forceinline__ SeqRaw seq_read(const SeqArgs& a, uint64_t t0, uint32_t lane, const uint8_t* kslot,
                                           const uint8_t* oslot) {
    SeqRaw r{0, Key{0ull, 0ull}};
    const uint64_t t = t0 + lane;
    if (t < a.n) {
        if (a.ops) {
            const uint64_t lo = reinterpret_cast<uintptr_t>(a.ops) & 15u;
            r.op = (int)(int8_t)oslot[((lo + t0) & 15u) + lane];
        } else {
            r.op = a.op_const;
        }
        if (r.op != 0) {
            const uint32_t kb = a.s.key_bytes;
            const uint8_t* sb;
            if (kb == 4 || kb == 8) {
                sb = kslot + lane * kb;
            } else {
                const uint64_t lo = reinterpret_cast<uintptr_t>(a.keys) & 15u;
                sb = kslot + ((lo + t0 * kb) & 15u) + (uint64_t)lane * kb;
            }
            const uint32_t n0 = kb < 8 ? kb : 8;
            for (uint32_t b = 0; b < n0; ++b) r.k.x0 |= (uint64_t)sb[b] << (8 * b);
            for (uint32_t b = 8; b < kb; ++b) r.k.x1 |= (uint64_t)sb[b] << (8 * (b - 8));
        }
    }
    return r;
}

// One window of up to 32 consecutive updates, one per lane.
struct SeqWin {
    int op;
    Key k;
    uint32_t h[kMaxD], f[kMaxD];
    uint32_t lr[kMaxD];   // windows without deletions: leader lane of this lane's Fat counter of row i | rank << 8
    uint32_t old[kMaxD];  // leader lanes: that counter's value before the window
    bool ins_only;        // the window holds no deletion
};

__device__ __forceinline__ void seq_prepare(const SeqArgs& a, const SeqRaw& r, uint32_t lane, SeqWin& W) {
    const SketchDesc& s = a.s;
    W.op = r.op;
    W.k = r.k;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
        W.h[i] = 0u;
        W.f[i] = 0u;
        W.lr[i] = lane;
        W.old[i] = 0u;
    }
    if (W.op != 0) {
        bool ok = true;
#pragma unroll
        for (int i = 0; i < kMaxD; ++i)
            if (i < (int)s.d) ok &= row_index(s, W.k, (uint32_t)i, &W.h[i], &W.f[i]);
        if (!ok) {
            atomicOr(a.ctrl + kCtrlErr, kErrBadKey);
            W.op = 0;
        }
    }
    W.ins_only = __all_sync(kFull, W.op >= 0);
}

// old = atomicAdd(addr, v) when p, else old unchanged, as one predicated instruction: the result
// register stays pending until it is read, instead of being merged (and waited for) right away.
__device__ __forceinline__ void atom_add_if(bool p, uint32_t* addr, uint32_t v, uint32_t& old) {
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.u32 q, %3, 0;\n\t"
        "@q atom.global.add.u32 %0, [%1], %2;\n\t}"
        : "+r"(old)
        : "l"(addr), "r"(v), "r"((uint32_t)p)
        : "memory");
}

// Window without deletions: one increment per distinct Fat counter, by the counter's lowest lane,
// whose return value stays pending until seq_fat_after.
__device__ __forceinline__ void seq_issue_fat(const SketchDesc& s, uint32_t lane, SeqWin& W) {
    const unsigned lt = (1u << lane) - 1u;
    // a row's counter index h*z + f, as 32 bits when every index of the row is below 2^31
    const bool narrow = (uint64_t)s.w * s.z <= 0x80000000ull;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
        if (i < (int)s.d) {
            uint32_t* c = fat_ptr(s, (uint32_t)i, W.h[i], W.f[i]);
            const uint64_t idx = (uint64_t)W.h[i] * s.z + W.f[i];
            // idle lanes carry values no counter index reaches, so they match nothing
            unsigned g;
            if (narrow) g = __match_any_sync(kFull, W.op > 0 ? (uint32_t)idx : 0x80000000u | lane);
            else g = __match_any_sync(kFull, W.op > 0 ? (unsigned long long)idx : ~(unsigned long long)lane);
            const uint32_t lead = (uint32_t)(__ffs(g) - 1);
            W.lr[i] = lead | ((uint32_t)__popc(g & lt) << 8);
            atom_add_if(W.op > 0 && lane == lead, c, (uint32_t)__popc(g), W.old[i]);
        }
    }
}

// Fat estimate after this lane's insertion: min over rows of (value before the window + rank + 1).
__device__ __forceinline__ uint32_t seq_fat_after(uint32_t d, const SeqWin& W) {
    uint32_t F = 0xFFFFFFFFu;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i) {
        if (i < (int)d) {
            const uint32_t o = __shfl_sync(kFull, W.old[i], W.lr[i] & 31u);
            F = min(F, o + (W.lr[i] >> 8) + 1u);
        }
    }
    return F;
}

// Lanes of the window sharing a bucket with this lane, in any row.
__device__ __forceinline__ unsigned seq_conflicts(uint32_t d, uint32_t lane, const SeqWin& W) {
    unsigned conf = 0u;
#pragma unroll
    for (int i = 0; i < kMaxD; ++i)  // one row at a time; h < w < 2^31, idle lanes take unique values above
        if (i < (int)d) conf |= __match_any_sync(kFull, W.op != 0 ? W.h[i] : 0x80000000u | lane);
    return conf;
}

// Steps of a window without deletions: the paper's insertion rule on the Slim, with F known.  The
// lanes of one step touch disjoint Slim counters, and __syncwarp orders one step's accesses before
// the next step's, so plain accesses suffice on shared memory (SlimPtr = uint32_t*); on global
// memory the accesses stay volatile (SlimPtr = volatile uint32_t*).
//
// A run of insertions of one key with no other update of its buckets in between collapses into
// its first lane (see above): r copies, F taken after the run's last insertion.
template <typename SlimPtr>
__device__ __forceinline__ void seq_slim_inserts(uint32_t d, uint32_t w, uint32_t key_bytes, SlimPtr A,
                                                 uint32_t lane, const SeqWin& W, uint32_t F, unsigned conf) {
    const unsigned dep = conf & ((1u << lane) - 1u);
    bool live = W.op > 0;
    unsigned same = __match_any_sync(kFull, W.k.x0);
    if (key_bytes > 8) same &= __match_any_sync(kFull, W.k.x1);
    const unsigned G = same & __ballot_sync(kFull, live);
    uint32_t r = 1;
    int last = (int)lane;
    if (live) {
        const int first = __ffs(G) - 1;
        last = 31 - __clz(G);
        const unsigned between = (last > first + 1) ? (((1u << last) - 1u) & ~((2u << first) - 1u)) : 0u;
        if ((conf & ~G & between) == 0u) {
            if (lane == (uint32_t)first) r = (uint32_t)__popc(G);
            else live = false;  // folded into the first insertion of the run
        } else {
            last = (int)lane;
        }
    }
    F = __shfl_sync(kFull, F, last);  // the first lane of a collapsed run takes F after the run
    unsigned pending = __ballot_sync(kFull, live);
    while (pending) {
        const bool ready = ((pending >> lane) & 1u) && (dep & pending) == 0u;
        if (ready) {
            uint32_t v[kMaxD], m = 0xFFFFFFFFu;
#pragma unroll
            for (int i = 0; i < kMaxD; ++i) {
                v[i] = i < (int)d ? A[(uint64_t)i * w + W.h[i]] : 0xFFFFFFFFu;
                m = min(m, v[i]);
            }
            const uint64_t m1 = (uint64_t)m + r;
            const uint32_t T = m1 < (uint64_t)F ? (uint32_t)m1 : F;
#pragma unroll
            for (int i = 0; i < kMaxD; ++i)
                if (i < (int)d && v[i] < T) A[(uint64_t)i * w + W.h[i]] = T;
        }
        __syncwarp();
        pending &= ~__ballot_sync(kFull, ready);
    }
}

// Steps of a window holding a deletion: Fat updates inside the steps, runs of same-key inserts
// collapsed (see above).
__device__ __forceinline__ void seq_mixed_window(const SketchDesc& s, volatile uint32_t* A, uint32_t lane,
                                                 const SeqWin& W, unsigned conf, bool* under) {
    const unsigned lt = (1u << lane) - 1u;
    int op = W.op;
    unsigned same = __match_any_sync(kFull, W.k.x0);
    if (s.key_bytes > 8) same &= __match_any_sync(kFull, W.k.x1);
    const unsigned insm = __ballot_sync(kFull, op > 0);
    uint32_t r = 1;
    if (op > 0) {
        const unsigned G = same & insm;
        const int first = __ffs(G) - 1, last = 31 - __clz(G);
        const unsigned between = (last > first + 1) ? (((1u << last) - 1u) & ~((2u << first) - 1u)) : 0u;
        if ((conf & ~G & between) == 0u) {
            if (lane == (uint32_t)first) r = (uint32_t)__popc(G);
            else op = 0;  // folded into the first insert of the run
        }
    }
    unsigned pending = __ballot_sync(kFull, op != 0);
    const unsigned dep = conf & lt;
    while (pending) {
        const bool ready = ((pending >> lane) & 1u) && (dep & pending) == 0u;
        if (ready) {
            if (op > 0) {
                uint32_t F = 0xFFFFFFFFu, m = 0xFFFFFFFFu;
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d) F = min(F, atomicAdd(fat_ptr(s, i, W.h[i], W.f[i]), r) + r);
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d) m = min(m, A[(uint64_t)i * s.w + W.h[i]]);
                const uint64_t mr = (uint64_t)m + r;
                const uint32_t T = mr < (uint64_t)F ? (uint32_t)mr : F;
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d && A[(uint64_t)i * s.w + W.h[i]] < T) A[(uint64_t)i * s.w + W.h[i]] = T;
            } else {
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d && atomicAdd(fat_ptr(s, i, W.h[i], W.f[i]), 0xFFFFFFFFu) == 0u) *under = true;
#pragma unroll
                for (int i = 0; i < kMaxD; ++i) {
                    if (i < (int)s.d) {
                        bool dummy = false;
                        const uint32_t M = bucket_bound_cg(s, i, W.h[i], W.f[i], &dummy);
                        if (A[(uint64_t)i * s.w + W.h[i]] > M) A[(uint64_t)i * s.w + W.h[i]] = M;
                    }
                }
            }
        }
        __syncwarp();
        pending &= ~__ballot_sync(kFull, ready);
    }
}

__global__ void __launch_bounds__(kSeqBlock, 1) seq_update_kernel(const SeqArgs a) {
    extern __shared__ uint32_t sA[];
    const SketchDesc& s = a.s;
    const uint64_t slim_n = (uint64_t)s.d * s.w;
    if (a.slim_in_smem) {
        for (uint64_t i = threadIdx.x; i < slim_n; i += blockDim.x) sA[i] = __ldcg(s.A + i);
        __syncthreads();
    }
    volatile uint32_t* A = a.slim_in_smem ? sA : s.A;
    __shared__ __align__(16) uint8_t s_kring[kSeqRing][kSeqKeyGran * 16];
    __shared__ __align__(16) uint8_t s_oring[kSeqRing][kSeqOpGran * 16];
    if (threadIdx.x < 32 && a.n > 0) {
        const uint32_t lane = threadIdx.x;
        bool under = false;
        SeqWin cur, nxt;
        // windows 0..2 in flight; window j uses ring slot j % kSeqRing
        for (int j = 0; j < 3; ++j) seq_stage(a, 32ull * j, lane, s_kring[j], s_oring[j]);
        cp_async_wait<2>();
        __syncwarp();
        seq_prepare(a, seq_read(a, 0, lane, s_kring[0], s_oring[0]), lane, cur);
        if (cur.ins_only) seq_issue_fat(s, lane, cur);
        for (uint64_t t0 = 0; t0 < a.n; t0 += 32) {
            const bool has_next = t0 + 32 < a.n;
            const uint32_t wi = (uint32_t)(t0 >> 5);
            const uint32_t F = cur.ins_only ? seq_fat_after(s.d, cur) : 0u;  // waits for the increments
            bool nxt_issued = false;
            if (has_next) {
                // windows up to wi + 2 are staged: wait for wi + 1, leave wi + 2 in flight
                cp_async_wait<1>();
                __syncwarp();
                const uint32_t sn = (wi + 1) % kSeqRing, sf = (wi + 3) % kSeqRing;
                seq_prepare(a, seq_read(a, t0 + 32, lane, s_kring[sn], s_oring[sn]), lane, nxt);
                // slot sf last held window wi - 1, read in an earlier iteration
                seq_stage(a, t0 + 96, lane, s_kring[sf], s_oring[sf]);
                // the current window's increments have returned, so the next window's follow them
                if (cur.ins_only && nxt.ins_only) {
                    seq_issue_fat(s, lane, nxt);
                    nxt_issued = true;
                }
            }
            const unsigned conf = seq_conflicts(s.d, lane, cur);
            if (cur.ins_only) {
                if (a.slim_in_smem) seq_slim_inserts(s.d, s.w, s.key_bytes, sA, lane, cur, F, conf);
                else seq_slim_inserts(s.d, s.w, s.key_bytes, A, lane, cur, F, conf);
            }
            else seq_mixed_window(s, A, lane, cur, conf, &under);
            if (has_next) {
                if (nxt.ins_only && !nxt_issued) seq_issue_fat(s, lane, nxt);
                cur = nxt;
            }
        }
        if (under) atomicOr(a.ctrl + kCtrlErr, kErrUnderflow);
    }
    if (a.slim_in_smem) {
        __syncthreads();
        for (uint64_t i = threadIdx.x; i < slim_n; i += blockDim.x) s.A[i] = sA[i];
    }
}

}  // namespace

cudaError_t launch_seq_update(const SeqArgs& a, cudaStream_t st, int smem_limit) {
    SeqArgs b = a;
    const uint64_t slim_bytes = (uint64_t)a.s.d * a.s.w * 4ull;
    size_t smem = 0;
    b.slim_in_smem = 0;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, seq_update_kernel) != cudaSuccess) return cudaErrorInvalidValue;
    // the Slim goes to shared memory when it fits beside the kernel's static shared memory
    if (slim_bytes + fa.sharedSizeBytes <= (uint64_t)smem_limit) {
        b.slim_in_smem = 1;
        smem = (size_t)slim_bytes;
        cudaError_t e = cudaFuncSetAttribute(seq_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    seq_update_kernel<<<1, kSeqBlock, smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace sfk
