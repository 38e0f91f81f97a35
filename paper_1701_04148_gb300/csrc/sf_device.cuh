// sf_device.cuh -- device-side building blocks of the SF-sketch kernels (sm_103a).
//
// Hashing: SplitMix64's output finaliser (Steele, Lea, Flood, OOPSLA 2014) applied to the key
// words xor a per-row seed, then multiply-shift range reduction (Lemire, ACM TOMACS 2019):
//   h_i = (hi32(H_i) * w) >> 32   (bucket / Slim counter, Sec. 3.4: h_i maps to [1, w])
//   f_i = (lo32(H_i) * z) >> 32   (counter inside the Fat bucket, Sec. 3.4: f_i maps to [1, z])
// The paper only asks for independent uniformly distributed hash functions (Sec. 3.1, 3.4).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sfk {

constexpr int kMaxD = 8;
constexpr int kMaxZ = 64;

// Error bits latched in the control block (read and cleared by sf_sync).
constexpr uint32_t kErrUnderflow = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrBadKey = 4u;
constexpr uint32_t kErrDictFull = 8u;

// Control block: the first 256 bytes of every scratch buffer.  Word 0 latches error bits;
// bytes 8..15 hold the 64-bit arrival counter of the grid barrier (monotonic across launches).
enum : uint32_t { kCtrlErr = 0, kCtrlBarrier64 = 2, kCtrlWords = 64 };

// Per-chunk key dictionary entry (32 bytes).  The key is claimed with one 128-bit CAS:
// key_lo = bytes 0..7, key_hi = bytes 8..14 with bit 63 set (so an occupied entry is never 0).
// The counters hold the key's inserts c_e and deletes in the chunk and m_e = min_i A0_i[h_i(e)];
// mask_slack holds the rows i with A0_i[h_i] = m_e (bits 0..7) and, in insertion-only launches,
// a slack sl (bits 8..31) with m_e + sl <= the key's chunk-end Fat minimum F_e.
constexpr unsigned long long kKeyTag = 1ull << 63;
constexpr uint32_t kSlackMax = 0xFFFFFFu;
struct alignas(32) DictEntry {
    unsigned long long key_lo;
    unsigned long long key_hi;
    uint32_t c_ins;
    uint32_t c_del;
    uint32_t m;
    uint32_t mask_slack;
};

struct SketchDesc {
    uint32_t* A;             // Slim, A[i*w + j]
    uint32_t* B;             // Fat,  B[(i*w + j)*z + k]
    uint32_t d, w, z, key_bytes;
    uint64_t rs[kMaxD];      // row seeds
    const uint32_t* idx_table;  // explicit-index mode table, else nullptr
    uint32_t n_ids;
    uint32_t sf4_delete;     // nonzero: deletions clamp to the bucket sum (SF_4), else to the maximum (SF_F)
};

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

struct Key {
    uint64_t x0, x1;
};

// Packed little-endian key t.  4/8-byte keys use one aligned read-only load.
__device__ __forceinline__ Key load_key(const uint8_t* __restrict__ keys, uint64_t t, uint32_t kb) {
    Key k{0ull, 0ull};
    if (kb == 4) {
        k.x0 = __ldg(reinterpret_cast<const uint32_t*>(keys) + t);
    } else if (kb == 8) {
        k.x0 = __ldg(reinterpret_cast<const unsigned long long*>(keys) + t);
    } else {
        const uint8_t* p = keys + t * kb;
        const uint32_t n0 = kb < 8 ? kb : 8;
        for (uint32_t b = 0; b < n0; ++b) k.x0 |= (uint64_t)__ldg(p + b) << (8 * b);
        for (uint32_t b = 8; b < kb; ++b) k.x1 |= (uint64_t)__ldg(p + b) << (8 * (b - 8));
    }
    return k;
}

// The kb-byte little-endian key that starts `off` bytes (0..7) into the consecutive 64-bit words
// w0, w1, w2 (w1 and w2 may be 0 where the key does not reach them).
__device__ __forceinline__ Key key_from_words(uint64_t w0, uint64_t w1, uint64_t w2, uint32_t off, uint32_t kb) {
    const uint32_t sh = 8u * off;
    Key k;
    k.x0 = sh ? (w0 >> sh) | (w1 << (64u - sh)) : w0;
    k.x1 = sh ? (w1 >> sh) | (w2 << (64u - sh)) : w1;
    if (kb < 8u) {
        k.x0 &= (1ull << (8u * kb)) - 1ull;
        k.x1 = 0ull;
    } else if (kb == 8u) {
        k.x1 = 0ull;
    } else if (kb < 16u) {
        k.x1 &= (1ull << (8u * (kb - 8u))) - 1ull;
    }
    return k;
}

// The kb-byte key at byte `off` of a 16-byte-aligned shared-memory stage, read as the (at most three)
// 64-bit words covering it; the caller keeps those words inside the stage.  Byte-wise reads of a
// warp's 13-byte keys meet bank conflicts on every one of their 13 loads; the word reads measured
// 3.5 % faster on the single-sketch 13-byte Zipf sweep (same counters).
__device__ __forceinline__ Key key_from_stage(const uint4* stage, uint32_t off, uint32_t kb) {
    const unsigned long long* sw = reinterpret_cast<const unsigned long long*>(stage) + (off >> 3);
    const uint32_t o8 = off & 7u, nw = (o8 + kb + 7u) >> 3;
    return key_from_words(sw[0], nw > 1u ? sw[1] : 0ull, nw > 2u ? sw[2] : 0ull, o8, kb);
}

// One packed key t from the aligned 8-byte words that cover it (widths other than 4 and 8 bytes):
// at most three 64-bit loads (a 15-byte key starting 7 bytes into a word spans 22 bytes).  A warp
// reading 13-byte keys byte by byte issues 13 loads, each touching the four or five 128-byte lines
// its 32 keys span; the word loads touch the same lines in three.  A key whose covering words reach
// outside [keys, keys + total_bytes) is read byte by byte, so no byte outside the caller's buffer is
// touched.
__device__ __forceinline__ Key load_key_words(const uint8_t* __restrict__ keys, uint64_t total_bytes, uint64_t t,
                                              uint32_t kb) {
    const uintptr_t base = reinterpret_cast<uintptr_t>(keys);
    const uintptr_t a = base + t * kb;
    const uintptr_t a0 = a & ~(uintptr_t)7;
    const uint32_t off = (uint32_t)(a & 7u);
    const uint32_t nw = (off + kb + 7u) >> 3;  // covering words, 1..3
    if (a0 < base || a0 + 8u * nw > base + total_bytes) return load_key(keys, t, kb);
    const unsigned long long* w = reinterpret_cast<const unsigned long long*>(a0);
    return key_from_words(__ldg(w), nw > 1u ? __ldg(w + 1) : 0ull, nw > 2u ? __ldg(w + 2) : 0ull, off, kb);
}

// Per-warp load of up to 32 packed keys of a width other than 4 or 8 bytes: the warp reads the
// 16-byte-aligned granules covering its keys with vector loads into shared memory (streaming,
// evict-first: each key byte is read once), and reads a granule that straddles either end of the
// caller's buffer byte by byte, so no byte outside [keys, keys + n*kb) is ever touched.
__device__ __forceinline__ Key load_key_staged(const uint8_t* __restrict__ keys, uint64_t total_bytes,
                                               uint64_t first, uint32_t nvalid, uint32_t kb, uint32_t lane,
                                               uint4* stage) {
    const uintptr_t kaddr = reinterpret_cast<uintptr_t>(keys);
    const uint8_t* kal = reinterpret_cast<const uint8_t*>(kaddr & ~(uintptr_t)15);
    const uint64_t lo = kaddr & 15u, hi = lo + total_bytes;  // valid bytes, relative to kal
    const uint64_t b0 = lo + first * kb, b1 = b0 + (uint64_t)nvalid * kb;
    const uint64_t g0 = b0 & ~15ull;
    const uint32_t ngran = (uint32_t)((b1 - g0 + 15) >> 4);  // <= 31 for kb <= 15
    if (lane < ngran) {
        const uint64_t gb = g0 + 16ull * lane;
        uint4 v;
        if (gb >= lo && gb + 16 <= hi) {
            v = __ldcs(reinterpret_cast<const uint4*>(kal + gb));
        } else {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            for (uint32_t q = 0; q < 16; ++q)
                if (gb + q >= lo && gb + q < hi) w[q >> 2] |= (uint32_t)__ldg(kal + gb + q) << (8 * (q & 3));
            v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        stage[lane] = v;
    }
    __syncwarp();
    Key k{0ull, 0ull};
    // (b0 - g0) + lane * kb + kb <= 15 + 32 * 15: the covering words stay inside the 512-byte stage
    if (lane < nvalid) k = key_from_stage(stage, (uint32_t)(b0 - g0) + lane * kb, kb);
    __syncwarp();
    return k;
}

__device__ __forceinline__ uint64_t row_hash(const Key& k, uint32_t kb, uint64_t seed) {
    uint64_t H = mix64(k.x0 ^ seed);
    if (kb > 8) H = mix64(H ^ k.x1);
    return H;
}

__device__ __forceinline__ uint32_t reduce_hi(uint64_t H, uint32_t range) {
    return (uint32_t)(((H >> 32) * (uint64_t)range) >> 32);
}

__device__ __forceinline__ uint32_t reduce_lo(uint64_t H, uint32_t range) {
    return (uint32_t)(((H & 0xFFFFFFFFull) * (uint64_t)range) >> 32);
}

// Row indices of one key for D rows (D = 0: the runtime s.d rows, at most kMaxD).  Returns
// false for a bad key id or table entry in explicit-index mode.  probe receives a well-mixed
// 64-bit value of the key for the dictionaries (row 0's hash, or a mix of the explicit id): its
// low half picks a slot, its high half serves as a fingerprint.
template <int D>
__device__ __forceinline__ bool key_indices(const SketchDesc& s, const Key& k, uint32_t* h, uint32_t* f,
                                            uint64_t* probe) {
    constexpr int N = D ? D : kMaxD;
    if (s.idx_table) {
        const uint64_t id = k.x0;
        if (id >= s.n_ids) return false;
        const uint32_t* row = s.idx_table + id * (uint64_t)s.d * 2;
        bool ok = true;
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (D || i < (int)s.d) {
                h[i] = __ldg(row + 2 * i);
                f[i] = __ldg(row + 2 * i + 1);
                ok &= (h[i] < s.w) && (f[i] < s.z);  // a bad table entry must not index out of bounds
            }
        *probe = mix64(id);
        return ok;
    }
    uint64_t H0 = 0;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (D || i < (int)s.d) {
            const uint64_t H = row_hash(k, s.key_bytes, s.rs[i]);
            if (i == 0) H0 = H;
            h[i] = reduce_hi(H, s.w);
            f[i] = reduce_lo(H, s.z);
        }
    *probe = H0;
    return true;
}

__device__ __forceinline__ bool key_equal(const uint8_t* __restrict__ keys, uint64_t t, uint32_t kb,
                                          const Key& k) {
    const Key o = load_key(keys, t, kb);
    return o.x0 == k.x0 && o.x1 == k.x1;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// L2 eviction-priority policies.  The Fat and the Slim are reused across chunks and should stay in
// L2 (evict_last); the chunk dictionary and the key stream are touched once or twice per chunk
// (evict_first), so they should not push counters out.
__device__ __forceinline__ unsigned long long l2_policy_keep() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ unsigned long long l2_policy_stream() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint32_t ld_cg_pol(const uint32_t* p, unsigned long long pol) {
    uint32_t v;
    asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ uint4 ld_cg_v4_pol(const void* p, unsigned long long pol) {
    uint4 v;
    asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ void red_add_pol(uint32_t* p, uint32_t v, unsigned long long pol) {
    asm volatile("red.global.add.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ uint32_t atom_add_pol(uint32_t* p, uint32_t v, unsigned long long pol) {
    uint32_t old;
    asm volatile("atom.global.add.L2::cache_hint.u32 %0, [%1], %2, %3;"
                 : "=r"(old)
                 : "l"(p), "r"(v), "l"(pol)
                 : "memory");
    return old;
}

__device__ __forceinline__ void red_max_pol(uint32_t* p, uint32_t v, unsigned long long pol) {
    asm volatile("red.global.max.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ void red_min_pol(uint32_t* p, uint32_t v, unsigned long long pol) {
    asm volatile("red.global.min.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

// 128-bit compare-and-swap in global memory (atom.cas.b128, sm_90 and later).
__device__ __forceinline__ void cas128(unsigned long long* addr, unsigned long long cmp_lo,
                                       unsigned long long cmp_hi, unsigned long long new_lo,
                                       unsigned long long new_hi, unsigned long long& old_lo,
                                       unsigned long long& old_hi) {
    asm volatile(
        "{\n\t.reg .b128 c, v, o;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.global.cas.b128 o, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, o;\n\t}"
        : "=l"(old_lo), "=l"(old_hi)
        : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(addr)
        : "memory");
}

// Split-phase grid barrier: grid_arrive announces this block (after all its threads' prior memory
// operations), grid_wait blocks until every block of the grid has arrived `target` times in total.
// Work placed between the two overlaps the wait.
//
// Ordering without extra fences: __syncthreads orders every thread's earlier accesses before
// thread 0's arrival, and the arrival is a gpu-scope release (red.release), which is cumulative
// over what precedes it; the waiter's gpu-scope acquire load that sees the final count, followed
// by __syncthreads, orders those accesses before every thread's later ones.  A fence.sc on either
// side adds nothing to this and was measured to cost about 0.2 us per barrier.
__device__ __forceinline__ void grid_arrive(uint32_t* ctrl) {
    __syncthreads();
    if (threadIdx.x == 0) red_release_gpu_add_u64(reinterpret_cast<unsigned long long*>(ctrl + kCtrlBarrier64), 1ull);
}

__device__ __forceinline__ bool grid_wait(uint32_t* ctrl, unsigned long long target, uint64_t timeout_ns) {
    __shared__ int s_ok_w;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(ctrl + kCtrlBarrier64);
        if (ld_acquire_gpu_u64(cnt) < target) {
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire_gpu_u64(cnt) < target) {
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicOr(ctrl + kCtrlErr, kErrTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok_w = ok;
    }
    __syncthreads();
    return s_ok_w != 0;
}

// Grid-wide barrier for a co-resident (cooperatively launched) grid.  Every block adds 1 to a
// monotonic 64-bit counter and waits until it reaches `target` = (barriers passed so far + 1) *
// gridDim.x.  The wait is bounded: after timeout_ns the block latches kErrTimeout and returns
// false, so the kernel leaves instead of hanging.
__device__ __forceinline__ bool grid_barrier(uint32_t* ctrl, unsigned long long target, uint64_t timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ctrl + kCtrlBarrier64);
        red_release_gpu_add_u64(cnt, 1ull);
        if (ld_acquire_gpu_u64(cnt) < target) {
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire_gpu_u64(cnt) < target) {
                if (globaltimer_ns() - t0 > timeout_ns) {
                    // give up: latch the error and leave; every other block then misses this one at
                    // its next barrier, times out the same way, and the launch ends
                    atomicOr(ctrl + kCtrlErr, kErrTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ uint32_t warp_min_u32(uint32_t v, uint32_t mask) {
    return __reduce_min_sync(mask, v);
}

// ---- counter addressing shared by the update kernels ---------------------------------------

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t* fat_ptr(const SketchDesc& s, uint32_t i, uint32_t h, uint32_t f) {
    return s.B + ((uint64_t)i * s.w + h) * s.z + f;
}

__device__ __forceinline__ uint32_t* slim_ptr(const SketchDesc& s, uint32_t i, uint32_t h) {
    return s.A + (uint64_t)i * s.w + h;
}

// The bound a deletion clamps Slim counter A_i[h] to, from the Fat bucket B_i[h][.]: its maximum
// max_k B_i[h][k] (SF_F, Sec. 3.5), or with s.sf4_delete its sum sum_k B_i[h][k] (SF_4, Sec. 3.4;
// a sum of 2^32 or more is returned as the 32-bit maximum, which no counter exceeds).  Also
// reports whether B_i[h][f] went negative (strict-turnstile violation).
__device__ __forceinline__ uint32_t bucket_bound_cg(const SketchDesc& s, uint32_t i, uint32_t h,
                                                    uint32_t f, bool* underflow,
                                                    unsigned long long pol = 0ull, bool hinted = false) {
    const uint32_t* bk = s.B + ((uint64_t)i * s.w + h) * s.z;
    uint32_t mx = 0;
    uint64_t sum = 0;
    if ((s.z & 3u) == 0u) {
        const uint4* b4 = reinterpret_cast<const uint4*>(bk);
        for (uint32_t q = 0; q < (s.z >> 2); ++q) {
            const uint4 v = hinted ? ld_cg_v4_pol(b4 + q, pol) : __ldcg(b4 + q);
            mx = max(max(mx, v.x), max(v.y, max(v.z, v.w)));
            sum += (uint64_t)v.x + v.y + v.z + v.w;
        }
    } else {
        for (uint32_t k = 0; k < s.z; ++k) {
            const uint32_t v = hinted ? ld_cg_pol(bk + k, pol) : __ldcg(bk + k);
            mx = max(mx, v);
            sum += v;
        }
    }
    if ((int32_t)(hinted ? ld_cg_pol(bk + f, pol) : __ldcg(bk + f)) < 0) *underflow = true;
    if (s.sf4_delete) return sum < 0xFFFFFFFFull ? (uint32_t)sum : 0xFFFFFFFFu;
    return mx;
}

// Indices of row i only (the sequential kernels take rows one at a time).
__device__ __forceinline__ bool row_index(const SketchDesc& s, const Key& k, uint32_t i, uint32_t* h,
                                          uint32_t* f) {
    if (s.idx_table) {
        if (k.x0 >= s.n_ids) return false;
        const uint32_t* row = s.idx_table + (k.x0 * s.d + i) * 2;
        *h = __ldg(row);
        *f = __ldg(row + 1);
        return *h < s.w && *f < s.z;
    }
    const uint64_t H = row_hash(k, s.key_bytes, s.rs[i]);
    *h = reduce_hi(H, s.w);
    *f = reduce_lo(H, s.z);
    return true;
}

}  // namespace sfk
