// sf_update.cu -- SF-sketch insert/delete kernels (sm_103a).
//
// Paper rules (Yang et al., SF-sketch):
//   insertion (Sec. 3.4, kept by SF_F in Sec. 3.5): B_i[h_i][f_i] += 1 for every row; with
//     Bmin the minimum of those d counters after the increment and m = min_i A_i[h_i], every
//     A_l[h_l] equal to m is incremented when m < Bmin.
//   deletion (Sec. 3.5): B_i[h_i][f_i] -= 1; A_i[h_i] is lowered to max_k B_i[h_i][k] when
//     larger (the paper's "if the maximum changed" test never matters because
//     A_i[j] <= max_k B_i[j][k] always holds, Appendix I).
//
// chunk_update_kernel implements the chunked schedule: per chunk of S updates
//   phase 1: Fat += every update (warp-aggregated atomics); a per-chunk dictionary collects each
//            distinct key's inserts c_e, deletes, and m_e = min_i A0_i[h_i(e)] (Slim untouched)
//   barrier
//   phase 2: one thread per distinct key: F_e = min_i B_i[h_i][f_i], T_e = min(m_e + c_e, F_e),
//            atomicMax(A_i[h_i], T_e); for deleted keys atomicMin(A_i[h_i], max_k B_i[h_i][k]);
//            the dictionary slot is cleared for the next chunk
//   barrier
// All clamps of one Slim counter in a chunk share the bound max_k B_i[j][k] of the chunk-end
// Fat, and every raise target satisfies T_e <= F_e <= that bound, so the raises and clamps of a
// counter commute: applying them with atomics in any order gives the stream-order result.
//
// seq_update_kernel is the S = 1 path: one warp walks the stream in order, lane i owning row i.
#include "sf_internal.h"

namespace sfk {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t* fat_ptr(const SketchDesc& s, uint32_t i, uint32_t h, uint32_t f) {
    return s.B + ((uint64_t)i * s.w + h) * s.z + f;
}

__device__ __forceinline__ uint32_t* slim_ptr(const SketchDesc& s, uint32_t i, uint32_t h) {
    return s.A + (uint64_t)i * s.w + h;
}

// max_k B_i[h][k] and whether B_i[h][f] went negative (strict-turnstile violation).
__device__ __forceinline__ uint32_t bucket_max_cg(const SketchDesc& s, uint32_t i, uint32_t h,
                                                  uint32_t f, bool* underflow) {
    const uint32_t* bk = s.B + ((uint64_t)i * s.w + h) * s.z;
    uint32_t mx = 0;
    if ((s.z & 3u) == 0u) {
        const uint4* b4 = reinterpret_cast<const uint4*>(bk);
        for (uint32_t q = 0; q < (s.z >> 2); ++q) {
            const uint4 v = __ldcg(b4 + q);
            mx = max(max(mx, v.x), max(v.y, max(v.z, v.w)));
        }
    } else {
        for (uint32_t k = 0; k < s.z; ++k) mx = max(mx, __ldcg(bk + k));
    }
    if ((int32_t)__ldcg(bk + f) < 0) *underflow = true;
    return mx;
}

__global__ void __launch_bounds__(kChunkBlock) chunk_update_kernel(const ChunkArgs a) {
    const SketchDesc& s = a.s;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
    const uint64_t nchunks = (a.n + a.S - 1) / a.S;

    for (uint64_t c = 0; c < nchunks; ++c) {
        const uint64_t base = c * (uint64_t)a.S;
        const uint64_t len = min((uint64_t)a.S, a.n - base);

        // ---- phase 1: Fat updates and the chunk dictionary --------------------------------
        for (uint64_t j = gwarp * 32; j < len; j += nwarps * 32) {
            const uint64_t rel = j + lane;
            uint32_t h[kMaxD], f[kMaxD], probe = 0;
            Key k{0ull, 0ull};
            int op = 0;
            if (rel < len) {
                op = a.ops ? (int)a.ops[base + rel] : a.op_const;
                if (op != 0) {
                    k = load_key(a.keys, base + rel, s.key_bytes);
                    if (!key_indices(s, k, h, f, &probe)) {
                        atomicOr(a.ctrl + kCtrlErr, kErrBadKey);
                        op = 0;
                    }
                }
            }
            const unsigned act = __ballot_sync(kFull, op != 0);
            if (act == 0u) continue;
            const unsigned ins = __ballot_sync(kFull, op > 0);
            unsigned grp = __match_any_sync(kFull, k.x0);
            if (s.key_bytes > 8) grp &= __match_any_sync(kFull, k.x1);
            grp &= act;
            if (op == 0 || lane != (uint32_t)(__ffs(grp) - 1)) continue;

            // one leader per distinct key of this warp
            const uint32_t ci = __popc(grp & ins), cd = __popc(grp & ~ins);
            const int32_t net = (int32_t)ci - (int32_t)cd;
            if (net != 0) {
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d) atomicAdd(fat_ptr(s, i, h[i], f[i]), (uint32_t)net);
            }
            uint32_t slot = probe & a.cap_mask;
            const uint32_t me = (uint32_t)rel + 1u;
            bool found = false;
            for (uint32_t p = 0; p <= a.cap_mask; ++p) {
                const uint32_t cur = atomicCAS(&a.dict[slot].owner, 0u, me);
                if (cur == 0u || key_equal(a.keys, base + cur - 1u, s.key_bytes, k)) {
                    found = true;
                    break;
                }
                slot = (slot + 1u) & a.cap_mask;
            }
            if (!found) {
                atomicOr(a.ctrl + kCtrlErr, kErrDictFull);
                continue;
            }
            if (ci) {
                atomicAdd(&a.dict[slot].c_ins, ci);
                uint32_t m = 0xFFFFFFFFu;
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d) m = min(m, __ldcg(slim_ptr(s, i, h[i])));
                __stcg(&a.dict[slot].m, m);  // every writer stores the same chunk-start value
            }
            if (cd) atomicAdd(&a.dict[slot].c_del, cd);
        }
        if (!grid_barrier(a.ctrl, gridDim.x, a.timeout_ns)) return;

        // ---- phase 2: Slim raises and clamps, one thread per distinct key -----------------
        for (uint64_t slot = gtid; slot <= a.cap_mask; slot += gthreads) {
            uint4* ep = reinterpret_cast<uint4*>(a.dict + slot);
            const uint4 e = __ldcg(ep);
            if (e.x == 0u) continue;
            const Key k = load_key(a.keys, base + e.x - 1u, s.key_bytes);
            uint32_t h[kMaxD], f[kMaxD], probe;
            key_indices(s, k, h, f, &probe);
            if (e.y) {
                uint32_t F = 0xFFFFFFFFu;
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d) F = min(F, __ldcg(fat_ptr(s, i, h[i], f[i])));
                const uint64_t mc = (uint64_t)e.w + e.y;
                const uint32_t T = mc < (uint64_t)F ? (uint32_t)mc : F;
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d) {
                        uint32_t* ap = slim_ptr(s, i, h[i]);
                        if (__ldcg(ap) < T) atomicMax(ap, T);
                    }
            }
            if (e.z) {
                bool under = false;
#pragma unroll
                for (int i = 0; i < kMaxD; ++i)
                    if (i < (int)s.d) {
                        const uint32_t M = bucket_max_cg(s, i, h[i], f[i], &under);
                        uint32_t* ap = slim_ptr(s, i, h[i]);
                        if (__ldcg(ap) > M) atomicMin(ap, M);
                    }
                if (under) atomicOr(a.ctrl + kCtrlErr, kErrUnderflow);
            }
            __stcg(ep, make_uint4(0u, 0u, 0u, 0u));
        }
        if (!grid_barrier(a.ctrl, gridDim.x, a.timeout_ns)) return;
    }
}

// Indices of row i only (the sequential kernel gives each lane one row).
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

__global__ void __launch_bounds__(kSeqBlock) seq_update_kernel(const SeqArgs a) {
    extern __shared__ uint32_t sA[];
    const SketchDesc& s = a.s;
    const uint64_t slim_n = (uint64_t)s.d * s.w;
    if (a.slim_in_smem) {
        for (uint64_t i = threadIdx.x; i < slim_n; i += blockDim.x) sA[i] = __ldcg(s.A + i);
        __syncthreads();
    }
    uint32_t* A = a.slim_in_smem ? sA : s.A;
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        const bool row = lane < s.d;
        bool under = false;
        for (uint64_t t = 0; t < a.n; ++t) {
            const int op = a.ops ? (int)a.ops[t] : a.op_const;
            if (op == 0) continue;
            const Key k = load_key(a.keys, t, s.key_bytes);
            uint32_t h = 0, f = 0;
            bool ok = true;
            if (row) ok = row_index(s, k, lane, &h, &f);
            if (!__all_sync(kFull, ok)) {
                if (lane == 0) atomicOr(a.ctrl + kCtrlErr, kErrBadKey);
                continue;
            }
            uint32_t* bp = row ? fat_ptr(s, lane, h, f) : nullptr;
            volatile uint32_t* ap = row ? A + (uint64_t)lane * s.w + h : nullptr;
            if (op > 0) {
                uint32_t nv = 0xFFFFFFFFu, av = 0xFFFFFFFFu;
                if (row) {
                    nv = atomicAdd(bp, 1u) + 1u;
                    av = *ap;
                }
                const uint32_t F = __reduce_min_sync(kFull, nv);
                const uint32_t m = __reduce_min_sync(kFull, av);
                if (row && m < F && av == m) *ap = m + 1u;
            } else {
                if (row) {
                    const uint32_t old = atomicAdd(bp, 0xFFFFFFFFu);
                    if (old == 0u) under = true;
                    bool dummy = false;
                    const uint32_t M = bucket_max_cg(s, lane, h, f, &dummy);
                    if (*ap > M) *ap = M;
                }
            }
            __syncwarp();
        }
        if (under) atomicOr(a.ctrl + kCtrlErr, kErrUnderflow);
    }
    if (a.slim_in_smem) {
        __syncthreads();
        for (uint64_t i = threadIdx.x; i < slim_n; i += blockDim.x) s.A[i] = sA[i];
    }
}

}  // namespace

int chunk_update_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, chunk_update_kernel, kChunkBlock, 0) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_chunk_update(const ChunkArgs& a, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kChunkBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, chunk_update_kernel, a);
}

cudaError_t launch_seq_update(const SeqArgs& a, cudaStream_t st, int smem_limit) {
    SeqArgs b = a;
    const uint64_t slim_bytes = (uint64_t)a.s.d * a.s.w * 4ull;
    size_t smem = 0;
    b.slim_in_smem = 0;
    if (slim_bytes <= (uint64_t)smem_limit) {
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
