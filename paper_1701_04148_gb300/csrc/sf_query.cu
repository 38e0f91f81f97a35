// sf_query.cu -- batched point queries on an exported Slim-subsketch (sm_103a).
//
// Query (Sec. 3.1, unchanged through SF_F, Sec. 3.5): the estimate of item e is the smallest
// of its d Slim counters, min_i A_i[h_i(e)]; the Fat is never read.  The paper's GPU version
// (Sec. 4.2) keeps all d arrays resident on the device and answers a batch per launch.
#include "sf_internal.h"

namespace sfk {

namespace {

// Key of slot t of a warp-iteration covering slots [base, base + 32) of one buffer of n keys.
// Widths other than 4 and 8 bytes are staged warp-cooperatively: 16-byte vector loads of the
// granules covering the warp's keys (load_key_staged) instead of kb single-byte loads per lane.
__device__ __forceinline__ Key warp_key(const uint8_t* keys, uint64_t n, uint64_t base, uint32_t kb, uint32_t lane,
                                        uint4* stage) {
    if (kb != 4 && kb != 8) {
        const uint64_t left = n > base ? n - base : 0;
        return load_key_staged(keys, n * kb, base, (uint32_t)(left < 32 ? left : 32), kb, lane, stage);
    }
    return base + lane < n ? load_key(keys, base + lane, kb) : Key{0ull, 0ull};
}

__device__ __forceinline__ uint32_t slim_min(const SketchDesc& s, const Key& k) {
    uint32_t h[kMaxD], f[kMaxD];
    uint64_t probe;
    uint32_t m = 0xFFFFFFFFu;
    if (key_indices<0>(s, k, h, f, &probe)) {
#pragma unroll
        for (int i = 0; i < kMaxD; ++i)
            if (i < (int)s.d) m = min(m, __ldg(s.A + (uint64_t)i * s.w + h[i]));
    }
    return m;
}

// Warps take 32 consecutive keys per iteration (a block reads a contiguous run of the key stream).
__global__ void __launch_bounds__(kQueryBlock) query_kernel(const QueryArgs q) {
    __shared__ uint4 s_stage[kQueryBlock / 32][32];
    const SketchDesc& s = q.s;
    const uint32_t lane = threadIdx.x & 31u;
    uint4* stage = s_stage[threadIdx.x >> 5];
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < q.n;
         base += nwarps * 32) {
        const Key k = warp_key(q.keys, q.n, base, s.key_bytes, lane, stage);
        if (base + lane < q.n) q.out[base + lane] = slim_min(s, k);
    }
}

// Many requests against many Slims in one launch: slot t belongs to the request whose answer range
// holds it (binary search over the out_off prefix).  A warp whose 32 slots all fall in one request
// (the common case) stages that request's keys together; a warp that straddles requests loads each
// lane's key on its own.
__global__ void __launch_bounds__(kQueryBlock) multi_query_kernel(const MultiQueryArgs q) {
    __shared__ uint4 s_stage[kQueryBlock / 32][32];
    const uint32_t lane = threadIdx.x & 31u;
    uint4* stage = s_stage[threadIdx.x >> 5];
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < q.total;
         base += nwarps * 32) {
        const uint64_t t = base + lane;
        const uint64_t ts = t < q.total ? t : q.total - 1;  // lanes past the end look up the last slot
        uint32_t lo = 0, hi = q.n_reqs;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(&q.reqs[mid].out_off) <= ts) lo = mid;
            else hi = mid;
        }
        const QueryReq& r = q.reqs[lo];
        SketchDesc s{};
        s.A = const_cast<uint32_t*>(r.A);
        s.d = r.d;
        s.w = r.w;
        s.z = 0xFFFFFFFFu;
        s.key_bytes = r.key_bytes;
#pragma unroll
        for (int i = 0; i < kMaxD; ++i) s.rs[i] = r.rs[i];
        const uint8_t* keys = q.keys + r.key_off;
        Key k{0ull, 0ull};
        if (__all_sync(kFull, lo == __shfl_sync(kFull, lo, 0))) {
            k = warp_key(keys, r.n, base - r.out_off, r.key_bytes, lane, stage);
        } else if (t < q.total) {
            k = load_key(keys, t - r.out_off, r.key_bytes);
        }
        if (t < q.total) q.out[t] = slim_min(s, k);
    }
}

}  // namespace

cudaError_t launch_multi_query(const MultiQueryArgs& a, int num_sms, cudaStream_t st) {
    if (a.total == 0) return cudaSuccess;
    const uint64_t want = (a.total + kQueryBlock - 1) / kQueryBlock;
    const uint64_t cap = (uint64_t)num_sms * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    multi_query_kernel<<<grid, kQueryBlock, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_query(const QueryArgs& a, int num_sms, cudaStream_t st) {
    if (a.n == 0) return cudaSuccess;
    const uint64_t want = (a.n + kQueryBlock - 1) / kQueryBlock;
    const uint64_t cap = (uint64_t)num_sms * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    query_kernel<<<grid, kQueryBlock, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sfk
