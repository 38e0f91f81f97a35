// sf_query.cu -- batched point queries on an exported Slim-subsketch (sm_103a).
//
// Query (Sec. 3.1, unchanged through SF_F, Sec. 3.5): the estimate of item e is the smallest
// of its d Slim counters, min_i A_i[h_i(e)]; the Fat is never read.  The paper's GPU version
// (Sec. 4.2) keeps all d arrays resident on the device and answers a batch per launch.
//
// Keys are read per thread, several in flight: one aligned load for 4/8-byte keys, otherwise the
// aligned 8-byte words covering the key (at most three loads; byte loads only where those words
// would reach past either end of the caller's buffer).  Measured on 10^6 13-byte keys, back-to-back
// launches: byte loads 23.0 us, word loads 22.4, word loads with the one-wave grid below 20.8.
// Staging a warp's keys through shared memory with 16-byte loads was no faster than byte loads: its
// byte reads from shared memory meet bank conflicts and cost as many L1 wavefronts.
#include "sf_internal.h"

namespace sfk {

namespace {

// Keys in flight per thread: each iteration loads K keys (t, t + stride, ...), hashes them, and
// issues all K * D gathers before it takes any minimum, so a thread keeps K independent chains of
// key load -> hash -> gathers going instead of one.  Measured on 10^6 13-byte keys (d = 4, 4 MiB
// Slim) / 2^24 8-byte keys (64 MiB Slim): K = 1 37.4 / 264 us, K = 2 34.8 / 254 us, K = 4 39.6 /
// 254 us (fewer threads).  The launches are bound by the L1 wavefronts of the gathers (each lane of a
// gather touches its own line), not by the chains.
constexpr int kQueryKeys = 2;

__device__ __forceinline__ Key query_key(const uint8_t* keys, uint64_t total_bytes, uint64_t t, uint32_t kb) {
    return (kb == 4u || kb == 8u) ? load_key(keys, t, kb) : load_key_words(keys, total_bytes, t, kb);
}

template <int D>
__global__ void __launch_bounds__(kQueryBlock) query_kernel(const QueryArgs q) {
    constexpr int K = kQueryKeys;
    const SketchDesc& s = q.s;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t0 < q.n; t0 += K * stride) {
        Key k[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint64_t t = t0 + (uint64_t)j * stride;
            k[j] = t < q.n ? query_key(q.keys, q.n * s.key_bytes, t, s.key_bytes) : Key{0ull, 0ull};
        }
        uint32_t h[K][D], f[D];
        bool ok[K];
        uint64_t probe;
#pragma unroll
        for (int j = 0; j < K; ++j) ok[j] = t0 + (uint64_t)j * stride < q.n && key_indices<D>(s, k[j], h[j], f, &probe);
        uint32_t v[K][D];
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int i = 0; i < D; ++i) v[j][i] = ok[j] ? __ldg(s.A + (uint64_t)i * s.w + h[j][i]) : 0xFFFFFFFFu;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint64_t t = t0 + (uint64_t)j * stride;
            if (t < q.n) {
                uint32_t m = 0xFFFFFFFFu;
#pragma unroll
                for (int i = 0; i < D; ++i) m = min(m, v[j][i]);
                q.out[t] = m;
            }
        }
    }
}

// The grid is one wave of resident blocks: the 13-byte form holds 40 registers (six blocks per
// SM), and a fixed eight blocks per SM left a partial second wave (measured: 22.4 -> 20.8 us for
// 10^6 13-byte keys, 269 -> 256 us for 2^24; capping registers at 32 spilled and ran slower).
template <int D>
cudaError_t launch_query_d(const QueryArgs& a, int num_sms, cudaStream_t st) {
    static int resident = 0;  // blocks per SM, asked once per process and row count
    if (resident == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, query_kernel<D>, kQueryBlock, 0) != cudaSuccess)
            return cudaGetLastError();
        resident = nb > 0 ? nb : 1;
    }
    const uint64_t want = (a.n + (uint64_t)kQueryBlock * kQueryKeys - 1) / ((uint64_t)kQueryBlock * kQueryKeys);
    const uint64_t cap = (uint64_t)num_sms * (uint64_t)resident;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    query_kernel<D><<<grid, kQueryBlock, 0, st>>>(a);
    return cudaGetLastError();
}

// Many requests against many Slims in one launch: thread t answers global slot t, finding its
// request by binary search over the out_off prefix (requests stay warp-coherent mostly).
__global__ void __launch_bounds__(kQueryBlock) multi_query_kernel(const MultiQueryArgs q) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < q.total; t += stride) {
        uint32_t lo = 0, hi = q.n_reqs;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(&q.reqs[mid].out_off) <= t) lo = mid;
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
        const Key k = query_key(q.keys + r.key_off, (uint64_t)r.n * r.key_bytes, t - r.out_off, r.key_bytes);
        uint32_t h[kMaxD], f[kMaxD];
        uint64_t probe;
        key_indices<0>(s, k, h, f, &probe);
        uint32_t m = 0xFFFFFFFFu;
#pragma unroll
        for (int i = 0; i < kMaxD; ++i)
            if (i < (int)s.d) m = min(m, __ldg(s.A + (uint64_t)i * s.w + h[i]));
        q.out[t] = m;
    }
}

}  // namespace

cudaError_t launch_multi_query(const MultiQueryArgs& a, int num_sms, cudaStream_t st) {
    if (a.total == 0) return cudaSuccess;
    static int resident = 0;  // one wave of resident blocks, as for query_kernel
    if (resident == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, multi_query_kernel, kQueryBlock, 0) != cudaSuccess)
            return cudaGetLastError();
        resident = nb > 0 ? nb : 1;
    }
    const uint64_t want = (a.total + kQueryBlock - 1) / kQueryBlock;
    const uint64_t cap = (uint64_t)num_sms * (uint64_t)resident;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    multi_query_kernel<<<grid, kQueryBlock, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_query(const QueryArgs& a, int num_sms, cudaStream_t st) {
    if (a.n == 0) return cudaSuccess;
    switch (a.s.d) {
        case 1: return launch_query_d<1>(a, num_sms, st);
        case 2: return launch_query_d<2>(a, num_sms, st);
        case 3: return launch_query_d<3>(a, num_sms, st);
        case 4: return launch_query_d<4>(a, num_sms, st);
        case 5: return launch_query_d<5>(a, num_sms, st);
        case 6: return launch_query_d<6>(a, num_sms, st);
        case 7: return launch_query_d<7>(a, num_sms, st);
        case 8: return launch_query_d<8>(a, num_sms, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sfk
