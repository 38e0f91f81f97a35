// sf_microbench.cu -- roofline denominators measured on the device (no sketch arithmetic).
//
// Built into its own library (libsfbench.so), apart from the sketch library: the benchmark and the
// bounded-wait failure test load it; nothing on the sketch path does.  It shares only the device
// header's building blocks (barrier, CAS forms) with the sketch kernels, compiled here on their own.
#include "sf_bench.h"
#include "sf_internal.h"

namespace sfk {

namespace {

// n_words a power of two: index = 40 LCG bits masked; otherwise (n_words <= 2^32) the top 32 bits
// scaled to [0, n_words) by a multiply-shift.
__global__ void __launch_bounds__(256) random_access_kernel(uint32_t* __restrict__ buf, uint64_t n_words,
                                                            uint64_t ops_per_thread, uint32_t kind,
                                                            uint32_t* __restrict__ sink) {
    const bool pow2 = (n_words & (n_words - 1)) == 0;
    const uint64_t mask = n_words - 1;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t x = tid * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    uint32_t acc = 0;
#pragma unroll 8
    for (uint64_t i = 0; i < ops_per_thread; ++i) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;  // Knuth's MMIX LCG
        const uint64_t idx = pow2 ? ((x >> 24) & mask) : (((x >> 32) * n_words) >> 32);
        switch (kind) {
            case SF_BENCH_RED_ADD: atomicAdd(buf + idx, 1u); break;
            case SF_BENCH_ATOM_ADD: acc += atomicAdd(buf + idx, 1u); break;
            case SF_BENCH_LOAD_CG: acc += __ldcg(buf + idx); break;
            case SF_BENCH_RED_MAX: atomicMax(buf + idx, (uint32_t)(x >> 40)); break;
            case SF_BENCH_MIX_RED_LD:  // odd warps load, even warps reduce
                if (threadIdx.x & 32u) acc += __ldcg(buf + idx);
                else atomicAdd(buf + idx, 1u);
                break;
            case SF_BENCH_CAS128: {
                unsigned long long ol, oh;
                cas128(reinterpret_cast<unsigned long long*>(buf + (idx & ~3ull)), 0ull, 0ull, x, tid, ol, oh);
                acc += (uint32_t)(ol ^ oh);
                break;
            }
            default: acc += atomicCAS(buf + idx, 0u, (uint32_t)tid); break;
        }
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps returned values live
}

__global__ void __launch_bounds__(kChunkBlock) barrier_kernel(uint32_t* ctrl, uint32_t n) {
    for (uint32_t i = 0; i < n; ++i)
        if (!grid_barrier(ctrl, (unsigned long long)(i + 1) * gridDim.x, kBarrierTimeoutNs)) return;
}

// Blocks >= gridDim.x - missing skip the barrier; the others wait for them until timeout_ns.
__global__ void __launch_bounds__(kChunkBlock) missing_arrival_kernel(uint32_t* ctrl, uint32_t missing,
                                                                      uint64_t timeout_ns) {
    if (blockIdx.x >= gridDim.x - missing) return;
    grid_barrier(ctrl, (unsigned long long)gridDim.x, timeout_ns);
}

}  // namespace

}  // namespace sfk

extern "C" {

sf_status sf_bench_random_access(uint32_t* buf_dev, uint64_t n_words, uint64_t total_ops, uint32_t kind,
                                 uint32_t grid_blocks, void* cuda_stream) {
    if (!buf_dev || n_words == 0 || kind > SF_BENCH_CAS128) return SF_ERR_INVALID;
    if (kind == SF_BENCH_CAS128 && (((uintptr_t)buf_dev & 15u) != 0 || (n_words & 3u) != 0)) return SF_ERR_INVALID;
    if ((n_words & (n_words - 1)) != 0 && n_words > (1ull << 32)) return SF_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SF_ERR_CUDA;
    const uint32_t grid = grid_blocks ? grid_blocks : (uint32_t)sms * 8u;
    const uint64_t threads = (uint64_t)grid * 256u;
    const uint64_t per = (total_ops + threads - 1) / threads;
    sfk::random_access_kernel<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(buf_dev, n_words, per, kind,
                                                                          buf_dev);
    return cudaGetLastError() == cudaSuccess ? SF_OK : SF_ERR_CUDA;
}

sf_status sf_bench_grid_barrier(void* scratch_dev, uint32_t n_barriers, void* cuda_stream) {
    if (!scratch_dev) return SF_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SF_ERR_CUDA;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sfk::barrier_kernel, sfk::kChunkBlock, 0) != cudaSuccess ||
        bps <= 0)
        return SF_ERR_CUDA;
    if (cudaMemsetAsync(scratch_dev, 0, 256, st) != cudaSuccess) return SF_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sms * (bps < 2 ? bps : 2)));
    cfg.blockDim = dim3(sfk::kChunkBlock);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, sfk::barrier_kernel, (uint32_t*)scratch_dev, n_barriers) != cudaSuccess)
        return SF_ERR_CUDA;
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, scratch_dev, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SF_ERR_CUDA;
    return (err & sfk::kErrTimeout) ? SF_ERR_TIMEOUT : SF_OK;
}

sf_status sf_bench_wait_timeout(void* scratch_dev, uint32_t missing_blocks, uint64_t timeout_ns, void* cuda_stream) {
    if (!scratch_dev || timeout_ns > 1000000000ull) return SF_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SF_ERR_CUDA;
    if (missing_blocks >= (uint32_t)sms) return SF_ERR_INVALID;
    if (cudaMemsetAsync(scratch_dev, 0, 256, st) != cudaSuccess) return SF_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sms);
    cfg.blockDim = dim3(sfk::kChunkBlock);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, sfk::missing_arrival_kernel, (uint32_t*)scratch_dev, missing_blocks, timeout_ns) !=
        cudaSuccess)
        return SF_ERR_CUDA;
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, scratch_dev, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SF_ERR_CUDA;
    return (err & sfk::kErrTimeout) ? SF_ERR_TIMEOUT : SF_OK;
}

}  // extern "C"
