/*
 * sf_bench.h -- measurement kernels of the GB300 SF-sketch library.
 *
 * The paper has no counterpart: these calls measure the roofline denominators the update and
 * query kernels are judged against (random 32-bit atomics and loads on an L2- or HBM-resident
 * buffer, and the cost of one grid-wide barrier of the persistent update kernel).  They touch
 * only the caller's buffer and never a sketch.
 */
#ifndef SF_BENCH_H_
#define SF_BENCH_H_

#include <stdint.h>

#include "sf.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SF_BENCH_RED_ADD   0u  /* atomicAdd, result unused (reduction)   */
#define SF_BENCH_ATOM_ADD  1u  /* atomicAdd, result used                 */
#define SF_BENCH_LOAD_CG   2u  /* 32-bit load bypassing L1               */
#define SF_BENCH_RED_MAX   3u  /* atomicMax, result unused               */
#define SF_BENCH_CAS       4u  /* atomicCAS, result used                 */
#define SF_BENCH_MIX_RED_LD 5u /* even warps atomicAdd (result unused), odd warps 32-bit load bypassing
                                  L1: the 1:1 read-modify-write / load mix of the sketch update (on a
                                  GB300 this schedule measured above alternating the two in one thread) */
#define SF_BENCH_CAS128    6u  /* 128-bit CAS on the 16-byte-aligned group holding the word (result
                                  used): the update's dictionary claim                            */

/*
 * Issues total_ops random 32-bit operations of `kind` on buf_dev[0 .. n_words) (device,
 * caller-owned, contents overwritten; n_words a power of two or at most 2^32, else
 * SF_ERR_INVALID; for SF_BENCH_CAS128 also a multiple of 4, with buf_dev 16-byte aligned) on
 * cuda_stream.  Addresses come from a 64-bit LCG per thread (uniform over the
 * buffer).  grid_blocks = 0 picks 8 blocks of
 * 256 threads per SM.  The caller times the call with CUDA events.
 */
sf_status sf_bench_random_access(uint32_t *buf_dev, uint64_t n_words, uint64_t total_ops, uint32_t kind,
                                 uint32_t grid_blocks, void *cuda_stream);

/*
 * Runs n_barriers grid-wide barriers of the persistent update kernel's kind (cooperative
 * launch, same grid shape), with no other work.  scratch_dev: >= 256 device bytes, zeroed by
 * the call.  Returns SF_ERR_TIMEOUT if a wait gave up (after synchronising the stream).
 */
sf_status sf_bench_grid_barrier(void *scratch_dev, uint32_t n_barriers, void *cuda_stream);

/*
 * Failure-detection check of the bounded device waits: the same barrier loop, but
 * `missing_blocks` blocks of the grid never arrive, so every other block's wait runs out after
 * timeout_ns (at most 1 s here) and the call returns SF_ERR_TIMEOUT with the context still usable.
 * missing_blocks = 0 is a normal run.  No fault and no unbounded wait is involved.
 */
sf_status sf_bench_wait_timeout(void *scratch_dev, uint32_t missing_blocks, uint64_t timeout_ns, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SF_BENCH_H_ */
