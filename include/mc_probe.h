/*
 * mc_probe.h -- measurement kernels of the benchmark (libmcprobe.so).
 *
 * None of these has a counterpart in the paper (arXiv 2201.13191) and none is
 * part of the method: they measure, on the GPU at hand, the ceilings against
 * which the benchmark states its rooflines.  They live in a library of their
 * own, beside the product library libmc.so (include/mc.h).
 *
 * Every entry point takes device pointers that belong to the caller, enqueues
 * one kernel on `stream` (a cudaStream_t passed as void*, NULL = legacy default
 * stream) without synchronising, and returns MC_PROBE_OK or a negative status.
 */
#ifndef MC_PROBE_H
#define MC_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_PROBE_OK 0
#define MC_PROBE_ERR_INVALID_ARG -1 /* argument out of range */
#define MC_PROBE_ERR_CUDA -3        /* the launch failed */

/* Streaming read bandwidth.  grid x block threads (block a multiple of 32,
 * <= 256) read buf[0 .. n_bytes) (device memory, 16-byte aligned, n_bytes a
 * multiple of 16) in coalesced 16-byte words, `passes` times over, and write
 * one folded word each to sink[thread] (device, grid x block words).  Bytes
 * read per launch: passes x n_bytes.  A buffer that fits in L2 is read from
 * L2 after the first pass; a buffer larger than L2 is read from HBM on every
 * pass.  Errors: INVALID_ARG, CUDA. */
int mc_probe_stream(const void *buf, uint64_t n_bytes, int passes, int grid, int block, uint32_t *sink,
                    void *stream);

/* Random-gather rate.  grid x block threads (block a multiple of 32, <= 256)
 * each perform 8 x rounds independent random 4-byte loads from
 * buf[0 .. n_words) (device memory, n_words < 2^32) and write one folded word
 * to sink[thread] (device, grid x block words).  Loads per launch:
 * 8 x rounds x grid x block, each touching its own 32-byte sector.
 * Errors: INVALID_ARG, CUDA. */
int mc_probe_gather(const void *buf, uint64_t n_words, int rounds, int grid, int block, uint32_t *sink,
                    void *stream);

/* Tensor-core issue rate.  grid CTAs (one per SM) each issue 4 x rounds
 * tcgen05.mma of shape M = 128, N = n (16, 32, 64, 128 or 256), K = 16 on BF16
 * operands resident in shared memory, then wait for them; *err (device int)
 * is set to 1 if a bounded wait gave up.  FLOPs per launch:
 * grid x rounds x 4 x 2 x 128 x n x 16.  Errors: INVALID_ARG, CUDA. */
int mc_probe_mma(int n, int grid, int rounds, int *err, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MC_PROBE_H */
