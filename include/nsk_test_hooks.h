/* nsk_test_hooks.h -- test-only entry points of libnsk.so.
 *
 * Not part of the solver's interface (include/nsk.h): these calls exist so that
 * the test suite can drive the library's failure detection from the host,
 * without faulting or hanging a GPU. Production code has no reason to call them.
 * Same conventions as nsk.h: plain C, status codes, never abort. */
#ifndef NSK_TEST_HOOKS_H
#define NSK_TEST_HOOKS_H

#include "nsk.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Failure-detection hook of a batch: writes an arrival count far above any grid
 * size into the batch's grid barrier, so the next barrier of the persistent
 * schedule can never complete. The next nsk_batch_step (persistent schedule)
 * then ends every block's bounded wait after the batch's timeout
 * (nsk_batch_set_timeout) and returns NSK_ERR_TIMEOUT; the batch clears its
 * barrier and error word and stays usable. Synchronises the batch's stream.
 * NSK_ERR_ARG for a NULL batch. */
int nsk_test_hook_block_batch_barrier(nsk_batch* batch);

/* Caps the grid of the persistent tensor-core kernels (the resident-weight
 * GEMM behind nsk_gemm_bf16 and the network's training GEMMs, and the fused
 * inference forward of nsk_mlp_forward) at max_ctas CTAs; 0 (the default)
 * removes the cap (one CTA per SM, or fewer when there are fewer 128-row
 * tiles). With a cap a small problem runs several row tiles per CTA, the
 * schedule of large problems: both TMEM accumulators in turn, and the next
 * tile's loads while the previous tile drains. Process-wide; results are
 * the same with and without a cap. NSK_ERR_ARG for a negative cap. */
int nsk_test_hook_tc_grid_cap(int max_ctas);

/* Selects the kernel of the fused inference forward (nsk_mlp_forward with the
 * fused forward on): 0 (the default) the warp-specialised kernel, whose operands
 * arrive by TMA and whose load, MMA and epilogue stages overlap, wherever it
 * applies (n_out <= 64 and its buffers fit in shared memory); 1 always the
 * kernel that runs the stages one after another. Both perform the same MMAs in
 * the same order with the same epilogue arithmetic. Process-wide. NSK_ERR_ARG
 * for another value. */
int nsk_test_hook_mlp_fwd_kernel(int which);

/* The FP64 reciprocal (fn = 0) and square root (fn = 1) the stage kernels use
 * (Newton-Raphson from the FP32 hardware approximations; CUDA's own division
 * and sqrt outside 2^-120 < x < 2^120), evaluated on the device arrays x -> y
 * of n values on stream, for their accuracy tests. Queued, no
 * synchronisation. NSK_ERR_ARG for another fn, NULL arrays or n < 0. */
int nsk_test_hook_math(int fn, const double* x, double* y, long long n, void* stream);

/* Bounds-checking build only (libnsk_check.so, compiled with -DNSK_BOUNDS_CHECK):
 * makes the context's neighbour strides point far outside the mesh, so that
 * the index checks of its next stage launches fire: they set the error word's
 * bounds bit, keep every access inside its array, and the call returns
 * NSK_ERR_BOUNDS. Use only with the model II stage kernels (separate, fused,
 * lean or single-block schedule), then destroy the context. In the regular
 * library, which has no index checks, it changes nothing and returns
 * NSK_ERR_STATE. */
int nsk_test_hook_corrupt_neighbours(nsk_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* NSK_TEST_HOOKS_H */
