// nsk_dg1.cu -- instantiation of the stage kernels for dimension 1 (one
// translation unit per dimension so the library builds in parallel).
#include "nsk_kernels.cuh"

int nsk_launch_stage_d1(const NskParams& p, int np, bool fp32, const NskBuffers& b, const NskLaunch& l,
                        cudaStream_t s) {
  return nsk::launch_stage_np<1>(p, np, fp32, b, l, s);
}

size_t nsk_block_bytes_d1(const NskParams& p, int np, bool fp32) { return nsk::block_bytes_np<1>(p, np, fp32); }
int nsk_launch_block_d1(const NskParams& p, int np, bool fp32, const NskBuffers& b, int mode, const NskLsrkCoef& coef,
                        double dt, int nsteps, void* Rout, cudaStream_t s) {
  return nsk::launch_block_np<1>(p, np, fp32, b, mode, coef, dt, nsteps, Rout, s);
}
