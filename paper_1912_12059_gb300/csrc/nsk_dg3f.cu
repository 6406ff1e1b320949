// nsk_dg3f.cu -- instantiation of the stage kernels for dimension 3 in FP32 (the FP32 operator,
// with the line-per-thread kernels at N = 3); dispatched from nsk_dg3.cu.
#include "nsk_kernels.cuh"

int nsk_launch_stage_d3_fp32(const NskParams& p, int np, const NskBuffers& b, const NskLaunch& l, cudaStream_t s) {
  return nsk::launch_stage_np_r<float, 3>(p, np, b, l, s);
}

size_t nsk_block_bytes_d3_fp32(const NskParams& p, int np) { return nsk::block_bytes_np_r<float, 3>(p, np); }
int nsk_launch_block_d3_fp32(const NskParams& p, int np, const NskBuffers& b, int mode, const NskLsrkCoef& coef,
                             double dt, int nsteps, void* Rout, cudaStream_t s) {
  return nsk::launch_block_np_r<float, 3>(p, np, b, mode, coef, dt, nsteps, Rout, s);
}
