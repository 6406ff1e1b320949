// nsk_dg3.cu -- instantiation of the stage kernels for dimension 3 in FP64, and the dispatch of
// the 3D stage launches to the precision's translation unit (the FP32 kernels are in
// nsk_dg3f.cu, so that the two build in parallel).
#include "nsk_kernels.cuh"

int nsk_launch_stage_d3_fp32(const NskParams& p, int np, const NskBuffers& b, const NskLaunch& l, cudaStream_t s);
size_t nsk_block_bytes_d3_fp32(const NskParams& p, int np);
int nsk_launch_block_d3_fp32(const NskParams& p, int np, const NskBuffers& b, int mode, const NskLsrkCoef& coef,
                             double dt, int nsteps, void* Rout, cudaStream_t s);

int nsk_launch_stage_d3(const NskParams& p, int np, bool fp32, const NskBuffers& b, const NskLaunch& l,
                        cudaStream_t s) {
  if (fp32) return nsk_launch_stage_d3_fp32(p, np, b, l, s);
  return nsk::launch_stage_np_r<double, 3>(p, np, b, l, s);
}

size_t nsk_block_bytes_d3(const NskParams& p, int np, bool fp32) {
  return fp32 ? nsk_block_bytes_d3_fp32(p, np) : nsk::block_bytes_np_r<double, 3>(p, np);
}
int nsk_launch_block_d3(const NskParams& p, int np, bool fp32, const NskBuffers& b, int mode, const NskLsrkCoef& coef,
                        double dt, int nsteps, void* Rout, cudaStream_t s) {
  if (fp32) return nsk_launch_block_d3_fp32(p, np, b, mode, coef, dt, nsteps, Rout, s);
  return nsk::launch_block_np_r<double, 3>(p, np, b, mode, coef, dt, nsteps, Rout, s);
}

// a part of a separate-face stage over an element range (FP64, N = 3, 128 or 256 threads)
int nsk_launch_stage_part_d3(const NskParams& p, int np, bool fp32, const NskBuffers& b, const NskLaunch& l,
                             cudaStream_t s, int part, long long e0, long long ne) {
  if (fp32 || np != 4) return NSK_ERR_ARG;
  constexpr int G128 = nsk::group_for<3, 4>(128), G256 = nsk::group_for<3, 4>(256);
  if (l.tpb == 128) return nsk::launch_stage_part<double, 3, 4, G128>(p, b, l, s, part, e0, ne);
  if (l.tpb == 256) return nsk::launch_stage_part<double, 3, 4, G256>(p, b, l, s, part, e0, ne);
  return NSK_ERR_ARG;
}
