// nsk_aux.cu -- time-step and diagnostics reductions, precision conversion.
#include "nsk_kernels.cuh"

namespace {

template <typename R>
__global__ void __launch_bounds__(256) k_convert(const R* __restrict__ src, void* __restrict__ dst, bool dst64,
                                                 long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (dst64)
      ((double*)dst)[i] = (double)src[i];
    else
      ((float*)dst)[i] = (float)src[i];
  }
}

unsigned reduce_grid(long long n) {
  long long g = (n + 255) / 256;
  return (unsigned)(g < 152 * 8 ? (g > 0 ? g : 1) : 152 * 8);
}

template <typename R, int D>
int launch_dt_t(const NskParams& p, int np, const NskBuffers& b, double cfl, cudaStream_t s) {
  long long npe = 1;
  for (int k = 0; k < D; ++k) npe *= np;
  const long long nn = p.E * npe;
  if (cudaMemsetAsync(b.lam, 0, sizeof(unsigned long long), s) != cudaSuccess) return NSK_ERR_CUDA;
  nsk::k_dt<R, D><<<reduce_grid(nn), 256, 0, s>>>(p, nn, (const R*)b.U, b.lam, b.err);
  nsk::k_dt_final<<<1, 1, 0, s>>>(p, D, np - 1, cfl, b.lam, b.dt);
  return cudaGetLastError() == cudaSuccess ? 2 : NSK_ERR_CUDA;
}

template <typename R, int D, int NP>
int launch_diag_t(const NskParams& p, const NskBuffers& b, cudaStream_t s) {
  nsk::k_diag<R, D, NP><<<b.nparts, 256, 0, s>>>(p, (const R*)b.U, (const R*)b.Q, b.part);
  nsk::k_diag_final<<<1, 256, 0, s>>>(b.nparts, b.part);
  return cudaGetLastError() == cudaSuccess ? 2 : NSK_ERR_CUDA;
}

template <typename R, int D>
int launch_diag_np(const NskParams& p, int np, const NskBuffers& b, cudaStream_t s) {
  switch (np) {
    case 2: return launch_diag_t<R, D, 2>(p, b, s);
    case 3: return launch_diag_t<R, D, 3>(p, b, s);
    case 4: return launch_diag_t<R, D, 4>(p, b, s);
    case 5: return launch_diag_t<R, D, 5>(p, b, s);
    case 6: return launch_diag_t<R, D, 6>(p, b, s);
    default: return NSK_ERR_ARG;
  }
}

}  // namespace

int nsk_launch_dt(const NskParams& p, int dim, int np, bool fp32, const NskBuffers& b, double cfl, cudaStream_t s) {
  switch (dim) {
    case 1: return fp32 ? launch_dt_t<float, 1>(p, np, b, cfl, s) : launch_dt_t<double, 1>(p, np, b, cfl, s);
    case 2: return fp32 ? launch_dt_t<float, 2>(p, np, b, cfl, s) : launch_dt_t<double, 2>(p, np, b, cfl, s);
    case 3: return fp32 ? launch_dt_t<float, 3>(p, np, b, cfl, s) : launch_dt_t<double, 3>(p, np, b, cfl, s);
    default: return NSK_ERR_ARG;
  }
}

int nsk_launch_diag(const NskParams& p, int dim, int np, bool fp32, const NskBuffers& b, cudaStream_t s) {
  switch (dim) {
    case 1: return fp32 ? launch_diag_np<float, 1>(p, np, b, s) : launch_diag_np<double, 1>(p, np, b, s);
    case 2: return fp32 ? launch_diag_np<float, 2>(p, np, b, s) : launch_diag_np<double, 2>(p, np, b, s);
    case 3: return fp32 ? launch_diag_np<float, 3>(p, np, b, s) : launch_diag_np<double, 3>(p, np, b, s);
    default: return NSK_ERR_ARG;
  }
}

int nsk_launch_convert(const void* src, bool src64, void* dst, bool dst64, long long n, cudaStream_t s) {
  if (n <= 0) return 0;
  if (src64)
    k_convert<double><<<reduce_grid(n), 256, 0, s>>>((const double*)src, dst, dst64, n);
  else
    k_convert<float><<<reduce_grid(n), 256, 0, s>>>((const float*)src, dst, dst64, n);
  return cudaGetLastError() == cudaSuccess ? 1 : NSK_ERR_CUDA;
}
