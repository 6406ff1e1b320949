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

// ---------------------------------------------------------------------------
// Arithmetic-rate probe (nsk_measure_fma_rate): the FMA throughput of this GPU
// in FP64 and FP32, the denominator of the ALU roofline of the FP64 stage
// kernels. Every thread runs CHAINS independent chains x <- x a + b (a, b
// runtime values: nothing folds) so the pipe, not the dependency latency, is
// the limit; |x| stays near b / (1 - a) = 1 (no overflow, no subnormals).
// ---------------------------------------------------------------------------
namespace {

constexpr int kProbeChains = 8;

template <typename R>
__global__ void __launch_bounds__(256) k_fma_rate(R* __restrict__ sink, const int iters, const R a, const R b) {
  R x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = R(threadIdx.x + c) * R(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += x[c];
  if (s == R(-1)) sink[threadIdx.x] = s;  // never true for these chains; keeps the work alive
}

template <typename R>
int fma_rate_t(int iters, double* tflops, double* ms_out, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return NSK_ERR_CUDA;
  const unsigned blocks = (unsigned)sms * 8;  // 64 resident warps per SM
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return NSK_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return NSK_ERR_CUDA;
  }
  const R a = R(0.999999), b = R(1e-6);
  k_fma_rate<R><<<blocks, 256, 0, s>>>(nullptr, iters / 8 > 0 ? iters / 8 : 1, a, b);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_rate<R><<<blocks, 256, 0, s>>>(nullptr, iters, a, b);
  cudaEventRecord(e1, s);
  int st = NSK_OK;
  float ms = 0.f;
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
    st = NSK_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  const double flops = 2.0 * kProbeChains * (double)iters * (double)blocks * 256.0;
  if (tflops) *tflops = flops / ((double)ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return NSK_OK;
}

}  // namespace

extern "C" int nsk_measure_fma_rate(int precision, int iters, double* tflops, double* ms, void* stream) {
  if (iters < 1 || iters > (1 << 24) || (precision != NSK_FP64 && precision != NSK_FP32_MIXED)) return NSK_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return precision == NSK_FP64 ? fma_rate_t<double>(iters, tflops, ms, s) : fma_rate_t<float>(iters, tflops, ms, s);
}

// ---------------------------------------------------------------------------
// Test hook (include/nsk_test_hooks.h): the stage kernels' FP64 reciprocal and square root on
// device arrays, for their accuracy tests.
// ---------------------------------------------------------------------------
namespace {
__global__ void __launch_bounds__(256) k_math_hook(const int fn, const double* __restrict__ x,
                                                   double* __restrict__ y, const long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fn == 0 ? nsk::rcp_nr(x[i]) : nsk::sqrt_nr(x[i]);
}
}  // namespace

extern "C" int nsk_test_hook_math(int fn, const double* x, double* y, long long n, void* stream) {
  if ((fn != 0 && fn != 1) || !x || !y || n < 0) return NSK_ERR_ARG;
  if (n == 0) return NSK_OK;
  k_math_hook<<<reduce_grid(n), 256, 0, (cudaStream_t)stream>>>(fn, x, y, n);
  return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

// ---- single-block schedule: dispatch by dimension ----
size_t nsk_block_bytes(int dim, const NskParams& p, int np, bool fp32) {
  switch (dim) {
    case 1: return nsk_block_bytes_d1(p, np, fp32);
    case 2: return nsk_block_bytes_d2(p, np, fp32);
    default: return nsk_block_bytes_d3(p, np, fp32);
  }
}

int nsk_launch_block(int dim, const NskParams& p, int np, bool fp32, const NskBuffers& b, int mode,
                     const NskLsrkCoef& coef, double dt, int nsteps, void* Rout, cudaStream_t s) {
  switch (dim) {
    case 1: return nsk_launch_block_d1(p, np, fp32, b, mode, coef, dt, nsteps, Rout, s);
    case 2: return nsk_launch_block_d2(p, np, fp32, b, mode, coef, dt, nsteps, Rout, s);
    default: return nsk_launch_block_d3(p, np, fp32, b, mode, coef, dt, nsteps, Rout, s);
  }
}
