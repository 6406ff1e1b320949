// nsk_mlp.cu -- tensor-core building blocks of the learned c-closure: the tcgen05 BF16
// GEMM exposed through the C ABI (nsk_gemm_bf16) for testing and reuse.
#include "nsk_kernels.cuh"
#include "nsk_nvtx.h"
#include "nsk_tc.cuh"
#include "nsk_test_hooks.h"

namespace nsk {
namespace tc {
int g_grid_cap = 0;
int g_fwd_kernel = 0;
}  // namespace tc
}  // namespace nsk

extern "C" int nsk_test_hook_mlp_fwd_kernel(int which) {
  if (which < 0 || which > 1) return NSK_ERR_ARG;
  nsk::tc::g_fwd_kernel = which;
  return NSK_OK;
}

extern "C" int nsk_test_hook_tc_grid_cap(int max_ctas) {
  if (max_ctas < 0) return NSK_ERR_ARG;
  nsk::tc::g_grid_cap = max_ctas;
  return NSK_OK;
}

namespace {
__device__ int g_gemm_err;  // error word of calls that pass none
int* default_err() {
  static int* p = nullptr;
  if (!p) {
    void* q = nullptr;
    if (cudaGetSymbolAddress(&q, g_gemm_err) != cudaSuccess) return nullptr;
    p = (int*)q;
  }
  return p;
}
}  // namespace

extern "C" int nsk_gemm_bf16(const void* A, const void* B, int M, int N, int K, int lda, int ldb, int k_split,
                             int epilogue, const float* bias, float* out, int ldo, void* hout, int ldh, void* hout_t,
                             int ldt, const float* zin, int ldz, float* bias_grad, int* err, void* stream) {
  if (!A || !B) return NSK_ERR_ARG;
  if (epilogue < 0 || epilogue > 3) return NSK_ERR_ARG;
  if ((epilogue == nsk::tc::EPI_STORE || epilogue == nsk::tc::EPI_ATOMIC) && !out) return NSK_ERR_ARG;
  if ((epilogue == nsk::tc::EPI_GELU || epilogue == nsk::tc::EPI_DGELU) && !hout) return NSK_ERR_ARG;
  if (epilogue == nsk::tc::EPI_DGELU && !zin) return NSK_ERR_ARG;
  nsk::tc::GemmArgs a;
  a.A = (const __nv_bfloat16*)A;
  a.B = (const __nv_bfloat16*)B;
  a.M = M;
  a.N = N;
  a.K = K;
  a.lda = lda;
  a.ldb = ldb;
  a.k_split = k_split > 0 ? k_split : K;
  a.epi = epilogue;
  a.bias = bias;
  a.out = out;
  a.ldo = ldo;
  a.hout = (__nv_bfloat16*)hout;
  a.ldh = ldh;
  a.hout_t = (__nv_bfloat16*)hout_t;
  a.ldt = ldt;
  a.zin = zin;
  a.ldz = ldz;
  a.bias_grad = bias_grad;
  a.err = err ? err : default_err();
  if (!a.err) return NSK_ERR_CUDA;
  return nsk::tc::launch_gemm(a, (cudaStream_t)stream);
}

// ===========================================================================
// Per-element network of the learned c-closure: n_in -> h1 -> h2 -> n_out,
// GELU hidden layers, BF16 weights and activations, FP32 accumulation on the
// tensor cores (k_gemm_tc), FP32 master parameters and Adam moments.
// ===========================================================================
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

struct nsk_mlp {
  int nin, nin_pad, h1, h2, nout, max_batch, max_rows, ldb;  // ldb: row stride of transposed activations
  cudaStream_t stream;
  size_t nparam, oW1, ob1, oW2, ob2, oW3, ob3;
  float *param, *grad, *m1, *m2;
  __nv_bfloat16 *W1, *W1t, *W2, *W2t, *W3, *W3t;
  // training activations (max_batch rows)
  __nv_bfloat16 *Xt, *H1, *H1t, *H2, *H2t, *dY, *dYt, *dZ2, *dZ2t, *dZ1, *dZ1t;
  float *Z1, *Z2, *Y;
  // inference activations (max_rows rows)
  __nv_bfloat16 *IH1, *IH2;
  double* loss;
  int* err;
  long long adam_step, launches;
  int fused_forward;  // 1 (default): inference forward in one kernel when the network fits
};

namespace {

int round16(int x) { return (x + 15) & ~15; }

__global__ void k_weights_bf16(const float* __restrict__ W, int N, int K, __nv_bfloat16* __restrict__ Wb,
                               __nv_bfloat16* __restrict__ Wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * K) return;
  const int n = i / K, k = i % K;
  const __nv_bfloat16 v = __float2bfloat16_rn(W[i]);
  Wb[i] = v;
  Wt[(size_t)k * N + n] = v;
}

__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ X, int rows, int cols, int ldx,
                                 __nv_bfloat16* __restrict__ Xt, int ldt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)rows * cols) return;
  const int r = (int)(i / cols), c = (int)(i % cols);
  Xt[(size_t)c * ldt + r] = X[(size_t)r * ldx + c];
}

// mean squared error L = sum (Y - T)^2 / (B n); dY = 2 (Y - T) / (B n) in BF16 (and transposed);
// column sums of dY are the gradient of the output bias
__global__ void k_loss_grad(const float* __restrict__ Y, const float* __restrict__ T, int B, int n,
                            __nv_bfloat16* __restrict__ dY, __nv_bfloat16* __restrict__ dYt, int ldt,
                            float* __restrict__ gb3, double* __restrict__ loss) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < (long long)B * n) {
    const int r = (int)(i / n), c = (int)(i % n);
    const float d = Y[i] - T[i];
    l = (double)d * d;
    const float g = 2.0f * d / ((float)B * (float)n);
    const __nv_bfloat16 gb = __float2bfloat16_rn(g);
    dY[i] = gb;
    dYt[(size_t)c * ldt + r] = gb;
    atomicAdd(&gb3[c], g);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

unsigned nb(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

nsk::tc::GemmArgs gemm_args(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                            int epi, int* err) {
  nsk::tc::GemmArgs a;
  memset(&a, 0, sizeof(a));
  a.A = A;
  a.B = B;
  a.lda = lda;
  a.ldb = ldb;
  a.M = M;
  a.N = N;
  a.K = K;
  a.k_split = K;
  a.epi = epi;
  a.err = err;
  return a;
}

int mlp_weights_to_bf16(nsk_mlp* m) {
  k_weights_bf16<<<nb((long long)m->h1 * m->nin_pad), 256, 0, m->stream>>>(m->param + m->oW1, m->h1, m->nin_pad,
                                                                          m->W1, m->W1t);
  k_weights_bf16<<<nb((long long)m->h2 * m->h1), 256, 0, m->stream>>>(m->param + m->oW2, m->h2, m->h1, m->W2, m->W2t);
  k_weights_bf16<<<nb((long long)m->nout * m->h2), 256, 0, m->stream>>>(m->param + m->oW3, m->nout, m->h2, m->W3,
                                                                       m->W3t);
  m->launches += 3;
  return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

// forward + backward of one batch; gradients into m->grad, loss (sum of squares) into m->loss
int mlp_grad(nsk_mlp* m, const __nv_bfloat16* X, const float* T, int B) {
  cudaStream_t s = m->stream;
  int* e = m->err;
  if (cudaMemsetAsync(m->grad, 0, sizeof(float) * m->nparam, s) != cudaSuccess ||
      cudaMemsetAsync(m->loss, 0, sizeof(double), s) != cudaSuccess)
    return NSK_ERR_CUDA;
  int st;
  k_transpose_bf16<<<nb((long long)B * m->nin_pad), 256, 0, s>>>(X, B, m->nin_pad, m->nin_pad, m->Xt, m->ldb);
  nsk::tc::GemmArgs a = gemm_args(X, m->nin_pad, m->W1, m->nin_pad, B, m->h1, m->nin_pad, nsk::tc::EPI_GELU, e);
  a.bias = m->param + m->ob1;
  a.out = m->Z1;
  a.ldo = m->h1;
  a.hout = m->H1;
  a.ldh = m->h1;
  a.hout_t = m->H1t;
  a.ldt = m->ldb;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  a = gemm_args(m->H1, m->h1, m->W2, m->h1, B, m->h2, m->h1, nsk::tc::EPI_GELU, e);
  a.bias = m->param + m->ob2;
  a.out = m->Z2;
  a.ldo = m->h2;
  a.hout = m->H2;
  a.ldh = m->h2;
  a.hout_t = m->H2t;
  a.ldt = m->ldb;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  a = gemm_args(m->H2, m->h2, m->W3, m->h2, B, m->nout, m->h2, nsk::tc::EPI_STORE, e);
  a.bias = m->param + m->ob3;
  a.out = m->Y;
  a.ldo = m->nout;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  k_loss_grad<<<nb((long long)B * m->nout), 256, 0, s>>>(m->Y, T, B, m->nout, m->dY, m->dYt, m->ldb,
                                                          m->grad + m->ob3, m->loss);
  // dZ2 = (dY W3) * GELU'(Z2)
  a = gemm_args(m->dY, m->nout, m->W3t, m->nout, B, m->h2, m->nout, nsk::tc::EPI_DGELU, e);
  a.zin = m->Z2;
  a.ldz = m->h2;
  a.hout = m->dZ2;
  a.ldh = m->h2;
  a.hout_t = m->dZ2t;
  a.ldt = m->ldb;
  a.bias_grad = m->grad + m->ob2;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  // dZ1 = (dZ2 W2) * GELU'(Z1)
  a = gemm_args(m->dZ2, m->h2, m->W2t, m->h2, B, m->h1, m->h2, nsk::tc::EPI_DGELU, e);
  a.zin = m->Z1;
  a.ldz = m->h1;
  a.hout = m->dZ1;
  a.ldh = m->h1;
  a.hout_t = m->dZ1t;
  a.ldt = m->ldb;
  a.bias_grad = m->grad + m->ob1;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  // weight gradients: reduction over the batch (split-K partial sums)
  const int ks = 256;
  a = gemm_args(m->dYt, m->ldb, m->H2t, m->ldb, m->nout, m->h2, B, nsk::tc::EPI_ATOMIC, e);
  a.out = m->grad + m->oW3;
  a.ldo = m->h2;
  a.k_split = ks;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  a = gemm_args(m->dZ2t, m->ldb, m->H1t, m->ldb, m->h2, m->h1, B, nsk::tc::EPI_ATOMIC, e);
  a.out = m->grad + m->oW2;
  a.ldo = m->h1;
  a.k_split = ks;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  a = gemm_args(m->dZ1t, m->ldb, m->Xt, m->ldb, m->h1, m->nin_pad, B, nsk::tc::EPI_ATOMIC, e);
  a.out = m->grad + m->oW1;
  a.ldo = m->nin_pad;
  a.k_split = ks;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  m->launches += 10;
  return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

// inference forward on a given stream and error word (used by the closure on the context's stream)
int mlp_forward_on(nsk_mlp* m, const __nv_bfloat16* X, int rows, float* Y, cudaStream_t s, int* err) {
  int st;
  if (m->fused_forward) {  // one kernel for the three layers when the network fits on chip
    nsk::tc::MlpFwdArgs f;
    f.X = X;
    f.W1 = m->W1;
    f.W2 = m->W2;
    f.W3 = m->W3;
    f.b1 = m->param + m->ob1;
    f.b2 = m->param + m->ob2;
    f.b3 = m->param + m->ob3;
    f.Y = Y;
    f.M = rows;
    f.ldx = m->nin_pad;
    f.ldy = m->nout;
    f.K1 = m->nin_pad;
    f.H1 = m->h1;
    f.H2 = m->h2;
    f.NO = m->nout;
    f.err = err;
    st = nsk::tc::launch_mlp_fwd3(f, s);
    if (st != NSK_ERR_ARG) {
      if (st == NSK_OK) m->launches += 1;
      return st;
    }
  }
  nsk::tc::GemmArgs a = gemm_args(X, m->nin_pad, m->W1, m->nin_pad, rows, m->h1, m->nin_pad, nsk::tc::EPI_GELU, err);
  a.bias = m->param + m->ob1;
  a.hout = m->IH1;
  a.ldh = m->h1;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  a = gemm_args(m->IH1, m->h1, m->W2, m->h1, rows, m->h2, m->h1, nsk::tc::EPI_GELU, err);
  a.bias = m->param + m->ob2;
  a.hout = m->IH2;
  a.ldh = m->h2;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  a = gemm_args(m->IH2, m->h2, m->W3, m->h2, rows, m->nout, m->h2, nsk::tc::EPI_STORE, err);
  a.bias = m->param + m->ob3;
  a.out = Y;
  a.ldo = m->nout;
  if ((st = nsk::tc::launch_gemm(a, s))) return st;
  m->launches += 3;
  return NSK_OK;
}

int mlp_check(nsk_mlp* m, double* loss_out, int B) {
  int h = 0;
  double l = 0.0;
  if (cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return NSK_ERR_CUDA;
  if (h) {
    cudaMemsetAsync(m->err, 0, sizeof(int), m->stream);
    return NSK_ERR_TIMEOUT;
  }
  if (loss_out) *loss_out = l / ((double)B * m->nout);
  return NSK_OK;
}

void mlp_free(nsk_mlp* m) {
  if (!m) return;
  void* ptrs[] = {m->param, m->grad, m->m1, m->m2, m->W1, m->W1t, m->W2, m->W2t, m->W3, m->W3t, m->Xt, m->H1,
                  m->H1t, m->H2, m->H2t, m->dY, m->dYt, m->dZ2, m->dZ2t, m->dZ1, m->dZ1t, m->Z1, m->Z2, m->Y,
                  m->IH1, m->IH2, m->loss, m->err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
}

}  // namespace

extern "C" {

int nsk_mlp_create(nsk_mlp** out, int n_in, int h1, int h2, int n_out, int max_batch, int max_rows, void* stream) {
  if (!out || n_in < 1 || h1 < 16 || h2 < 16 || n_out < 16 || h1 > 256 || h2 > 256 || n_out > 256 || (h1 % 16) ||
      (h2 % 16) || (n_out % 16) || round16(n_in) > 256 || max_batch < 16 || (max_batch % 16) || max_rows < 1)
    return NSK_ERR_ARG;
  *out = nullptr;
  nsk_mlp* m = new (std::nothrow) nsk_mlp();
  if (!m) return NSK_ERR_NOMEM;
  m->nin = n_in;
  m->nin_pad = round16(n_in);
  m->fused_forward = 1;
  m->h1 = h1;
  m->h2 = h2;
  m->nout = n_out;
  m->max_batch = max_batch;
  m->max_rows = max_rows;
  m->ldb = max_batch;
  m->stream = (cudaStream_t)stream;
  m->oW1 = 0;
  m->ob1 = m->oW1 + (size_t)h1 * m->nin_pad;
  m->oW2 = m->ob1 + h1;
  m->ob2 = m->oW2 + (size_t)h2 * h1;
  m->oW3 = m->ob2 + h2;
  m->ob3 = m->oW3 + (size_t)n_out * h2;
  m->nparam = m->ob3 + n_out;
  const size_t B = max_batch, R = max_rows, bf = sizeof(__nv_bfloat16), f4 = sizeof(float);
  struct {
    void** p;
    size_t bytes;
  } al[] = {
      {(void**)&m->param, f4 * m->nparam}, {(void**)&m->grad, f4 * m->nparam},
      {(void**)&m->m1, f4 * m->nparam},    {(void**)&m->m2, f4 * m->nparam},
      {(void**)&m->W1, bf * h1 * m->nin_pad}, {(void**)&m->W1t, bf * h1 * m->nin_pad},
      {(void**)&m->W2, bf * h2 * h1},      {(void**)&m->W2t, bf * h2 * h1},
      {(void**)&m->W3, bf * n_out * h2},   {(void**)&m->W3t, bf * n_out * h2},
      {(void**)&m->Xt, bf * m->nin_pad * B}, {(void**)&m->H1, bf * B * h1},
      {(void**)&m->H1t, bf * B * h1},      {(void**)&m->H2, bf * B * h2},
      {(void**)&m->H2t, bf * B * h2},      {(void**)&m->dY, bf * B * n_out},
      {(void**)&m->dYt, bf * B * n_out},   {(void**)&m->dZ2, bf * B * h2},
      {(void**)&m->dZ2t, bf * B * h2},     {(void**)&m->dZ1, bf * B * h1},
      {(void**)&m->dZ1t, bf * B * h1},     {(void**)&m->Z1, f4 * B * h1},
      {(void**)&m->Z2, f4 * B * h2},       {(void**)&m->Y, f4 * B * n_out},
      {(void**)&m->IH1, bf * R * h1},      {(void**)&m->IH2, bf * R * h2},
      {(void**)&m->loss, sizeof(double)},  {(void**)&m->err, sizeof(int)},
  };
  for (auto& a : al)
    if (cudaMalloc(a.p, a.bytes) != cudaSuccess) {
      cudaGetLastError();
      mlp_free(m);
      return NSK_ERR_NOMEM;
    }
  if (cudaMemset(m->param, 0, f4 * m->nparam) != cudaSuccess || cudaMemset(m->m1, 0, f4 * m->nparam) != cudaSuccess ||
      cudaMemset(m->m2, 0, f4 * m->nparam) != cudaSuccess || cudaMemset(m->err, 0, sizeof(int)) != cudaSuccess) {
    mlp_free(m);
    return NSK_ERR_CUDA;
  }
  *out = m;
  return NSK_OK;
}

long long nsk_mlp_num_params(nsk_mlp* m) { return m ? (long long)m->nparam : -1; }

// flat FP32 layout: W1 [h1][n_in_pad], b1 [h1], W2 [h2][h1], b2 [h2], W3 [n_out][h2], b3 [n_out]
int nsk_mlp_set_params(nsk_mlp* m, const float* host, long long n) {
  if (!m || !host || n != (long long)m->nparam) return NSK_ERR_ARG;
  if (cudaMemcpyAsync(m->param, host, sizeof(float) * m->nparam, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->m1, 0, sizeof(float) * m->nparam, m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->m2, 0, sizeof(float) * m->nparam, m->stream) != cudaSuccess)
    return NSK_ERR_CUDA;
  m->adam_step = 0;
  const int st = mlp_weights_to_bf16(m);
  if (st) return st;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

int nsk_mlp_get_params(nsk_mlp* m, float* host, long long n) {
  if (!m || !host || n != (long long)m->nparam) return NSK_ERR_ARG;
  if (cudaMemcpyAsync(host, m->param, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess)
    return NSK_ERR_CUDA;
  return NSK_OK;
}

int nsk_mlp_set_fused_forward(nsk_mlp* m, int on) {
  if (!m) return NSK_ERR_ARG;
  m->fused_forward = on ? 1 : 0;
  return NSK_OK;
}

int nsk_mlp_forward(nsk_mlp* m, const void* X, int rows, float* Y) {
  const NskRange nvtx_range("nsk_mlp_forward");
  if (!m || !X || !Y || rows < 1 || rows > m->max_rows) return NSK_ERR_ARG;
  return mlp_forward_on(m, (const __nv_bfloat16*)X, rows, Y, m->stream, m->err);
}

int nsk_mlp_gradients(nsk_mlp* m, const void* X, const float* T, int batch, float* grads_host, double* loss) {
  if (!m || !X || !T || batch < 16 || batch > m->max_batch || (batch % 16)) return NSK_ERR_ARG;
  int st = mlp_grad(m, (const __nv_bfloat16*)X, T, batch);
  if (st) return st;
  if (grads_host &&
      cudaMemcpyAsync(grads_host, m->grad, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return NSK_ERR_CUDA;
  return mlp_check(m, loss, batch);
}

int nsk_mlp_train_step(nsk_mlp* m, const void* X, const float* T, int batch, double lr, double* loss) {
  const NskRange nvtx_range("nsk_mlp_train_step");
  if (!m || !X || !T || batch < 16 || batch > m->max_batch || (batch % 16) || !(lr > 0.0)) return NSK_ERR_ARG;
  int st = mlp_grad(m, (const __nv_bfloat16*)X, T, batch);
  if (st) return st;
  m->adam_step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)m->adam_step), c2 = 1.0f - powf(b2, (float)m->adam_step);
  k_adam<<<nb((long long)m->nparam), 256, 0, m->stream>>>(m->param, m->grad, m->m1, m->m2, (long long)m->nparam,
                                                          (float)lr, b1, b2, 1e-8f, c1, c2);
  m->launches += 1;
  if ((st = mlp_weights_to_bf16(m))) return st;
  return loss ? mlp_check(m, loss, batch) : NSK_OK;
}

long long nsk_mlp_launch_count(nsk_mlp* m) { return m ? m->launches : -1; }

void nsk_mlp_destroy(nsk_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  mlp_free(m);
}

}  // extern "C"

// ===========================================================================
// Learned c-closure of a context
// ===========================================================================
namespace {

constexpr float kFeatScale = 0.5f;  // feature scale: density deviations within an element

// Features of element e: the nodal densities minus the element mean, then the means of the
// 2 dim face neighbours minus the element mean (order x-, x+, y-, y+, z-, z+), each divided
// by kFeatScale; every value v is passed as two BF16 numbers, hi = bf16(v) and
// lo = bf16(v - hi) (columns [0, nf) and [nf, 2 nf)), so the tensor cores see about 16
// significant bits of the input. The quasi-equilibrium c - rho is invariant under adding a
// constant to rho, so the element mean itself is not an input.
// element means of rho, one thread per element (16-byte loads where the element's values fill
// whole 16-byte units: many loads in flight per thread)
template <typename R>
__global__ void __launch_bounds__(256) k_elem_mean(const long long E, const int npe, const R* __restrict__ U,
                                                   float* __restrict__ mean) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const R* u = U + e * npe;
  float acc = 0.f;
  if (sizeof(R) == 4 && (npe & 3) == 0) {
    const float4* u4 = reinterpret_cast<const float4*>(u);
    for (int q = 0; q < npe / 4; ++q) {
      const float4 v = u4[q];
      acc += (v.x + v.y) + (v.z + v.w);
    }
  } else {
    for (int n = 0; n < npe; ++n) acc += (float)u[n];
  }
  mean[e] = acc / (float)npe;
}

// the same for FP32 elements of 64 nodes, half a warp per element (lane q loads nodes 4q..4q+3:
// 16-byte loads that together read the element's 256 bytes at once); the sum in the same order,
// ((0 + s_0) + s_1) + ... + s_15 with s_q = (u_4q + u_4q+1) + (u_4q+2 + u_4q+3), gathered by
// shuffles within the half warp
__global__ void __launch_bounds__(256) k_elem_mean64(const long long E, const float* __restrict__ U,
                                                     float* __restrict__ mean) {
  const long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  if (e >= E) return;  // whole half warps: E is counted in elements
  const int q = threadIdx.x & 15;
  const unsigned half = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
  const float4 v = reinterpret_cast<const float4*>(U + e * 64)[q];
  const float sq = (v.x + v.y) + (v.z + v.w);
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) acc += __shfl_sync(half, sq, k, 16);
  if (q == 0) mean[e] = acc / 64.0f;
}

// four elements per warp (their loads issued together), lane f taking features f, f + 32, ... of
// each (no division per value; the face neighbours from the element's Cartesian position)
constexpr int kFeatEpw = 4;
template <typename R, int D>
__global__ void __launch_bounds__(256) k_closure_features(const NskParams p, const int npe, const R* __restrict__ U,
                                                          const float* __restrict__ mean_e,
                                                          __nv_bfloat16* __restrict__ X, const int nin_pad) {
  const long long e0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kFeatEpw;
  const int lane = threadIdx.x & 31;
  const int nf = npe + 2 * D;
#pragma unroll
  for (int q = 0; q < kFeatEpw; ++q) {
    const long long e = e0 + q;
    if (e >= p.E) return;  // uniform over the warp
    const float mean = mean_e[e];
    const nsk::ElemIdx ex = nsk::elem_idx<D>(p, (int)e);
    __nv_bfloat16* row = X + e * nin_pad;
    for (int f = lane; f < nf; f += 32) {
      float v;
      if (f < npe) {
        v = (float)U[e * npe + f] - mean;
      } else {
        const int j = f - npe;
        v = mean_e[nsk::nbr_of(p, ex, j >> 1, (j & 1) ? 1 : -1)] - mean;
      }
      v /= kFeatScale;
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      row[f] = hi;
      row[nf + f] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
    for (int f = 2 * nf + lane; f < nin_pad; f += 32) row[f] = __float2bfloat16_rn(0.f);  // zero padding columns
  }
}

// FP32 3D elements with N = 3 (64 nodes, 70 features, rows of 144 BF16 = 288 bytes): half a
// warp per element; lane q takes nodes 4q..4q+3 (one 16-byte load), writes their four high parts
// (columns 4q.., 8 bytes) and four low parts (columns 70 + 4q.., two 4-byte stores), lanes 0-5
// the face-neighbour means (columns 64 + q and 134 + q), lanes 6-7 the zero padding (140-143):
// every store of a half warp lands in the element's row. The same operations per value as
// k_closure_features.
__global__ void __launch_bounds__(256) k_closure_features64(const NskParams p, const float* __restrict__ U,
                                                            const float* __restrict__ mean_e,
                                                            __nv_bfloat16* __restrict__ X) {
  constexpr int NPE = 64, NF = NPE + 6, PAD = 144;
  const long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  if (e >= p.E) return;
  const int q = threadIdx.x & 15;
  const float mean = mean_e[e];
  unsigned char* row = reinterpret_cast<unsigned char*>(X + e * PAD);
  auto hi_lo = [](float v, uint32_t& hb, uint32_t& lb) {
    const float s = v / kFeatScale;
    const __nv_bfloat16 hi = __float2bfloat16_rn(s);
    hb = __bfloat16_as_ushort(hi);
    lb = __bfloat16_as_ushort(__float2bfloat16_rn(s - __bfloat162float(hi)));
  };
  const float4 t = reinterpret_cast<const float4*>(U + e * NPE)[q];
  uint32_t h[4], l[4];
  hi_lo(t.x - mean, h[0], l[0]);
  hi_lo(t.y - mean, h[1], l[1]);
  hi_lo(t.z - mean, h[2], l[2]);
  hi_lo(t.w - mean, h[3], l[3]);
  *reinterpret_cast<uint2*>(row + 8 * q) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
  *reinterpret_cast<uint32_t*>(row + 2 * NF + 8 * q) = l[0] | (l[1] << 16);
  *reinterpret_cast<uint32_t*>(row + 2 * NF + 8 * q + 4) = l[2] | (l[3] << 16);
  if (q < 6) {
    const nsk::ElemIdx ex = nsk::elem_idx<3>(p, (int)e);
    uint32_t hb, lb;
    hi_lo(mean_e[nsk::nbr_of(p, ex, q >> 1, (q & 1) ? 1 : -1)] - mean, hb, lb);
    *reinterpret_cast<unsigned short*>(row + 2 * (NPE + q)) = (unsigned short)hb;
    *reinterpret_cast<unsigned short*>(row + 2 * (NF + NPE + q)) = (unsigned short)lb;
  } else if (q < 8) {
    *reinterpret_cast<uint32_t*>(row + 2 * (2 * NF) + 4 * (q - 6)) = 0u;
  }
}

template <typename R>
int launch_features(const nsk_ctx* c, const R* U, const float* mean, __nv_bfloat16* X, int nin_pad) {
  if (sizeof(R) == 4 && c->dim == 3 && c->npe == 64 && nin_pad == 144 && ((uintptr_t)X & 15u) == 0) {
    k_closure_features64<<<(unsigned)((c->E * 16 + 255) / 256), 256, 0, c->stream>>>(c->p, (const float*)U, mean, X);
    return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
  }
  const unsigned g = nb((c->E + kFeatEpw - 1) / kFeatEpw * 32);
  if (c->dim == 1)
    k_closure_features<R, 1><<<g, 256, 0, c->stream>>>(c->p, c->npe, U, mean, X, nin_pad);
  else if (c->dim == 2)
    k_closure_features<R, 2><<<g, 256, 0, c->stream>>>(c->p, c->npe, U, mean, X, nin_pad);
  else
    k_closure_features<R, 3><<<g, 256, 0, c->stream>>>(c->p, c->npe, U, mean, X, nin_pad);
  return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

template <typename R>
__global__ void k_closure_apply(const long long nn, const int dim, R* __restrict__ U, const float* __restrict__ Y,
                                const float s) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < nn) U[(long long)(dim + 1) * nn + g] = U[g] + (R)(s * Y[g]);
}

template <typename R>
__global__ void k_closure_targets(const long long nn, const int dim, const R* __restrict__ U, float* __restrict__ Y,
                                  const double inv_s) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < nn) Y[g] = (float)(((double)U[(long long)(dim + 1) * nn + g] - (double)U[g]) * inv_s);
}

// sums of ((beta/alpha) R_c)^2 and (c - rho)^2 over all nodes (FP64)
template <typename R>
__global__ void __launch_bounds__(256) k_closure_judge(const long long nn, const int dim, const R* __restrict__ U,
                                                       const R* __restrict__ Rr, const double ba,
                                                       double* __restrict__ red) {
  double a = 0.0, b = 0.0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nn; g += (long long)gridDim.x * blockDim.x) {
    const double r = ba * (double)Rr[(long long)(dim + 1) * nn + g];
    const double d = (double)U[(long long)(dim + 1) * nn + g] - (double)U[g];
    a += r * r;
    b += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&red[0], a);
    atomicAdd(&red[1], b);
  }
}

double closure_scale(const nsk_ctx* c) { return c->p.kappa / c->p.alpha * c->p.rh[0] * c->p.rh[0]; }

int closure_features(nsk_ctx* c, void* X) {
  const int nin_pad = round16(2 * (c->npe + 2 * c->dim));
  if (!c->cl_mean && cudaMalloc((void**)&c->cl_mean, sizeof(float) * c->E) != cudaSuccess) {
    cudaGetLastError();
    return NSK_ERR_NOMEM;
  }
  float* mean = c->cl_mean;
  int st;
  if (c->precision == NSK_FP32_MIXED) {
    if (c->npe == 64 && ((uintptr_t)c->b.U & 15u) == 0)
      k_elem_mean64<<<(unsigned)((c->E * 16 + 255) / 256), 256, 0, c->stream>>>(c->E, (const float*)c->b.U, mean);
    else
      k_elem_mean<float><<<nb(c->E), 256, 0, c->stream>>>(c->E, c->npe, (const float*)c->b.U, mean);
    st = launch_features<float>(c, (const float*)c->b.U, mean, (__nv_bfloat16*)X, nin_pad);
  } else {
    k_elem_mean<double><<<nb(c->E), 256, 0, c->stream>>>(c->E, c->npe, (const double*)c->b.U, mean);
    st = launch_features<double>(c, (const double*)c->b.U, mean, (__nv_bfloat16*)X, nin_pad);
  }
  c->launches += 2;
  return st;
}

}  // namespace

// c := rho + s y at the nodes of G elements per block, and the traces of the new c on the
// element's faces (the c component of Utr; same arithmetic as the prolongation, so the other
// trace components written by the previous stage stay consistent with it)
template <typename R, int D, int NP, int G>
__global__ void __launch_bounds__(G * nsk::Shape<D, NP>::NPE)
    k_closure_apply_tr(const NskParams p, R* __restrict__ U, const float* __restrict__ Y, const float s,
                       R* __restrict__ Utr) {
  using S = nsk::Shape<D, NP>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NF = S::NF;
  __shared__ R sc[G * NPE];
  const int le = threadIdx.x / NPE, n = threadIdx.x % NPE;
  const int e = blockIdx.x * G + le;
  const bool valid = le < G && e < p.E;
  const size_t nn = (size_t)p.nne;
  const int g = e * NPE + n;
  if (valid) {
    const R cv = U[g] + (R)(s * Y[g]);
    U[(D + 1) * nn + g] = cv;
    sc[le * NPE + n] = cv;
  }
  __syncthreads();
  if (valid) {
    const auto& t = TabSel<R>::get(p);
    R* o = Utr + (size_t)(D + 1) * NF * p.nfe + (e * NFN);
    for (int it = n; it < NF * NFN; it += NPE) {
      const int slot = it / NFN, fn = it % NFN, k = slot >> 1;
      const R* L = (slot & 1) ? t.lp : t.lm;
      const int n0 = nsk::line_base<D, NP>(fn, k), st = nsk::node_stride<NP>(k);
      R acc = 0;
#pragma unroll
      for (int j = 0; j < NP; ++j) acc = fma(L[j], sc[le * NPE + n0 + j * st], acc);
      o[(size_t)slot * p.nfe + fn] = acc;
    }
  }
}

// the same for FP32 3D elements with N = 3, one thread per x-line of 4 nodes (16 per element,
// G elements per block): 16-byte loads and stores, the x-face traces from the thread's own line,
// the y- and z-face traces four face nodes per thread from the staged c (same arithmetic)
template <int G>
__global__ void __launch_bounds__(G * 16)
    k_closure_apply_line(const NskParams p, float* __restrict__ U, const float* __restrict__ Y, const float s,
                         float* __restrict__ Utr) {
  constexpr int NPE = 64, NFN = 16;
  __shared__ __align__(16) float sc[G * NPE];
  const int le = threadIdx.x >> 4, t = threadIdx.x & 15;
  const int e = blockIdx.x * G + le;
  const bool valid = e < p.E;
  const size_t nn = (size_t)p.nne;
  const int g0 = e * NPE + 4 * t;
  const auto& T = TabSel<float>::get(p);
  float* o = Utr + (size_t)4 * 6 * p.nfe + (size_t)e * NFN;  // the c plane of the traces
  float cv[4];
  if (valid) {
    const float4 r = *reinterpret_cast<const float4*>(U + g0);
    const float4 y = *reinterpret_cast<const float4*>(Y + g0);
    cv[0] = r.x + s * y.x;
    cv[1] = r.y + s * y.y;
    cv[2] = r.z + s * y.z;
    cv[3] = r.w + s * y.w;
    const float4 c4 = make_float4(cv[0], cv[1], cv[2], cv[3]);
    *reinterpret_cast<float4*>(U + 4 * nn + g0) = c4;
    *reinterpret_cast<float4*>(sc + le * NPE + 4 * t) = c4;
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {  // x faces at face node t
      const float* L = sd ? T.lp : T.lm;
      float acc = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) acc = fmaf(L[i], cv[i], acc);
      o[(size_t)sd * p.nfe + t] = acc;
    }
  }
  __syncthreads();
  if (valid) {  // y and z faces: four face nodes of one slot per thread
    const int slot = 2 + (t >> 2), k = slot >> 1, g = t & 3;
    const float* L = (slot & 1) ? T.lp : T.lm;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const float4 ln = *reinterpret_cast<const float4*>(sc + le * NPE + 4 * (k == 1 ? jj + 4 * g : g + 4 * jj));
      acc[0] = fmaf(L[jj], ln.x, acc[0]);
      acc[1] = fmaf(L[jj], ln.y, acc[1]);
      acc[2] = fmaf(L[jj], ln.z, acc[2]);
      acc[3] = fmaf(L[jj], ln.w, acc[3]);
    }
    *reinterpret_cast<float4*>(o + (size_t)slot * p.nfe + 4 * g) = make_float4(acc[0], acc[1], acc[2], acc[3]);
  }
}

template <typename R, int D, int NP>
int launch_apply_tr(const nsk_ctx* c, float s, void* utr) {
  if constexpr (std::is_same<R, float>::value && D == 3 && NP == 4) {
    constexpr int GL = 16;
    k_closure_apply_line<GL><<<(unsigned)((c->E + GL - 1) / GL), GL * 16, 0, c->stream>>>(c->p, (float*)c->b.U, c->cl_Y,
                                                                                         s, (float*)utr);
    return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
  }
  constexpr int G = nsk::group_for<D, NP>(256);
  k_closure_apply_tr<R, D, NP, G><<<(unsigned)((c->E + G - 1) / G), G * nsk::Shape<D, NP>::NPE, 0, c->stream>>>(
      c->p, (R*)c->b.U, c->cl_Y, s, (R*)utr);
  return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

template <typename R, int D>
int launch_apply_tr_np(const nsk_ctx* c, float s, void* utr) {
  switch (c->np) {
    case 2: return launch_apply_tr<R, D, 2>(c, s, utr);
    case 3: return launch_apply_tr<R, D, 3>(c, s, utr);
    case 4: return launch_apply_tr<R, D, 4>(c, s, utr);
    case 5: return launch_apply_tr<R, D, 5>(c, s, utr);
    case 6: return launch_apply_tr<R, D, 6>(c, s, utr);
    default: return NSK_ERR_ARG;
  }
}

template <typename R>
int launch_apply_tr_d(const nsk_ctx* c, float s, void* utr) {
  if (c->dim == 1) return launch_apply_tr_np<R, 1>(c, s, utr);
  if (c->dim == 2) return launch_apply_tr_np<R, 2>(c, s, utr);
  return launch_apply_tr_np<R, 3>(c, s, utr);
}

int nsk_closure_apply_ctx(nsk_ctx* c, void* utr) {
  if (!c->mlp || !c->cl_X || !c->cl_Y) return NSK_ERR_STATE;
  int st = closure_features(c, c->cl_X);
  if (st) return st;
  st = mlp_forward_on(c->mlp, (const __nv_bfloat16*)c->cl_X, (int)c->E, c->cl_Y, c->stream, c->b.err);
  if (st) return st;
  c->launches += 3;
  const float s = (float)closure_scale(c);
  if (utr) {
    st = c->precision == NSK_FP32_MIXED ? launch_apply_tr_d<float>(c, s, utr) : launch_apply_tr_d<double>(c, s, utr);
  } else {
    if (c->precision == NSK_FP32_MIXED)
      k_closure_apply<float><<<nb(c->nn), 256, 0, c->stream>>>(c->nn, c->dim, (float*)c->b.U, c->cl_Y, s);
    else
      k_closure_apply<double><<<nb(c->nn), 256, 0, c->stream>>>(c->nn, c->dim, (double*)c->b.U, c->cl_Y, s);
    st = cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
  }
  c->launches += 1;
  return st;
}

int nsk_closure_judge_ctx(nsk_ctx* c) {
  NskLaunch l = {NSK_MODE_RHS, c->rbuf, 0.0, 0.0, nullptr, 0.0, nullptr, c->tpb, c->fused_face};
  int st = nsk_ctx_launch_stage(c, l);
  if (st) return st;
  if (cudaMemsetAsync(c->cl_red, 0, 2 * sizeof(double), c->stream) != cudaSuccess) return NSK_ERR_CUDA;
  const unsigned grid = (unsigned)std::min<long long>((c->nn + 255) / 256, 152 * 8);
  const double ba = c->p.beta / c->p.alpha;
  if (c->precision == NSK_FP32_MIXED)
    k_closure_judge<float><<<grid, 256, 0, c->stream>>>(c->nn, c->dim, (const float*)c->b.U, (const float*)c->rbuf,
                                                        ba, c->cl_red);
  else
    k_closure_judge<double><<<grid, 256, 0, c->stream>>>(c->nn, c->dim, (const double*)c->b.U,
                                                         (const double*)c->rbuf, ba, c->cl_red);
  c->launches += 1;
  double h[2];
  if (cudaMemcpyAsync(h, c->cl_red, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return NSK_ERR_CUDA;
  c->last_eta = h[1] > 0.0 ? sqrt(h[0] / h[1]) : (h[0] > 0.0 ? INFINITY : 0.0);
  if (c->closure_mode == NSK_C_LEARNED && !(c->last_eta <= c->eta_max)) {
    c->closure_mode = NSK_C_EXPLICIT;  // fallback: the explicit c equation takes over from the closure's c
    c->p.closure = 0;
    c->fallbacks += 1;
  }
  return NSK_OK;
}

extern "C" {

int nsk_set_closure(nsk_ctx* c, int mode, nsk_mlp* mlp, int judge_every, double eta_max) {
  if (!c || (mode != NSK_C_EXPLICIT && mode != NSK_C_LEARNED) || judge_every < 0) return NSK_ERR_ARG;
  if (mode == NSK_C_LEARNED && c->p.model == NSK_MODEL_NSK) return NSK_ERR_STATE;  // no c to close
  if (mode == NSK_C_LEARNED && c->fv_path()) return NSK_ERR_STATE;  // sub-cell path: explicit c only
  if (mode == NSK_C_EXPLICIT) {
    c->closure_mode = NSK_C_EXPLICIT;
    c->p.closure = 0;
    return NSK_OK;
  }
  if (!mlp || !(eta_max > 0.0) || !c->params_set) return mlp ? NSK_ERR_STATE : NSK_ERR_ARG;
  if (mlp->nin != 2 * (c->npe + 2 * c->dim) || mlp->nout != c->npe || mlp->max_rows < c->E) return NSK_ERR_ARG;
  for (int k = 1; k < c->dim; ++k)
    if (fabs(c->h[k] - c->h[0]) > 1e-12 * c->h[0]) return NSK_ERR_ARG;  // cubic elements only
  if (!c->cl_X) {  // the context takes the three buffers together or none of them
    const size_t bytes[3] = {sizeof(__nv_bfloat16) * c->E * mlp->nin_pad, sizeof(float) * c->nn, 2 * sizeof(double)};
    void* got[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < 3; ++i) {
      void* q = nullptr;
      if (cudaMalloc(&q, bytes[i]) != cudaSuccess) {
        cudaGetLastError();
        for (int j = 0; j < i; ++j) cudaFree(got[j]);
        return NSK_ERR_NOMEM;
      }
      got[i] = q;
    }
    c->cl_X = got[0];
    c->cl_Y = (float*)got[1];
    c->cl_red = (double*)got[2];
  }
  c->mlp = mlp;
  c->closure_mode = NSK_C_LEARNED;
  c->p.closure = 1;
  c->judge_every = judge_every;
  c->eta_max = eta_max;
  c->last_eta = 0.0;
  c->steps_since_judge = 0;
  return NSK_OK;
}

int nsk_closure_status(nsk_ctx* c, int* mode, double* last_eta, long long* fallbacks) {
  if (!c) return NSK_ERR_ARG;
  if (mode) *mode = c->closure_mode;
  if (last_eta) *last_eta = c->last_eta;
  if (fallbacks) *fallbacks = c->fallbacks;
  return NSK_OK;
}

int nsk_closure_features(nsk_ctx* c, void* X) {
  if (!c || !X) return NSK_ERR_ARG;
  if (!c->state_set) return NSK_ERR_STATE;
  const int st = closure_features(c, X);
  if (st) return st;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

int nsk_closure_targets(nsk_ctx* c, float* Y) {
  if (!c || !Y) return NSK_ERR_ARG;
  if (!c->state_set || !c->params_set) return NSK_ERR_STATE;
  const double inv_s = 1.0 / closure_scale(c);
  if (c->precision == NSK_FP32_MIXED)
    k_closure_targets<float><<<nb(c->nn), 256, 0, c->stream>>>(c->nn, c->dim, (const float*)c->b.U, Y, inv_s);
  else
    k_closure_targets<double><<<nb(c->nn), 256, 0, c->stream>>>(c->nn, c->dim, (const double*)c->b.U, Y, inv_s);
  c->launches += 1;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

int nsk_closure_apply(nsk_ctx* c) {
  if (!c) return NSK_ERR_ARG;
  if (!c->state_set || c->closure_mode != NSK_C_LEARNED) return NSK_ERR_STATE;
  const int st = nsk_closure_apply_ctx(c, nullptr);
  if (st) return st;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

int nsk_closure_judge(nsk_ctx* c, double* eta) {
  if (!c || !eta) return NSK_ERR_ARG;
  if (!c->state_set || !c->cl_red) return NSK_ERR_STATE;
  const int st = nsk_closure_judge_ctx(c);
  if (st) return st;
  *eta = c->last_eta;
  return NSK_OK;
}

}  // extern "C"
