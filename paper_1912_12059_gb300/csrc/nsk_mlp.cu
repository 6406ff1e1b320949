// nsk_mlp.cu -- tensor-core building blocks of the learned c-closure: the tcgen05 BF16
// GEMM exposed through the C ABI (nsk_gemm_bf16) for testing and reuse.
#include "nsk_tc.cuh"

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
