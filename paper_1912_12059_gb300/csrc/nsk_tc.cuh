// nsk_tc.cuh -- BF16 GEMM on the sm_103a tensor cores (tcgen05, accumulators in TMEM).
//
//   C[M x N] = A[M x K] . B[N x K]^T      (A and B BF16, K contiguous; FP32 accumulation)
//
// One CTA of 128 threads owns a 128-row tile of C and the whole N (16 <= N <= 256,
// N % 16 == 0) and a range of K (split-K over gridDim.y). K is consumed in chunks of
// 64: all threads stage the A and B chunks in shared memory in the canonical
// K-major, no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix), one
// elected thread issues the tcgen05.mma instructions (M = 128, K = 16 each) into a
// TMEM accumulator of N FP32 columns, and tcgen05.commit arrives on an mbarrier that
// all threads wait on (bounded in time) before the chunk buffers are reused. The
// epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31,
// i.e. rows 32w..32w+31 of the tile) and applies one of the fused epilogues below.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "nsk_internal.h"

namespace nsk {
namespace tc {

constexpr int kBM = 128;      // rows of C per CTA (TMEM lanes)
constexpr int kKC = 64;       // K chunk staged per pipeline step
constexpr int kMaxN = 256;    // TMEM columns allocated
constexpr int kThreads = 128;
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound of every mbarrier wait

// Upper bound on the grid of the persistent kernels (k_gemm_tc_rb, k_mlp_fwd3), 0 = none (one CTA
// per SM, or fewer when there are fewer row tiles). Set only by the test hook
// nsk_test_hook_tc_grid_cap, so that small problems run several row tiles per CTA.
extern int g_grid_cap;
inline unsigned persistent_grid(int ntiles, int sms) {
  int g = ntiles < sms ? ntiles : sms;
  if (g_grid_cap > 0 && g > g_grid_cap) g = g_grid_cap;
  return (unsigned)g;
}

enum Epilogue : int {
  EPI_STORE = 0,   // C (+ bias) -> FP32 out
  EPI_ATOMIC = 1,  // atomicAdd(out, C): split-K partial sums
  EPI_GELU = 2,    // z = C + bias: z -> zout (FP32, optional), GELU(z) -> hout (BF16), optional transposed copy
  EPI_DGELU = 3,   // dz = C * GELU'(zin): dz -> hout (BF16) and transposed copy, column sums -> bias_grad
};

struct GemmArgs {
  const __nv_bfloat16* A;  // [M][lda]
  const __nv_bfloat16* B;  // [N][ldb]
  int M, N, K, lda, ldb;
  int k_split;             // K per gridDim.y slice (multiple of kKC), or K
  int epi;
  const float* bias;       // [N] or NULL
  float* out;              // FP32 [M][ldo] (STORE, ATOMIC) or z [M][ldo] (GELU, optional)
  int ldo;
  __nv_bfloat16* hout;     // BF16 [M][ldh] (GELU, DGELU)
  int ldh;
  __nv_bfloat16* hout_t;   // BF16 [N][ldt] transposed copy (optional)
  int ldt;
  const float* zin;        // FP32 [M][ldz] pre-activation (DGELU)
  int ldz;
  float* bias_grad;        // [N] column sums (DGELU, optional)
  int* err;                // error word (NSK_EBIT_TIMEOUT on an expired wait)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long tc_global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle. lbo = byte distance between
// core matrices adjacent in K, sbo = between core matrices adjacent in M (or N).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // fixed constant 0b001 in bits 46-48; swizzle mode (61-63) = 0
  return d;
}

// the same for a K-major operand in a swizzled layout (what a TMA box with that swizzle writes):
// rows of 32 (kSw32) or 128 (kSw128) bytes along K, their 16-byte chunks permuted within each
// group of 8 rows, groups sbo bytes apart; a K step inside a row is an offset of the start
// address (the permutation follows the address bits, so the group base must be aligned to the
// group size: 256 or 1024 bytes). The leading byte offset is unused (16 bytes, encoded 1).
constexpr uint32_t kSw32 = 6u, kSw128 = 2u;  // layout type, descriptor bits 61-63
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr, uint32_t sbo, uint32_t layout) {
  return sdesc(saddr, 16u, sbo) | ((uint64_t)layout << 61);
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, shape M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) of a [rows x kKC] chunk in the core-matrix layout
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)((((r >> 3) * (kKC / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// erf after Abramowitz and Stegun, Handbook of Mathematical Functions, Eq. 7.1.26 (a rational
// approximation due to Hastings): erf(y) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-y^2),
// t = 1 / (1 + p y) for y >= 0, odd extension; absolute error <= 1.5e-7 (plus FP32 rounding).
// The GELU epilogues are bound by it, so it is written for few instructions: the argument is
// scaled once, w = x sqrt(log2(e) / 2), so that exp(-y^2) = 2^(-w^2) and p y = (p / sqrt(log2 e)) |w|
// with y = |x| / sqrt 2; the reciprocal and the power of two are the hardware approximations
// (about 1 and 2 ulp), denormal results flushed to zero.
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fast_ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2
__device__ __forceinline__ float gelu(float x) {
  constexpr float kW = 0.84932180028801904f;   // sqrt(log2(e) / 2)
  constexpr float kP = 0.27273748087922250f;   // 0.3275911 / sqrt(log2(e))
  // every product rounded on its own (no contraction), as gelu2 below repeats it
  const float w = __fmul_rn(x, kW);
  const float aw = fabsf(w);
  const float t = fast_rcp(fmaf(kP, aw, 1.0f));
  const float poly = __fmul_rn(
      t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f));
  const float erf_abs = fmaf(-poly, fast_ex2(-__fmul_rn(w, w)), 1.0f);  // erf(|x| / sqrt 2)
  const float h = __fmul_rn(0.5f, x);
  return fmaf(h, copysignf(erf_abs, x), h);
}
// the same GELU on two values at once, operation for operation (the packed FP32 instructions round
// each lane as the scalar ones do, so the results equal gelu's bit for bit): half the FP32
// instructions of two scalar evaluations; the Horner coefficients are negated so that the
// negation of the polynomial is exact and free
__device__ __forceinline__ float2 f2s(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 gelu2(float2 x) {
  const float2 w = __fmul2_rn(x, f2s(0.84932180028801904f));
  const float2 aw = make_float2(fabsf(w.x), fabsf(w.y));
  const float2 d = __ffma2_rn(f2s(0.27273748087922250f), aw, f2s(1.0f));
  const float2 t = make_float2(fast_rcp(d.x), fast_rcp(d.y));
  float2 pn = __ffma2_rn(t, f2s(-1.061405429f), f2s(1.453152027f));
  pn = __ffma2_rn(t, pn, f2s(-1.421413741f));
  pn = __ffma2_rn(t, pn, f2s(0.284496736f));
  pn = __ffma2_rn(t, pn, f2s(-0.254829592f));
  const float2 poly_neg = __fmul2_rn(t, pn);  // -poly of gelu
  const float2 ww = __fmul2_rn(w, w);
  const float2 e = make_float2(fast_ex2(-ww.x), fast_ex2(-ww.y));
  const float2 erf_abs = __ffma2_rn(poly_neg, e, f2s(1.0f));
  const float2 h = __fmul2_rn(x, f2s(0.5f));
  return __ffma2_rn(h, make_float2(copysignf(erf_abs.x, x.x), copysignf(erf_abs.y, x.y)), h);
}
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.3989422804014327f * __expf(-0.5f * x * x);
}

// stage rows [0, nrows) of a chunk of a K-major BF16 matrix (row stride ld) at column k0
// into shared memory; rows beyond `valid_rows` and columns beyond `kmax` are zero
__device__ __forceinline__ void stage_chunk(unsigned char* s, const __nv_bfloat16* g, int ld, int nrows,
                                            int valid_rows, int k0, int kmax) {
  for (int idx = threadIdx.x; idx < nrows * (kKC / 8); idx += kThreads) {
    const int r = idx / (kKC / 8), j = idx % (kKC / 8);
    const int k = k0 + j * 8;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r < valid_rows && k < kmax) v = *reinterpret_cast<const uint4*>(g + (size_t)r * ld + k);
    *reinterpret_cast<uint4*>(s + core_off(r, j * 8)) = v;
  }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, int* err) {
  const unsigned long long t0 = tc_global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
    if (tc_global_ns() - t0 > kWaitNs) {
      atomicOr(err, NSK_EBIT_TIMEOUT);
      return false;
    }
  }
}

// epilogue of 32 accumulator columns [c0, c0 + 32) of row m (valid if rv) held in v
__device__ __forceinline__ void epilogue_chunk(const GemmArgs& a, const int m, const bool rv, const int c0,
                                               const uint32_t* v, const int lane) {
  const int ncol = min(32, a.N - c0);
  float colsum[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    colsum[j] = 0.f;
    if (j >= ncol) continue;
    const int n = c0 + j;
    float x = __uint_as_float(v[j]);
    if (a.epi == EPI_STORE) {
      if (rv) a.out[(size_t)m * a.ldo + n] = x + (a.bias ? a.bias[n] : 0.f);
    } else if (a.epi == EPI_ATOMIC) {
      if (rv) atomicAdd(&a.out[(size_t)m * a.ldo + n], x);
    } else if (a.epi == EPI_GELU) {
      const float z = x + (a.bias ? a.bias[n] : 0.f);
      if (rv) {
        if (a.out) a.out[(size_t)m * a.ldo + n] = z;
        const __nv_bfloat16 h = __float2bfloat16_rn(gelu(z));
        a.hout[(size_t)m * a.ldh + n] = h;
        if (a.hout_t) a.hout_t[(size_t)n * a.ldt + m] = h;
      }
    } else {  // EPI_DGELU
      const float dz = rv ? x * gelu_grad(a.zin[(size_t)m * a.ldz + n]) : 0.f;
      if (rv) {
        const __nv_bfloat16 h = __float2bfloat16_rn(dz);
        a.hout[(size_t)m * a.ldh + n] = h;
        if (a.hout_t) a.hout_t[(size_t)n * a.ldt + m] = h;
      }
      colsum[j] = dz;
    }
  }
  if (a.epi == EPI_DGELU && a.bias_grad) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float s = colsum[j];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0 && j < ncol) atomicAdd(&a.bias_grad[c0 + j], s);
    }
  }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                         // kBM x kKC BF16 = 16 KB
  unsigned char* sB = smem + kBM * kKC * 2;         // kMaxN x kKC BF16 = 32 KB
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int aborted;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM;
  const int kb = blockIdx.y * a.k_split;
  const int ke = min(a.K, kb + a.k_split);
  const int rowsA = min(kBM, a.M - m0);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kMaxN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    aborted = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(kBM, a.N);
  uint32_t phase = 0;

  for (int k0 = kb; k0 < ke; k0 += kKC) {
    stage_chunk(sA, a.A + (size_t)m0 * a.lda, a.lda, kBM, rowsA, k0, ke);
    stage_chunk(sB, a.B, a.ldb, a.N, a.N, k0, ke);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int nk = min(kKC, ke - k0) / 16;
      for (int s = 0; s < nk; ++s) {
        // a K step of 16 spans two core matrices along K (2 x 128 bytes)
        const uint64_t ad = sdesc(smem_u32(sA) + s * 256, 128, (kKC / 8) * 128);
        const uint64_t bd = sdesc(smem_u32(sB) + s * 256, 128, (kKC / 8) * 128);
        const uint32_t acc = (k0 > kb || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar)));
    }
    const bool ok = mbar_wait(smem_u32(&mbar), phase, a.err);
    phase ^= 1u;
    if (!ok) aborted = 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (aborted) break;
  }

  if (!aborted && ke > kb) {
    const int r = warp * 32 + lane;  // row of the tile owned by this thread
    const int m = m0 + r;
    const bool rv = m < a.M;
    for (int c0 = 0; c0 < a.N; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
            "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
            "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      epilogue_chunk(a, m, rv, c0, v, lane);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMaxN));
}

// 48 KB of operand chunks; the launch requests 80 KB so that at most two CTAs share an SM
// and their two 256-column TMEM allocations never contend (512 columns per SM)
constexpr int kSmemBytes = 80 * 1024;

// ---------------------------------------------------------------------------
// Persistent variant for a weight matrix B that fits in shared memory (K <= 256,
// N % 64 == 0): B is staged once per CTA and stays resident; the CTA walks over
// 128-row tiles of A with two TMEM accumulators (all 512 columns) so that the
// epilogue of tile i-1 (8 warps: warp w reads lanes 32 (w % 4).. and the column
// half w / 4) runs while the tensor cores compute tile i. Operands are staged
// with cp.async (16-byte copies straight into the core-matrix layout).
// ---------------------------------------------------------------------------
constexpr int kRbThreads = 256;
constexpr int kRbSmemMin = 116 * 1024;  // forces one CTA per SM: it owns all 512 TMEM columns
constexpr int kRbStageBytes = 8 * 32 * 33 * 4;  // eight warps' epilogue staging blocks
constexpr int kRbSmemMax = 256 * 256 * 2 + 128 * 256 * 2 + kRbStageBytes;  // B, A tiles at K = N = 256, staging

__device__ __forceinline__ uint32_t core_off_k(int r, int k, int K) {
  return (uint32_t)((((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(src_bytes) : "memory");
}

__host__ __device__ constexpr int rb_b_bytes(int N, int K) { return ((N * K * 2) + 1023) & ~1023; }

constexpr int kStage = 32 * 33;  // floats of one warp's 32 x 32 staging block (padded rows)

// write the 32 x 32 block held transposed in `st` (st[r * 33 + c], row r = lane of the producer)
// to rows row0.. of a row-major matrix with 16-byte vector stores (rows beyond rows_valid skipped)
__device__ __forceinline__ void store_block_f32(const float* st, float* out, size_t ld, int row0, int col0,
                                                int rows_valid, int lane) {
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int r = it * 4 + (lane >> 3), c = (lane & 7) * 4;
    if (r < rows_valid) {
      const float4 v = make_float4(st[r * 33 + c], st[r * 33 + c + 1], st[r * 33 + c + 2], st[r * 33 + c + 3]);
      *reinterpret_cast<float4*>(out + (size_t)(row0 + r) * ld + col0 + c) = v;
    }
  }
}
__device__ __forceinline__ void store_block_bf16(const float* st, __nv_bfloat16* out, size_t ld, int row0, int col0,
                                                 int rows_valid, int lane) {
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int r = it * 8 + (lane >> 2), c = (lane & 3) * 8;
    if (r < rows_valid) {
      __align__(16) __nv_bfloat16 h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) h[j] = __float2bfloat16_rn(st[r * 33 + c + j]);
      *reinterpret_cast<uint4*>(out + (size_t)(row0 + r) * ld + col0 + c) = *reinterpret_cast<const uint4*>(h);
    }
  }
}

// epilogue of the resident-B kernel for 32 columns [c0, c0 + 32) of the warp's 32 rows
// (row0 = first row, lane = row offset); outputs go through the warp's staging block
__device__ __forceinline__ void epilogue_chunk_rb(const GemmArgs& a, const int row0, const int lane, const int c0,
                                                  const uint32_t* v, float* st) {
  const int m = row0 + lane;
  const int rows_valid = a.M - row0;
  const bool rv = lane < rows_valid;
  float x[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) x[j] = __uint_as_float(v[j]) + ((a.epi != EPI_DGELU && a.bias) ? a.bias[c0 + j] : 0.f);
  if (a.epi == EPI_STORE || (a.epi == EPI_GELU && a.out)) {
#pragma unroll
    for (int j = 0; j < 32; ++j) st[lane * 33 + j] = x[j];
    __syncwarp();
    store_block_f32(st, a.out, a.ldo, row0, c0, rows_valid, lane);
    __syncwarp();
    if (a.epi == EPI_STORE) return;
  }
  if (a.epi == EPI_DGELU) {  // stage the pre-activations of the block (coalesced loads)
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int r = it * 4 + (lane >> 3), c = (lane & 7) * 4;
      if (r < rows_valid) {
        const float4 z = *reinterpret_cast<const float4*>(a.zin + (size_t)(row0 + r) * a.ldz + c0 + c);
        st[r * 33 + c] = z.x;
        st[r * 33 + c + 1] = z.y;
        st[r * 33 + c + 2] = z.z;
        st[r * 33 + c + 3] = z.w;
      }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = rv ? x[j] * gelu_grad(st[lane * 33 + j]) : 0.f;
    __syncwarp();
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = gelu(x[j]);
  }
  if (a.epi == EPI_DGELU && a.bias_grad) {  // column sums of the FP32 values
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float sum = x[j];
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) atomicAdd(&a.bias_grad[c0 + j], sum);
    }
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) st[lane * 33 + j] = x[j];
  __syncwarp();
  store_block_bf16(st, a.hout, a.ldh, row0, c0, rows_valid, lane);
  __syncwarp();
  if (a.hout_t && rv) {
#pragma unroll
    for (int j = 0; j < 32; ++j) a.hout_t[(size_t)(c0 + j) * a.ldt + m] = __float2bfloat16_rn(x[j]);
  }
}

__global__ void __launch_bounds__(kRbThreads, 1) k_gemm_tc_rb(const GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int K = a.K, N = a.N;
  unsigned char* sB = smem;
  unsigned char* sA = smem + rb_b_bytes(N, K);
  float* stage = reinterpret_cast<float*>(sA + kBM * K * 2) + (threadIdx.x >> 5) * kStage;
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int aborted;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, half = warp >> 2;
  const int ntiles = (a.M + kBM - 1) / kBM;
  const int kc = K >> 3;  // 16-byte chunks per row

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    aborted = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // resident B
  const uint32_t sBa = smem_u32(sB), sAa = smem_u32(sA);
  for (int idx = threadIdx.x; idx < N * kc; idx += kRbThreads) {
    const int r = idx / kc, j = idx % kc;
    cp_async16(sBa + core_off_k(r, j * 8, K), a.B + (size_t)r * a.ldb + j * 8, 16);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(kBM, N);
  uint32_t ph[2] = {0u, 0u};
  int prev_tile = -1;

  for (int t = blockIdx.x, i = 0;; t += gridDim.x, ++i) {
    const bool have = t < ntiles;
    if (i > 0) {  // the MMAs of tile i-1 must be done before its A buffer is refilled
      const int b = (i - 1) & 1;
      const bool ok = mbar_wait(smem_u32(&mbar[b]), ph[b], a.err);
      ph[b] ^= 1u;
      if (!ok) aborted = 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (have) {
      const int m0 = t * kBM;
      for (int idx = threadIdx.x; idx < kBM * kc; idx += kRbThreads) {
        const int r = idx / kc, j = idx % kc;
        const bool v = m0 + r < a.M;
        cp_async16(sAa + core_off_k(r, j * 8, K), v ? (const void*)(a.A + (size_t)(m0 + r) * a.lda + j * 8)
                                                    : (const void*)a.A, v ? 16 : 0);
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (aborted) break;
    if (have && threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t d = tmem + (uint32_t)((i & 1) * 256);
      for (int st = 0; st < K / 16; ++st) {
        const uint64_t ad = sdesc(sAa + st * 256, 128, kc * 128);
        const uint64_t bd = sdesc(sBa + st * 256, 128, kc * 128);
        const uint32_t acc = st > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar[i & 1])));
    }
    if (prev_tile >= 0) {  // epilogue of the previous tile overlaps the MMAs just issued
      const int row0 = prev_tile * kBM + q * 32;
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(((i - 1) & 1) * 256);
      for (int c0 = half * (N / 2); c0 < (half + 1) * (N / 2); c0 += 32) {
        uint32_t v[32];
        tmem_ld32(base + (uint32_t)c0, v);
        epilogue_chunk_rb(a, row0, lane, c0, v, stage);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
    if (!have) break;
    prev_tile = t;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------------------
// Fused inference forward of the closure network, Y = W3 g(W2 g(W1 X + b1) + b2) + b3
// (g = GELU), for one 128-row tile at a time: the hidden activations never leave the SM.
// One CTA of 512 threads per SM owns all 512 TMEM columns: layer 1 accumulates in columns
// [0, H1), layer 2 in [256, 256 + H2), layer 3 in [0, NO) again (layer 1 is drained by then).
// Shared memory: W2 resident ([H2][H1], loaded once), the row tile (X, then g(layer 1), then
// g(layer 2), each in the K-major core-matrix layout the next MMA reads), and one streaming
// buffer for the 64-column chunks of W1 and then for W3 (the next tile's rows and first W1
// chunk are loaded while layer 3 drains). The epilogues of warp w read TMEM lanes 32 (w % 4)..
// and 32-column chunks w / 4, w / 4 + 4, ...; GELU and the BF16 rounding
// are the same as the per-layer kernels', and so is the order of the MMAs along K, so the
// result equals the three-GEMM chain.
// ---------------------------------------------------------------------------
struct MlpFwdArgs {
  const __nv_bfloat16* X;  // [M][ldx], columns [0, K1) used
  const __nv_bfloat16* W1; // [H1][K1]
  const __nv_bfloat16* W2; // [H2][H1]
  const __nv_bfloat16* W3; // [NO][H2]
  const float *b1, *b2, *b3;
  float* Y;                // [M][ldy]
  int M, ldx, ldy, K1, H1, H2, NO;
  int* err;
};
constexpr int kFwThreads = 512;
constexpr int kFwWarps = kFwThreads / 32;
constexpr int kFwChunk = 64;  // K columns of W1 per streaming step

__host__ __device__ inline int fw_align(int b) { return (b + 1023) & ~1023; }
__host__ __device__ inline int fw_w2_bytes(const MlpFwdArgs& a) { return fw_align(a.H2 * a.H1 * 2); }
__host__ __device__ inline int fw_xh_bytes(const MlpFwdArgs& a) {
  const int kx = a.K1 > a.H1 ? (a.K1 > a.H2 ? a.K1 : a.H2) : (a.H1 > a.H2 ? a.H1 : a.H2);
  return fw_align(kBM * kx * 2);
}
__host__ __device__ inline int fw_ws_bytes(const MlpFwdArgs& a) {
  const int w1 = a.H1 * kFwChunk * 2, w3 = a.NO * a.H2 * 2;
  return fw_align(w1 > w3 ? w1 : w3);
}
__host__ __device__ inline int fw_smem_bytes(const MlpFwdArgs& a) {
  return fw_w2_bytes(a) + fw_xh_bytes(a) + fw_ws_bytes(a);
}

// accumulator columns [0, N) of the warp's 32 rows -> + bias -> GELU -> BF16 into the row tile
// (layout with K = N) in shared memory; warp w: TMEM lanes 32 (w % 4).., 32-column chunks
// w / 4, w / 4 + 4, ...
// (the warp's lanes share the columns: lane j loads the bias of column c0 + j, shuffles broadcast it)
__device__ __forceinline__ void fw_gelu_to_smem(uint32_t tacc, int N, const float* __restrict__ bias,
                                                unsigned char* sxh, int warp, int lane) {
  const int q = warp & 3, part = warp >> 2, r = q * 32 + lane;
  for (int c0 = part * 32; c0 < N; c0 += 32 * (kFwWarps / 4)) {
    const float bl = c0 + lane < N ? bias[c0 + lane] : 0.f;
    uint32_t v[32];
    tmem_ld32(tacc + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const int c = c0 + g * 8;
      __align__(16) __nv_bfloat16 h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        h[j] = __float2bfloat16_rn(gelu(__uint_as_float(v[g * 8 + j]) + __shfl_sync(0xffffffffu, bl, g * 8 + j)));
      if (c < N) *reinterpret_cast<uint4*>(sxh + core_off_k(r, c, N)) = *reinterpret_cast<const uint4*>(h);
    }
  }
}

__device__ __forceinline__ void fw_mma(uint32_t d, uint32_t sa, uint32_t sb, int lda_k, int ldb_k, int ksteps,
                                       uint32_t idesc, bool accumulate) {
  for (int s = 0; s < ksteps; ++s) {
    const uint64_t ad = sdesc(sa + s * 256, 128, (uint32_t)(lda_k / 8) * 128);
    const uint64_t bd = sdesc(sb + s * 256, 128, (uint32_t)(ldb_k / 8) * 128);
    const uint32_t acc = (accumulate || s > 0) ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void fw_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

// cp.async of the row tile t of X and of the first 64-column chunk of W1
__device__ __forceinline__ void fw_load_tile(const MlpFwdArgs& a, int t, uint32_t aXH, uint32_t aWs) {
  const int m0 = t * kBM;
  for (int idx = threadIdx.x; idx < kBM * (a.K1 / 8); idx += kFwThreads) {
    const int r = idx / (a.K1 / 8), j = idx % (a.K1 / 8);
    const bool v = m0 + r < a.M;
    cp_async16(aXH + core_off_k(r, j * 8, a.K1), v ? (const void*)(a.X + (size_t)(m0 + r) * a.ldx + j * 8)
                                                   : (const void*)a.X, v ? 16 : 0);
  }
}
__device__ __forceinline__ void fw_load_w1(const MlpFwdArgs& a, int kc, uint32_t aWs) {
  const int kw = min(kFwChunk, a.K1 - kc);
  for (int idx = threadIdx.x; idx < a.H1 * (kw / 8); idx += kFwThreads) {
    const int r = idx / (kw / 8), j = idx % (kw / 8);
    cp_async16(aWs + core_off_k(r, j * 8, kFwChunk), a.W1 + (size_t)r * a.K1 + kc + j * 8, 16);
  }
}

__global__ void __launch_bounds__(kFwThreads, 1) k_mlp_fwd3(const MlpFwdArgs a) {
  // its own dynamic-shared-memory symbol: the 16-byte alignment keeps the static area at a few
  // bytes (tcgen05 no-swizzle operands and cp.async need 16-byte alignment only)
  extern __shared__ __align__(16) unsigned char fw_smem[];
  unsigned char* sW2 = fw_smem;
  unsigned char* sXH = fw_smem + fw_w2_bytes(a);
  unsigned char* sWs = sXH + fw_xh_bytes(a);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int aborted;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (a.M + kBM - 1) / kBM;
  const uint32_t aW2 = smem_u32(sW2), aXH = smem_u32(sXH), aWs = smem_u32(sWs);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    aborted = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  for (int idx = threadIdx.x; idx < a.H2 * (a.H1 / 8); idx += kFwThreads) {  // resident W2
    const int r = idx / (a.H1 / 8), j = idx % (a.H1 / 8);
    cp_async16(aW2 + core_off_k(r, j * 8, a.H1), a.W2 + (size_t)r * a.H1 + j * 8, 16);
  }
  if ((int)blockIdx.x < ntiles) {
    fw_load_tile(a, blockIdx.x, aXH, aWs);
    fw_load_w1(a, 0, aWs);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tm = tmem_slot;
  uint32_t ph = 0;

  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int m0 = t * kBM;
    // layer 1: W1 streamed in 64-column chunks of K (the tile and chunk 0 are already on their way)
    for (int kc = 0; kc < a.K1; kc += kFwChunk) {
      const int kw = min(kFwChunk, a.K1 - kc);
      if (kc > 0) fw_load_w1(a, kc, aWs);
      asm volatile("cp.async.wait_all;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        fw_mma(tm, aXH + (uint32_t)(kc / 8) * 128, aWs, a.K1, kFwChunk, kw / 16, idesc_bf16(kBM, a.H1), kc > 0);
        fw_commit(&mbar);
      }
      if (!mbar_wait(smem_u32(&mbar), ph, a.err)) aborted = 1;
      ph ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
    __syncthreads();
    if (aborted) break;
    for (int idx = threadIdx.x; idx < a.NO * (a.H2 / 8); idx += kFwThreads) {  // W3 (lands during epilogues)
      const int r = idx / (a.H2 / 8), j = idx % (a.H2 / 8);
      cp_async16(aWs + core_off_k(r, j * 8, a.H2), a.W3 + (size_t)r * a.H2 + j * 8, 16);
    }
    fw_gelu_to_smem(tm, a.H1, a.b1, sXH, warp, lane);
    asm volatile("tcgen05.fence::before_thread_sync;");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // layer 2: g(layer 1) x W2^T -> columns [256, 256 + H2)
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      fw_mma(tm + 256u, aXH, aW2, a.H1, a.H1, a.H1 / 16, idesc_bf16(kBM, a.H2), false);
      fw_commit(&mbar);
    }
    if (!mbar_wait(smem_u32(&mbar), ph, a.err)) aborted = 1;
    ph ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (aborted) break;
    fw_gelu_to_smem(tm + 256u, a.H2, a.b2, sXH, warp, lane);
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // layer 3: g(layer 2) x W3^T -> columns [0, NO)
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      fw_mma(tm, aXH, aWs, a.H2, a.H2, a.H2 / 16, idesc_bf16(kBM, a.NO), false);
      fw_commit(&mbar);
    }
    if (!mbar_wait(smem_u32(&mbar), ph, a.err)) aborted = 1;
    ph ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (aborted) break;
    // the row tile and the streaming buffer are free: start the next tile's loads, then drain layer 3
    if (t + (int)gridDim.x < ntiles) {
      fw_load_tile(a, t + gridDim.x, aXH, aWs);
      fw_load_w1(a, 0, aWs);
    }
    {
      const int q = warp & 3, part = warp >> 2, r = q * 32 + lane;
      const bool rv = m0 + r < a.M;
      for (int c0 = part * 32; c0 < a.NO; c0 += 32 * (kFwWarps / 4)) {
        const float bl = c0 + lane < a.NO ? a.b3[c0 + lane] : 0.f;
        uint32_t v[32];
        tmem_ld32(tm + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        float o[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) o[j] = __uint_as_float(v[j]) + __shfl_sync(0xffffffffu, bl, j);
        if (rv) {
          float* y = a.Y + (size_t)(m0 + r) * a.ldy + c0;
#pragma unroll
          for (int g = 0; g < 8; ++g)
            if (c0 + g * 4 < a.NO)
              *reinterpret_cast<float4*>(y + g * 4) = make_float4(o[g * 4], o[g * 4 + 1], o[g * 4 + 2], o[g * 4 + 3]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // TMEM columns are reused by the next tile
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(512));
}

// ---------------------------------------------------------------------------
// Warp-specialised fused forward: the same network, the same MMAs in the same K order and the
// same GELU and BF16 rounding as k_mlp_fwd3, with the stages overlapped:
//  - operands arrive by TMA (cp.async.bulk.tensor, boxes 8 K columns wide that land directly in
//    the K-major no-swizzle core-matrix layout below); one warp loads the row tiles and W1, one
//    W2 and W3, one warp issues the MMAs of layers 2 and 3, one those of layer 1, and
//    kWsEpiWarps warps run the epilogues; every role blocks only on its own barriers;
//  - W2 stays resident; the row tile X and W1 stream together through a ring of entries, one
//    16-column slab of each per layer-1 K step, and W3 through a ring of two 64-column chunks;
//  - a layer's activations are written in 64-column chunks into a two-slot ring, and the next
//    layer's MMAs consume chunk c while the epilogue produces chunk c + 1;
//  - layer 1 of the next tile accumulates in TMEM columns [0, H1) while the epilogue works on
//    layer 2 ([256, 256 + H2)) and drains layer 3 ([256, 256 + NO), NO <= 64: inside layer 2's
//    first chunk, which the epilogue has read before the first layer-3 MMA is issued); the two
//    MMA warps issue independently (disjoint accumulators; each commit tracks its own thread's
//    MMAs), so that layer 1 of the next tile streams while layer 3 waits for activations;
//  - the epilogue stages its layer-3 block in the activation slots (in bytes only its own warp
//    writes there) and stores it 64 bytes per row, eight rows per warp instruction.
// Operand layouts in shared memory, chosen for few TMA requests (one per box row): the row-tile
// and W1 slabs are boxes of 16 K columns (32-byte rows, 32-byte swizzle), W2 and the W3 chunks
// boxes of 64 K columns (128-byte rows, 128-byte swizzle, W2's boxes side by side along K); the
// activation slots, written by the epilogue, are in the no-swizzle core-matrix layout: element
// (r, k) at (k / 8) 128 16 + r 16 + (k % 8) 2 bytes, core matrices adjacent along K 2048 bytes
// apart (the descriptor's leading byte offset) and along M 128 bytes apart (its stride offset).
// ---------------------------------------------------------------------------
constexpr int kWsEpiWarps = 16;                       // 4 per TMEM lane quarter
constexpr int kWsThreads = (kWsEpiWarps + 4) * 32;    // + two TMA warps and two MMA warps
constexpr int kWsHChunk = 64;                         // activation columns per ring slot
constexpr int kWsHSlot = kBM * kWsHChunk * 2;         // bytes of one activation slot
constexpr int kWsMaxRing = 6;
constexpr int kWsXSlab = kBM * 16 * 2;                // bytes of a 16-column slab of the row tile

struct FwdMaps {
  // X [M][ldx] and W1 [H1][K1]: boxes of 16 columns x 128 / H1 rows, 32-byte swizzle; W2 [H2][H1]
  // and W3 [NO][H2]: boxes of 64 columns x H2 / NO rows, 128-byte swizzle
  CUtensorMap x, w1, w2, w3;
};

// shared memory: W2 [H2][H1] | two activation slots | ns row-tile/W1 entries | two W3 chunks |
// b1 b2; a ring entry holds a 16-column slab of the row tile X with the matching W1 slab (H1
// rows), a W3 chunk the NO rows of 64 columns of W3 (b3 is read from global memory)
__host__ __device__ inline int ws_slot_bytes(const MlpFwdArgs& a) { return kWsXSlab + a.H1 * 32; }
__host__ __device__ inline int ws_w3_slot_bytes(const MlpFwdArgs& a) { return a.NO * kWsHChunk * 2; }
// W2 in boxes of 64 K columns (the last one zero-filled beyond H1)
__host__ __device__ inline int ws_w2_bytes(const MlpFwdArgs& a) { return (a.H1 + 63) / 64 * a.H2 * 128; }
__host__ __device__ inline int ws_off_h(const MlpFwdArgs& a) { return fw_align(ws_w2_bytes(a)); }
__host__ __device__ inline int ws_off_w(const MlpFwdArgs& a) { return ws_off_h(a) + 2 * kWsHSlot; }
__host__ __device__ inline int ws_off_w3(const MlpFwdArgs& a, int ns) {
  return fw_align(ws_off_w(a) + ns * ws_slot_bytes(a));
}
__host__ __device__ inline int ws_off_bias(const MlpFwdArgs& a, int ns) {
  return ws_off_w3(a, ns) + 2 * ws_w3_slot_bytes(a);
}
__host__ __device__ inline int ws_smem_bytes(const MlpFwdArgs& a, int ns) {
  return ws_off_bias(a, ns) + (a.H1 + a.H2) * 4;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// whether the phase of parity `parity` of an mbarrier has completed (does not block)
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void ws_mma(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void ws_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

// Wait for the phase of parity `parity` of an mbarrier, bounded in time; gives up early when
// another role has already aborted (flag set), and sets the flag and the error word on a timeout.
__device__ __forceinline__ bool ws_wait(uint32_t bar, uint32_t parity, int* err, volatile int* abort_flag) {
  if (mbar_test(bar, parity)) return true;  // the common case: the phase has completed; no clock read
  const unsigned long long t0 = tc_global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort_flag) return false;
    if (tc_global_ns() - t0 > kWaitNs) {
      atomicOr(err, NSK_EBIT_TIMEOUT);
      *abort_flag = 1;
      return false;
    }
  }
}
// the same for all lanes of a warp, with a warp-uniform result
__device__ __forceinline__ bool ws_wait_warp(uint32_t bar, uint32_t parity, int* err, volatile int* abort_flag) {
  const bool ok = ws_wait(bar, parity, err, abort_flag);
  return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// GELU(accumulator + bias) of 16 columns of the warp's 32 rows as BF16 into an activation slot:
// the thread's row r, slot-local columns [kk, kk + 16) (kk a multiple of 16); bias: the 16 biases
// in shared memory at shared-window address `bias` (every lane reads the same addresses: broadcast loads)
// four floats from shared memory (a shared-window address: ld.shared, not a generic load)
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
  float4 r;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(a));
  return r;
}
__device__ __forceinline__ void ws_gelu16(uint32_t taddr, uint32_t bias, unsigned char* slot, int r, int kk) {
  float b[16];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const float4 t = lds_f4(bias + 16u * g);
    b[4 * g] = t.x;
    b[4 * g + 1] = t.y;
    b[4 * g + 2] = t.z;
    b[4 * g + 3] = t.w;
  }
  uint32_t v[16];
  tmem_ld16(taddr, v);
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    uint32_t pk[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // columns 8 g + 2 j, + 1: the same values as gelu(acc + b), paired
      const int c = g * 8 + 2 * j;
      const float2 y = gelu2(__fadd2_rn(make_float2(__uint_as_float(v[c]), __uint_as_float(v[c + 1])),
                                        make_float2(b[c], b[c + 1])));
      const __nv_bfloat162 hb = __floats2bfloat162_rn(y.x, y.y);
      pk[j] = *reinterpret_cast<const uint32_t*>(&hb);
    }
    *reinterpret_cast<uint4*>(slot + ((kk >> 3) + g) * (kBM * 16) + r * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

// barrier indices in the kernel's array
enum WsBar : int {
  WB_W2 = 0, WB_A1FULL, WB_A1FREE, WB_A2FULL, WB_A2FREE, WB_A3FULL, WB_FINAL, WB_FINAL1,
  WB_HFULL, WB_HFREE = WB_HFULL + 2, WB_3FULL = WB_HFREE + 2, WB_3FREE = WB_3FULL + 2,
  WB_WFULL = WB_3FREE + 2, WB_WFREE = WB_WFULL + kWsMaxRing,
  WB_COUNT = WB_WFREE + kWsMaxRing
};

__global__ void __launch_bounds__(kWsThreads, 1)
    k_mlp_fwd3_ws(const MlpFwdArgs a, const int ns, const __grid_constant__ FwdMaps maps) {
  extern __shared__ __align__(1024) unsigned char ws_smem[];
  __shared__ __align__(8) uint64_t bars[WB_COUNT];
  // the 128-byte-swizzled operands (W2 at the base, the W3 chunks) need their 1024-byte pattern
  // aligned in the shared window: checked before any copy is issued
  if ((smem_u32(ws_smem) & 1023u) != 0u) {
    if (threadIdx.x == 0) atomicOr(a.err, NSK_EBIT_BOUNDS);
    return;
  }
  __shared__ uint32_t tmem_slot;
  __shared__ int aborted_s;
  volatile int* aborted = &aborted_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (a.M + kBM - 1) / kBM;
  const int slotb = ws_slot_bytes(a);
  const uint32_t aW2 = smem_u32(ws_smem), aW3 = smem_u32(ws_smem + ws_off_w3(a, ns));
  const uint32_t aH = smem_u32(ws_smem + ws_off_h(a)), aW = smem_u32(ws_smem + ws_off_w(a));
  const int w3b = ws_w3_slot_bytes(a);
  unsigned char* sH = ws_smem + ws_off_h(a);
  float* sB = reinterpret_cast<float*>(ws_smem + ws_off_bias(a, ns));  // b1 | b2
  auto bar = [&](int i) { return smem_u32(&bars[i]); };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    aborted_s = 0;
    for (int i = 0; i < WB_COUNT; ++i) {
      const bool epi = i == WB_A1FREE || i == WB_A2FREE || i == WB_HFULL || i == WB_HFULL + 1;
      mbar_init(bar(i), epi ? kWsEpiWarps : 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  for (int i = threadIdx.x; i < a.H1 + a.H2; i += kWsThreads) sB[i] = i < a.H1 ? a.b1[i] : a.b2[i - a.H1];
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tm = tmem_slot;

  if (warp == kWsEpiWarps) {
    // ---- TMA producer of the ring: the X and W1 slabs of every tile of this CTA in order (the order
    // in which the layer-1 MMA warp consumes them) ----
    if (lane == 0) {
      uint32_t r = 0u;
      int armed[kWsMaxRing];
      for (int i = 0; i < kWsMaxRing; ++i) armed[i] = 0;
      bool ok = true;
      // X columns [k0, k0 + 16) of row tile t (rows beyond M read as zero), then the W1 slab
      auto load_xw1 = [&](int t, int k0) {
        const uint32_t s = r % (uint32_t)ns;
        ok = ok && ws_wait(bar(WB_WFREE + s), ((r / ns) & 1u) ^ 1u, a.err, aborted);
        if (!ok) return;
        const uint32_t dst = aW + s * (uint32_t)slotb, w1 = dst + (uint32_t)kWsXSlab;
        mbar_expect_tx(bar(WB_WFULL + s), (uint32_t)(kWsXSlab + a.H1 * 32));
        tma_load_2d(dst, &maps.x, k0, t * kBM, bar(WB_WFULL + s));
        tma_load_2d(w1, &maps.w1, k0, 0, bar(WB_WFULL + s));
        armed[s] = (int)(r / ns) + 1;
        ++r;
      };
      for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x)
        for (int k0 = 0; ok && k0 < a.K1; k0 += 16) load_xw1(t, k0);
      // every copy this thread started has landed before the CTA exits (bounded waits; all have on
      // the normal path, where the MMA warp consumed them)
      volatile int never = 0;
      for (int s = 0; s < ns; ++s)
        if (armed[s] > 0) ws_wait(bar(WB_WFULL + s), (uint32_t)(armed[s] - 1) & 1u, a.err, &never);
    }
  } else if (warp == kWsEpiWarps + 3) {
    // ---- TMA producer of the weights: W2 once, then per tile the W3 chunks through their ring ----
    if (lane == 0) {
      uint32_t r3 = 0u;
      int armed[2] = {0, 0};
      bool ok = true;
      mbar_expect_tx(bar(WB_W2), (uint32_t)ws_w2_bytes(a));
      for (int b = 0; b < (a.H1 + 63) / 64; ++b)
        tma_load_2d(aW2 + (uint32_t)(b * a.H2 * 128), &maps.w2, 64 * b, 0, bar(WB_W2));
      for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x)
        for (int k0 = 0; ok && k0 < a.H2; k0 += kWsHChunk) {  // W3 columns [k0, k0 + 64): one box
          const uint32_t s = r3 & 1u;
          ok = ws_wait(bar(WB_3FREE + s), ((r3 >> 1) & 1u) ^ 1u, a.err, aborted);
          if (!ok) break;
          mbar_expect_tx(bar(WB_3FULL + s), (uint32_t)w3b);
          tma_load_2d(aW3 + s * (uint32_t)w3b, &maps.w3, k0, 0, bar(WB_3FULL + s));
          armed[s] = (int)(r3 >> 1) + 1;
          ++r3;
        }
      // every copy this thread started has landed before the CTA exits (bounded waits)
      volatile int never = 0;
      ws_wait(bar(WB_W2), 0u, a.err, &never);
      for (int s = 0; s < 2; ++s)
        if (armed[s] > 0) ws_wait(bar(WB_3FULL + s), (uint32_t)(armed[s] - 1) & 1u, a.err, &never);
    }
  } else if (warp == kWsEpiWarps + 1) {
    // ---- MMA issuer of layers 2 and 3: per tile, L2 chunk by chunk (resident W2), then L3 chunk
    // by chunk (W3 from its ring), each chunk as soon as its activations are in ----
    if (lane == 0) {
      uint32_t a2f = 1u, v = 0u, r3 = 0u;
      const uint32_t id2 = idesc_bf16(kBM, a.H2), id3 = idesc_bf16(kBM, a.NO);
      bool ok = ws_wait(bar(WB_W2), 0u, a.err, aborted);
      for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        ok = ws_wait(bar(WB_A2FREE), a2f, a.err, aborted);
        a2f ^= 1u;
        for (int c = 0; ok && c < a.H1; c += kWsHChunk) {  // layer 2: activation chunks x W2
          const uint32_t hs = v & 1u;
          ok = ws_wait(bar(WB_HFULL + hs), (v >> 1) & 1u, a.err, aborted);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int w = min(kWsHChunk, a.H1 - c);
          for (int s = 0; s < w / 16; ++s)
            ws_mma(tm + 256u, sdesc(aH + hs * kWsHSlot + (uint32_t)(s * 2 * kBM * 16), kBM * 16, 128),
                   sdesc_sw(aW2 + (uint32_t)(((c + 16 * s) / 64) * a.H2 * 128 + ((c + 16 * s) % 64) * 2), 1024u,
                            kSw128),
                   id2, (c > 0 || s > 0) ? 1u : 0u);
          ws_commit(bar(WB_HFREE + hs));
          ++v;
        }
        if (!ok) break;
        ws_commit(bar(WB_A2FULL));
        for (int c = 0; ok && c < a.H2; c += kWsHChunk) {  // layer 3: activation chunks x W3 chunks
          const uint32_t hs = v & 1u, s3 = r3 & 1u;
          ok = ws_wait(bar(WB_HFULL + hs), (v >> 1) & 1u, a.err, aborted) &&
               ws_wait(bar(WB_3FULL + s3), (r3 >> 1) & 1u, a.err, aborted);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int w = min(kWsHChunk, a.H2 - c);
          for (int s = 0; s < w / 16; ++s)
            ws_mma(tm + 256u, sdesc(aH + hs * kWsHSlot + (uint32_t)(s * 2 * kBM * 16), kBM * 16, 128),
                   sdesc_sw(aW3 + s3 * (uint32_t)w3b + (uint32_t)(s * 32), 1024u, kSw128), id3, (c > 0 || s > 0) ? 1u : 0u);
          ws_commit(bar(WB_3FREE + s3));
          ws_commit(bar(WB_HFREE + hs));
          ++r3;
          ++v;
        }
        if (ok) ws_commit(bar(WB_A3FULL));
      }
      // every MMA this thread issued has completed before TMEM is released (bounded wait)
      ws_commit(bar(WB_FINAL));
      volatile int never = 0;
      ws_wait(bar(WB_FINAL), 0u, a.err, &never);
    }
  } else if (warp == kWsEpiWarps + 2) {
    // ---- MMA issuer of layer 1: per tile, once the epilogue has released the accumulator, one K
    // step per ring entry (X slab, W1 slab) as the entries land ----
    if (lane == 0) {
      uint32_t a1f = 1u, r = 0u;
      const uint32_t id1 = idesc_bf16(kBM, a.H1);
      bool ok = true;
      for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        ok = ws_wait(bar(WB_A1FREE), a1f, a.err, aborted);
        a1f ^= 1u;
        for (int s = 0; ok && s < a.K1 / 16; ++s) {
          const uint32_t rs = r % (uint32_t)ns;
          ok = ws_wait(bar(WB_WFULL + rs), (r / ns) & 1u, a.err, aborted);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t e0 = aW + rs * (uint32_t)slotb;
          ws_mma(tm, sdesc_sw(e0, 256u, kSw32), sdesc_sw(e0 + (uint32_t)kWsXSlab, 256u, kSw32), id1, s > 0 ? 1u : 0u);
          ws_commit(bar(WB_WFREE + rs));
          ++r;
        }
        if (ok) ws_commit(bar(WB_A1FULL));
      }
      ws_commit(bar(WB_FINAL1));
      volatile int never = 0;
      ws_wait(bar(WB_FINAL1), 0u, a.err, &never);
    }
  } else {
    // ---- epilogue warps: warp w reads TMEM lanes 32 (w % 4).. (rows q 32 + lane) and the 16-column
    // block w / 4 of each 64-column chunk ----
    const int q = warp & 3, sub = warp >> 2, r = q * 32 + lane;
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    uint32_t f1 = 0u, f2 = 0u, f3 = 0u, u = 0u;
    bool ok = true;
    const uint32_t aB = smem_u32(sB);
    auto gelu_layer = [&](uint32_t col0, int H, uint32_t bias) {
      for (int c = 0; ok && c < H; c += kWsHChunk) {
        const uint32_t hs = u & 1u;
        ok = ws_wait_warp(bar(WB_HFREE + hs), ((u >> 1) & 1u) ^ 1u, a.err, aborted);
        if (!ok) break;
        const int cc = c + sub * 16;
        if (cc < H) ws_gelu16(tm + lanes + col0 + (uint32_t)cc, bias + 4u * cc, sH + hs * kWsHSlot, r, sub * 16);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(WB_HFULL + hs));
        ++u;
      }
    };
    for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
      ok = ws_wait_warp(bar(WB_A1FULL), f1, a.err, aborted);
      f1 ^= 1u;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      gelu_layer(0u, a.H1, aB);
      if (!ok) break;
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(WB_A1FREE));
      ok = ws_wait_warp(bar(WB_A2FULL), f2, a.err, aborted);
      f2 ^= 1u;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      gelu_layer(256u, a.H2, aB + 4u * a.H1);
      if (!ok) break;
      float b3[16];  // requested before the wait for layer 3, used after it
      if (sub * 16 < a.NO)
#pragma unroll
        for (int i = 0; i < 16; ++i) b3[i] = __ldg(a.b3 + sub * 16 + i);
      ok = ws_wait_warp(bar(WB_A3FULL), f3, a.err, aborted);
      f3 ^= 1u;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint32_t v[16];
      if (sub * 16 < a.NO) tmem_ld16(tm + lanes + 256u + (uint32_t)(sub * 16), v);
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(WB_A2FREE));  // layer 2's and 3's accumulator read
      if (sub * 16 < a.NO) {  // layer 3: + b3 -> Y
        // the warp's 32 rows x 16 columns, staged by 16-byte column group j in 512 bytes of the
        // activation slots that this warp alone writes (its bytes of activation chunks 0 and 1;
        // every MMA reading them has completed), then stored 64 bytes per row, 8 rows per
        // instruction
        auto piece = [&](int j) {
          return sH + (j >> 1) * kWsHSlot + (2 * sub + (j & 1)) * (kBM * 16) + q * 512;
        };
#pragma unroll
        for (int j = 0; j < 4; ++j)
          *reinterpret_cast<float4*>(piece(j) + lane * 16) =
              make_float4(__uint_as_float(v[4 * j]) + b3[4 * j], __uint_as_float(v[4 * j + 1]) + b3[4 * j + 1],
                          __uint_as_float(v[4 * j + 2]) + b3[4 * j + 2], __uint_as_float(v[4 * j + 3]) + b3[4 * j + 3]);
        __syncwarp();
        const int j = lane >> 3;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int rr = 8 * i + (lane & 7), m = t * kBM + q * 32 + rr;
          const float4 y = *reinterpret_cast<const float4*>(piece(j) + rr * 16);
          if (m < a.M) *reinterpret_cast<float4*>(a.Y + (size_t)m * a.ldy + sub * 16 + 4 * j) = y;
        }
        __syncwarp();
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(512));
  }
}

// cuTensorMapEncodeTiled, taken from the driver through the runtime (no link-time dependency)
typedef CUresult (*TmapEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline TmapEncodeFn tmap_encode_fn() {
  static TmapEncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TmapEncodeFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}
// 2D BF16 tensor map of a row-major [rows][ld] matrix, columns [0, cols) used; boxes of
// box_cols x box_rows with the given swizzle; elements beyond the matrix read as zero
inline bool bf16_tmap(CUtensorMap* m, const void* base, int cols, int rows, int ld, int box_cols, int box_rows,
                      CUtensorMapSwizzle swizzle) {
  const TmapEncodeFn fn = tmap_encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// which fused forward launch_mlp_fwd3 uses: 0 the warp-specialised kernel where it applies,
// 1 always k_mlp_fwd3 (set only by the test hook nsk_test_hook_mlp_fwd_kernel)
extern int g_fwd_kernel;

// fused forward when the network fits (NSK_ERR_ARG otherwise: the caller uses the per-layer GEMMs)
inline int launch_mlp_fwd3(const MlpFwdArgs& a, cudaStream_t s) {
  auto a16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  if (a.M < 1 || a.K1 < 16 || a.K1 > 256 || (a.K1 % 16) || a.H1 < 16 || a.H1 > 256 || (a.H1 % 16) ||
      a.H2 < 16 || a.H2 > 256 || (a.H2 % 16) || a.NO < 16 || a.NO > 256 || (a.NO % 16) || (a.ldx % 8) ||
      a.ldx < a.K1 || (a.ldy % 4) || a.ldy < a.NO || !a16(a.X) || !a16(a.W1) || !a16(a.W2) || !a16(a.W3) ||
      !a16(a.Y))
    return NSK_ERR_ARG;
  constexpr int kFwSmemMax = 226 * 1024;  // the per-block limit (227 KB) minus the static area (1 KB)
  int smem = fw_smem_bytes(a);
  if (smem > kFwSmemMax) return NSK_ERR_ARG;
  smem = smem < kRbSmemMin ? kRbSmemMin : smem;  // one CTA per SM: it owns all 512 TMEM columns
  static bool attr_done = false;
  static int sms = 0;
  if (!attr_done) {
    int dev = 0;
    if (cudaFuncSetAttribute(k_mlp_fwd3, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwSmemMax) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return NSK_ERR_CUDA;
    }
    attr_done = true;
  }
  const int ntiles = (a.M + kBM - 1) / kBM;
  // the warp-specialised kernel: layer 3 fits in layer 2's first activation chunk, W2 and W3 fit
  // resident beside a ring of at least 2 row-tile/W1 slabs (the largest that fits, up to
  // kWsMaxRing), and the tensor maps can be made
  if (g_fwd_kernel == 0 && a.NO <= kWsHChunk) {
    int ns = kWsMaxRing;
    while (ns >= 2 && ws_smem_bytes(a, ns) > kFwSmemMax) --ns;
    FwdMaps maps;
    constexpr CUtensorMapSwizzle k32 = CU_TENSOR_MAP_SWIZZLE_32B, k128 = CU_TENSOR_MAP_SWIZZLE_128B;
    if (ns >= 2 && bf16_tmap(&maps.x, a.X, a.K1, a.M, a.ldx, 16, kBM, k32) &&
        bf16_tmap(&maps.w1, a.W1, a.K1, a.H1, a.K1, 16, a.H1, k32) &&
        bf16_tmap(&maps.w2, a.W2, a.H1, a.H2, a.H1, 64, a.H2, k128) &&
        bf16_tmap(&maps.w3, a.W3, a.H2, a.NO, a.H2, 64, a.NO, k128)) {
      static bool ws_attr = false;
      if (!ws_attr) {
        if (cudaFuncSetAttribute(k_mlp_fwd3_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwSmemMax) !=
            cudaSuccess) {
          cudaGetLastError();
          return NSK_ERR_CUDA;
        }
        ws_attr = true;
      }
      k_mlp_fwd3_ws<<<persistent_grid(ntiles, sms), kWsThreads, ws_smem_bytes(a, ns), s>>>(a, ns, maps);
      return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
    }
  }
  k_mlp_fwd3<<<persistent_grid(ntiles, sms), kFwThreads, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

// host launcher (grid: ceil(M/128) x ceil(K/k_split))
inline int launch_gemm(const GemmArgs& a, cudaStream_t s) {
  if (a.M < 1 || a.N < 16 || a.N > kMaxN || (a.N % 16) || a.K < 16 || (a.K % 16) || (a.lda % 8) || (a.ldb % 8) ||
      a.lda < a.K || a.ldb < a.K || a.k_split < 16 || (a.k_split % kKC && a.k_split < a.K))
    return NSK_ERR_ARG;
  static bool attr_done = false;
  static int sms = 0;
  if (!attr_done) {
    int dev = 0;
    if (cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_gemm_tc_rb, cudaFuncAttributeMaxDynamicSharedMemorySize, kRbSmemMax) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return NSK_ERR_CUDA;
    }
    attr_done = true;
  }
  // resident-B kernel: 16-byte aligned rows of every output it writes with vector stores
  auto a16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  const bool aligned = (a.epi == EPI_STORE ? (a.ldo % 4) == 0 && a16(a.out) : (a.ldh % 8) == 0 && a16(a.hout)) &&
                       (!(a.epi == EPI_GELU && a.out) || ((a.ldo % 4) == 0 && a16(a.out))) &&
                       (a.epi != EPI_DGELU || ((a.ldz % 4) == 0 && a16(a.zin)));
  const bool resident = a.epi != EPI_ATOMIC && a.k_split >= a.K && a.K <= 256 && (a.N % 64) == 0 && aligned;
  if (resident) {
    int smem = rb_b_bytes(a.N, a.K) + kBM * a.K * 2 + kRbStageBytes;
    smem = smem < kRbSmemMin ? kRbSmemMin : smem;
    const int ntiles = (a.M + kBM - 1) / kBM;
    if (smem > kRbSmemMax) return NSK_ERR_ARG;
    k_gemm_tc_rb<<<persistent_grid(ntiles, sms), kRbThreads, smem, s>>>(a);
  } else {
    dim3 grid((unsigned)((a.M + kBM - 1) / kBM), (unsigned)((a.K + a.k_split - 1) / a.k_split));
    k_gemm_tc<<<grid, kThreads, kSmemBytes, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

}  // namespace tc
}  // namespace nsk
