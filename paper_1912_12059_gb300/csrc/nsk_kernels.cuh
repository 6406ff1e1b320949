// nsk_kernels.cuh -- sm_103a kernels of one explicit DGSEM stage of relaxation
// model II (arXiv:1912.12059, Sec. 2.3 and Sec. 3.1), templated on the arithmetic
// type R of the DG operator (double, or float with the equation of state in
// double), the dimension D and the number of nodes per direction NP = N + 1.
//
// One stage is four launches (three with the fused face schedule, one fewer again
// when the previous stage's volume kernel already wrote the traces of its output):
//   k_prolong  U -> traces of U on every element face (GL: l_j(+-1) dot a line)
//   k_lift     U, traces -> BR1 gradients Q of (v, c) and the face-normal
//              viscous-flux traces of the element's own faces
//   k_face     traces -> local Lax-Friedrichs convective flux minus the BR1
//              mean viscous flux, once per face (separate schedule only)
//   k_volume   U, Q, face fluxes -> weak-form volume integral, surface lifting,
//              relaxation sources, then the residual or the fused LSRK update;
//              with the fused face schedule it evaluates its own faces' fluxes;
//              optionally it also writes the traces of the updated state
// The grid-wide dependencies of BR1 (a face needs both neighbours' traces,
// twice per residual) are the launch boundaries.
#pragma once

#include "nsk_internal.h"
#include <type_traits>

namespace nsk {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <int D, int NP>
struct Shape {
  static constexpr int NPE = ipow(NP, D);      // nodes per element
  static constexpr int NFN = ipow(NP, D - 1);  // nodes per face
  static constexpr int NV = D + 2;             // conservative variables
  static constexpr int NW = D + 1;             // lifted primitive variables (v, c)
  static constexpr int NQ = D * (D + 1);       // gradient components
  static constexpr int NVF = D * (D + 1) / 2 + D;  // viscous form: symmetric stress / mu and grad c
  static constexpr int NF = 2 * D;             // faces per element
  static constexpr int G = (256 / NPE) > 0 ? 256 / NPE : 1;  // elements per block
  static constexpr int TPB = G * NPE;
};

// index of node n along direction k
template <int NP>
__device__ __forceinline__ int coord(int n, int k) {
  int s = 1;
  for (int q = 0; q < k; ++q) s *= NP;
  return (n / s) % NP;
}

// face-node index of node n on the faces normal to direction k
template <int D, int NP>
__device__ __forceinline__ int face_node(int n, int k) {
  if (D == 1) return 0;
  const int i0 = n % NP, i1 = (n / NP) % NP;
  if (D == 2) return k == 0 ? i1 : i0;
  const int i2 = n / (NP * NP);
  return k == 0 ? i1 + NP * i2 : (k == 1 ? i0 + NP * i2 : i0 + NP * i1);
}

// first node of the line in direction k through face node fn
template <int D, int NP>
__device__ __forceinline__ int line_base(int fn, int k) {
  if (D == 1) return 0;
  if (D == 2) return k == 0 ? fn * NP : fn;
  const int a = fn % NP, b = fn / NP;
  return k == 0 ? NP * (a + NP * b) : (k == 1 ? a + NP * NP * b : a + NP * b);
}

template <int NP>
__device__ __forceinline__ int node_stride(int k) {
  return k == 0 ? 1 : (k == 1 ? NP : NP * NP);
}

// Bounds-checking build (-DNSK_BOUNDS_CHECK, libnsk_check.so): every neighbour index is checked
// against the element count; a failing check sets NSK_EBIT_BOUNDS in the error word p.berr and
// the index becomes 0, so the access stays inside its array (no fault, no trap). All other
// indices of the stage kernels follow from loop bounds and the element index.
__device__ __forceinline__ long long chk_elem(const NskParams& p, long long e) {
#ifdef NSK_BOUNDS_CHECK
  if ((unsigned long long)e >= (unsigned long long)p.E) {
    if (p.berr) atomicOr(p.berr, NSK_EBIT_BOUNDS);
    return 0;
  }
#endif
  (void)p;
  return e;
}

// periodic neighbour of element e in direction k, side dir = -1 / +1 (element indices fit
// in 32 bits: nsk_init_mesh rejects meshes with E * nodes per element above 2^31)
__device__ __forceinline__ long long nbr_elem(const NskParams& p, long long e, int k, int dir) {
  unsigned s = 1;
  for (int q = 0; q < k; ++q) s *= (unsigned)p.ne[q];
  const int n = p.ne[k];
  const int c = (int)(((unsigned)e / s) % (unsigned)n);
  int cn = c + dir;
  cn += (cn < 0) ? n : 0;
  cn -= (cn >= n) ? n : 0;
  return chk_elem(p, e + (long long)(cn - c) * (long long)s);
}

// Cartesian position of an element for the stage kernels: 32-bit index and coordinates
// (fast division by the invariant ne[0], ne[1]); its neighbours are a compare and an add.
struct ElemIdx {
  int e, c0, c1, c2;
};
template <int D>
__device__ __forceinline__ ElemIdx elem_idx(const NskParams& p, int e) {
  ElemIdx x{e, e, 0, 0};
  if constexpr (D >= 2) {
    const unsigned t = fdiv((unsigned)e, p.fd_ne0);
    x.c0 = e - (int)t * p.ne[0];
    if constexpr (D == 2) {
      x.c1 = (int)t;
    } else {
      const unsigned z = fdiv(t, p.fd_ne1);
      x.c1 = (int)t - (int)z * p.ne[1];
      x.c2 = (int)z;
    }
  }
  return x;
}
// periodic neighbour of x in direction k, side dir = -1 / +1 (same result as nbr_elem)
__device__ __forceinline__ int nbr_of(const NskParams& p, const ElemIdx& x, int k, int dir) {
  const int c = k == 0 ? x.c0 : (k == 1 ? x.c1 : x.c2);
  if (dir > 0) return (int)chk_elem(p, c == p.ne[k] - 1 ? x.e - p.ewrap[k] : x.e + p.est[k]);
  return (int)chk_elem(p, c == 0 ? x.e + p.ewrap[k] : x.e - p.est[k]);
}

// ---- FP64 reciprocal and square root with few FP64 instructions ----
// The stage kernels are bound by the FP64 pipe (two FP64 operations per SM and clock on this
// GPU), where a correctly rounded division or square root costs about ten of them. Here both are
// Newton-Raphson iterations seeded by the FP32 hardware approximations (rcp.approx,
// rsqrt.approx, relative error about 2^-23): the seed's conversions to and from FP32 are integer
// operations on the bit patterns (off the FP64 pipe), and two Newton corrections bring the error
// from 2^-22 to 2^-44 to below one unit in the last place (a faithful result, not always the
// correctly rounded one; the tests bound it by one ulp against CUDA's division and sqrt).
// Domain: positive normal x with 2^-120 < x < 2^120 (the FP32 range of the seed); elsewhere
// the CUDA functions are used.

// |x| truncated to FP32 (round toward zero), from the bit pattern; x in the domain above
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  return __uint_as_float((((hi & 0x7FFFFFFFu) - ((1023u - 127u) << 20)) << 3) | (lo >> 29));
}
// a positive normal FP32 value as FP64 (exact)
__device__ __forceinline__ double f64_exact(float y) {
  const unsigned b = __float_as_uint(y);
  return __hiloint2double((int)((((b >> 23) + (1023u - 127u)) << 20) | ((b & 0x7FFFFFu) >> 3)), (int)(b << 29));
}
__device__ __forceinline__ bool nr_domain(double x) {
  return (unsigned)__double2hiint(x) - ((1023u - 120u) << 20) < (240u << 20);
}
__device__ __forceinline__ float rcp_approx_f32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx_f32(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// 1/a: y <- y + y (1 - a y), twice, from the FP32 seed
__device__ __forceinline__ double rcp_nr(double a) {
  if (!nr_domain(a)) return 1.0 / a;
  double y = f64_exact(rcp_approx_f32(f32_trunc(a)));
  y = fma(y, fma(-a, y, 1.0), y);
  return fma(y, fma(-a, y, 1.0), y);
}
// sqrt(x): s <- s + (x - s^2) h with h ~ 1/(2 sqrt x) from the FP32 seed of 1/sqrt(x), twice
__device__ __forceinline__ double sqrt_nr(double x) {
  if (!nr_domain(x)) return sqrt(x);
  const float y0 = rsqrt_approx_f32(f32_trunc(x));
  const double h = f64_exact(0.5f * y0);  // exact: a power-of-two scaling
  double s = x * f64_exact(y0);
  s = fma(fma(-s, s, x), h, s);
  return fma(fma(-s, s, x), h, s);
}
// the arithmetic type's reciprocal and square root in the stage kernels: FP64 through the
// Newton-Raphson forms above, FP32 as the hardware computes them
__device__ __forceinline__ double rcp_s(double a) { return rcp_nr(a); }
__device__ __forceinline__ float rcp_s(float a) { return 1.0f / a; }
__device__ __forceinline__ double sqrt_s(double x) { return sqrt_nr(x); }
__device__ __forceinline__ float sqrt_s(float x) { return sqrtf(x); }

// ---- Van-der-Waals EoS, Sec. 2.1 (reduced: p = 8 T rho / (3 - rho) - 3 rho^2) ----
// Modified pressure p_alpha = p + alpha rho^2 / 2 (Eq. modified_pressure) and its derivative
// with one reciprocal q = 1 / (3 - rho):
//   p_alpha = 8 T rho q + (alpha/2 - 3) rho^2,   p_alpha' = 24 T q^2 + (alpha - 6) rho.
// Expressions with two products are written as explicit fused multiply-adds so
// that every kernel that inlines them rounds identically (results then do not
// depend on the schedule or on which kernel evaluates them).
__device__ __forceinline__ double eos_pa64(const NskParams& p, double rho) {
  const double q = 1.0 / (3.0 - rho);
  return fma(p.t8 * rho, q, (p.pa2 * rho) * rho);
}
__device__ __forceinline__ void eos_both64(const NskParams& p, double rho, double& pa, double& dpa) {
  const double q = 1.0 / (3.0 - rho);
  pa = fma(p.t8 * rho, q, (p.pa2 * rho) * rho);
  dpa = fma(p.t24 * q, q, p.dpa1 * rho);
}
// 1/(3 - rho) in FP64 for the FP32 operator's rho: FP32 seed q0, then one Newton-Raphson
// step for the reciprocal, q = q0 + q0 (1 - a q0), which squares the seed's relative error
// (<= 2^-23 -> <= 2^-46; the FP64 value is rounded to FP32 afterwards). a = 3 - rho is exact
// in FP64.
__device__ __forceinline__ double recip_3m(float rho) {
  const double a = 3.0 - (double)rho;
  const double q0 = (double)(1.0f / (float)a);
  return fma(q0, fma(-a, q0, 1.0), q0);
}
__device__ __forceinline__ double eos_pa64f(const NskParams& p, float rho) {
  const double r = rho, q = recip_3m(rho);
  return fma(p.t8 * r, q, (p.pa2 * r) * r);
}
__device__ __forceinline__ void eos_both64f(const NskParams& p, float rho, double& pa, double& dpa) {
  const double r = rho, q = recip_3m(rho);
  pa = fma(p.t8 * r, q, (p.pa2 * r) * r);
  dpa = fma(p.t24 * q, q, p.dpa1 * r);
}
// Precision policy of the FP32 operator: FP32 EoS, except inside the spinodal interval and
// wherever p_alpha' cancels (alpha close to alpha_*), where it is evaluated in FP64.
__device__ __forceinline__ bool eos_needs64(const NskParams& p, float rho) {
  return rho > p.spin_lof && rho < p.spin_hif;
}
template <typename R> struct Eos;
template <> struct Eos<double> {
  __device__ static __forceinline__ double pa(const NskParams& p, double rho) { return eos_pa64(p, rho); }
  __device__ static __forceinline__ void both(const NskParams& p, double rho, double& pa, double& dpa) {
    eos_both64(p, rho, pa, dpa);
  }
  // with q = 1/(3 - rho) already known
  __device__ static __forceinline__ double pa_q(const NskParams& p, double rho, double q) {
    return fma(p.t8 * rho, q, (p.pa2 * rho) * rho);
  }
  __device__ static __forceinline__ void both_q(const NskParams& p, double rho, double q, double& pa, double& dpa) {
    pa = fma(p.t8 * rho, q, (p.pa2 * rho) * rho);
    dpa = fma(p.t24 * q, q, p.dpa1 * rho);
  }
};
template <> struct Eos<float> {
  __device__ static __forceinline__ float pa(const NskParams& p, float rho) {
    if (eos_needs64(p, rho)) return (float)eos_pa64f(p, rho);
    const float q = 1.0f / (3.0f - rho);
    return fmaf(p.t8f * rho, q, (p.pa2f * rho) * rho);
  }
  __device__ static __forceinline__ void both(const NskParams& p, float rho, float& pa, float& dpa) {
    if (!eos_needs64(p, rho)) {
      const float q = 1.0f / (3.0f - rho);
      const float a = (p.t24f * q) * q, b = p.dpa1f * rho;
      pa = fmaf(p.t8f * rho, q, (p.pa2f * rho) * rho);
      dpa = fmaf(p.t24f * q, q, b);
      if (fabsf(dpa) >= 1e-3f * (fabsf(a) + fabsf(b))) return;
    }
    double pd, dd;
    eos_both64f(p, rho, pd, dd);
    pa = (float)pd;
    dpa = (float)dd;
  }
};
__device__ __forceinline__ double eos_free_energy(const NskParams& p, double rho) {
  // W = rho R T ln(rho / (1 - b rho)) - a rho^2, Eq. (vdw_freeenergy)
  return (8.0 / 3.0) * p.T * rho * log(3.0 * rho / (3.0 - rho)) - 3.0 * rho * rho;
}
// 0 < rho < 3 tested on the bit pattern (positive IEEE numbers order like their bits; zero,
// negatives, NaN and 3 or more fall outside), which keeps the test off the FP64 pipe. In FP64
// the high word decides: it accepts rho >= 2^-1042 (smaller positive subnormals are flagged).
__device__ __forceinline__ bool rho_ok(double rho) {
  return (unsigned)__double2hiint(rho) - 1u < 0x40080000u - 1u;
}
__device__ __forceinline__ bool rho_ok(float rho) { return __float_as_uint(rho) - 1u < 0x40400000u - 1u; }
template <typename R>
__device__ __forceinline__ int rho_flags(R rho) {
  if (rho_ok(rho)) return 0;
  return (rho != rho) ? (NSK_EBIT_RHO | NSK_EBIT_NAN) : NSK_EBIT_RHO;
}
// p_alpha' >= 0 and finite, on the bit pattern (a negative sign, NaN or infinity fail; so does -0)
__device__ __forceinline__ bool sound_ok(double d) { return (unsigned)__double2hiint(d) < 0x7FF00000u; }
__device__ __forceinline__ bool sound_ok(float d) { return __float_as_uint(d) < 0x7F800000u; }

// Asynchronous global -> shared copy of one 4- or 8-byte value (cp.async, L1-allocating form);
// both addresses are aligned to the value's size.
template <typename R>
__device__ __forceinline__ void cp_async_elem(R* sdst, const R* gsrc) {
  static_assert(sizeof(R) == 4 || sizeof(R) == 8, "cp.async copies 4 or 8 bytes here");
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gsrc), "n"((int)sizeof(R)) : "memory");
}
// the same for 16 bytes (cp.async.cg, L2 only: each face value is read by two elements of
// different blocks, so L1 allocation does not pay); both addresses 16-byte aligned
__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}
// W values from src to the shared buffer dst: asynchronously (cp.async, src in global memory)
// or, ASYNC false, with plain loads and stores (src may then be in shared memory, which cp.async
// cannot read)
template <bool ASYNC, int W, typename R>
__device__ __forceinline__ void stage_copy(R* dst, const R* src) {
  if constexpr (ASYNC) {
    if constexpr (W > 1)
      cp_async_16(dst, src);
    else
      cp_async_elem(dst, src);
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) dst[w] = src[w];
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// nanoseconds of the global timer
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident), bounded: a block that waits
// longer than timeout_ns sets NSK_EBIT_TIMEOUT and every block then returns false (bar[0]: arrivals,
// bar[1]: generation; both start at zero).
inline __device__ bool grid_barrier(unsigned* bar, int* err, const unsigned long long timeout_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*vgen == gen) {
        if (global_ns() - t0 > timeout_ns) {
          atomicOr(err, NSK_EBIT_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int*)err & NSK_EBIT_TIMEOUT) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// --------------------------------------------------------------------------
// Stage bodies. Every stage kernel below (and the batched persistent kernel in
// nsk_batch.cu) is a thin wrapper around these device functions:
//   prolong_item  one (element, face slot, face node) trace of U
//   lift_group    BR1 lifting of G consecutive elements
//   face_item     numerical flux of one face node
//   volume_group  volume integral + surface lifting + sources + update of G elements
// Element groups use threads [0, G*NPE) of the block; the remaining threads
// only take part in the block barriers.
// --------------------------------------------------------------------------

// Utr[v][slot][E][nfn], slot = 2k + (0: face xi_k = -1, 1: xi_k = +1): the trace
// sum_j l_j(+-1) U_j along the line in direction k through face node fn of element e.
// `u` points at node 0 of the element's first variable, variables `vs` apart (the
// global array, or an element staged in shared memory: both give the same bits).
// NVAR conservative variables (d + 2 for model II, d + 1 for the original NSK equations).
// The NVAR traces of one (face slot, face node) of an element, and in FP64 also the planes
// 1/rho and 1/(3 - rho) of the trace: out[NVAR + TraceComps<R>::extra]. `u` points at node 0
// of the element's first variable, variables `vs` apart (the global array, or an element
// staged in shared memory: both give the same bits).
template <typename R, int D, int NP, int NVAR = Shape<D, NP>::NV>
__device__ __forceinline__ void trace_vals(const NskParams& p, const R* __restrict__ u, const size_t vs,
                                           const int slot, const int fn, R* out) {
  const auto& t = TabSel<R>::get(p);
  const int k = slot >> 1;
  const R* L = (slot & 1) ? t.lp : t.lm;
  const int n0 = line_base<D, NP>(fn, k), st = node_stride<NP>(k);
  const R* ul = u + n0;
#pragma unroll
  for (int v = 0; v < NVAR; ++v) {
    R acc = 0;
#pragma unroll
    for (int j = 0; j < NP; ++j) acc = fma(L[j], ul[v * vs + j * st], acc);
    out[v] = acc;
  }
  if constexpr (TraceComps<R>::extra > 0) {
    // one division: d = 1/(rho (3 - rho)) gives 1/rho = (3 - rho) d and 1/(3 - rho) = rho d
    const R rho = out[0];
    const R d = rcp_s(rho * (R(3) - rho));
    out[NVAR] = (R(3) - rho) * d;
    out[NVAR + 1] = rho * d;
  }
}

// Utr[v][slot][E][nfn], slot = 2k + (0: face xi_k = -1, 1: xi_k = +1): the trace
// sum_j l_j(+-1) U_j along the line in direction k through face node fn of element e
// (trace_vals, stored).
// NVAR conservative variables (d + 2 for model II, d + 1 for the original NSK equations).
template <typename R, int D, int NP, int NVAR = Shape<D, NP>::NV>
__device__ __forceinline__ void prolong_trace(const NskParams& p, const R* __restrict__ u, const size_t vs,
                                              R* __restrict__ Utr, const int e, const int slot, const int fn) {
  using S = Shape<D, NP>;
  constexpr int NT = NVAR + TraceComps<R>::extra;
  const size_t pl = (size_t)S::NF * p.nfe;  // distance between the planes of two variables
  R* o = Utr + (size_t)slot * p.nfe + (e * S::NFN + fn);
  R vals[NT];
  trace_vals<R, D, NP, NVAR>(p, u, vs, slot, fn, vals);
#pragma unroll
  for (int v = 0; v < NT; ++v) o[v * pl] = vals[v];
}

// one (element, face slot, face node) item of the prolongation, idx = (slot, e, fn) flattened
// (idx / nfn < 2^31 for every mesh nsk_init_mesh accepts)
template <typename R, int D, int NP>
__device__ __forceinline__ void prolong_item(const NskParams& p, const R* __restrict__ U, R* __restrict__ Utr,
                                             const long long idx) {
  using S = Shape<D, NP>;
  const int fn = (int)(idx % S::NFN);
  const unsigned r = (unsigned)(idx / S::NFN);
  const unsigned slot = fdiv(r, p.fd_E);
  const int e = (int)(r - slot * (unsigned)p.E);
  prolong_trace<R, D, NP>(p, U + (size_t)e * S::NPE, (size_t)p.nne, Utr, e, (int)slot, fn);
}

// Shared-memory copy of the direction operators (2/h_k folded in) of one precision:
// [D][NP][NP] dk, then [D][NP] lpk, then [D][NP] lmk. Every thread of a warp reads its own
// row i; from shared memory the distinct rows are served in one pass, where the kernel
// parameter bank would serialise them. dk is scaled by sd, lpk and lmk by sl: the kernels
// whose face values are stored doubled (the lifting's sums of two traces, the face fluxes
// 2 F*) take sl = 1/2 (an exact scaling); the Runge-Kutta update folds dt into both.
template <int D, int NP>
__host__ __device__ constexpr int tab_smem() {
  return D * NP * NP + 2 * D * NP;
}
template <typename R, int D, int NP>
__device__ __forceinline__ void stage_tables(const NskTab<R>& t, R* tb, const R sd = R(1), const R sl = R(1)) {
  for (int x = threadIdx.x; x < D * NP * NP; x += blockDim.x) {
    const int k = x / (NP * NP), r = x % (NP * NP);
    tb[x] = sd * t.dk[k][(r / NP) * NSK_MAXNP + r % NP];
  }
  for (int x = threadIdx.x; x < D * NP; x += blockDim.x) {
    tb[D * NP * NP + x] = sl * t.lpk[x / NP][x % NP];
    tb[D * NP * NP + D * NP + x] = sl * t.lmk[x / NP][x % NP];
  }
}

// the NP values of one line from shared memory: 16-byte loads when a line fills whole
// 16-byte units (f is then 16-byte aligned), else one value at a time
template <typename R, int NP>
__device__ __forceinline__ void load_line(const R* f, R (&x)[NP]) {
  if constexpr ((NP * sizeof(R)) % 16 == 0) {
    using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
    constexpr int W = 16 / (int)sizeof(R);
#pragma unroll
    for (int j = 0; j < NP; j += W) {
      const V t = *reinterpret_cast<const V*>(f + j);
      const R* tv = reinterpret_cast<const R*>(&t);
#pragma unroll
      for (int w = 0; w < W; ++w) x[j + w] = tv[w];
    }
  } else {
#pragma unroll
    for (int j = 0; j < NP; ++j) x[j] = f[j];
  }
}

// node n at position i_k of line face_node(n, k): the nodes laid out with the lines in
// direction k contiguous (k = 0 is the natural order)
template <int D, int NP>
__device__ __forceinline__ int line_pos(int n, int k) {
  return face_node<D, NP>(n, k) * NP + coord<NP>(n, k);
}

// distance between two faces' central fluxes in the lifting's shared buffer: for faces of 16
// nodes or more it is congruent to NFN modulo 32, so the face slots one warp writes in turn
// fall on consecutive banks
template <int D, int NP>
__host__ __device__ constexpr int lift_slot_stride() {
  using S = Shape<D, NP>;
  return S::NFN >= 16 ? S::NW * S::NFN + ((S::NFN - S::NW * S::NFN) % 32 + 32) % 32 : S::NW * S::NFN;
}
// the lifting keeps one copy of the primitive variables per direction, lines contiguous, when
// its lines load 16 bytes at a time and the block's buffers stay within 40 KB
template <typename R, int D, int NP, int G>
__host__ __device__ constexpr bool lift_lines() {
  using S = Shape<D, NP>;
  return D >= 2 && (NP * sizeof(R)) % 16 == 0 &&
         (G * D * S::NW * S::NPE + G * S::NF * lift_slot_stride<D, NP>()) * (int)sizeof(R) <= 40 * 1024;
}
// shared memory (in units of R) of lift_group
template <typename R, int D, int NP, int G>
__host__ __device__ constexpr int lift_work_smem() {
  using S = Shape<D, NP>;
  constexpr int front = G * (lift_lines<R, D, NP, G>() ? D : 1) * S::NW * S::NPE + G * S::NF * lift_slot_stride<D, NP>();
  return front > G * D * S::NW * S::NPE ? front : G * D * S::NW * S::NPE;
}
template <typename R, int D, int NP, int G>
__host__ __device__ constexpr int lift_smem() {
  return lift_work_smem<R, D, NP, G>() + tab_smem<D, NP>();
}

// ---- parts of the BR1 lifting, shared by the stage kernels (so every schedule rounds alike) ----

// The primitive variables w = (v, c) (MODEL 1: (v, rho)) of node n of a lifting element, stored in
// the lifting's shared buffer sw once per direction copy (lines of direction k contiguous when
// LINES). u points at the node's first variable, variables vs apart.
template <typename R, int D, int NP, int G, int MODEL = 0>
__device__ __forceinline__ void lift_store_w(const R* __restrict__ u, const size_t vs, R* sw, const int le,
                                             const int n, int& eflag) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NW = S::NW;
  constexpr bool LINES = lift_lines<R, D, NP, G>();
  constexpr int NCOPY = LINES ? D : 1;
  const R rho = u[0];
  eflag |= rho_flags(rho);
  const R inv = rcp_s(rho);
  R wn[NW];
#pragma unroll
  for (int a = 0; a < D; ++a) wn[a] = u[(1 + a) * vs] * inv;
  wn[D] = MODEL == 1 ? rho : u[(D + 1) * vs];
#pragma unroll
  for (int c = 0; c < NCOPY; ++c) {
    const int pos = LINES ? line_pos<D, NP>(n, c) : n;
#pragma unroll
    for (int w = 0; w < NW; ++w) sw[((le * NCOPY + c) * NW + w) * NPE + pos] = wn[w];
  }
}

// 2 w* of one (face slot, face node) from the element's own trace uo and its neighbour's un
// (the 1/2 of the central flux is in the staged lpk, lmk: an exact scaling), each with NV
// conservative values and, in FP64, 1/rho and 1/(3 - rho) after them; ws: NW values NFN apart.
template <typename R, int D, int NFN, int NV, int MODEL = 0>
__device__ __forceinline__ void lift_wstar(const R* uo, const R* un, R* ws, int& eflag) {
  eflag |= rho_flags(uo[0]) | rho_flags(un[0]);
  R io, in;
  if constexpr (TraceComps<R>::extra > 0) {
    io = uo[NV];
    in = un[NV];
  } else {
    io = R(1) / uo[0];
    in = R(1) / un[0];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) ws[a * NFN] = fma(uo[1 + a], io, un[1 + a] * in);
  ws[D * NFN] = MODEL == 1 ? uo[0] + un[0] : uo[D + 1] + un[D + 1];
}

// The lifted gradients q[k NW + w] of node n (weak form, central flux; the direction operators
// with 2/h_k folded in and the 1/2 of w* in lpk, lmk staged at tb), from sw and the 2 w* in sws.
template <typename R, int D, int NP, int G>
__device__ __forceinline__ void lift_q(const R* tb, const R* sw, const R* sws, const int le, const int n,
                                       R (&q)[Shape<D, NP>::NQ]) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NW = S::NW, NF = S::NF;
  constexpr bool LINES = lift_lines<R, D, NP, G>();
  constexpr int NCOPY = LINES ? D : 1, SWS = lift_slot_stride<D, NP>();
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int i = coord<NP>(n, k), fn = face_node<D, NP>(n, k);
    const int n0 = line_base<D, NP>(fn, k), st = node_stride<NP>(k);
    R dk[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) dk[j] = tb[(k * NP + i) * NP + j];
    const R lpk = tb[D * NP * NP + k * NP + i], lmk = tb[D * NP * NP + D * NP + k * NP + i];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      R wl[NP];
      if (LINES || k == 0) {  // the line is contiguous
        load_line<R, NP>(sw + ((le * NCOPY + (LINES ? k : 0)) * NW + w) * NPE + (LINES ? fn * NP : n0), wl);
      } else {
#pragma unroll
        for (int j = 0; j < NP; ++j) wl[j] = sw[(le * NW + w) * NPE + n0 + j * st];
      }
      R vol = 0;
#pragma unroll
      for (int j = 0; j < NP; ++j) vol = fma(dk[j], wl[j], vol);
      const R wp = sws[(le * NF + 2 * k + 1) * SWS + w * NFN + fn];
      const R wm = sws[(le * NF + 2 * k) * SWS + w * NFN + fn];
      q[k * NW + w] = fma(wp, lpk, fma(-wm, lmk, -vol));
    }
  }
}

// the viscous stress without mu from the lifted velocity gradients (symmetric: each
// off-diagonal sum once)
template <typename R, int D>
__device__ __forceinline__ void stress_of(const R* q, R (&tau)[D][D]) {
  constexpr int NW = D + 1;
  R div = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) div += q[a * NW + a];
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int a = k; a < D; ++a) {
      const R sum = q[k * NW + a] + q[a * NW + k];
      tau[k][a] = (a == k) ? fma(-R(2.0 / 3.0), div, sum) : sum;
      tau[a][k] = tau[k][a];
    }
  }
}

// The viscous form of the lifted gradients that the volume kernel needs: the stress without mu
// (its D(D+1)/2 independent components, row by row from the diagonal: (k, a) for a >= k) and
// grad c; stored by the lifting in place of the gradients (fewer values, and the stress is
// formed once).
template <typename R, int D>
__device__ __forceinline__ void visc_store(const R (&tau)[D][D], const R* gc, R* __restrict__ Q, const size_t nn,
                                           const int g) {
  int c = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int a = k; a < D; ++a) Q[(c++) * nn + g] = tau[k][a];
  }
#pragma unroll
  for (int k = 0; k < D; ++k) Q[(c++) * nn + g] = gc[k];
}
template <typename R, int D>
__device__ __forceinline__ void visc_load(const R* __restrict__ Q, const size_t nn, const int g, R (&tau)[D][D],
                                          R* gc) {
  int c = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int a = k; a < D; ++a) {
      tau[k][a] = Q[(c++) * nn + g];
      tau[a][k] = tau[k][a];
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) gc[k] = Q[(c++) * nn + g];
}
// the stress (without mu) and grad c of a node's lifted gradients q
template <typename R, int D>
__device__ __forceinline__ void visc_of(const R* q, R (&tau)[D][D], R* gc) {
  stress_of<R, D>(q, tau);
#pragma unroll
  for (int k = 0; k < D; ++k) gc[k] = q[k * (D + 1) + D];
}

// The face-normal viscous flux F^v_k = (tau_{.k}, (kappa/beta) c_{x_k}) traced onto the element's
// own faces: the nodal fluxes (without mu and kappa/beta, lines of direction k contiguous) go to
// sfv, then, after a block barrier, each face value is the trace with mu l(+-1) or
// (kappa/beta) l(+-1). TO_SMEM: into fo[((le NF + slot) NW + c) NFN + fn]; else into
// FVtr[c][slot][E][nfn]. Ends with a block barrier.
template <typename R, int D, int NP, int G, bool TO_SMEM = false>
__device__ __forceinline__ void lift_fv_traces(const NskParams& p, const R (&tau)[D][D], const R* gc, R* sfv,
                                               const bool valid, const int le, const int n, const int e,
                                               R* __restrict__ FVtr, R* fo) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NW = S::NW, NF = S::NF;
  const auto& t = TabSel<R>::get(p);
  if (valid) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int pos = line_pos<D, NP>(n, k);
#pragma unroll
      for (int a = 0; a < D; ++a) sfv[((le * D + k) * NW + a) * NPE + pos] = tau[k][a];
      sfv[((le * D + k) * NW + D) * NPE + pos] = gc[k];
    }
  }
  __syncthreads();
  if (valid) {
    const size_t pl = (size_t)NF * p.nfe;  // distance between the planes of two trace variables
    for (int it = n; it < NF * NFN; it += NPE) {
      const int slot = it / NFN, fn = it % NFN, k = slot >> 1;
      const R* Lmu = (slot & 1) ? t.lpmu : t.lmmu;  // mu l(+-1)
      const R* Lkb = (slot & 1) ? t.lpkb : t.lmkb;  // (kappa/beta) l(+-1)
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        R f[NP];
        load_line<R, NP>(sfv + ((le * D + k) * NW + c) * NPE + fn * NP, f);
        const R* L = c < D ? Lmu : Lkb;
        R acc = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) acc = fma(L[j], f[j], acc);
        if constexpr (TO_SMEM)
          fo[((le * NF + slot) * NW + c) * NFN + fn] = acc;
        else
          FVtr[(size_t)slot * p.nfe + (e * NFN + fn) + c * pl] = acc;
      }
    }
  }
  __syncthreads();
}

// BR1 lifting (Sec. 3.1) in weak form with the central flux,
//   Q_{k,w}(i) = (2/h_k) [ -sum_j (w_j/w_i) l_i'(xi_j) w_j + (w*_{k,+} l_i(1) - w*_{k,-} l_i(-1)) / w_i ]
// (evaluated with the 2/h_k-scaled tables dk, lpk, lmk),
// w = (v, c) formed from the conservative traces on both sides of each face; then the
// face-normal viscous flux F^v_k = (tau_{.k}, (kappa/beta) c_{x_k}) traced onto the
// element's own faces (FVtr[c][slot][E][nfn]) for the face flux.
// MODEL 1 (original NSK equations, state (rho, m)): w = (v, rho), and instead of the viscous
// flux traces the kernel writes into FVtr the trace of (grad rho)_k on the element's faces of
// direction k ([2d][E][nfn], one component), the input of the second lifting.
// QF (model II only): Q receives the viscous form (visc_store) instead of the gradients, for the
// volume kernel of a residual or Runge-Kutta stage; without it the gradients (nsk_lift, the
// diagnostics).
template <typename R, int D, int NP, int G, int MODEL = 0, bool QF = (MODEL == 0)>
__device__ __forceinline__ void lift_group(const NskParams& p, const R* __restrict__ U, const R* __restrict__ Utr,
                                           R* __restrict__ Q, R* __restrict__ FVtr, const long long e0, R* sm,
                                           int& eflag) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NW = S::NW, NF = S::NF, NQ = S::NQ;
  constexpr int NV = MODEL == 1 ? D + 1 : S::NV;  // conservative variables
  constexpr int NT = NV + TraceComps<R>::extra;
  constexpr bool LINES = lift_lines<R, D, NP, G>();
  constexpr int NCOPY = LINES ? D : 1, SWS = lift_slot_stride<D, NP>();
  R* sw = sm;                           // [G][NCOPY][NW][NPE] primitive variables at the nodes
  R* sws = sm + G * NCOPY * NW * NPE;   // [G][NF][SWS >= NW NFN] central flux w* on the faces
  R* tb = sm + lift_work_smem<R, D, NP, G>();  // direction operators
  const auto& t = TabSel<R>::get(p);
  const int le = threadIdx.x / NPE, n = threadIdx.x % NPE;
  const int e = (int)e0 + le;
  const bool valid = le < G && e < p.E;
  const size_t nn = (size_t)p.nne;             // distance between the planes of two nodal variables
  const size_t pl = (size_t)NF * p.nfe;        // distance between the planes of two trace variables
  const int g = e * NPE + n;

  stage_tables<R, D, NP>(t, tb, R(1), R(0.5));
  if (valid) {
    lift_store_w<R, D, NP, G, MODEL>(U + g, nn, sw, le, n, eflag);
    const ElemIdx ex = elem_idx<D>(p, e);
    // a fixed trip count (the last round predicated): the gathers of all rounds are in flight together
#pragma unroll
    for (int r = 0; r < (NF * NFN + NPE - 1) / NPE; ++r) {
      const int it = n + r * NPE;
      if (it >= NF * NFN) break;
      const int slot = it / NFN, fn = it % NFN, k = slot >> 1, s = slot & 1;
      const int en = nbr_of(p, ex, k, s ? 1 : -1);
      const int oslot = 2 * k + (1 - s);
      const R* to = Utr + (size_t)slot * p.nfe + (e * NFN + fn);
      const R* tn = Utr + (size_t)oslot * p.nfe + (en * NFN + fn);
      R uo[NT], un[NT];
#pragma unroll
      for (int v = 0; v < NT; ++v) {
        uo[v] = to[v * pl];
        un[v] = tn[v * pl];
      }
      lift_wstar<R, D, NFN, NV, MODEL>(uo, un, sws + (le * NF + slot) * SWS + fn, eflag);
    }
  }
  __syncthreads();

  R q[NQ];
  if (valid) {
    lift_q<R, D, NP, G>(tb, sw, sws, le, n, q);
    if constexpr (!QF) {
#pragma unroll
      for (int c = 0; c < NQ; ++c) Q[c * nn + g] = q[c];
    }
  }
  __syncthreads();  // shared memory is reused below

  if constexpr (MODEL == 1) {
    R* sg = sm;  // [G][D][NPE] grad rho at the nodes, lines in direction k contiguous
    if (valid) {
#pragma unroll
      for (int k = 0; k < D; ++k) sg[(le * D + k) * NPE + line_pos<D, NP>(n, k)] = q[k * NW + D];
    }
    __syncthreads();
    if (valid) {
      for (int it = n; it < NF * NFN; it += NPE) {
        const int slot = it / NFN, fn = it % NFN, k = slot >> 1;
        const R* L = (slot & 1) ? t.lp : t.lm;
        R f[NP];
        load_line<R, NP>(sg + (le * D + k) * NPE + fn * NP, f);
        R acc = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) acc = fma(L[j], f[j], acc);
        FVtr[(size_t)slot * p.nfe + (e * NFN + fn)] = acc;
      }
    }
    __syncthreads();  // the caller may reuse shared memory
    return;
  }
  // [G][D][NW][NPE] the viscous flux F^v_k at the nodes without its coefficients (the stress
  // tau / mu and grad c), lines in direction k contiguous; mu and kappa/beta are folded into
  // the face interpolation
  R tau[D][D], gc[D];
  if (valid) {
    visc_of<R, D>(q, tau, gc);
    if constexpr (QF) visc_store<R, D>(tau, gc, Q, nn, g);
  }
  lift_fv_traces<R, D, NP, G>(p, tau, gc, sm, valid, le, n, e, FVtr, nullptr);
}

// a[1 + k] for a runtime direction k through selects over compile-time indices, so that the
// arrays stay in registers (an index unknown at compile time sends an array to local memory)
template <int D, typename R>
__device__ __forceinline__ R comp1(const R* a, const int k) {
  R r = a[1];
  if constexpr (D > 1) r = k == 1 ? a[2] : r;
  if constexpr (D > 2) r = k == 2 ? a[3] : r;
  return r;
}

// The flux of face_flux (below) from the two sides' trace values: UL, UR the conservative traces (and
// in FP64 the planes 1/rho, 1/(3 - rho) after them), VL, VR the face-normal viscous fluxes.
template <typename R, int D, int NP>
__device__ __forceinline__ void face_flux_vals(const NskParams& p, const R* UL, const R* UR, const R* VL,
                                               const R* VR, const int k, R* F, int& eflag) {
  using S = Shape<D, NP>;
  constexpr int NV = S::NV;
  R pl, dl, pr, dr, il, ir;
  if constexpr (TraceComps<R>::extra > 0) {
    il = UL[NV];
    ir = UR[NV];
    Eos<R>::both_q(p, UL[0], UL[NV + 1], pl, dl);
    Eos<R>::both_q(p, UR[0], UR[NV + 1], pr, dr);
  } else {
    Eos<R>::both(p, UL[0], pl, dl);
    Eos<R>::both(p, UR[0], pr, dr);
    il = R(1) / UL[0];
    ir = R(1) / UR[0];
  }
  eflag |= rho_flags(UL[0]) | rho_flags(UR[0]);
  if (!sound_ok(dl) || !sound_ok(dr)) eflag |= NSK_EBIT_SOUND;
  if (p.flux == NSK_FLUX_HLLC) {
    // HLLC of the barotropic system (rho, m) with p_alpha (see nsk_set_flux): the physical flux
    // of the upwind side K, plus S_K (U*_K - U_K) inside the star region; c is not transported
    const R mL = comp1<D>(UL, k), mR = comp1<D>(UR, k);
    const R ul = mL * il, ur = mR * ir;
    const R al = sqrt_s(dl), ar = sqrt_s(dr);
    const R SL = fmin(ul - al, ur - ar), SR = fmax(ul + al, ur + ar);
    const R wl = UL[0] * (SL - ul), wr = UR[0] * (SR - ur);  // rho_K (S_K - u_K), wl < 0 < wr
    const R Ss = (pr - pl + fma(wl, ul, -(wr * ur))) / (wl - wr);
    const bool star = SL < R(0) && SR > R(0);
    const bool left = SL >= R(0) || (star && Ss >= R(0));
    R uk[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) uk[v] = left ? UL[v] : UR[v];
    const R ik = left ? il : ir, pk = left ? pl : pr;
    const R mk = left ? mL : mR, vk = left ? ul : ur;  // vk = mk ik: the upwind normal velocity
    // the direction k is a runtime value: the normal component is formed once and each component
    // selects it, the tangential ones from the upwind velocities v_a = m_a ik (same products)
    R va[D];
#pragma unroll
    for (int a = 0; a < D; ++a) va[a] = uk[1 + a] * ik;
    F[0] = mk;
    const R fnn = fma(mk, vk, pk);
#pragma unroll
    for (int a = 0; a < D; ++a) F[1 + a] = (a == k) ? fnn : mk * va[a];
    if (star) {
      const R SK = left ? SL : SR;
      const R coef = (left ? wl : wr) / (SK - Ss);  // rho of U*_K
      F[0] = fma(SK, coef - uk[0], F[0]);
      const R usn = coef * Ss;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const R us = (a == k) ? usn : coef * va[a];
        F[1 + a] = fma(SK, us - uk[1 + a], F[1 + a]);
      }
    }
    F[0] = R(2) * F[0];
#pragma unroll
    for (int a = 0; a < D; ++a) F[1 + a] = fma(R(2), F[1 + a], -(VL[a] + VR[a]));
    F[D + 1] = -(VL[D] + VR[D]);
    return;
  }
  const R mL = comp1<D>(UL, k), mR = comp1<D>(UR, k);  // normal momenta
  const R vl = mL * il, vr = mR * ir;                  // normal velocities
  const R lam_l = fabs(vl) + sqrt_s(dl), lam_r = fabs(vr) + sqrt_s(dr);
  const R lam = lam_l > lam_r ? lam_l : lam_r;
  F[0] = mL + mR;
  // m_k v_a summed over both sides: the normal component m_k v_k + p_alpha once, the tangential
  // ones as v_k m_a (the direction k is a runtime value: each component selects between them)
  const R fnn = fma(mL, vl, pl) + fma(mR, vr, pr);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const R sum = (a == k) ? fnn : fma(vl, UL[1 + a], vr * UR[1 + a]);
    F[1 + a] = sum - (VL[a] + VR[a]);
  }
  F[D + 1] = -(VL[D] + VR[D]);
#pragma unroll
  for (int v = 0; v < NV - 1; ++v) F[v] = fma(-lam, UR[v] - UL[v], F[v]);
  if (p.c_diss) F[NV - 1] = fma(-lam, UR[NV - 1] - UL[NV - 1], F[NV - 1]);
}


// Numerical flux on the face between eL (its +1 side, slot 2k+1) and eR (its -1 side,
// slot 2k), face node fn (HLLC instead of the Lax-Friedrichs flux when p.flux says so,
// see nsk_set_flux):
//   F* = (F^c_k(U_L) + F^c_k(U_R))/2 - lambda/2 (U_R - U_L) - (F^v_L + F^v_R)/2,
//   lambda = max(|v_{L,k}| + sqrt(p_alpha'(rho_L)), |v_{R,k}| + sqrt(p_alpha'(rho_R)))
// (local Lax-Friedrichs with the model II wave speeds, Eq. parabolic_eigenvalues_model2;
// BR1 viscous flux). The jump term acts on rho and momentum (c has no convective flux)
// unless c_diss is set. F receives 2 F* (the 1/2 is applied by the volume kernel's staged
// surface operators; scaling by 2 is exact, so the residual is unchanged bit for bit).
template <typename R, int D, int NP>
__device__ __forceinline__ void face_flux(const NskParams& p, const R* __restrict__ Utr, const R* __restrict__ FVtr,
                                          const int eL, const int eR, const int k, const int fn,
                                          R* F, int& eflag) {
  using S = Shape<D, NP>;
  constexpr int NFN = S::NFN, NF = S::NF, NV = S::NV, NW = S::NW, NT = NV + TraceComps<R>::extra;
  const size_t ps = (size_t)NF * p.nfe;  // distance between the planes of two trace variables
  const size_t oL = (size_t)(2 * k + 1) * p.nfe + (eL * NFN + fn), oR = (size_t)(2 * k) * p.nfe + (eR * NFN + fn);
  const R* tL = Utr + oL;
  const R* tR = Utr + oR;
  R UL[NT], UR[NT], VL[NW], VR[NW];
#pragma unroll
  for (int v = 0; v < NT; ++v) {
    UL[v] = tL[v * ps];
    UR[v] = tR[v * ps];
  }
#pragma unroll
  for (int c = 0; c < NW; ++c) {
    VL[c] = FVtr[oL + c * ps];
    VR[c] = FVtr[oR + c * ps];
  }
  face_flux_vals<R, D, NP>(p, UL, UR, VL, VR, k, F, eflag);
}

// Fstar[v][k][E][nfn]: twice the flux on face (e, +k) at face node fn.
template <typename R, int D, int NP>
__device__ __forceinline__ void face_at(const NskParams& p, const R* __restrict__ Utr, const R* __restrict__ FVtr,
                                        R* __restrict__ Fstar, const int k, const int e, const int fn, int& eflag) {
  using S = Shape<D, NP>;
  constexpr int NFN = S::NFN, NV = S::NV;
  R F[NV];
  face_flux<R, D, NP>(p, Utr, FVtr, e, nbr_of(p, elem_idx<D>(p, e), k, 1), k, fn, F, eflag);
  R* o = Fstar + (size_t)k * p.nfe + (e * NFN + fn);
#pragma unroll
  for (int v = 0; v < NV; ++v) o[(size_t)v * D * p.nfe] = F[v];
}

// one item of the face pass, idx = (k, e, fn) flattened (idx / nfn < 2^31)
template <typename R, int D, int NP>
__device__ __forceinline__ void face_item(const NskParams& p, const R* __restrict__ Utr, const R* __restrict__ FVtr,
                                          R* __restrict__ Fstar, const long long idx, int& eflag) {
  using S = Shape<D, NP>;
  const int fn = (int)(idx % S::NFN);
  const unsigned r = (unsigned)(idx / S::NFN);
  const unsigned k = fdiv(r, p.fd_E);
  const int e = (int)(r - k * (unsigned)p.E);
  face_at<R, D, NP>(p, Utr, FVtr, Fstar, (int)k, e, fn, eflag);
}

// shared memory (in units of R) of volume_group
template <typename R, int D, int NP, int G, bool FUSED>
__host__ __device__ constexpr int volume_smem() {
  using S = Shape<D, NP>;
  return G * D * S::NV * S::NPE + G * S::NF * S::NV * S::NFN + tab_smem<D, NP>() + 2;
}

// ---- parts of the volume kernel, shared by the stage kernels (so every schedule rounds alike) ----

// direction operators for the residual (scaled by sc: 1 for a residual, dt in a Runge-Kutta
// stage, where the contraction then yields dt R), then alpha sc and (alpha/beta) sc
template <typename R, int D, int NP>
__device__ __forceinline__ void volume_tables(const NskTab<R>& t, R* tb, const R sc) {
  stage_tables<R, D, NP>(t, tb, sc, R(0.5) * sc);
  if (threadIdx.x == 0) {
    tb[tab_smem<D, NP>()] = t.alpha * sc;
    tb[tab_smem<D, NP>() + 1] = t.ab * sc;
  }
}

// The nodal fluxes F_k = F^c_k - F^v_k of node n (c flux without its factor -kappa/beta, which
// is applied after the sum), stored with the lines of direction k contiguous:
// sf[((le D + k) NV + v) NPE + face_node(n, k) NP + i_k]. u: the conservative variables, tau the
// stress without mu and gc the gradient of c at the node.
template <typename R, int D, int NP>
__device__ __forceinline__ void volume_node_fluxes(const NskParams& p, const R* u, const R (&tau)[D][D],
                                                   const R* gc, R* sf, const int le, const int n) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NV = S::NV;
  const auto& t = TabSel<R>::get(p);
  R inv, pa;
  if constexpr (TraceComps<R>::extra > 0) {  // FP64: one division for 1/rho and 1/(3 - rho)
    const R dd = rcp_s(u[0] * (R(3) - u[0]));
    inv = (R(3) - u[0]) * dd;
    pa = Eos<R>::pa_q(p, u[0], u[0] * dd);
  } else {
    inv = R(1) / u[0];
    pa = Eos<R>::pa(p, u[0]);
  }
  const R mu = t.mu;
  // the convective momentum flux m_k v_a + p_alpha delta_ka: symmetric, so each pair k < a is
  // formed once as m_k v_a and serves (a, k) as well
  R vel[D], off[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) vel[a] = u[1 + a] * inv;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i + 1; j < D; ++j) off[i][j] = u[1 + i] * vel[j];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    // node n sits at position i_k of line face_node(n, k) in direction k
    R* f = sf + ((le * D + k) * NV) * NPE + face_node<D, NP>(n, k) * NP + coord<NP>(n, k);
    f[0] = u[1 + k];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const R fc = (a == k) ? fma(u[1 + k], vel[k], pa) : (k < a ? off[k][a] : off[a][k]);
      f[(1 + a) * NPE] = fma(-mu, tau[k][a], fc);
    }
    f[(D + 1) * NPE] = gc[k];  // the c flux -(kappa/beta) grad c, its factor applied after the sum
  }
}

// The residual of node n from the staged nodal fluxes sf and face fluxes sfs (2 F*), plus the
// sources, then: mode RHS, Rout = R; else K <- A K + dt R, U <- U + B K (u updated in place).
template <typename R, int D, int NP, int G>
__device__ __forceinline__ void volume_residual_update(const NskParams& p, const R* tb, const R* sf, const R* sfs,
                                                       R* u, const R* gc, const R* kin, const int mode, const R A,
                                                       const R B, R* __restrict__ U, R* __restrict__ K,
                                                       R* __restrict__ Rout, const int g, const int le,
                                                       const int n) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NV = S::NV, NF = S::NF;
  const auto& t = TabSel<R>::get(p);
  const size_t nn = (size_t)p.nne;  // distance between the planes of two nodal variables
  // res_v = sum_k [ sum_j dk[i][j] F_k(j) - F*_{k,+} lpk[i] + F*_{k,-} lmk[i] ]  (2/h_k folded in),
  // accumulated over k in ascending order
  // (the c equation's volume part, a sum over grad c, is kept apart and scaled by
  // -kappa/beta once)
  R res[NV], volc = 0;
#pragma unroll
  for (int v = 0; v < NV; ++v) res[v] = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int i = coord<NP>(n, k), fn = face_node<D, NP>(n, k);
    R dk[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) dk[j] = tb[(k * NP + i) * NP + j];
    const R lpk = tb[D * NP * NP + k * NP + i], lmk = tb[D * NP * NP + D * NP + k * NP + i];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      R fl[NP];
      load_line<R, NP>(sf + ((le * D + k) * NV + v) * NPE + fn * NP, fl);
      R acc = v == NV - 1 ? volc : res[v];
#pragma unroll
      for (int j = 0; j < NP; ++j) acc = fma(dk[j], fl[j], acc);
      const R fp = sfs[((le * NF + 2 * k + 1) * NV + v) * NFN + fn];
      const R fm = sfs[((le * NF + 2 * k) * NV + v) * NFN + fn];
      if (v == NV - 1) {
        volc = acc;
        res[v] = fma(fm, lmk, fma(-fp, lpk, res[v]));
      } else {
        res[v] = fma(fm, lmk, fma(-fp, lpk, acc));
      }
    }
  }
  res[NV - 1] = fma(-t.kb, volc, res[NV - 1]);
  const R alpha = tb[tab_smem<D, NP>()], ab = tb[tab_smem<D, NP>() + 1];  // scaled like the operators
#pragma unroll
  for (int a = 0; a < D; ++a) res[1 + a] = fma(alpha * u[0], gc[a], res[1 + a]);
  res[D + 1] = fma(ab, u[0] - u[D + 1], res[D + 1]);

  if (mode == NSK_MODE_RHS) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Rout[v * nn + g] = res[v];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R kv = fma(A, kin[v], res[v]);  // res holds dt R
      K[v * nn + g] = kv;
      u[v] = fma(B, kv, u[v]);
      U[v * nn + g] = u[v];
    }
  }
}

// The traces of the element's (new) state u on its own faces into UtrNext, through shared
// memory su ([G][NV][NPE]); starts and ends with a block barrier.
template <typename R, int D, int NP, int G>
__device__ __forceinline__ void volume_write_traces(const NskParams& p, const R* u, R* su, R* __restrict__ UtrNext,
                                                    const bool valid, const int le, const int n, const int e) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NV = S::NV, NF = S::NF;
  __syncthreads();  // su may alias buffers still being read
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) su[(le * NV + v) * NPE + n] = u[v];
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int r = 0; r < (NF * NFN + NPE - 1) / NPE; ++r) {
      const int it = n + r * NPE;
      if (it >= NF * NFN) break;
      prolong_trace<R, D, NP>(p, su + le * NV * NPE, NPE, UtrNext, e, it / NFN, it % NFN);
    }
  }
  __syncthreads();
}

// Weak-form volume integral and surface lifting (Eq. weakformulation),
//   R_i = sum_k (2/h_k) [ sum_j (w_j/w_i) l_i'(xi_j) F_k(U_j, Q_j) - (F*_{k,+} l_i(1) - F*_{k,-} l_i(-1)) / w_i ] + S_i,
// F_k = F^c_k - F^v_k, S = (0, alpha rho grad c, (alpha/beta)(rho - c)); then
// mode RHS: Rout = R; mode LSRK: K <- A K + dt R, U <- U + B K (dt folded into the staged
// operators and source coefficients, so the contraction yields dt R).
// The fluxes of the element's 2d faces are staged in shared memory: read from Fstar with
// coalesced loads, or, FUSED, evaluated by the element itself (each face is then
// evaluated by both neighbours, bit-identically). Both hold 2 F*: the staged lpk, lmk
// carry the 1/2.
// UtrNext (optional): the traces of the element's new state (LSRK) or of its state (RHS)
// are written there from shared memory, so the next stage needs no prolongation pass.
// It must not alias Utr when FUSED (neighbours still read Utr).
// ASYNC (separate face schedule): Fstar is in global memory and staged with cp.async; false when
// it is in shared memory (the single-block kernel), where plain copies stage it.
template <typename R, int D, int NP, int G, bool FUSED, bool QF = true, bool ASYNC = true>
__device__ __forceinline__ void volume_group(const NskParams& p, R* __restrict__ U, const R* __restrict__ Q,
                                             const R* __restrict__ Fstar, const R* __restrict__ Utr,
                                             const R* __restrict__ FVtr, R* __restrict__ K, R* __restrict__ Rout,
                                             const int mode, const R A, const R B, const R dt, const long long e0,
                                             R* sm, int& eflag, R* __restrict__ UtrNext = nullptr) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NV = S::NV, NQ = S::NQ, NF = S::NF;
  R* sf = sm;                          // [G][D][NV][NFN][NP] fluxes F_k at the nodes, lines in k contiguous
  R* sfs = sm + G * D * NV * NPE;      // [G][NF][NV][NFN] fluxes of the element's faces
  R* tb = sfs + G * NF * NV * NFN;     // direction operators, then the source coefficients
  const auto& t = TabSel<R>::get(p);
  const int le = threadIdx.x / NPE, n = threadIdx.x % NPE;
  const int e = (int)e0 + le;
  const bool valid = le < G && e < p.E;
  const size_t nn = (size_t)p.nne;  // distance between the planes of two nodal variables
  const int g = e * NPE + n;

  if constexpr (!FUSED) {
    // Fstar[v][k][E][nfn] holds the flux on face (e, +k): slot 2k+1 is the element's own
    // entry, slot 2k its -k neighbour's. Copied global -> shared asynchronously, so that the
    // copies are in flight during the nodal loads and flux arithmetic below and hold no registers.
    // A face's NFN values of one variable are contiguous on both sides: copied 16 bytes at a
    // time when NFN values fill whole 16-byte units (the offsets below are then multiples of 16
    // bytes: Fstar and the shared buffer start 16-byte aligned and nfe = E NFN).
    // Each thread keeps one (variable, piece) and walks the NF face slots.
    constexpr int W = (NFN * (int)sizeof(R)) % 16 == 0 ? 16 / (int)sizeof(R) : 1;
    constexpr int NFW = NFN / W, NQV = NV * NFW, PER = NPE / NQV;
    if constexpr (PER >= 1) {
      if (valid && n < PER * NQV) {
        const ElemIdx ex = elem_idx<D>(p, e);
        const int q = n % NQV, v = q / NFW, fn = (q % NFW) * W;
        R* sb = sfs + (le * NF * NV + v) * NFN + fn;
        for (int slot = n / NQV; slot < NF; slot += PER) {
          const int k = slot >> 1;
          const int src = (slot & 1) ? e : nbr_of(p, ex, k, -1);
          R* dst = sb + slot * NV * NFN;
          const R* srcp = Fstar + (size_t)(v * D + k) * p.nfe + (src * NFN + fn);
          stage_copy<ASYNC, W>(dst, srcp);
        }
      }
    } else if (valid) {
      const ElemIdx ex = elem_idx<D>(p, e);
      for (int it = n; it < NF * NV * NFW; it += NPE) {
        const int fn = (it % NFW) * W, v = (it / NFW) % NV, slot = it / (NV * NFW), k = slot >> 1;
        const int src = (slot & 1) ? e : nbr_of(p, ex, k, -1);
        R* dst = sfs + ((le * NF + slot) * NV + v) * NFN + fn;
        const R* srcp = Fstar + (size_t)(v * D + k) * p.nfe + (src * NFN + fn);
        stage_copy<ASYNC, W>(dst, srcp);
      }
    }
    if constexpr (ASYNC) cp_async_commit();
  }
  volume_tables<R, D, NP>(t, tb, mode == NSK_MODE_RHS ? R(1) : dt);
  R u[NV], kin[NV], tau[D][D], gc[D];
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = U[v * nn + g];
    if (mode != NSK_MODE_RHS) {  // the RK register is needed only at the end: load it early
#pragma unroll
      for (int v = 0; v < NV; ++v) kin[v] = K[v * nn + g];
    }
    if constexpr (QF) {  // the lifting stored the viscous form
      visc_load<R, D>(Q, nn, g, tau, gc);
    } else {
      R q[NQ];
#pragma unroll
      for (int c = 0; c < NQ; ++c) q[c] = Q[c * nn + g];
      visc_of<R, D>(q, tau, gc);
    }
    volume_node_fluxes<R, D, NP>(p, u, tau, gc, sf, le, n);
    if constexpr (FUSED) {
      const ElemIdx ex = elem_idx<D>(p, e);
      for (int it = n; it < NF * NFN; it += NPE) {
        const int slot = it / NFN, fn = it % NFN, k = slot >> 1;
        R F[NV];
        if (slot & 1)
          face_flux<R, D, NP>(p, Utr, FVtr, e, nbr_of(p, ex, k, 1), k, fn, F, eflag);
        else
          face_flux<R, D, NP>(p, Utr, FVtr, nbr_of(p, ex, k, -1), e, k, fn, F, eflag);
#pragma unroll
        for (int v = 0; v < NV; ++v) sfs[((le * NF + slot) * NV + v) * NFN + fn] = F[v];
      }
    }
  }
  if constexpr (!FUSED && ASYNC) cp_async_wait_all();
  __syncthreads();

  if (valid) volume_residual_update<R, D, NP, G>(p, tb, sf, sfs, u, gc, kin, mode, A, B, U, K, Rout, g, le, n);
  if (UtrNext != nullptr)  // uniform over the block
    volume_write_traces<R, D, NP, G>(p, u, sm, UtrNext, valid, le, n, e);
  else
    __syncthreads();  // the caller may reuse shared memory
}

// ---- lean stage (schedule fused_face = 2): two launches, no gradients or face fluxes in HBM ----
// Of everything the lifting computes, only the face-normal viscous flux F^v of an element's own
// faces is needed by another element (its face neighbour's flux), so the lean lifting writes
// just those traces; the lean volume kernel then recomputes the element's lifting on chip from
// its state and the neighbours' stored state traces, evaluates its 2d faces' fluxes with the
// neighbours' F^v traces, and does the volume integral, sources and update. Each element's own
// traces are prolonged on chip from its staged state. Every value is computed by the same
// functions as in the other schedules, so the results are the same bit for bit.

// shared memory (units of R) of lift_lean_group: the lifting's buffers and tables, then the
// element's staged state [G][NV][NPE]
template <typename R, int D, int NP, int G>
__host__ __device__ constexpr int lift_lean_smem() {
  return lift_smem<R, D, NP, G>() + G * Shape<D, NP>::NV * Shape<D, NP>::NPE;
}

template <typename R, int D, int NP, int G>
__device__ __forceinline__ void lift_lean_group(const NskParams& p, const R* __restrict__ U,
                                                const R* __restrict__ Utr, R* __restrict__ FVtr, const long long e0,
                                                R* sm, int& eflag) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NW = S::NW, NF = S::NF, NQ = S::NQ, NV = S::NV;
  constexpr int NT = NV + TraceComps<R>::extra;
  constexpr bool LINES = lift_lines<R, D, NP, G>();
  constexpr int NCOPY = LINES ? D : 1, SWS = lift_slot_stride<D, NP>();
  R* sw = sm;                                   // [G][NCOPY][NW][NPE] primitive variables
  R* sws = sm + G * NCOPY * NW * NPE;           // [G][NF][SWS] 2 w* on the faces
  R* tb = sm + lift_work_smem<R, D, NP, G>();   // direction operators
  R* su = tb + tab_smem<D, NP>();               // [G][NV][NPE] the element's state
  const auto& t = TabSel<R>::get(p);
  const int le = threadIdx.x / NPE, n = threadIdx.x % NPE;
  const int e = (int)e0 + le;
  const bool valid = le < G && e < p.E;
  const size_t nn = (size_t)p.nne;
  const size_t pl = (size_t)NF * p.nfe;
  const int g = e * NPE + n;

  stage_tables<R, D, NP>(t, tb, R(1), R(0.5));
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) su[(le * NV + v) * NPE + n] = U[v * nn + g];
  }
  __syncthreads();
  if (valid) {
    const R* ue = su + le * NV * NPE;
    lift_store_w<R, D, NP, G>(ue + n, NPE, sw, le, n, eflag);
    const ElemIdx ex = elem_idx<D>(p, e);
#pragma unroll
    for (int r = 0; r < (NF * NFN + NPE - 1) / NPE; ++r) {
      const int it = n + r * NPE;
      if (it >= NF * NFN) break;
      const int slot = it / NFN, fn = it % NFN, k = slot >> 1, s = slot & 1;
      const int en = nbr_of(p, ex, k, s ? 1 : -1);
      const R* tn = Utr + (size_t)(2 * k + (1 - s)) * p.nfe + (en * NFN + fn);
      R uo[NT], un[NT];
#pragma unroll
      for (int v = 0; v < NT; ++v) un[v] = tn[v * pl];
      trace_vals<R, D, NP>(p, ue, NPE, slot, fn, uo);
      lift_wstar<R, D, NFN, NV>(uo, un, sws + (le * NF + slot) * SWS + fn, eflag);
    }
  }
  __syncthreads();
  R q[NQ], tau[D][D], gc[D];
  if (valid) {
    lift_q<R, D, NP, G>(tb, sw, sws, le, n, q);
    visc_of<R, D>(q, tau, gc);
  }
  __syncthreads();
  lift_fv_traces<R, D, NP, G>(p, tau, gc, sm, valid, le, n, e, FVtr, nullptr);
}

// shared memory layout (units of R) of volume_lean_group
template <typename R, int D, int NP, int G>
struct LeanSmem {
  using S = Shape<D, NP>;
  static constexpr int NT = S::NV + TraceComps<R>::extra;
  static constexpr bool LINES = lift_lines<R, D, NP, G>();
  static constexpr int NCOPY = LINES ? D : 1;
  static constexpr int so = 0;                                  // [G][NF][NT][NFN] own state traces
  static constexpr int sn = so + G * S::NF * NT * S::NFN;       // [G][NF][NT][NFN] the neighbours' traces
  static constexpr int fo = sn + G * S::NF * NT * S::NFN;       // [G][NF][NW][NFN] own F^v traces
  static constexpr int fnb = fo + G * S::NF * S::NW * S::NFN;   // [G][NF][NW][NFN] the neighbours' F^v traces
  static constexpr int lift_work = G * NCOPY * S::NW * S::NPE + G * S::NF * lift_slot_stride<D, NP>();
  static constexpr int vol_work = G * D * S::NV * S::NPE;
  static constexpr int fv_work = G * D * S::NW * S::NPE;
  static constexpr int wmax = lift_work > vol_work ? (lift_work > fv_work ? lift_work : fv_work)
                                                   : (vol_work > fv_work ? vol_work : fv_work);
  static constexpr int work = fnb + G * S::NF * S::NW * S::NFN;  // lifting, then F^v at nodes, then sf
  static constexpr int sfs = work + ((wmax + 3) & ~3);          // [G][NF][NV][NFN] 2 F* of the faces
  static constexpr int t1 = sfs + G * S::NF * S::NV * S::NFN;   // lifting operators
  static constexpr int t2 = t1 + tab_smem<D, NP>();             // residual operators and source factors
  static constexpr int su = ((t2 + tab_smem<D, NP>() + 2) + 3) & ~3;  // [G][NV][NPE] the element's state
  static constexpr int total = su + G * S::NV * S::NPE;
};

template <typename R, int D, int NP, int G>
__host__ __device__ constexpr int volume_lean_smem() {
  return LeanSmem<R, D, NP, G>::total;
}

// Lean volume kernel body (see above): lifting on chip, face fluxes from the neighbours' state
// and F^v traces, volume integral + surface lifting + sources + update (modes RHS or LSRK), and
// the traces of the new state into UtrNext (optional; must not alias Utr).
template <typename R, int D, int NP, int G>
__device__ __forceinline__ void volume_lean_group(const NskParams& p, R* __restrict__ U, const R* __restrict__ Utr,
                                                  const R* __restrict__ FVtr, R* __restrict__ K, R* __restrict__ Rout,
                                                  const int mode, const R A, const R B, const R dt,
                                                  const long long e0, R* sm, int& eflag, R* __restrict__ UtrNext) {
  using S = Shape<D, NP>;
  using L = LeanSmem<R, D, NP, G>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NW = S::NW, NV = S::NV, NQ = S::NQ, NF = S::NF, NT = L::NT;
  constexpr int SWS = lift_slot_stride<D, NP>();
  R* so = sm + L::so;
  R* sn = sm + L::sn;
  R* fo = sm + L::fo;
  R* fnb = sm + L::fnb;
  R* work = sm + L::work;
  R* sw = work;                                 // lifting: [G][NCOPY][NW][NPE]
  R* sws = work + G * L::NCOPY * NW * NPE;       //          [G][NF][SWS]
  R* sfs = sm + L::sfs;
  R* t1 = sm + L::t1;
  R* t2 = sm + L::t2;
  R* su = sm + L::su;
  const auto& t = TabSel<R>::get(p);
  const int le = threadIdx.x / NPE, n = threadIdx.x % NPE;
  const int e = (int)e0 + le;
  const bool valid = le < G && e < p.E;
  const size_t nn = (size_t)p.nne;
  const size_t pl = (size_t)NF * p.nfe;
  const int g = e * NPE + n;

  // the neighbours' state and F^v traces of every face, global -> shared asynchronously (16 bytes
  // at a time when a face's NFN values fill whole 16-byte units; the offsets are then multiples
  // of 16 bytes), stored under the element's own face slot
  {
    constexpr int W = (NFN * (int)sizeof(R)) % 16 == 0 ? 16 / (int)sizeof(R) : 1;
    constexpr int NFW = NFN / W;
    if (valid) {
      const ElemIdx ex = elem_idx<D>(p, e);
      for (int it = n; it < NF * (NT + NW) * NFW; it += NPE) {
        const int piece = it % NFW, c = (it / NFW) % (NT + NW), slot = it / ((NT + NW) * NFW);
        const int k = slot >> 1, s = slot & 1;
        const int en = nbr_of(p, ex, k, s ? 1 : -1);
        const size_t src = (size_t)(2 * k + (1 - s)) * p.nfe + (en * NFN + piece * W);
        R* dst;
        const R* srcp;
        if (c < NT) {
          dst = sn + ((le * NF + slot) * NT + c) * NFN + piece * W;
          srcp = Utr + src + c * pl;
        } else {
          dst = fnb + ((le * NF + slot) * NW + (c - NT)) * NFN + piece * W;
          srcp = FVtr + src + (c - NT) * pl;
        }
        if constexpr (W > 1)
          cp_async_16(dst, srcp);
        else
          cp_async_elem(dst, srcp);
      }
    }
    cp_async_commit();
  }
  stage_tables<R, D, NP>(t, t1, R(1), R(0.5));
  volume_tables<R, D, NP>(t, t2, mode == NSK_MODE_RHS ? R(1) : dt);
  R u[NV], kin[NV], tau[D][D], gc[D];
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u[v] = U[v * nn + g];
      su[(le * NV + v) * NPE + n] = u[v];
    }
    if (mode != NSK_MODE_RHS) {
#pragma unroll
      for (int v = 0; v < NV; ++v) kin[v] = K[v * nn + g];
    }
  }
  __syncthreads();
  if (valid) {  // own traces on chip, and the primitive variables for the lifting
    const R* ue = su + le * NV * NPE;
    lift_store_w<R, D, NP, G>(ue + n, NPE, sw, le, n, eflag);
    for (int it = n; it < NF * NFN; it += NPE) {
      const int slot = it / NFN, fn = it % NFN;
      R uo[NT];
      trace_vals<R, D, NP>(p, ue, NPE, slot, fn, uo);
#pragma unroll
      for (int v = 0; v < NT; ++v) so[((le * NF + slot) * NT + v) * NFN + fn] = uo[v];
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (valid) {  // 2 w* of every face node
    for (int it = n; it < NF * NFN; it += NPE) {
      const int slot = it / NFN, fn = it % NFN;
      R uo[NT], un[NT];
#pragma unroll
      for (int v = 0; v < NT; ++v) {
        uo[v] = so[((le * NF + slot) * NT + v) * NFN + fn];
        un[v] = sn[((le * NF + slot) * NT + v) * NFN + fn];
      }
      lift_wstar<R, D, NFN, NV>(uo, un, sws + (le * NF + slot) * SWS + fn, eflag);
    }
  }
  __syncthreads();
  if (valid) {
    R q[NQ];
    lift_q<R, D, NP, G>(t1, sw, sws, le, n, q);
    visc_of<R, D>(q, tau, gc);
  }
  __syncthreads();
  lift_fv_traces<R, D, NP, G, true>(p, tau, gc, work, valid, le, n, e, nullptr, fo);  // ends with a barrier
  if (valid) {
    for (int it = n; it < NF * NFN; it += NPE) {  // the fluxes of the element's faces
      const int slot = it / NFN, fn = it % NFN, k = slot >> 1;
      // +k face (odd slot): the element is the left state, its neighbour the right one
      const bool plus = (slot & 1) != 0;
      R UL[NT], UR[NT], VL[NW], VR[NW], F[NV];
#pragma unroll
      for (int v = 0; v < NT; ++v) {
        const R o = so[((le * NF + slot) * NT + v) * NFN + fn], x = sn[((le * NF + slot) * NT + v) * NFN + fn];
        UL[v] = plus ? o : x;
        UR[v] = plus ? x : o;
      }
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        const R o = fo[((le * NF + slot) * NW + c) * NFN + fn], x = fnb[((le * NF + slot) * NW + c) * NFN + fn];
        VL[c] = plus ? o : x;
        VR[c] = plus ? x : o;
      }
      face_flux_vals<R, D, NP>(p, UL, UR, VL, VR, k, F, eflag);
#pragma unroll
      for (int v = 0; v < NV; ++v) sfs[((le * NF + slot) * NV + v) * NFN + fn] = F[v];
    }
    volume_node_fluxes<R, D, NP>(p, u, tau, gc, work, le, n);
  }
  __syncthreads();
  if (valid) volume_residual_update<R, D, NP, G>(p, t2, work, sfs, u, gc, kin, mode, A, B, U, K, Rout, g, le, n);
  if (UtrNext != nullptr)  // uniform over the block
    volume_write_traces<R, D, NP, G>(p, u, su, UtrNext, valid, le, n, e);
}

// ---- stand-alone stage kernels ---------------------------------------------
// blk_off (every stage kernel): the index of the grid's first block, for launches over a range
// of whole blocks of the mesh (the host-state step's slabs); the bounds checks stay the mesh's.
// grid (ceil(E nfn / 256), 2d): blockIdx.y is the face slot
template <typename R, int D, int NP>
__global__ void __launch_bounds__(256) k_prolong(const NskParams p, const R* __restrict__ U, R* __restrict__ Utr,
                                                 const int blk_off = 0) {
  using S = Shape<D, NP>;
  const int idx = (blockIdx.x + blk_off) * blockDim.x + threadIdx.x;
  if (idx < p.nfe) {
    const int e = idx / S::NFN;
    prolong_trace<R, D, NP>(p, U + (size_t)e * S::NPE, (size_t)p.nne, Utr, e, blockIdx.y, idx % S::NFN);
  }
}

// blocks of TPB threads that fit in the given number of resident warps (a block holds whole
// warps), at least one
template <int TPB>
__host__ __device__ constexpr int blocks_in_warps(int warps) {
  return warps / ((TPB + 31) / 32) > 0 ? warps / ((TPB + 31) / 32) : 1;
}

// FP32 lifting: 48 resident warps, three quarters of an SM (the loads of the face loop need
// the latency hiding)
template <typename R, int TPB>
__host__ __device__ constexpr int lift_min_blocks() {
  return sizeof(R) == 4 ? blocks_in_warps<TPB>(48) : 1;
}

// QF: store the viscous form for a volume kernel (residual and Runge-Kutta stages), else the
// gradients (a lifting-only stage)
template <typename R, int D, int NP, int G, bool QF>
__global__ void __launch_bounds__(G * Shape<D, NP>::NPE, (lift_min_blocks<R, G * Shape<D, NP>::NPE>()))
    k_lift(const NskParams p, const R* __restrict__ U, const R* __restrict__ Utr, R* __restrict__ Q,
           R* __restrict__ FVtr, int* __restrict__ err, const int blk_off = 0) {
  __shared__ __align__(16) R sm[lift_smem<R, D, NP, G>()];
  int eflag = 0;
  lift_group<R, D, NP, G, 0, QF>(p, U, Utr, Q, FVtr, (long long)(blockIdx.x + blk_off) * G, sm, eflag);
  if (eflag) atomicOr(err, eflag);
}

// grid (ceil(E nfn / 256), d): blockIdx.y is the face direction; FP32: 75% of an SM's threads
template <typename R, int D, int NP>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 ? 6 : 1)) k_face(const NskParams p, const R* __restrict__ Utr,
                                              const R* __restrict__ FVtr, R* __restrict__ Fstar,
                                              int* __restrict__ err, const int blk_off = 0) {
  using S = Shape<D, NP>;
  const int idx = (blockIdx.x + blk_off) * blockDim.x + threadIdx.x;
  int eflag = 0;
  if (idx < p.nfe) face_at<R, D, NP>(p, Utr, FVtr, Fstar, blockIdx.y, idx / S::NFN, idx % S::NFN, eflag);
  if (eflag) atomicOr(err, eflag);
}

// FP32 volume kernel (separate face schedule): 48 resident warps, three quarters of an SM
template <typename R, int TPB, bool FUSED>
__host__ __device__ constexpr int volume_min_blocks() {
  return (sizeof(R) == 4 && !FUSED) ? blocks_in_warps<TPB>(48) : 1;
}

template <typename R, int D, int NP, int G, bool FUSED>
__global__ void __launch_bounds__(G * Shape<D, NP>::NPE, (volume_min_blocks<R, G * Shape<D, NP>::NPE, FUSED>()))
    k_volume(const NskParams p, R* __restrict__ U, const R* __restrict__ Q, const R* __restrict__ Fstar,
             const R* __restrict__ Utr, const R* __restrict__ FVtr, R* __restrict__ K, R* __restrict__ Rout,
             const int mode, const R A, const R B, const double* __restrict__ dtp, const R dtv,
             int* __restrict__ err, R* __restrict__ UtrNext, const int blk_off = 0) {
  __shared__ __align__(16) R sm[volume_smem<R, D, NP, G, FUSED>()];
  const R dt = dtp ? (R)*dtp : dtv;
  int eflag = 0;
  volume_group<R, D, NP, G, FUSED>(p, U, Q, Fstar, Utr, FVtr, K, Rout, mode, A, B, dt,
                                   (long long)(blockIdx.x + blk_off) * G, sm, eflag, UtrNext);
  if (eflag) atomicOr(err, eflag);
}

// lean schedule kernels (dynamic shared memory: their buffers can exceed the 48 KB static limit)
template <typename R, int D, int NP, int G>
__global__ void __launch_bounds__(G * Shape<D, NP>::NPE)
    k_lift_lean(const NskParams p, const R* __restrict__ U, const R* __restrict__ Utr, R* __restrict__ FVtr,
                int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char lean_smem_raw[];
  R* sm = reinterpret_cast<R*>(lean_smem_raw);
  int eflag = 0;
  lift_lean_group<R, D, NP, G>(p, U, Utr, FVtr, (long long)blockIdx.x * G, sm, eflag);
  if (eflag) atomicOr(err, eflag);
}

template <typename R, int D, int NP, int G>
__global__ void __launch_bounds__(G * Shape<D, NP>::NPE)
    k_volume_lean(const NskParams p, R* __restrict__ U, const R* __restrict__ Utr, const R* __restrict__ FVtr,
                  R* __restrict__ K, R* __restrict__ Rout, const int mode, const R A, const R B,
                  const double* __restrict__ dtp, const R dtv, int* __restrict__ err, R* __restrict__ UtrNext) {
  extern __shared__ __align__(16) unsigned char lean_smem_raw[];
  R* sm = reinterpret_cast<R*>(lean_smem_raw);
  const R dt = dtp ? (R)*dtp : dtv;
  int eflag = 0;
  volume_lean_group<R, D, NP, G>(p, U, Utr, FVtr, K, Rout, mode, A, B, dt, (long long)blockIdx.x * G, sm, eflag,
                                 UtrNext);
  if (eflag) atomicOr(err, eflag);
}

// ---- single-block schedule (fused_face = 3): a small mesh's whole call in one launch ----
// One block runs the stages of every step of a call (or one residual) phase after phase
// (prolongation, lifting, face fluxes, volume + update; block barriers between them) on copies of
// the context's arrays in shared memory, laid out with the same plane strides (nne, nfe), so the
// stage bodies run on them unchanged and round exactly as in the other schedules. The state and
// the RK register are copied in at the start and out at the end (the residual goes straight to
// global memory). Keeping the arrays on chip also keeps every value written and read again within
// the launch out of the read-only cache path that global loads may take.
template <typename R, int D, int NP, int G>
struct BlockLayout {
  using S = Shape<D, NP>;
  static constexpr int NT = S::NV + TraceComps<R>::extra;
  static constexpr int work = lift_smem<R, D, NP, G>() > volume_smem<R, D, NP, G, false>()
                                  ? lift_smem<R, D, NP, G>()
                                  : volume_smem<R, D, NP, G, false>();
  // offsets in units of R for a mesh of E elements (every array starts 16-byte aligned)
  static __host__ __device__ size_t up(size_t x) { return (x + 15) & ~(size_t)15; }
  static __host__ __device__ size_t U(long long) { return 0; }
  static __host__ __device__ size_t K(long long E) { return U(E) + up((size_t)S::NV * E * S::NPE); }
  static __host__ __device__ size_t Q(long long E) { return K(E) + up((size_t)S::NV * E * S::NPE); }
  static __host__ __device__ size_t Utr(long long E) { return Q(E) + up((size_t)S::NVF * E * S::NPE); }
  static __host__ __device__ size_t FVtr(long long E) { return Utr(E) + up((size_t)NT * S::NF * E * S::NFN); }
  static __host__ __device__ size_t Fstar(long long E) { return FVtr(E) + up((size_t)S::NW * S::NF * E * S::NFN); }
  static __host__ __device__ size_t Work(long long E) { return Fstar(E) + up((size_t)S::NV * D * E * S::NFN); }
  static __host__ __device__ size_t total(long long E) { return Work(E) + work; }
};

template <typename R, int D, int NP, int G>
__global__ void __launch_bounds__(G * Shape<D, NP>::NPE, 1)
    k_block_steps(const NskParams p, R* __restrict__ Ug, R* __restrict__ Kg, R* __restrict__ Rout, const int mode,
                  const NskLsrkCoef coef, const R dt, const int nsteps, int* __restrict__ err) {
  using S = Shape<D, NP>;
  using L = BlockLayout<R, D, NP, G>;
  extern __shared__ __align__(16) unsigned char block_smem_raw[];
  R* sm = reinterpret_cast<R*>(block_smem_raw);
  const long long E = p.E;
  R* U = sm + L::U(E);
  R* K = sm + L::K(E);
  R* Q = sm + L::Q(E);
  R* Utr = sm + L::Utr(E);
  R* FVtr = sm + L::FVtr(E);
  R* Fstar = sm + L::Fstar(E);
  R* work = sm + L::Work(E);
  const int nv = S::NV * p.nne;
  const bool rk = mode != NSK_MODE_RHS;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    U[i] = Ug[i];
    if (rk) K[i] = Kg[i];
  }
  __syncthreads();
  const int ngroups = (int)((E + G - 1) / G);
  const int nstage = rk ? 5 : 1;
  int eflag = 0;
  for (int step = 0; step < nsteps; ++step) {
    for (int st = 0; st < nstage; ++st) {
      if (step == 0 && st == 0) {  // later stages take the traces the volume phase wrote
        for (long long idx = threadIdx.x; idx < (long long)S::NF * p.nfe; idx += blockDim.x)
          prolong_item<R, D, NP>(p, U, Utr, idx);
        __syncthreads();
      }
      for (int gi = 0; gi < ngroups; ++gi)  // ends with a block barrier
        lift_group<R, D, NP, G, 0, true>(p, U, Utr, Q, FVtr, (long long)gi * G, work, eflag);
      for (long long idx = threadIdx.x; idx < (long long)D * p.nfe; idx += blockDim.x)
        face_item<R, D, NP>(p, Utr, FVtr, Fstar, idx, eflag);
      __syncthreads();
      const bool last = step == nsteps - 1 && st == nstage - 1;
      for (int gi = 0; gi < ngroups; ++gi)  // ends with a block barrier; traces written in place
        volume_group<R, D, NP, G, false, true, false>(p, U, Q, Fstar, Utr, FVtr, K, Rout, mode, (R)coef.A[st],
                                               (R)coef.B[st], dt, (long long)gi * G, work, eflag,
                                               last ? nullptr : Utr);
    }
  }
  if (rk) {
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      Ug[i] = U[i];
      Kg[i] = K[i];
    }
  }
  if (eflag) atomicOr(err, eflag);
}

// --------------------------------------------------------------------------
// k_dt: max over nodes of sum_k (|v_k| + sqrt(p_alpha'(rho))) / h_k (FP64), as
// the bits of a non-negative double (monotone as unsigned integers).
// --------------------------------------------------------------------------
template <typename R, int D>
__global__ void __launch_bounds__(256) k_dt(const NskParams p, const long long nn, const R* __restrict__ U,
                                            unsigned long long* __restrict__ lam, int* __restrict__ err) {
  double m = 0.0;
  int eflag = 0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nn; g += (long long)gridDim.x * blockDim.x) {
    const double rho = (double)U[g];
    eflag |= rho_flags(rho);
    double pa, dp;
    eos_both64(p, rho, pa, dp);
    if (!(dp >= 0.0)) eflag |= NSK_EBIT_SOUND;
    const double a = sqrt(dp);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) s += (fabs((double)U[(1 + k) * nn + g] / rho) + a) * (0.5 * p.rh[k]);
    m = s > m ? s : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
    atomicMax(lam, (unsigned long long)__double_as_longlong(m));
  }
  if (eflag) atomicOr(err, eflag);
}

// dt = min(convective, viscous, source) bounds; see nsk_compute_dt in nsk.h
static __global__ void k_dt_final(const NskParams p, const int dim, const int N, const double cfl,
                           const unsigned long long* __restrict__ lam, double* __restrict__ dt) {
  const double lmax = __longlong_as_double((long long)*lam);
  const double tn = 2.0 * N + 1.0;
  double r = cfl / (tn * lmax);
  // with the learned closure the c equation (diffusion kappa/beta, source alpha/beta) is not integrated
  const double lamv = p.closure ? p.mu : (p.mu > p.kappa / p.beta ? p.mu : p.kappa / p.beta);
  double ih2 = 0.0;
  for (int k = 0; k < dim; ++k) ih2 += 0.25 * p.rh[k] * p.rh[k];
  if (lamv > 0.0) {
    const double dv = cfl / (tn * tn * lamv * ih2);
    r = dv < r ? dv : r;
  }
  if (!p.closure) {
    const double ds = cfl * 4.6 * p.beta / p.alpha;
    r = ds < r ? ds : r;
  }
  *dt = r;
}

// --------------------------------------------------------------------------
// k_diag: per-block partial quadrature sums (mass, energy, ||rho - c||^2), FP64,
// summed in a fixed order by k_diag_final (deterministic).
// --------------------------------------------------------------------------
template <typename R, int D, int NP>
__global__ void __launch_bounds__(256) k_diag(const NskParams p, const R* __restrict__ U, const R* __restrict__ Q,
                                              double* __restrict__ part) {
  using S = Shape<D, NP>;
  const long long nn = p.E * S::NPE;
  double sm = 0.0, se = 0.0, sl = 0.0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nn; g += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(g % S::NPE);
    double wq = p.jac;
#pragma unroll
    for (int k = 0; k < D; ++k) wq *= p.td.w[coord<NP>(n, k)];
    // the original NSK state has no c: its capillary energy uses grad rho (same slot of Q)
    const double rho = (double)U[g], c = p.model == NSK_MODEL_NSK ? rho : (double)U[(D + 1) * nn + g];
    double m2 = 0.0, g2 = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double m = (double)U[(1 + a) * nn + g];
      const double gc = (double)Q[(long long)(a * S::NW + D) * nn + g];
      m2 += m * m;
      g2 += gc * gc;
    }
    sm += wq * rho;
    se += wq * (m2 / (2.0 * rho) + eos_free_energy(p, rho) + 0.5 * p.alpha * (rho - c) * (rho - c) +
                0.5 * p.kappa * g2);
    sl += wq * (rho - c) * (rho - c);
  }
  __shared__ double red[3][256];
  red[0][threadIdx.x] = sm;
  red[1][threadIdx.x] = se;
  red[2][threadIdx.x] = sl;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) part[blockIdx.x * 3 + c] = red[c][0];
}

static __global__ void __launch_bounds__(256) k_diag_final(const int nparts, double* __restrict__ part) {
  __shared__ double red[3][256];
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x)
    for (int c = 0; c < 3; ++c) s[c] += part[b * 3 + c];
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) part[nparts * 3 + c] = red[c][0];
}

// ---- launch helpers ------------------------------------------------------
inline unsigned grid_for(long long items, int tpb) { return (unsigned)((items + tpb - 1) / tpb); }

// elements per block for a block-size choice tpb (at least one element)
template <int D, int NP>
__host__ __device__ constexpr int group_for(int tpb) {
  return tpb / Shape<D, NP>::NPE > 0 ? tpb / Shape<D, NP>::NPE : 1;
}

}  // namespace nsk
#include "nsk_line.cuh"
namespace nsk {

template <typename R, int D, int NP, int G, bool FUSED>
int launch_stage_g(const NskParams& p, const NskBuffers& b, const NskLaunch& l, cudaStream_t s) {
  using S = Shape<D, NP>;
  int nl = 0;
  if (l.ev) cudaEventRecord(l.ev[0], s);
  if (!l.traces_ready) {
    k_prolong<R, D, NP><<<dim3(grid_for(p.nfe, 256), S::NF), 256, 0, s>>>(p, (const R*)b.U, (R*)b.Utr);
    ++nl;
  }
  if (l.ev) cudaEventRecord(l.ev[1], s);
  const unsigned eb = (unsigned)((p.E + G - 1) / G);
  if (l.mode == NSK_MODE_LIFT)
    k_lift<R, D, NP, G, false><<<eb, G * S::NPE, 0, s>>>(p, (const R*)b.U, (const R*)b.Utr, (R*)b.Q, (R*)b.FVtr,
                                                          b.err);
  else
    k_lift<R, D, NP, G, true><<<eb, G * S::NPE, 0, s>>>(p, (const R*)b.U, (const R*)b.Utr, (R*)b.Q, (R*)b.FVtr,
                                                         b.err);
  if (l.ev) cudaEventRecord(l.ev[2], s);
  ++nl;
  if (l.mode != NSK_MODE_LIFT) {
    if (!FUSED) {
      k_face<R, D, NP><<<dim3(grid_for(p.nfe, 256), D), 256, 0, s>>>(p, (const R*)b.Utr, (const R*)b.FVtr,
                                                                       (R*)b.Fstar, b.err);
      ++nl;
    }
    if (l.ev) cudaEventRecord(l.ev[3], s);
    k_volume<R, D, NP, G, FUSED><<<eb, G * S::NPE, 0, s>>>(
        p, (R*)b.U, (const R*)b.Q, (const R*)b.Fstar, (const R*)b.Utr, (const R*)b.FVtr, (R*)b.K, (R*)l.Rout,
        l.mode, (R)l.A, (R)l.B, l.dt_dev, (R)l.dt_val, b.err, (R*)l.utr_next);
    if (l.ev) cudaEventRecord(l.ev[4], s);
    ++nl;
  }
  if (cudaGetLastError() != cudaSuccess) return NSK_ERR_CUDA;
  return nl;
}

// One part of a separate-face Runge-Kutta stage over the elements [e0, e0 + ne) (the host-state
// step's slab launches): part 0 the prolongation, 1 the lifting (viscous form stored), 2 the
// face pass over the faces (e, +k) of those elements, 3 the volume kernel with the update l
// describes. The range must be whole blocks of every kernel: e0 and ne multiples of G and of the
// 256 / nfn elements of a prolongation or face-pass block. Returns 1 (launches made),
// NSK_ERR_ARG, or NSK_ERR_CUDA.
template <typename R, int D, int NP, int G>
int launch_stage_part(const NskParams& p, const NskBuffers& b, const NskLaunch& l, cudaStream_t s, int part,
                      long long e0, long long ne) {
  using S = Shape<D, NP>;
  const long long f0 = e0 * S::NFN, nf = ne * S::NFN;
  if (e0 < 0 || ne <= 0 || e0 + ne > p.E || e0 % G || ne % G || f0 % 256 || nf % 256) return NSK_ERR_ARG;
  const unsigned fb = (unsigned)(nf / 256), eb = (unsigned)(ne / G);
  const int foff = (int)(f0 / 256), eoff = (int)(e0 / G);
  switch (part) {
    case 0:
      k_prolong<R, D, NP><<<dim3(fb, S::NF), 256, 0, s>>>(p, (const R*)b.U, (R*)b.Utr, foff);
      break;
    case 1:
      k_lift<R, D, NP, G, true><<<eb, G * S::NPE, 0, s>>>(p, (const R*)b.U, (const R*)b.Utr, (R*)b.Q, (R*)b.FVtr,
                                                           b.err, eoff);
      break;
    case 2:
      k_face<R, D, NP><<<dim3(fb, D), 256, 0, s>>>(p, (const R*)b.Utr, (const R*)b.FVtr, (R*)b.Fstar, b.err, foff);
      break;
    case 3:
      k_volume<R, D, NP, G, false><<<eb, G * S::NPE, 0, s>>>(
          p, (R*)b.U, (const R*)b.Q, (const R*)b.Fstar, (const R*)b.Utr, (const R*)b.FVtr, (R*)b.K, (R*)l.Rout,
          l.mode, (R)l.A, (R)l.B, l.dt_dev, (R)l.dt_val, b.err, (R*)l.utr_next, eoff);
      break;
    default:
      return NSK_ERR_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? 1 : NSK_ERR_CUDA;
}

// the lean schedule's two launches (a residual-free lifting stage, mode LIFT, takes the
// separate schedule's lifting kernel, which stores the gradients)
template <typename R, int D, int NP, int G>
int launch_stage_lean(const NskParams& p, const NskBuffers& b, const NskLaunch& l, cudaStream_t s) {
  using S = Shape<D, NP>;
  if (l.mode == NSK_MODE_LIFT) return launch_stage_g<R, D, NP, G, false>(p, b, l, s);
  constexpr int smem_lift = (int)sizeof(R) * lift_lean_smem<R, D, NP, G>();
  constexpr int smem_vol = (int)sizeof(R) * volume_lean_smem<R, D, NP, G>();
  static const bool attr_ok =
      cudaFuncSetAttribute(k_lift_lean<R, D, NP, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_lift) ==
          cudaSuccess &&
      cudaFuncSetAttribute(k_volume_lean<R, D, NP, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_vol) ==
          cudaSuccess;
  if (!attr_ok) return NSK_ERR_CUDA;
  int nl = 0;
  if (l.ev) cudaEventRecord(l.ev[0], s);
  if (!l.traces_ready) {
    k_prolong<R, D, NP><<<dim3(grid_for(p.nfe, 256), S::NF), 256, 0, s>>>(p, (const R*)b.U, (R*)b.Utr);
    ++nl;
  }
  if (l.ev) cudaEventRecord(l.ev[1], s);
  const unsigned eb = (unsigned)((p.E + G - 1) / G);
  k_lift_lean<R, D, NP, G><<<eb, G * S::NPE, smem_lift, s>>>(p, (const R*)b.U, (const R*)b.Utr, (R*)b.FVtr, b.err);
  ++nl;
  if (l.ev) cudaEventRecord(l.ev[2], s);
  if (l.ev) cudaEventRecord(l.ev[3], s);
  k_volume_lean<R, D, NP, G><<<eb, G * S::NPE, smem_vol, s>>>(p, (R*)b.U, (const R*)b.Utr, (const R*)b.FVtr, (R*)b.K,
                                                              (R*)l.Rout, l.mode, (R)l.A, (R)l.B, l.dt_dev,
                                                              (R)l.dt_val, b.err, (R*)l.utr_next);
  ++nl;
  if (l.ev) cudaEventRecord(l.ev[4], s);
  if (cudaGetLastError() != cudaSuccess) return NSK_ERR_CUDA;
  return nl;
}

// schedule: tpb in {128, 256} (elements per block = tpb / nodes per element); face fluxes in
// their own pass (fused_face 0), inside the volume kernel (1), the lean two-launch stage (2), or
// the separate face pass with line-per-thread lifting and volume kernels (4, FP32 3D N = 3)
template <typename R, int D, int NP>
int launch_stage(const NskParams& p, const NskBuffers& b, const NskLaunch& l, cudaStream_t s) {
  constexpr int G128 = group_for<D, NP>(128), G256 = group_for<D, NP>(256);
  if (l.fused_face == 2)
    return l.tpb == 128 ? launch_stage_lean<R, D, NP, G128>(p, b, l, s) : launch_stage_lean<R, D, NP, G256>(p, b, l, s);
  if constexpr (std::is_same<R, float>::value && D == 3 && NP == 4) {
    // line schedule (fused_face 4): 16 threads per element, 8 or 16 elements per block; for other
    // precisions and shapes it is the separate face pass
    if (l.fused_face == 4) return l.tpb == 128 ? launch_stage_line<8>(p, b, l, s) : launch_stage_line<16>(p, b, l, s);
  }
  const bool fused = l.fused_face == 1;
  if (l.tpb == 128)
    return fused ? launch_stage_g<R, D, NP, G128, true>(p, b, l, s) : launch_stage_g<R, D, NP, G128, false>(p, b, l, s);
  return fused ? launch_stage_g<R, D, NP, G256, true>(p, b, l, s) : launch_stage_g<R, D, NP, G256, false>(p, b, l, s);
}

template <int D>
int launch_stage_np(const NskParams& p, int np, bool fp32, const NskBuffers& b, const NskLaunch& l, cudaStream_t s) {
  switch (np) {
#define NSK_CASE(NPV)                                                                                     \
  case NPV:                                                                                               \
    return fp32 ? launch_stage<float, D, NPV>(p, b, l, s) : launch_stage<double, D, NPV>(p, b, l, s);
    NSK_CASE(2)
    NSK_CASE(3)
    NSK_CASE(4)
    NSK_CASE(5)
    NSK_CASE(6)
#undef NSK_CASE
    default:
      return NSK_ERR_ARG;
  }
}

// the stage launches of one precision (a translation unit per precision builds in parallel)
template <typename R, int D>
int launch_stage_np_r(const NskParams& p, int np, const NskBuffers& b, const NskLaunch& l, cudaStream_t s) {
  switch (np) {
    case 2: return launch_stage<R, D, 2>(p, b, l, s);
    case 3: return launch_stage<R, D, 3>(p, b, l, s);
    case 4: return launch_stage<R, D, 4>(p, b, l, s);
    case 5: return launch_stage<R, D, 5>(p, b, l, s);
    case 6: return launch_stage<R, D, 6>(p, b, l, s);
    default: return NSK_ERR_ARG;
  }
}

// shared memory the single-block schedule needs for a mesh (0 when N is not compiled here)
template <typename R, int D, int NP>
size_t block_bytes_t(const NskParams& p) {
  return sizeof(R) * BlockLayout<R, D, NP, group_for<D, NP>(256)>::total(p.E);
}

template <typename R, int D, int NP>
int launch_block_t(const NskParams& p, const NskBuffers& b, int mode, const NskLsrkCoef& coef, double dt,
                   int nsteps, void* Rout, cudaStream_t s) {
  constexpr int G = group_for<D, NP>(256);
  static const bool attr_ok = cudaFuncSetAttribute(k_block_steps<R, D, NP, G>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   kBlockSmemMax) == cudaSuccess;
  if (!attr_ok) return NSK_ERR_CUDA;
  const size_t bytes = block_bytes_t<R, D, NP>(p);
  if (bytes > (size_t)kBlockSmemMax) return NSK_ERR_ARG;
  k_block_steps<R, D, NP, G><<<1, G * Shape<D, NP>::NPE, bytes, s>>>(p, (R*)b.U, (R*)b.K, (R*)Rout, mode, coef,
                                                                        (R)dt, nsteps, b.err);
  return cudaGetLastError() == cudaSuccess ? 1 : NSK_ERR_CUDA;
}

// the single-block schedule of one precision
template <typename R, int D>
size_t block_bytes_np_r(const NskParams& p, int np) {
  switch (np) {
    case 2: return block_bytes_t<R, D, 2>(p);
    case 3: return block_bytes_t<R, D, 3>(p);
    case 4: return block_bytes_t<R, D, 4>(p);
    case 5: return block_bytes_t<R, D, 5>(p);
    case 6: return block_bytes_t<R, D, 6>(p);
    default: return (size_t)-1;
  }
}
template <typename R, int D>
int launch_block_np_r(const NskParams& p, int np, const NskBuffers& b, int mode, const NskLsrkCoef& coef, double dt,
                      int nsteps, void* Rout, cudaStream_t s) {
  switch (np) {
    case 2: return launch_block_t<R, D, 2>(p, b, mode, coef, dt, nsteps, Rout, s);
    case 3: return launch_block_t<R, D, 3>(p, b, mode, coef, dt, nsteps, Rout, s);
    case 4: return launch_block_t<R, D, 4>(p, b, mode, coef, dt, nsteps, Rout, s);
    case 5: return launch_block_t<R, D, 5>(p, b, mode, coef, dt, nsteps, Rout, s);
    case 6: return launch_block_t<R, D, 6>(p, b, mode, coef, dt, nsteps, Rout, s);
    default: return NSK_ERR_ARG;
  }
}

template <int D>
size_t block_bytes_np(const NskParams& p, int np, bool fp32) {
  switch (np) {
#define NSK_CASE(NPV) \
  case NPV:           \
    return fp32 ? block_bytes_t<float, D, NPV>(p) : block_bytes_t<double, D, NPV>(p);
    NSK_CASE(2)
    NSK_CASE(3)
    NSK_CASE(4)
    NSK_CASE(5)
    NSK_CASE(6)
#undef NSK_CASE
    default:
      return (size_t)-1;
  }
}

template <int D>
int launch_block_np(const NskParams& p, int np, bool fp32, const NskBuffers& b, int mode, const NskLsrkCoef& coef,
                    double dt, int nsteps, void* Rout, cudaStream_t s) {
  switch (np) {
#define NSK_CASE(NPV)                                                                        \
  case NPV:                                                                                  \
    return fp32 ? launch_block_t<float, D, NPV>(p, b, mode, coef, dt, nsteps, Rout, s)      \
                : launch_block_t<double, D, NPV>(p, b, mode, coef, dt, nsteps, Rout, s);
    NSK_CASE(2)
    NSK_CASE(3)
    NSK_CASE(4)
    NSK_CASE(5)
    NSK_CASE(6)
#undef NSK_CASE
    default:
      return NSK_ERR_ARG;
  }
}

}  // namespace nsk
