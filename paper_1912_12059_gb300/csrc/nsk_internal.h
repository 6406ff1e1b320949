// nsk_internal.h -- shared declarations of the CUDA library (host + device).
// Not part of the public ABI (include/nsk.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "nsk.h"

#define NSK_MAXNP 6  // polynomial degree N <= 5

// Error-word bits set by kernels (atomicOr) and read back by the host.
enum : int {
  NSK_EBIT_RHO = 1,       // density outside (0, 3)
  NSK_EBIT_SOUND = 2,     // p_alpha'(rho) < 0 (hyperbolicity lost)
  NSK_EBIT_NAN = 4,       // NaN / Inf met
  NSK_EBIT_TIMEOUT = 8,   // a bounded device wait expired
  NSK_EBIT_BOUNDS = 16,   // an index check of the bounds-checking build failed
};

// 1D nodal tables of the tensor-product basis (Sec. 3.1), in both precisions.
// dvol[i*NSK_MAXNP + j] = (w_j / w_i) l_i'(xi_j): weak-form volume operator;
// lm/lp[j] = l_j(-1) / l_j(+1): prolongation to the faces;
// lmw/lpw[i] = l_i(-1) / w_i, l_i(+1) / w_i: surface lifting.
template <typename R>
struct NskTab {
  R dvol[NSK_MAXNP * NSK_MAXNP];
  R lm[NSK_MAXNP], lp[NSK_MAXNP];
  R lmw[NSK_MAXNP], lpw[NSK_MAXNP];
  R w[NSK_MAXNP];  // quadrature weights
  // model coefficients in the operator's precision (no per-thread conversions or divisions)
  R rh[3];         // 2 / h_k
  R mu, kb, alpha, ab;  // mu, kappa / beta, alpha, alpha / beta
  // the operators of direction k with the metric factor 2/h_k folded in (one rounding of
  // the product, fewer instructions in the contractions): dk = (2/h_k) dvol,
  // lpk = (2/h_k) lpw, lmk = (2/h_k) lmw
  R dk[3][NSK_MAXNP * NSK_MAXNP];
  R lpk[3][NSK_MAXNP], lmk[3][NSK_MAXNP];
  // face interpolation with the viscous coefficients folded in (the lifting's traces of
  // F^v: mu l(+-1) for the stress, (kappa/beta) l(+-1) for the c flux)
  R lpmu[NSK_MAXNP], lmmu[NSK_MAXNP], lpkb[NSK_MAXNP], lmkb[NSK_MAXNP];
};

// Components of a face trace: the conservative variables, and in FP64 also
// 1/rho and 1/(3 - rho) of the trace (shared by the lifting and face kernels,
// so the FP64 path divides once per trace instead of four times).
template <typename R> struct TraceComps { static constexpr int extra = 0; };
template <> struct TraceComps<double> { static constexpr int extra = 2; };

// Division by an invariant divisor d >= 1 as a multiply and a shift (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): with l = ceil(log2 d),
// s = 31 + l and m = ceil(2^s / d) (< 2^32), x / d = (x m) >> s exactly for 0 <= x < 2^31.
struct FastDiv {
  unsigned m;
  int s;
};
inline FastDiv make_fastdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  const int s = 31 + l;
  return FastDiv{(unsigned)(((1ull << s) + d - 1) / d), s};
}
__host__ __device__ __forceinline__ unsigned fdiv(unsigned x, FastDiv f) {
  return (unsigned)(((unsigned long long)x * f.m) >> f.s);
}

// Everything a kernel needs besides its buffers; passed by value.
struct NskParams {
  long long E;     // number of elements
  int ne[3];       // elements per direction (1 beyond dim)
  // 32-bit index arithmetic (nsk_init_mesh keeps E * nodes per element below 2^31)
  int nne, nfe;    // E * nodes per element, E * nodes per face: the size of one variable's plane
  int est[3];      // element-index stride of direction k (1, ne0, ne0 ne1)
  int ewrap[3];    // (ne[k] - 1) est[k]: the periodic jump across direction k
  FastDiv fd_ne0, fd_ne1, fd_E;
  double rh[3];    // 2 / h_k (Cartesian metric terms)
  double T, kappa, alpha, beta, mu;
  double jac;      // J = prod_k h_k / 2
  int closure;     // 1: the c equation is replaced by the learned closure (dt without its bounds)
  int model;       // NSK_MODEL_RELAXATION (state rho, m, c) or NSK_MODEL_NSK (state rho, m)
  // EoS constants: p_alpha = t8 rho q + pa2 rho^2, p_alpha' = t24 q^2 + dpa1 rho, q = 1/(3 - rho)
  double t8, t24, pa2, dpa1;
  float t8f, t24f, pa2f, dpa1f;
  double spin_lo, spin_hi;  // spinodal interval (p' < 0): the FP32 operator evaluates the EoS in FP64 there
  float spin_lof, spin_hif; // the same bounds rounded outward to FP32
  int c_diss;      // Lax-Friedrichs jump on c as well
  int flux;        // NSK_FLUX_LF or NSK_FLUX_HLLC
  int* berr;       // error word of the bounds-checking build's index checks (NULL: none)
  NskTab<double> td;
  NskTab<float> tf;
};

template <typename R> struct TabSel;
template <> struct TabSel<double> {
  __host__ __device__ static const NskTab<double>& get(const NskParams& p) { return p.td; }
};
template <> struct TabSel<float> {
  __host__ __device__ static const NskTab<float>& get(const NskParams& p) { return p.tf; }
};

// Device buffers of one context (type-erased: FP64 or FP32 per precision mode).
struct NskBuffers {
  void* U;       // [nvar][E][npe] state
  void* K;       // [nvar][E][npe] low-storage RK register
  void* Q;       // [nq][E][npe] lifted gradients
  void* Utr;     // [nvar + extra][2d][E][nfn] traces of U on the element's own faces
  void* FVtr;    // [d+1][2d][E][nfn] face-normal viscous flux traces (own side)
  void* Fstar;   // [nvar][d][E][nfn] numerical flux on face (e, +k)
  int* err;      // error word
  unsigned long long* lam;  // dt reduction target (bits of a non-negative double)
  double* dt;    // device time step
  double* part;  // diagnostics partial sums [nblocks][3]
  int nparts;
  // original NSK equations only (NULL otherwise)
  void* Gtr;     // [2d][E][nfn] traces of (grad rho)_k on the faces of direction k
  void* Q2;      // [E][npe] lap rho from the second lifting
};

// What one stage pipeline launch should do.
enum { NSK_MODE_RHS = 0, NSK_MODE_LSRK = 1, NSK_MODE_LIFT = 2 };

struct NskLaunch {
  int mode;
  void* Rout;              // residual output (mode RHS), precision of the context
  double A, B;             // LSRK stage coefficients (mode LSRK)
  const double* dt_dev;    // device dt (NULL: use dt_val)
  double dt_val;
  cudaEvent_t* ev;         // NULL, or NSK_NKERN + 1 events bracketing the kernels
  int tpb;                 // block-size schedule: 128 or 256 threads (elements per block follow)
  int fused_face;          // 1: face fluxes evaluated inside the volume kernel
  int traces_ready = 0;    // 1: Utr already holds the traces of U (no prolongation pass)
  void* utr_next = nullptr;  // non-NULL: the volume kernel writes the traces of its output state here
};

#define NSK_NKERN 5  // prolong, lift, face, volume, single-block stage/step kernel

// LSRK stage coefficients passed by value to the single-block kernel
struct NskLsrkCoef {
  double A[5], B[5];
};
// dynamic shared memory the single-block schedule may use (the per-block limit, 227 KB, less a margin)
constexpr int kBlockSmemMax = 200 * 1024;

// Per-dimension launchers (nsk_dg1.cu, nsk_dg2.cu, nsk_dg3.cu). Return the
// number of kernels launched, or a negative NSK_ERR_* code.
int nsk_launch_stage_d1(const NskParams& p, int np, bool fp32, const NskBuffers& b, const NskLaunch& l,
                        cudaStream_t s);
int nsk_launch_stage_d2(const NskParams& p, int np, bool fp32, const NskBuffers& b, const NskLaunch& l,
                        cudaStream_t s);
// original NSK equations (FP64), nsk_orig.cu
int nsk_launch_stage_nsk(int dim, const NskParams& p, int np, const NskBuffers& b, const NskLaunch& l,
                         cudaStream_t s);
int nsk_launch_dt_nsk(const NskParams& p, int dim, const NskBuffers& b, double cfl, int N, cudaStream_t s);
int nsk_launch_stage_d3(const NskParams& p, int np, bool fp32, const NskBuffers& b, const NskLaunch& l,
                        cudaStream_t s);
// one part (0 prolongation, 1 lifting, 2 face pass, 3 volume) of a separate-face 3D stage over the
// elements [e0, e0 + ne), whole blocks of every kernel (FP64, N = 3); launches made or an error
int nsk_launch_stage_part_d3(const NskParams& p, int np, bool fp32, const NskBuffers& b, const NskLaunch& l,
                             cudaStream_t s, int part, long long e0, long long ne);
// Single-block schedule (nsk_set_schedule fused_face = 3): the bytes of shared memory a mesh
// needs, and one launch running nsteps LSRK steps (mode LSRK, fixed dt) or one residual (mode
// RHS, into Rout) in one block; returns 1 (launches), NSK_ERR_ARG when the mesh does not fit.
size_t nsk_block_bytes(int dim, const NskParams& p, int np, bool fp32);
int nsk_launch_block(int dim, const NskParams& p, int np, bool fp32, const NskBuffers& b, int mode,
                     const NskLsrkCoef& coef, double dt, int nsteps, void* Rout, cudaStream_t s);
size_t nsk_block_bytes_d1(const NskParams& p, int np, bool fp32);
size_t nsk_block_bytes_d2(const NskParams& p, int np, bool fp32);
size_t nsk_block_bytes_d3(const NskParams& p, int np, bool fp32);
int nsk_launch_block_d1(const NskParams& p, int np, bool fp32, const NskBuffers& b, int mode, const NskLsrkCoef& coef,
                        double dt, int nsteps, void* Rout, cudaStream_t s);
int nsk_launch_block_d2(const NskParams& p, int np, bool fp32, const NskBuffers& b, int mode, const NskLsrkCoef& coef,
                        double dt, int nsteps, void* Rout, cudaStream_t s);
int nsk_launch_block_d3(const NskParams& p, int np, bool fp32, const NskBuffers& b, int mode, const NskLsrkCoef& coef,
                        double dt, int nsteps, void* Rout, cudaStream_t s);
// dt: reduces max_nodes sum_k (|v_k| + sqrt(p_alpha'))/h_k into b.lam and writes b.dt.
int nsk_launch_dt(const NskParams& p, int dim, int np, bool fp32, const NskBuffers& b, double cfl,
                  cudaStream_t s);
// diagnostics: needs b.Q current (run a LIFT stage first); writes b.part, final sums in b.part[0..2].
int nsk_launch_diag(const NskParams& p, int dim, int np, bool fp32, const NskBuffers& b, cudaStream_t s);
// precision conversion of nodal arrays (FP32 mode boundary)
int nsk_launch_convert(const void* src, bool src64, void* dst, bool dst64, long long n, cudaStream_t s);

// One context (the opaque nsk_ctx of the ABI): mesh, parameters, device buffers.
// Device buffers of the 1D sub-cell path (nsk_fv.cu)
struct FvBuffers {
  int* flags;    // [E] 1: the element holds N+1 sub-cell means
  double* ind;   // [E] last Persson indicator
  double* Uf;    // [E][2][3] face states
  double* Gf;    // [E][2][2] (v_x, c_x) of each element side of its faces
  double* SL;    // [E][N+1][3] MinMod slopes of the FV elements
  double* Fh;    // [E+1][3] element-face fluxes
  unsigned* bar; // [2] grid barrier of the cooperative small-mesh launch (arrivals, generation)
};
int nsk_fv_launch_stage(const NskParams& p, const void* fvp, int np, const FvBuffers& fb, const NskBuffers& b,
                        int mode, double* Rout, double A, double B, const double* dtp, double dtv, cudaStream_t s);
int nsk_fv_launch_switch(const NskParams& p, const void* fvp, int np, const FvBuffers& fb, double* U,
                         cudaStream_t s);
size_t nsk_fv_params_size();
int nsk_fv_coop_max_elements();
int nsk_fv_launch_coop(const NskParams& p, const void* fvp, int np, const FvBuffers& fb, const NskBuffers& b,
                       int nsteps, int switching, double dt, const double* A, const double* B, cudaStream_t s);
int nsk_fv_fill_params(void* fvp, int np, const double* xi, const double* gauss_x, const double* gauss_w, double h,
                       int dirichlet, const double* Ub_lo, const double* Ub_hi, double upper, double lower);

// z-slabs of the host-state step's overlapped copies
constexpr int NSK_IO_SLABS = 8;

struct nsk_ctx {
  int dim, N, np, npe, nfn, nvar, nq, node_type, precision;
  long long E, nn;
  int ne[3];
  double lo[3], hi[3], h[3];
  double xi[NSK_MAXNP], w[NSK_MAXNP];
  cudaStream_t stream;
  NskParams p;
  NskBuffers b;
  void* rbuf;        // residual scratch, context precision, nvar*nn
  void* utr_alt;     // second trace buffer (same shape as b.Utr): the fused-face schedule writes
                     // the next stage's traces there while neighbours still read b.Utr
  double* stage64;   // FP64 staging for transfers, max(nvar, nq, dim)*nn
  bool params_set, state_set;
  long long launches;
  size_t rsize;      // bytes per value in context precision
  // per-kernel profiling (nsk_set_profiling)
  bool prof_on;
  std::vector<cudaEvent_t> prof_pool;  // groups of NSK_NKERN + 1 events
  std::vector<int> prof_nk;            // bit k set: kernel k launched between events k and k+1
  size_t prof_used;                    // groups recorded since the last sync
  double prof_ms[NSK_NKERN];
  long long prof_cnt[NSK_NKERN];
  int tpb, fused_face;  // stage schedule (nsk_set_schedule / nsk_autotune)
  // learned c-closure (nsk_set_closure)
  int closure_mode;            // NSK_C_EXPLICIT or NSK_C_LEARNED
  struct nsk_mlp* mlp;         // borrowed network
  int judge_every;             // steps between two judge evaluations (0: never)
  double eta_max, last_eta;    // fallback threshold, last judged error
  long long fallbacks, steps_since_judge;
  void* cl_X;                  // BF16 features [E][n_in_pad]
  float* cl_Y;                 // network output [E][npe]
  double* cl_red;              // judge sums
  float* cl_mean;              // element mean densities (features)
  // 1D sub-cell shock capturing and Dirichlet boundaries (nsk_set_subcell, nsk_set_dirichlet)
  int fv_on, fv_dirichlet;     // switching on; Dirichlet (else periodic) boundaries
  double fv_upper, fv_lower;   // indicator thresholds
  double fv_Ub[2][3];          // boundary states
  void* fv_params;             // host copy of the kernels' parameter block
  FvBuffers fvb;
  // the host-state step (nsk_step_host): its copy stream and events, made on first use
  cudaStream_t io_stream;
  cudaEvent_t io_ev[2 * NSK_IO_SLABS + 1];
  bool fv_path() const { return fv_on || fv_dirichlet; }
};

// host helpers shared by the translation units of the library
int nsk_ctx_launch_stage(nsk_ctx* c, NskLaunch l);  // queues one stage on the context's stream
int nsk_ctx_sync_check(nsk_ctx* c);                  // synchronise the stream, read and clear the error word
// c := rho + s * network(features(rho)); utr non-NULL: also the traces of the new c there
int nsk_closure_apply_ctx(nsk_ctx* c, void* utr);
int nsk_closure_judge_ctx(nsk_ctx* c);               // judge + fallback (synchronises)
