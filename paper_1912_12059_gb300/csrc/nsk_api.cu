// nsk_api.cu -- host side of libnsk.so: the C ABI declared in include/nsk.h.
// Builds the nodal tables and the mesh, owns the device buffers of a context,
// validates arguments and call order, and queues the stage kernels.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>
#include <utility>
#include <vector>

#include "nsk_internal.h"
#include "nsk_nvtx.h"
#include "nsk_test_hooks.h"

namespace {

// ---- nodal basis (Sec. 3.1): Gauss-Legendre / Gauss-Lobatto nodes and weights ----

// P_n(x) and P_{n-1}(x) by the Bonnet recurrence.
void legendre_pair(int n, double x, double* pn, double* pnm1) {
  double a = 1.0, b = x;  // P_0, P_1
  if (n == 0) {
    *pn = 1.0;
    *pnm1 = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    const double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    a = b;
    b = c;
  }
  *pn = b;
  *pnm1 = a;
}

// Gauss-Legendre: the n = N+1 roots of P_n, Newton from Tricomi's estimate;
// weights 2 (1 - x^2) / (n P_{n-1}(x))^2.
void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.141592653589793238462643;
  for (int i = 0; i < n; ++i) {
    const double theta = pi * (4.0 * (n - i) - 1.0) / (4.0 * n + 2.0);
    double z = (1.0 - 1.0 / (8.0 * n * n) + 1.0 / (8.0 * n * n * n)) * cos(theta);
    for (int it = 0; it < 60; ++it) {
      double pn, pm;
      legendre_pair(n, z, &pn, &pm);
      const double dp = n * (pm - z * pn) / (1.0 - z * z);
      const double dz = pn / dp;
      z -= dz;
      if (fabs(dz) <= 1e-17) break;
    }
    double pn, pm;
    legendre_pair(n, z, &pn, &pm);
    x[i] = z;
    w[i] = 2.0 * (1.0 - z * z) / ((n * pm) * (n * pm));
  }
}

// Gauss-Lobatto with N+1 nodes: +-1 and the roots of P_N'; Newton with
// P_N'' from Legendre's differential equation; weights 2 / (N (N+1) P_N(x)^2).
void gauss_lobatto(int N, double* x, double* w) {
  const double pi = 3.141592653589793238462643;
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double z = -cos(pi * i / N);
    for (int it = 0; it < 60; ++it) {
      double pn, pm;
      legendre_pair(N, z, &pn, &pm);
      const double d1 = N * (pm - z * pn) / (1.0 - z * z);
      const double d2 = (2.0 * z * d1 - N * (N + 1.0) * pn) / (1.0 - z * z);
      const double dz = d1 / d2;
      z -= dz;
      if (fabs(dz) <= 1e-17) break;
    }
    x[i] = z;
  }
  for (int i = 0; i <= N; ++i) {
    double pn, pm;
    legendre_pair(N, x[i], &pn, &pm);
    w[i] = 2.0 / (N * (N + 1.0) * pn * pn);
  }
}

// Barycentric weights, derivative matrix D_ij = l_j'(x_i) and l_j(x0).
void barycentric(int n, const double* x, double* lam) {
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) p *= x[j] - x[m];
    lam[j] = 1.0 / p;
  }
}
double lagrange_at(int n, const double* x, const double* lam, int j, double x0) {
  for (int m = 0; m < n; ++m)
    if (x0 == x[m]) return m == j ? 1.0 : 0.0;
  double s = 0.0;
  for (int m = 0; m < n; ++m) s += lam[m] / (x0 - x[m]);
  return lam[j] / (x0 - x[j]) / s;
}

template <typename R>
void fill_tab(NskTab<R>& t, int n, const double* x, const double* w) {
  double lam[NSK_MAXNP], D[NSK_MAXNP][NSK_MAXNP];
  barycentric(n, x, lam);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      D[i][j] = lam[j] / lam[i] / (x[i] - x[j]);
      diag -= D[i][j];
    }
    D[i][i] = diag;
  }
  memset(&t, 0, sizeof(t));
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) t.dvol[i * NSK_MAXNP + j] = (R)(w[j] / w[i] * D[j][i]);
    const double lm = lagrange_at(n, x, lam, i, -1.0), lp = lagrange_at(n, x, lam, i, 1.0);
    t.lm[i] = (R)lm;
    t.lp[i] = (R)lp;
    t.lmw[i] = (R)(lm / w[i]);
    t.lpw[i] = (R)(lp / w[i]);
    t.w[i] = (R)w[i];
  }
}

// Spinodal densities of the reduced VdW fluid: p'(rho) = 0 <=> rho (3 - rho)^2 = 4 T, one root
// in (0, 1) and one in (1, 3) for 0 < T < 1 (bisection).
void spinodal_interval(double T, double* lo, double* hi) {
  auto g = [T](double r) { return r * (3.0 - r) * (3.0 - r) - 4.0 * T; };
  double a = 0.0, b = 1.0;  // g(a) < 0 < g(b)
  for (int it = 0; it < 200; ++it) {
    const double m = 0.5 * (a + b);
    (g(m) < 0.0 ? a : b) = m;
  }
  *lo = 0.5 * (a + b);
  a = 1.0;
  b = 3.0;  // g(a) > 0 > g(b)
  for (int it = 0; it < 200; ++it) {
    const double m = 0.5 * (a + b);
    (g(m) > 0.0 ? a : b) = m;
  }
  *hi = 0.5 * (a + b);
}

// model coefficients of both operator precisions (after the mesh and the parameters are known)
template <typename R>
void fill_coef(NskTab<R>& t, const NskParams& p) {
  const NskTab<double>& td = p.td;  // the FP64 operator tables (already filled)
  for (int k = 0; k < 3; ++k) {
    t.rh[k] = (R)p.rh[k];
    for (int i = 0; i < NSK_MAXNP; ++i) {
      for (int j = 0; j < NSK_MAXNP; ++j) t.dk[k][i * NSK_MAXNP + j] = (R)(p.rh[k] * td.dvol[i * NSK_MAXNP + j]);
      t.lpk[k][i] = (R)(p.rh[k] * td.lpw[i]);
      t.lmk[k][i] = (R)(p.rh[k] * td.lmw[i]);
    }
  }
  t.mu = (R)p.mu;
  t.kb = (R)(p.kappa / p.beta);
  for (int i = 0; i < NSK_MAXNP; ++i) {
    t.lpmu[i] = (R)(p.mu * td.lp[i]);
    t.lmmu[i] = (R)(p.mu * td.lm[i]);
    t.lpkb[i] = (R)(p.kappa / p.beta * td.lp[i]);
    t.lmkb[i] = (R)(p.kappa / p.beta * td.lm[i]);
  }
  t.alpha = (R)p.alpha;
  t.ab = (R)(p.alpha / p.beta);
}

// index constants of the kernels (after E and ne are known)
void set_index_constants(NskParams& p, int npe, int nfn) {
  p.nne = (int)(p.E * npe);
  p.nfe = (int)(p.E * nfn);
  int st = 1;
  for (int k = 0; k < 3; ++k) {
    p.est[k] = st;
    p.ewrap[k] = (p.ne[k] - 1) * st;
    st *= p.ne[k];
  }
  p.fd_ne0 = make_fastdiv((unsigned)p.ne[0]);
  p.fd_ne1 = make_fastdiv((unsigned)p.ne[1]);
  p.fd_E = make_fastdiv((unsigned)p.E);
}

void set_eos_constants(NskParams& p) {
  fill_coef<double>(p.td, p);
  fill_coef<float>(p.tf, p);
  p.t8 = 8.0 * p.T;
  p.t24 = 24.0 * p.T;
  p.pa2 = 0.5 * p.alpha - 3.0;
  p.dpa1 = p.alpha - 6.0;
  p.t8f = (float)p.t8;
  p.t24f = (float)p.t24;
  p.pa2f = (float)p.pa2;
  p.dpa1f = (float)p.dpa1;
  spinodal_interval(p.T, &p.spin_lo, &p.spin_hi);
  p.spin_lof = nextafterf((float)p.spin_lo, 0.0f);
  p.spin_hif = nextafterf((float)p.spin_hi, 4.0f);
}

// Carpenter-Kennedy RK4(3)5[2N] (the published rational coefficients).
const double kA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                      -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                      1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                      2277821191437.0 / 14882151754819.0};

}  // namespace



namespace {

// events for the next profiled stage (NULL when profiling is off)
cudaEvent_t* prof_group(nsk_ctx* c, int mask) {
  if (!c->prof_on) return nullptr;
  const size_t g = c->prof_used;
  if ((g + 1) * (NSK_NKERN + 1) > c->prof_pool.size()) {
    for (int i = 0; i < NSK_NKERN + 1; ++i) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
      c->prof_pool.push_back(ev);
    }
  }
  if (c->prof_nk.size() <= g) c->prof_nk.resize(g + 1);
  c->prof_nk[g] = mask;
  c->prof_used = g + 1;
  return &c->prof_pool[g * (NSK_NKERN + 1)];
}

// after a stream synchronisation: fold the recorded event pairs into the totals
void prof_collect(nsk_ctx* c) {
  for (size_t g = 0; g < c->prof_used; ++g) {
    cudaEvent_t* ev = &c->prof_pool[g * (NSK_NKERN + 1)];
    for (int k = 0; k < NSK_NKERN; ++k) {
      if (!((c->prof_nk[g] >> k) & 1)) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) == cudaSuccess) {
        c->prof_ms[k] += ms;
        c->prof_cnt[k] += 1;
      }
    }
  }
  c->prof_used = 0;
}

int sync_and_check(nsk_ctx* c) {
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NSK_ERR_CUDA;
  prof_collect(c);
  int h = 0;
  if (cudaMemcpy(&h, c->b.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NSK_ERR_CUDA;
  if (h) {
    int z = 0;
    if (cudaMemcpy(c->b.err, &z, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return NSK_ERR_CUDA;
    if (h & NSK_EBIT_TIMEOUT) return NSK_ERR_TIMEOUT;
    if (h & NSK_EBIT_BOUNDS) return NSK_ERR_BOUNDS;
    return NSK_ERR_NONPHYSICAL;
  }
  return NSK_OK;
}

// the single-block schedule applies: relaxation model II, no sub-cells, and the mesh's arrays fit
// in one block's shared memory
bool block_eligible(const nsk_ctx* c) {
  return c->p.model == NSK_MODEL_RELAXATION && !c->fv_path() &&
         nsk_block_bytes(c->dim, c->p, c->np, c->precision == NSK_FP32_MIXED) <= (size_t)kBlockSmemMax;
}

// one launch of the single-block kernel: nsteps LSRK steps at the fixed dt, or (nsteps = 0) one
// residual into l.Rout; profiled as kernel 4
int launch_block(nsk_ctx* c, int nsteps, double dt, void* Rout) {
  cudaEvent_t* ev = prof_group(c, 16);
  if (ev) cudaEventRecord(ev[4], c->stream);
  NskLsrkCoef coef;
  for (int i = 0; i < 5; ++i) {
    coef.A[i] = kA[i];
    coef.B[i] = kB[i];
  }
  const int r = nsk_launch_block(c->dim, c->p, c->np, c->precision == NSK_FP32_MIXED, c->b,
                                 nsteps > 0 ? NSK_MODE_LSRK : NSK_MODE_RHS, coef, dt, nsteps > 0 ? nsteps : 1, Rout,
                                 c->stream);
  if (ev) cudaEventRecord(ev[5], c->stream);
  if (r < 0) return r;
  c->launches += r;
  return NSK_OK;
}

// the line schedule (fused_face 4) has kernels for the FP32 operator of relaxation model II on
// 3D elements with N = 3 (elsewhere it runs as the separate face pass)
bool line_eligible(const nsk_ctx* c) {
  return c->precision == NSK_FP32_MIXED && c->dim == 3 && c->np == 4 && c->p.model != NSK_MODEL_NSK && !c->fv_path();
}

int launch_stage(nsk_ctx* c, NskLaunch l) {
  if (l.fused_face == 3) {  // single-block schedule: a residual in one launch; otherwise the separate face pass
    if (l.mode == NSK_MODE_RHS && block_eligible(c)) return launch_block(c, 0, 0.0, l.Rout);
    l.fused_face = 0;
  }
  // kernels 0..3 = prolong, lift, face, volume
  const int mask = c->p.model == NSK_MODEL_NSK ? (l.mode == NSK_MODE_LIFT ? 3 : 15)
                                                : ((l.traces_ready ? 0 : 1) | 2 |
                                                   (l.mode == NSK_MODE_LIFT
                                                        ? 0
                                                        : (((l.fused_face == 0 || l.fused_face == 4) ? 4 : 0) | 8)));
  l.ev = prof_group(c, mask);
  int r;
  const bool f32 = c->precision == NSK_FP32_MIXED;
  if (c->p.model == NSK_MODEL_NSK) {  // the original NSK equations: their own stage kernels
    r = nsk_launch_stage_nsk(c->dim, c->p, c->np, c->b, l, c->stream);
    if (r < 0) return r;
    c->launches += r;
    return NSK_OK;
  }
  switch (c->dim) {
    case 1: r = nsk_launch_stage_d1(c->p, c->np, f32, c->b, l, c->stream); break;
    case 2: r = nsk_launch_stage_d2(c->p, c->np, f32, c->b, l, c->stream); break;
    default: r = nsk_launch_stage_d3(c->p, c->np, f32, c->b, l, c->stream); break;
  }
  if (r < 0) return r;
  c->launches += r;
  return NSK_OK;
}

// copy an internal nodal array (context precision, ncomp*nn values) out to dst
int export_nodal(nsk_ctx* c, const void* src, int ncomp, double* dst, int where) {
  const long long n = (long long)ncomp * c->nn;
  const size_t bytes = sizeof(double) * (size_t)n;
  if (c->precision == NSK_FP64) {
    const cudaMemcpyKind kind = where == NSK_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cudaMemcpyAsync(dst, src, bytes, kind, c->stream) != cudaSuccess) return NSK_ERR_CUDA;
  } else {
    double* tgt = where == NSK_DEVICE ? dst : c->stage64;
    int r = nsk_launch_convert(src, false, tgt, true, n, c->stream);
    if (r < 0) return r;
    c->launches += r;
    if (where == NSK_HOST &&
        cudaMemcpyAsync(dst, c->stage64, bytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      return NSK_ERR_CUDA;
  }
  return NSK_OK;
}

void free_ctx(nsk_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->b.U, c->b.K, c->b.Q, c->b.Utr, c->utr_alt, c->b.FVtr, c->b.Fstar, c->b.Q2, c->b.Gtr,
                  c->b.err, c->b.lam,
                  c->b.dt, c->b.part, c->rbuf, c->stage64, c->cl_X, c->cl_Y, c->cl_red, c->cl_mean,
                  c->fvb.flags, c->fvb.ind, c->fvb.Uf, c->fvb.Gf, c->fvb.SL, c->fvb.Fh, c->fvb.bar};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (c->io_stream) cudaStreamDestroy(c->io_stream);
  for (cudaEvent_t ev : c->io_ev)
    if (ev) cudaEventDestroy(ev);
  free(c->fv_params);
  for (cudaEvent_t ev : c->prof_pool) cudaEventDestroy(ev);
  delete c;
}

}  // namespace

int nsk_ctx_launch_stage(nsk_ctx* c, NskLaunch l) { return launch_stage(c, l); }
int nsk_ctx_sync_check(nsk_ctx* c) { return sync_and_check(c); }

namespace {
// device time step of the context's model (kernel launches issued, or an NSK_ERR_* code)
int launch_dt(nsk_ctx* c, double cfl) {
  if (c->p.model == NSK_MODEL_NSK) return nsk_launch_dt_nsk(c->p, c->dim, c->b, cfl, c->np - 1, c->stream);
  return nsk_launch_dt(c->p, c->dim, c->np, c->precision == NSK_FP32_MIXED, c->b, cfl, c->stream);
}
}  // namespace

extern "C" {

const char* nsk_error_string(int code) {
  switch (code) {
    case NSK_OK: return "ok";
    case NSK_ERR_ARG: return "invalid argument";
    case NSK_ERR_CUDA: return "CUDA runtime error";
    case NSK_ERR_NONPHYSICAL: return "non-physical state (rho outside (0,3), p_alpha' < 0 or NaN)";
    case NSK_ERR_TIMEOUT: return "bounded device wait expired";
    case NSK_ERR_STATE: return "call order violated";
    case NSK_ERR_NOMEM: return "device allocation failed";
    case NSK_ERR_IO: return "checkpoint file error (unwritable, unreadable, short or for another mesh)";
    case NSK_ERR_BOUNDS: return "index check of the bounds-checking build failed";
    default: return "unknown error";
  }
}

int nsk_init_mesh(nsk_ctx** out, int dim, const int nelem[3], const double lo[3], const double hi[3], int N,
                  int node_type, int precision, void* cuda_stream) {
  if (!out || !nelem || !lo || !hi) return NSK_ERR_ARG;
  *out = nullptr;
  if (dim < 1 || dim > 3 || N < 1 || N + 1 > NSK_MAXNP) return NSK_ERR_ARG;
  if (node_type != NSK_NODES_GAUSS && node_type != NSK_NODES_GAUSS_LOBATTO) return NSK_ERR_ARG;
  if (precision != NSK_FP64 && precision != NSK_FP32_MIXED) return NSK_ERR_ARG;
  nsk_ctx* c = new (std::nothrow) nsk_ctx();
  if (!c) return NSK_ERR_NOMEM;
  c->dim = dim;
  c->N = N;
  c->np = N + 1;
  c->node_type = node_type;
  c->precision = precision;
  c->nvar = dim + 2;
  c->nq = dim * (dim + 1);
  c->npe = 1;
  c->nfn = 1;
  c->E = 1;
  for (int k = 0; k < 3; ++k) {
    if (k < dim) {
      if (nelem[k] < 1 || !(hi[k] > lo[k]) || !isfinite(lo[k]) || !isfinite(hi[k])) {
        delete c;
        return NSK_ERR_ARG;
      }
      c->ne[k] = nelem[k];
      c->lo[k] = lo[k];
      c->hi[k] = hi[k];
      c->h[k] = (hi[k] - lo[k]) / nelem[k];
      c->npe *= c->np;
      if (k > 0) c->nfn *= c->np;
    } else {
      c->ne[k] = 1;
      c->lo[k] = 0.0;
      c->hi[k] = 1.0;
      c->h[k] = 2.0;
    }
    c->E *= c->ne[k];
  }
  if (c->E > (1LL << 31) / c->npe) {  // keep every per-variable index in 32-bit blocks of the grid
    delete c;
    return NSK_ERR_ARG;
  }
  c->nn = c->E * c->npe;
  c->stream = (cudaStream_t)cuda_stream;
  c->rsize = precision == NSK_FP64 ? sizeof(double) : sizeof(float);
  // default schedule (nsk_autotune picks per mesh): 256 threads, each face evaluated once
  c->tpb = 256;
  c->fused_face = 0;
  if (node_type == NSK_NODES_GAUSS)
    gauss_legendre(c->np, c->xi, c->w);
  else
    gauss_lobatto(N, c->xi, c->w);

  NskParams& p = c->p;
  memset(&p, 0, sizeof(p));
  p.E = c->E;
  p.jac = 1.0;
  for (int k = 0; k < 3; ++k) {
    p.ne[k] = c->ne[k];
    p.rh[k] = k < dim ? 2.0 / c->h[k] : 0.0;
    if (k < dim) p.jac *= c->h[k] / 2.0;
  }
  set_index_constants(p, c->npe, c->nfn);
  fill_tab<double>(p.td, c->np, c->xi, c->w);
  fill_tab<float>(p.tf, c->np, c->xi, c->w);

  const size_t rs = c->rsize;
  const long long nn = c->nn;
  const long long faces = c->E * 2 * dim * c->nfn;
  long long g = (nn + 255) / 256;
  c->b.nparts = (int)(g < 152 * 8 ? (g > 0 ? g : 1) : 152 * 8);
  int maxc = c->nq > c->nvar ? c->nq : c->nvar;
  struct {
    void** ptr;
    size_t bytes;
  } allocs[] = {
      {&c->b.U, rs * c->nvar * nn},
      {&c->b.K, rs * c->nvar * nn},
      {&c->b.Q, rs * c->nq * nn},
      {&c->b.Utr, rs * (c->nvar + (precision == NSK_FP64 ? TraceComps<double>::extra : 0)) * faces},
      {&c->utr_alt, rs * (c->nvar + (precision == NSK_FP64 ? TraceComps<double>::extra : 0)) * faces},
      {&c->b.FVtr, rs * (dim + 1) * faces},
      {&c->b.Fstar, rs * c->nvar * c->E * dim * c->nfn},
      {(void**)&c->b.err, sizeof(int)},
      {(void**)&c->b.lam, 2 * sizeof(unsigned long long)},
      {(void**)&c->b.dt, sizeof(double)},
      {(void**)&c->b.part, sizeof(double) * (3 * (size_t)c->b.nparts + 3)},
      {&c->rbuf, rs * c->nvar * nn},
      {(void**)&c->stage64, sizeof(double) * maxc * nn},
  };
  for (auto& a : allocs) {
    if (cudaMalloc(a.ptr, a.bytes) != cudaSuccess) {
      cudaGetLastError();
      free_ctx(c);
      return NSK_ERR_NOMEM;
    }
  }
  c->p.berr = c->b.err;  // the bounds-checking build's index checks report here
  if (cudaMemset(c->b.err, 0, sizeof(int)) != cudaSuccess || cudaMemset(c->b.K, 0, rs * c->nvar * nn) != cudaSuccess ||
      cudaMemset(c->b.dt, 0, sizeof(double)) != cudaSuccess) {
    free_ctx(c);
    return NSK_ERR_CUDA;
  }
  *out = c;
  return NSK_OK;
}

int nsk_set_params(nsk_ctx* c, double T, double kappa, double alpha, double beta, double mu) {
  if (!c) return NSK_ERR_ARG;
  if (!(T > 0.0 && T < 1.0) || !(kappa > 0.0) || !(beta > 0.0) || !(mu >= 0.0) || !isfinite(alpha) ||
      !isfinite(kappa) || !isfinite(beta) || !isfinite(mu))
    return NSK_ERR_ARG;
  // Reduced VdW: W'' = p'/rho = 24 T / (rho (3 - rho)^2) - 6; rho (3 - rho)^2 peaks at
  // rho = 1, so min W'' = 6 T - 6 and alpha_* = 3 (1 - T) (Eq. alpha_fullyhyperbolic_limit).
  const double alpha_star = 3.0 * (1.0 - T);
  if (!(alpha > alpha_star)) return NSK_ERR_ARG;
  c->p.T = T;
  c->p.kappa = kappa;
  c->p.alpha = alpha;
  c->p.beta = beta;
  c->p.mu = mu;
  set_eos_constants(c->p);
  c->params_set = true;
  return NSK_OK;
}

int nsk_set_c_dissipation(nsk_ctx* c, int on) {
  if (!c) return NSK_ERR_ARG;
  c->p.c_diss = on ? 1 : 0;
  return NSK_OK;
}

int nsk_set_model(nsk_ctx* c, int model) {
  if (!c || (model != NSK_MODEL_RELAXATION && model != NSK_MODEL_NSK)) return NSK_ERR_ARG;
  if (model == NSK_MODEL_NSK) {
    if (c->precision != NSK_FP64) return NSK_ERR_ARG;
    if (c->closure_mode == NSK_C_LEARNED || c->fv_path()) return NSK_ERR_STATE;
    if (!c->b.Q2) {  // lap rho, and the traces of grad rho; the context takes both or neither
      const size_t faces = (size_t)c->E * 2 * c->dim * c->nfn;
      void *q2 = nullptr, *gtr = nullptr;
      if (cudaMalloc(&q2, sizeof(double) * (size_t)c->nn) != cudaSuccess) {
        cudaGetLastError();
        return NSK_ERR_NOMEM;
      }
      if (cudaMalloc(&gtr, sizeof(double) * faces) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(q2);
        return NSK_ERR_NOMEM;
      }
      c->b.Q2 = q2;
      c->b.Gtr = gtr;
    }
  }
  c->p.model = model;
  c->nvar = model == NSK_MODEL_NSK ? c->dim + 1 : c->dim + 2;
  c->state_set = false;  // the state layout changed
  return NSK_OK;
}

int nsk_set_flux(nsk_ctx* c, int flux) {
  if (!c || (flux != NSK_FLUX_LF && flux != NSK_FLUX_HLLC)) return NSK_ERR_ARG;
  c->p.flux = flux;
  return NSK_OK;
}

int nsk_set_state(nsk_ctx* c, const double* U, int where) {
  const NskRange nvtx_range("nsk_set_state");
  if (!c || !U || (where != NSK_HOST && where != NSK_DEVICE)) return NSK_ERR_ARG;
  if (!c->params_set) return NSK_ERR_STATE;
  const long long n = (long long)c->nvar * c->nn;
  const size_t bytes = sizeof(double) * (size_t)n;
  const cudaMemcpyKind kind = where == NSK_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (c->precision == NSK_FP64) {
    if (cudaMemcpyAsync(c->b.U, U, bytes, kind, c->stream) != cudaSuccess) return NSK_ERR_CUDA;
  } else {
    const double* src = U;
    if (where == NSK_HOST) {
      if (cudaMemcpyAsync(c->stage64, U, bytes, kind, c->stream) != cudaSuccess) return NSK_ERR_CUDA;
      src = c->stage64;
    }
    int r = nsk_launch_convert(src, true, c->b.U, false, n, c->stream);
    if (r < 0) return r;
    c->launches += r;
  }
  if (cudaMemsetAsync(c->b.K, 0, c->rsize * (size_t)n, c->stream) != cudaSuccess) return NSK_ERR_CUDA;
  if (c->fvb.flags && cudaMemsetAsync(c->fvb.flags, 0, sizeof(int) * (size_t)c->E, c->stream) != cudaSuccess)
    return NSK_ERR_CUDA;  // the given state is nodal (DG) everywhere
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NSK_ERR_CUDA;
  c->state_set = true;
  return NSK_OK;
}

int nsk_get_state(nsk_ctx* c, double* U, int where) {
  const NskRange nvtx_range("nsk_get_state");
  if (!c || !U || (where != NSK_HOST && where != NSK_DEVICE)) return NSK_ERR_ARG;
  if (!c->state_set) return NSK_ERR_STATE;
  int r = export_nodal(c, c->b.U, c->nvar, U, where);
  if (r) return r;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

int nsk_node_coords(nsk_ctx* c, double* x, int where) {
  if (!c || !x || (where != NSK_HOST && where != NSK_DEVICE)) return NSK_ERR_ARG;
  const long long nn = c->nn;
  double* hx = (double*)malloc(sizeof(double) * c->dim * nn);
  if (!hx) return NSK_ERR_NOMEM;
  for (long long e = 0; e < c->E; ++e) {
    long long ec[3] = {e % c->ne[0], (e / c->ne[0]) % c->ne[1], e / ((long long)c->ne[0] * c->ne[1])};
    for (int n = 0; n < c->npe; ++n) {
      int idx = n;
      for (int k = 0; k < c->dim; ++k) {
        const int i = idx % c->np;
        idx /= c->np;
        hx[k * nn + e * c->npe + n] = c->lo[k] + c->h[k] * (ec[k] + 0.5 * (c->xi[i] + 1.0));
      }
    }
  }
  int st = NSK_OK;
  const cudaMemcpyKind kind = where == NSK_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  if (cudaMemcpy(x, hx, sizeof(double) * c->dim * nn, kind) != cudaSuccess) st = NSK_ERR_CUDA;
  free(hx);
  return st;
}

// one stage of the 1D sub-cell path (nsk_fv.cu)
int fv_stage(nsk_ctx* c, int mode, double* Rout, double A, double B, const double* dtp, double dtv) {
  const int r = nsk_fv_launch_stage(c->p, c->fv_params, c->np, c->fvb, c->b, mode, Rout, A, B, dtp, dtv, c->stream);
  if (r < 0) return r;
  c->launches += r;
  return NSK_OK;
}

int nsk_rhs(nsk_ctx* c, double t, double* Ut, int where) {
  const NskRange nvtx_range("nsk_rhs");
  (void)t;
  if (!c || !Ut || (where != NSK_HOST && where != NSK_DEVICE)) return NSK_ERR_ARG;
  if (!c->state_set) return NSK_ERR_STATE;
  if (c->fv_path()) {
    int r = fv_stage(c, NSK_MODE_RHS, (double*)c->rbuf, 0.0, 0.0, nullptr, 0.0);
    if (r) return r;
    r = export_nodal(c, c->rbuf, c->nvar, Ut, where);
    if (r) return r;
    return sync_and_check(c);
  }
  NskLaunch l = {NSK_MODE_RHS, c->rbuf, 0.0, 0.0, nullptr, 0.0, nullptr, c->tpb, c->fused_face};
  int r = launch_stage(c, l);
  if (r) return r;
  r = export_nodal(c, c->rbuf, c->nvar, Ut, where);
  if (r) return r;
  return sync_and_check(c);
}

int nsk_lift(nsk_ctx* c, double* Q, int where) {
  const NskRange nvtx_range("nsk_lift");
  if (!c || !Q || (where != NSK_HOST && where != NSK_DEVICE)) return NSK_ERR_ARG;
  if (!c->state_set || c->fv_path()) return NSK_ERR_STATE;
  NskLaunch l = {NSK_MODE_LIFT, nullptr, 0.0, 0.0, nullptr, 0.0, nullptr, c->tpb, c->fused_face};
  int r = launch_stage(c, l);
  if (r) return r;
  r = export_nodal(c, c->b.Q, c->nq, Q, where);
  if (r) return r;
  return sync_and_check(c);
}

int nsk_compute_dt(nsk_ctx* c, double cfl, double* dt_out) {
  const NskRange nvtx_range("nsk_compute_dt");
  if (!c || !dt_out || !(cfl > 0.0)) return NSK_ERR_ARG;
  if (!c->state_set) return NSK_ERR_STATE;
  int r = launch_dt(c, cfl);
  if (r < 0) return r;
  c->launches += r;
  if (cudaMemcpyAsync(dt_out, c->b.dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return NSK_ERR_CUDA;
  return sync_and_check(c);
}

int nsk_step(nsk_ctx* c, double dt, int nsteps) {
  const NskRange nvtx_range("nsk_step");
  if (!c || nsteps < 0 || !isfinite(dt) || dt == 0.0) return NSK_ERR_ARG;
  if (!c->state_set) return NSK_ERR_STATE;
  const bool adaptive = dt < 0.0;
  if (c->fv_path()) {  // 1D sub-cell path: switches before every step, then the five stages
    if (!adaptive && c->E <= nsk_fv_coop_max_elements()) {  // small mesh: the whole call in one launch
      int r = nsk_fv_launch_coop(c->p, c->fv_params, c->np, c->fvb, c->b, nsteps, c->fv_on, dt, kA, kB, c->stream);
      if (r < 0) return r;
      if (r > 0) {
        c->launches += r;
        return sync_and_check(c);
      }
    }
    for (int s = 0; s < nsteps; ++s) {
      if (adaptive) {
        int r = launch_dt(c, -dt);
        if (r < 0) return r;
        c->launches += r;
      }
      if (c->fv_on) {
        int r = nsk_fv_launch_switch(c->p, c->fv_params, c->np, c->fvb, (double*)c->b.U, c->stream);
        if (r < 0) return r;
        c->launches += r;
      }
      for (int st = 0; st < 5; ++st) {
        int r = fv_stage(c, NSK_MODE_LSRK, nullptr, kA[st], kB[st], adaptive ? c->b.dt : nullptr, dt);
        if (r) return r;
      }
    }
    return sync_and_check(c);
  }
  if (c->fused_face == 3 && !adaptive && c->closure_mode != NSK_C_LEARNED && block_eligible(c)) {
    // single-block schedule: every stage of every step in one launch
    const int r = launch_block(c, nsteps, dt, nullptr);
    if (r) return r;
    return sync_and_check(c);
  }
  bool ready = false;  // b.Utr holds the traces of U
  for (int s = 0; s < nsteps; ++s) {
    if (adaptive) {
      int r = launch_dt(c, -dt);
      if (r < 0) return r;
      c->launches += r;
    }
    const bool learned = c->closure_mode == NSK_C_LEARNED;
    for (int st = 0; st < 5; ++st) {
      if (learned) {  // the closure rewrites c before every stage, and the c traces with it
        const int r = nsk_closure_apply_ctx(c, ready ? c->b.Utr : nullptr);
        if (r) return r;
      }
      // (the single-block schedule, where it does not apply, steps with the separate face pass)
      const int ff = c->fused_face == 3 ? 0 : c->fused_face;
      NskLaunch l = {NSK_MODE_LSRK, nullptr, kA[st], kB[st], adaptive ? c->b.dt : nullptr, dt, nullptr, c->tpb, ff};
      // the volume kernel writes the traces of the updated state for the next stage of this call
      const bool write = c->p.model != NSK_MODEL_NSK && !(s == nsteps - 1 && st == 4);
      l.traces_ready = ready;
      l.utr_next = write ? (ff ? c->utr_alt : c->b.Utr) : nullptr;
      int r = launch_stage(c, l);
      if (r) return r;
      if (write && ff) std::swap(c->b.Utr, c->utr_alt);
      ready = write;
    }
    if (learned && c->judge_every > 0 && ++c->steps_since_judge >= c->judge_every) {
      c->steps_since_judge = 0;
      int r = nsk_closure_apply_ctx(c, nullptr);  // judge the closure's c of the current state
      if (r) return r;
      r = nsk_closure_judge_ctx(c);
      if (r) return r;
      ready = false;
    }
  }
  if (c->closure_mode == NSK_C_LEARNED) {  // the stored state carries the closure's c
    const int r = nsk_closure_apply_ctx(c, nullptr);
    if (r) return r;
  }
  return sync_and_check(c);
}

// ---- the host-state step: the state in from host memory, the steps, the state out ----
namespace {
// the overlapped path applies: FP64 relaxation model without closure or sub-cells, 3D, N = 3,
// the separate face pass, no profiling, and NSK_IO_SLABS z-slabs of whole blocks of every
// stage kernel (each slab whole z planes, a multiple of the 16 elements of a 256-thread
// prolongation or face-pass block; the lifting and volume blocks hold 2 or 4 elements)
bool host_overlap_eligible(const nsk_ctx* c) {
  if (c->precision != NSK_FP64 || c->dim != 3 || c->np != 4 || c->p.model == NSK_MODEL_NSK || c->fv_path() ||
      c->closure_mode == NSK_C_LEARNED || c->fused_face != 0 || (c->tpb != 128 && c->tpb != 256) || c->prof_on)
    return false;
  return c->ne[2] % NSK_IO_SLABS == 0 && (c->E / NSK_IO_SLABS) % 16 == 0;
}
int io_setup(nsk_ctx* c) {
  if (!c->io_stream) {
    if (cudaStreamCreateWithFlags(&c->io_stream, cudaStreamNonBlocking) != cudaSuccess) {
      c->io_stream = nullptr;
      cudaGetLastError();
      return NSK_ERR_CUDA;
    }
  }
  for (cudaEvent_t& ev : c->io_ev)
    if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      ev = nullptr;
      cudaGetLastError();
      return NSK_ERR_CUDA;
    }
  return NSK_OK;
}
// the queued steps of the overlapped path (the copies on io_stream, the kernels on the context's
// stream); returns at the first error, with work possibly still queued
int host_steps(nsk_ctx* c, const double* U_in, double* U_out, double dt, int nsteps) {
  constexpr int NS = NSK_IO_SLABS;
  const long long slab = c->E / NS, sn = slab * c->npe;
  const size_t sbytes = sizeof(double) * (size_t)sn;
  double* U = (double*)c->b.U;
  cudaEvent_t* ev = c->io_ev;  // [0, NS): slab k in; [NS, 2 NS): slab k written; 2 NS: prior work
  auto copy = [&](double* dst, const double* src, int k, cudaMemcpyKind kind) -> int {
    for (int v = 0; v < c->nvar; ++v) {
      const size_t off = (size_t)v * (size_t)c->nn + (size_t)k * (size_t)sn;
      if (cudaMemcpyAsync(dst + off, src + off, sbytes, kind, c->io_stream) != cudaSuccess) return NSK_ERR_CUDA;
    }
    return NSK_OK;
  };
  auto part = [&](const NskLaunch& l, int which, int k0, int nk) -> int {
    const int r = nsk_launch_stage_part_d3(c->p, c->np, false, c->b, l, c->stream, which, (long long)k0 * slab,
                                           (long long)nk * slab);
    if (r < 0) return r;
    c->launches += r;
    return NSK_OK;
  };
  // the copies in, slab by slab, once the context's stream has finished what it holds
  if (cudaEventRecord(ev[2 * NS], c->stream) != cudaSuccess || cudaStreamWaitEvent(c->io_stream, ev[2 * NS], 0))
    return NSK_ERR_CUDA;
  for (int k = 0; k < NS; ++k) {
    if (copy(U, U_in, k, cudaMemcpyHostToDevice) || cudaEventRecord(ev[k], c->io_stream) != cudaSuccess)
      return NSK_ERR_CUDA;
  }
  if (cudaMemsetAsync(c->b.K, 0, c->rsize * (size_t)c->nvar * (size_t)c->nn, c->stream) != cudaSuccess)
    return NSK_ERR_CUDA;
  bool ready = false;  // b.Utr holds the traces of U
  for (int s = 0; s < nsteps; ++s)
    for (int st = 0; st < 5; ++st) {
      NskLaunch l = {NSK_MODE_LSRK, nullptr, kA[st], kB[st], nullptr, dt, nullptr, c->tpb, 0};
      const bool first = s == 0 && st == 0, last = s == nsteps - 1 && st == 4;
      l.traces_ready = ready;
      l.utr_next = last ? nullptr : c->b.Utr;  // the volume kernel writes the next stage's traces
      int r = NSK_OK;
      if (first) {
        // the prolongation of slab k once it has arrived, the lifting of slab k - 1 once slabs
        // k - 2 .. k have their traces (z neighbours; periodic, so slabs NS - 1 and 0 last), then
        // the face pass and the volume kernel over the mesh
        for (int k = 0; k < NS && r == NSK_OK; ++k) {
          if (cudaStreamWaitEvent(c->stream, ev[k], 0) != cudaSuccess) return NSK_ERR_CUDA;
          r = part(l, 0, k, 1);
          if (r == NSK_OK && k >= 2) r = part(l, 1, k - 1, 1);
        }
        if (r == NSK_OK) r = part(l, 1, NS - 1, 1);
        if (r == NSK_OK) r = part(l, 1, 0, 1);
        if (r == NSK_OK) r = part(l, 2, 0, NS);
        if (r == NSK_OK) r = part(l, 3, 0, NS);
      } else if (last) {
        // the lifting and face pass over the mesh, then the volume kernel slab by slab, each slab
        // copied out once written
        r = part(l, 1, 0, NS);
        if (r == NSK_OK) r = part(l, 2, 0, NS);
        for (int k = 0; k < NS && r == NSK_OK; ++k) {
          r = part(l, 3, k, 1);
          if (r == NSK_OK && (cudaEventRecord(ev[NS + k], c->stream) != cudaSuccess ||
                              cudaStreamWaitEvent(c->io_stream, ev[NS + k], 0) != cudaSuccess))
            r = NSK_ERR_CUDA;
          if (r == NSK_OK) r = copy(U_out, U, k, cudaMemcpyDeviceToHost);
        }
      } else {
        r = launch_stage(c, l);
      }
      if (r) return r;
      ready = !last;
    }
  return NSK_OK;
}
}  // namespace

int nsk_step_host(nsk_ctx* c, const double* U_in, double* U_out, double dt, int nsteps) {
  const NskRange nvtx_range("nsk_step_host");
  if (!c || !U_in || !U_out || nsteps < 1 || !isfinite(dt) || dt <= 0.0) return NSK_ERR_ARG;
  if (!c->params_set) return NSK_ERR_STATE;
  if (!host_overlap_eligible(c) || io_setup(c) != NSK_OK) {  // the three calls in turn
    int r = nsk_set_state(c, U_in, NSK_HOST);
    if (r == NSK_OK) r = nsk_step(c, dt, nsteps);
    if (r == NSK_OK) r = nsk_get_state(c, U_out, NSK_HOST);
    return r;
  }
  c->state_set = true;
  const int r = host_steps(c, U_in, U_out, dt, nsteps);
  // the caller's host buffers are not touched once the call returns, whatever happened
  const bool io_ok = cudaStreamSynchronize(c->io_stream) == cudaSuccess;
  const int rc = sync_and_check(c);
  if (r) return r;
  return io_ok ? rc : NSK_ERR_CUDA;
}

// ---- 1D sub-cell shock capturing and Dirichlet boundaries ----
static int fv_refresh(nsk_ctx* c) {
  if (!c->fv_params) {
    c->fv_params = malloc(nsk_fv_params_size());
    if (!c->fv_params) return NSK_ERR_NOMEM;
  }
  if (!c->fvb.flags) {  // the context takes the whole group, allocated and cleared, or none of it
    const size_t E = (size_t)c->E;
    FvBuffers fb = {};
    struct {
      void** ptr;
      size_t bytes;
    } allocs[] = {{(void**)&fb.flags, sizeof(int) * E},          {(void**)&fb.ind, sizeof(double) * E},
                  {(void**)&fb.Uf, sizeof(double) * 6 * E},      {(void**)&fb.Gf, sizeof(double) * 4 * E},
                  {(void**)&fb.SL, sizeof(double) * 3 * E * c->np}, {(void**)&fb.Fh, sizeof(double) * 3 * (E + 1)},
                  {(void**)&fb.bar, sizeof(unsigned) * 2}};
    int st = NSK_OK;
    for (auto& a : allocs) {
      void* q = nullptr;
      if (cudaMalloc(&q, a.bytes) != cudaSuccess) {
        cudaGetLastError();
        st = NSK_ERR_NOMEM;
        break;
      }
      *a.ptr = q;
    }
    if (st == NSK_OK && (cudaMemset(fb.flags, 0, sizeof(int) * E) != cudaSuccess ||
                         cudaMemset(fb.ind, 0, sizeof(double) * E) != cudaSuccess ||
                         cudaMemset(fb.bar, 0, sizeof(unsigned) * 2) != cudaSuccess))
      st = NSK_ERR_CUDA;
    if (st != NSK_OK) {
      for (auto& a : allocs)
        if (*a.ptr) cudaFree(*a.ptr);
      return st;
    }
    c->fvb = fb;
  }
  double gx[NSK_MAXNP], gw[NSK_MAXNP];
  gauss_legendre(c->np, gx, gw);
  return nsk_fv_fill_params(c->fv_params, c->np, c->xi, gx, gw, c->h[0], c->fv_dirichlet, c->fv_Ub[0], c->fv_Ub[1],
                            c->fv_upper, c->fv_lower);
}

static bool fv_allowed(const nsk_ctx* c) {
  return c->dim == 1 && c->precision == NSK_FP64 && c->p.model == NSK_MODEL_RELAXATION &&
         c->closure_mode == NSK_C_EXPLICIT && c->np <= 6;
}

int nsk_set_subcell(nsk_ctx* c, int on, double ind_upper, double ind_lower) {
  if (!c || (on && (isnan(ind_upper) || isnan(ind_lower) || ind_lower > ind_upper))) return NSK_ERR_ARG;
  if (on && !fv_allowed(c)) return NSK_ERR_ARG;
  if (!on && c->fvb.flags) {  // elements holding means cannot continue as nodal values
    std::vector<int> f((size_t)c->E);
    if (cudaMemcpy(f.data(), c->fvb.flags, sizeof(int) * f.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return NSK_ERR_CUDA;
    for (int x : f)
      if (x) return NSK_ERR_STATE;
  }
  c->fv_on = on ? 1 : 0;
  c->fv_upper = ind_upper;
  c->fv_lower = ind_lower;
  return c->fv_path() ? fv_refresh(c) : NSK_OK;
}

int nsk_set_dirichlet(nsk_ctx* c, int on, const double Ub_lo[3], const double Ub_hi[3]) {
  if (!c || (on && (!Ub_lo || !Ub_hi))) return NSK_ERR_ARG;
  if (on && !fv_allowed(c)) return NSK_ERR_ARG;
  if (on)
    for (int v = 0; v < 3; ++v) {
      if (!isfinite(Ub_lo[v]) || !isfinite(Ub_hi[v])) return NSK_ERR_ARG;
      c->fv_Ub[0][v] = Ub_lo[v];
      c->fv_Ub[1][v] = Ub_hi[v];
    }
  if (!on && c->fv_on) {
    c->fv_dirichlet = 0;
    return fv_refresh(c);
  }
  c->fv_dirichlet = on ? 1 : 0;
  return c->fv_path() ? fv_refresh(c) : NSK_OK;
}

int nsk_set_subcell_flags(nsk_ctx* c, const int* flags) {
  if (!c || !flags) return NSK_ERR_ARG;
  if (!c->fv_path()) return NSK_ERR_STATE;
  for (long long e = 0; e < c->E; ++e)
    if (flags[e] != 0 && flags[e] != 1) return NSK_ERR_ARG;
  if (cudaMemcpy(c->fvb.flags, flags, sizeof(int) * (size_t)c->E, cudaMemcpyHostToDevice) != cudaSuccess)
    return NSK_ERR_CUDA;
  return NSK_OK;
}

int nsk_get_subcell(nsk_ctx* c, int* flags, double* ind) {
  if (!c || (!flags && !ind)) return NSK_ERR_ARG;
  if (!c->fv_path()) return NSK_ERR_STATE;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NSK_ERR_CUDA;
  if (flags && cudaMemcpy(flags, c->fvb.flags, sizeof(int) * (size_t)c->E, cudaMemcpyDeviceToHost) != cudaSuccess)
    return NSK_ERR_CUDA;
  if (ind && cudaMemcpy(ind, c->fvb.ind, sizeof(double) * (size_t)c->E, cudaMemcpyDeviceToHost) != cudaSuccess)
    return NSK_ERR_CUDA;
  return NSK_OK;
}

int nsk_subcell_switch(nsk_ctx* c) {
  if (!c) return NSK_ERR_ARG;
  if (!c->fv_on) return NSK_ERR_STATE;
  if (!c->state_set) return NSK_ERR_STATE;
  const int r = nsk_fv_launch_switch(c->p, c->fv_params, c->np, c->fvb, (double*)c->b.U, c->stream);
  if (r < 0) return r;
  c->launches += r;
  return sync_and_check(c);
}

int nsk_diagnostics(nsk_ctx* c, double* mass, double* energy, double* l2) {
  const NskRange nvtx_range("nsk_diagnostics");
  if (!c) return NSK_ERR_ARG;
  if (!c->state_set) return NSK_ERR_STATE;
  NskLaunch l = {NSK_MODE_LIFT, nullptr, 0.0, 0.0, nullptr, 0.0, nullptr, c->tpb, c->fused_face};
  int r = launch_stage(c, l);
  if (r) return r;
  r = nsk_launch_diag(c->p, c->dim, c->np, c->precision == NSK_FP32_MIXED, c->b, c->stream);
  if (r < 0) return r;
  c->launches += r;
  double h[3];
  if (cudaMemcpyAsync(h, c->b.part + 3 * c->b.nparts, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return NSK_ERR_CUDA;
  r = sync_and_check(c);
  if (r) return r;
  if (mass) *mass = h[0];
  if (energy) *energy = h[1];
  if (l2) *l2 = sqrt(h[2]);
  return NSK_OK;
}

int nsk_get_sizes(nsk_ctx* c, long long* n_elem, int* nodes_per_elem, int* nvar) {
  if (!c) return NSK_ERR_ARG;
  if (n_elem) *n_elem = c->E;
  if (nodes_per_elem) *nodes_per_elem = c->npe;
  if (nvar) *nvar = c->nvar;
  return NSK_OK;
}

long long nsk_launch_count(nsk_ctx* c) { return c ? c->launches : -1; }

int nsk_set_schedule(nsk_ctx* c, int tpb, int fused_face) {
  if (!c || (tpb != 128 && tpb != 256) || fused_face < 0 || fused_face > 4) return NSK_ERR_ARG;
  c->tpb = tpb;
  c->fused_face = fused_face;
  return NSK_OK;
}

int nsk_get_schedule(nsk_ctx* c, int* tpb, int* fused_face) {
  if (!c) return NSK_ERR_ARG;
  if (tpb) *tpb = c->tpb;
  if (fused_face) *fused_face = c->fused_face;
  return NSK_OK;
}

int nsk_autotune(nsk_ctx* c, int* tpb_out, int* fused_out, double* ms_out) {
  const NskRange nvtx_range("nsk_autotune");
  if (!c) return NSK_ERR_ARG;
  if (!c->state_set) return NSK_ERR_STATE;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return NSK_ERR_CUDA;
  const int tpbs[2] = {128, 256};
  double best = 1e300;
  int bt = c->tpb, bf = c->fused_face, st = NSK_OK;
  const bool prof = c->prof_on;
  c->prof_on = false;
  // the lean two-launch stage applies to relaxation model II only (the original NSK equations
  // have their own stage kernels and take the schedule's block size alone)
  // and the line schedule to the FP32 operator on 3D elements with N = 3
  int sched[5], nsched = 0;
  sched[nsched++] = 0;
  sched[nsched++] = 1;
  if (c->p.model != NSK_MODEL_NSK) sched[nsched++] = 2;
  if (c->p.model != NSK_MODEL_NSK && block_eligible(c)) sched[nsched++] = 3;
  if (line_eligible(c)) sched[nsched++] = 4;
  for (int it = 0; it < 2 && st == NSK_OK; ++it)
    for (int f = 0; f < nsched && st == NSK_OK; ++f) {
      c->tpb = tpbs[it];
      c->fused_face = sched[f];
      NskLaunch l = {NSK_MODE_RHS, c->rbuf, 0.0, 0.0, nullptr, 0.0, nullptr, c->tpb, c->fused_face};
      st = launch_stage(c, l);  // warm-up; leaves b.Utr holding the traces of U
      if (st) break;
      // time what a stage inside nsk_step runs: no prolongation pass, traces written by the
      // volume kernel (to the spare buffer: U does not change in RHS mode)
      l.traces_ready = 1;
      l.utr_next = c->utr_alt;
      cudaEventRecord(e0, c->stream);
      for (int r = 0; r < 3 && st == NSK_OK; ++r) st = launch_stage(c, l);
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = NSK_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (st == NSK_OK && ms / 3.0 < best) {
        best = ms / 3.0;
        bt = c->tpb;
        bf = c->fused_face;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->prof_on = prof;
  c->tpb = bt;
  c->fused_face = bf;
  if (st) return st;
  if (tpb_out) *tpb_out = bt;
  if (fused_out) *fused_out = bf;
  if (ms_out) *ms_out = best;
  return sync_and_check(c);
}

int nsk_set_profiling(nsk_ctx* c, int on) {
  if (!c) return NSK_ERR_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NSK_ERR_CUDA;
  prof_collect(c);
  c->prof_on = on != 0;
  return NSK_OK;
}

int nsk_get_profile(nsk_ctx* c, double* ms, long long* launches, int n, int reset) {
  if (!c || n < 0) return NSK_ERR_ARG;
  for (int k = 0; k < n && k < NSK_NKERN; ++k) {
    if (ms) ms[k] = c->prof_ms[k];
    if (launches) launches[k] = c->prof_cnt[k];
  }
  if (reset)
    for (int k = 0; k < NSK_NKERN; ++k) {
      c->prof_ms[k] = 0.0;
      c->prof_cnt[k] = 0;
    }
  return NSK_NKERN;
}

int nsk_test_hook_corrupt_neighbours(nsk_ctx* c) {
  if (!c) return NSK_ERR_ARG;
#ifdef NSK_BOUNDS_CHECK
  for (int k = 0; k < c->dim; ++k) {
    c->p.est[k] = 1 << 29;
    c->p.ewrap[k] = -(1 << 29);
  }
  return NSK_OK;
#else
  return NSK_ERR_STATE;
#endif
}

// ---- checkpoint and resume ----
}  // extern "C"

namespace {
struct CkptHead {  // written field by field (no padding in the file)
  int32_t dim, N, node_type, precision, model, flux, c_diss, nflags, nelem[3];
  double lo[3], hi[3], T, kappa, alpha, beta, mu, t;
  int64_t step, nvals;
};
const char kCkptMagic[8] = {'N', 'S', 'K', 'C', 'K', 'P', 'T', 0};
const uint32_t kCkptVersion = 1;

template <typename X>
bool put(FILE* f, const X* x, size_t n) { return fwrite(x, sizeof(X), n, f) == n; }
template <typename X>
bool get(FILE* f, X* x, size_t n) { return fread(x, sizeof(X), n, f) == n; }

bool write_head(FILE* f, const CkptHead& h) {
  return put(f, kCkptMagic, 8) && put(f, &kCkptVersion, 1) && put(f, &h.dim, 1) && put(f, &h.N, 1) &&
         put(f, &h.node_type, 1) && put(f, &h.precision, 1) && put(f, &h.model, 1) && put(f, &h.flux, 1) &&
         put(f, &h.c_diss, 1) && put(f, &h.nflags, 1) && put(f, h.nelem, 3) && put(f, h.lo, 3) && put(f, h.hi, 3) &&
         put(f, &h.T, 1) && put(f, &h.kappa, 1) && put(f, &h.alpha, 1) && put(f, &h.beta, 1) && put(f, &h.mu, 1) &&
         put(f, &h.t, 1) && put(f, &h.step, 1) && put(f, &h.nvals, 1);
}
bool read_head(FILE* f, CkptHead& h) {
  char magic[8];
  uint32_t ver = 0;
  return get(f, magic, 8) && memcmp(magic, kCkptMagic, 8) == 0 && get(f, &ver, 1) && ver == kCkptVersion &&
         get(f, &h.dim, 1) && get(f, &h.N, 1) && get(f, &h.node_type, 1) && get(f, &h.precision, 1) &&
         get(f, &h.model, 1) && get(f, &h.flux, 1) && get(f, &h.c_diss, 1) && get(f, &h.nflags, 1) &&
         get(f, h.nelem, 3) && get(f, h.lo, 3) && get(f, h.hi, 3) && get(f, &h.T, 1) && get(f, &h.kappa, 1) &&
         get(f, &h.alpha, 1) && get(f, &h.beta, 1) && get(f, &h.mu, 1) && get(f, &h.t, 1) && get(f, &h.step, 1) &&
         get(f, &h.nvals, 1);
}
}  // namespace

extern "C" {

int nsk_save_checkpoint(nsk_ctx* c, const char* path, double t, long long step) {
  const NskRange nvtx_range("nsk_save_checkpoint");
  if (!c || !path) return NSK_ERR_ARG;
  if (!c->state_set || !c->params_set) return NSK_ERR_STATE;
  CkptHead h;
  memset(&h, 0, sizeof(h));
  h.dim = c->dim;
  h.N = c->N;
  h.node_type = c->node_type;
  h.precision = c->precision;
  h.model = c->p.model;
  h.flux = c->p.flux;
  h.c_diss = c->p.c_diss;
  h.nflags = c->fv_on ? (int32_t)c->E : 0;
  for (int k = 0; k < 3; ++k) {
    h.nelem[k] = c->ne[k];
    h.lo[k] = c->lo[k];
    h.hi[k] = c->hi[k];
  }
  h.T = c->p.T;
  h.kappa = c->p.kappa;
  h.alpha = c->p.alpha;
  h.beta = c->p.beta;
  h.mu = c->p.mu;
  h.t = t;
  h.step = step;
  h.nvals = (int64_t)c->nvar * c->nn;
  std::vector<double> U((size_t)h.nvals);
  int r = nsk_get_state(c, U.data(), NSK_HOST);
  if (r) return r;
  std::vector<int> flags((size_t)h.nflags);
  if (h.nflags && (r = nsk_get_subcell(c, flags.data(), nullptr))) return r;
  FILE* f = fopen(path, "wb");
  if (!f) return NSK_ERR_IO;
  bool ok = write_head(f, h) && put(f, U.data(), U.size());
  if (ok && h.nflags) {
    std::vector<int32_t> f32(flags.begin(), flags.end());
    ok = put(f, f32.data(), f32.size());
  }
  ok = (fclose(f) == 0) && ok;
  return ok ? NSK_OK : NSK_ERR_IO;
}

int nsk_load_checkpoint(nsk_ctx* c, const char* path, double* t, long long* step) {
  const NskRange nvtx_range("nsk_load_checkpoint");
  if (!c || !path) return NSK_ERR_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return NSK_ERR_IO;
  CkptHead h;
  bool ok = read_head(f, h);
  ok = ok && h.dim == c->dim && h.N == c->N && h.node_type == c->node_type && h.precision == c->precision &&
       h.model == c->p.model && h.nvals == (int64_t)c->nvar * c->nn && (h.nflags == 0 || h.nflags == c->E);
  for (int k = 0; k < 3 && ok; ++k)
    ok = h.nelem[k] == c->ne[k] && h.lo[k] == c->lo[k] && h.hi[k] == c->hi[k];
  std::vector<double> U;
  std::vector<int32_t> flags;
  if (ok) {
    U.resize((size_t)h.nvals);
    flags.resize((size_t)h.nflags);
    ok = get(f, U.data(), U.size()) && (h.nflags == 0 || get(f, flags.data(), flags.size()));
  }
  fclose(f);
  if (!ok) return NSK_ERR_IO;
  int r = nsk_set_params(c, h.T, h.kappa, h.alpha, h.beta, h.mu);
  if (r) return r;
  if ((r = nsk_set_flux(c, h.flux)) || (r = nsk_set_c_dissipation(c, h.c_diss))) return r;
  if ((r = nsk_set_state(c, U.data(), NSK_HOST))) return r;
  if (h.nflags) {
    std::vector<int> fl(flags.begin(), flags.end());
    if ((r = nsk_set_subcell_flags(c, fl.data()))) return r;
  }
  if (t) *t = h.t;
  if (step) *step = h.step;
  return NSK_OK;
}

void nsk_destroy(nsk_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free residual (nsk_rhs_static_scratch). The scratch of the four
// stage kernels (face traces, lifted gradients, face fluxes, error word) lives
// in one file-scope device array, so a call allocates nothing. In host code
// the array's name is only a host-side stand-in: its device address is looked
// up once per device with cudaGetSymbolAddress and cached.
// ---------------------------------------------------------------------------
#define NSK_STATIC_SCRATCH_BYTES (64ull << 20)
#define NSK_STATIC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char nsk_static_scratch[NSK_STATIC_SCRATCH_BYTES];

namespace {

// device address per device, set on first use; atomic, so host threads that make their first
// calls concurrently each look the address up (the same value) without a data race
std::atomic<void*> g_static_scratch[NSK_STATIC_MAX_DEVICES];

int static_scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return NSK_ERR_CUDA;
  if (dev < 0 || dev >= NSK_STATIC_MAX_DEVICES) return NSK_ERR_ARG;
  void* p = g_static_scratch[dev].load(std::memory_order_acquire);
  if (!p) {
    if (cudaGetSymbolAddress(&p, nsk_static_scratch) != cudaSuccess || !p) return NSK_ERR_CUDA;
    g_static_scratch[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return NSK_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" long long nsk_static_scratch_bytes(void) { return (long long)NSK_STATIC_SCRATCH_BYTES; }

extern "C" int nsk_rhs_static_scratch(int dim, const int nelem[3], const double lo[3], const double hi[3], int N,
                                      int node_type, double T, double kappa, double alpha, double beta, double mu,
                                      const double* U, double* Ut, void* cuda_stream) {
  // U is read by every stage kernel while Ut is written: the two must not alias
  if (!nelem || !lo || !hi || !U || !Ut || (const void*)U == (const void*)Ut) return NSK_ERR_ARG;
  if (dim < 1 || dim > 3 || N < 1 || N + 1 > NSK_MAXNP) return NSK_ERR_ARG;
  if (node_type != NSK_NODES_GAUSS && node_type != NSK_NODES_GAUSS_LOBATTO) return NSK_ERR_ARG;
  if (!(T > 0.0 && T < 1.0) || !(kappa > 0.0) || !(beta > 0.0) || !(mu >= 0.0) || !isfinite(alpha) ||
      !isfinite(kappa) || !isfinite(beta) || !isfinite(mu) || !(alpha > 3.0 * (1.0 - T)))
    return NSK_ERR_ARG;
  const int np = N + 1;
  long long E = 1, npe = 1, nfn = 1;
  double h[3];
  for (int k = 0; k < dim; ++k) {
    if (nelem[k] < 1 || !(hi[k] > lo[k]) || !isfinite(lo[k]) || !isfinite(hi[k])) return NSK_ERR_ARG;
    if (E > (1LL << 40) / nelem[k]) return NSK_ERR_ARG;
    E *= nelem[k];
    h[k] = (hi[k] - lo[k]) / nelem[k];
    npe *= np;
    if (k > 0) nfn *= np;
  }
  const long long nn = E * npe;
  const int nvar = dim + 2, nw = dim + 1, nq = dim * (dim + 1), nf = 2 * dim;
  // scratch layout: error word | Q | Utr | FVtr | Fstar, each 256-byte aligned
  const size_t b_err = 256;
  const size_t b_q = align256(sizeof(double) * (size_t)nq * nn);
  const size_t b_utr = align256(sizeof(double) * (size_t)(nvar + TraceComps<double>::extra) * nf * E * nfn);
  const size_t b_fv = align256(sizeof(double) * (size_t)nw * nf * E * nfn);
  const size_t b_fs = align256(sizeof(double) * (size_t)nvar * dim * E * nfn);
  if ((double)b_q + b_utr + b_fv + b_fs + b_err > (double)NSK_STATIC_SCRATCH_BYTES) return NSK_ERR_ARG;

  NskParams p;
  memset(&p, 0, sizeof(p));
  double xi[NSK_MAXNP], w[NSK_MAXNP];
  if (node_type == NSK_NODES_GAUSS)
    gauss_legendre(np, xi, w);
  else
    gauss_lobatto(N, xi, w);
  p.E = E;
  p.jac = 1.0;
  for (int k = 0; k < 3; ++k) {
    p.ne[k] = k < dim ? nelem[k] : 1;
    p.rh[k] = k < dim ? 2.0 / h[k] : 0.0;
    if (k < dim) p.jac *= h[k] / 2.0;
  }
  set_index_constants(p, (int)npe, (int)nfn);
  p.T = T;
  p.kappa = kappa;
  p.alpha = alpha;
  p.beta = beta;
  p.mu = mu;
  fill_tab<double>(p.td, np, xi, w);
  fill_tab<float>(p.tf, np, xi, w);
  set_eos_constants(p);

  void* base = nullptr;
  int st = static_scratch_address(&base);
  if (st) return st;
  unsigned char* s8 = (unsigned char*)base;
  NskBuffers b;
  memset(&b, 0, sizeof(b));
  b.U = (void*)U;
  b.err = (int*)s8;
  p.berr = b.err;
  b.Q = s8 + b_err;
  b.Utr = s8 + b_err + b_q;
  b.FVtr = s8 + b_err + b_q + b_utr;
  b.Fstar = s8 + b_err + b_q + b_utr + b_fv;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(b.err, 0, sizeof(int), stream) != cudaSuccess) return NSK_ERR_CUDA;
  NskLaunch l = {NSK_MODE_RHS, Ut, 0.0, 0.0, nullptr, 0.0, nullptr, 256, 0};
  int r;
  switch (dim) {
    case 1: r = nsk_launch_stage_d1(p, np, false, b, l, stream); break;
    case 2: r = nsk_launch_stage_d2(p, np, false, b, l, stream); break;
    default: r = nsk_launch_stage_d3(p, np, false, b, l, stream); break;
  }
  if (r < 0) return r;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, b.err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return NSK_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return NSK_ERR_CUDA;
  if (herr & NSK_EBIT_TIMEOUT) return NSK_ERR_TIMEOUT;
  return herr ? NSK_ERR_NONPHYSICAL : NSK_OK;
}
