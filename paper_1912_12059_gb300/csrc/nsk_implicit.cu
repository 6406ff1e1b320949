// nsk_implicit.cu -- implicit time integration: the six-stage, fourth-order ESDIRK that Sec. 3.1
// cites (the implicit tableau of Kennedy and Carpenter's ARK4(3)6L[2]SA, gamma = 1/4, stiffly
// accurate) with Jacobian-free Newton-Krylov on the residual kernels of the context.
//
// Every implicit stage G(X) = X - dt gamma R(X) - S_i = 0, S_i = U_n + dt sum_{j<i} a_ij R_j, is
// solved by Newton's method from the previous stage's value until ||G|| <= newton_tol ||S_i||;
// each Newton system (I - dt gamma J) d = -G by restarted GMRES(m) (Gram-Schmidt applied twice
// with batched projections, Givens rotations, relative residual krylov_tol, optionally right
// preconditioned by the inverses of the element blocks of I - dt gamma J(U_n)) with the
// matrix-free product J v ~ (R(X + eps v) - R(X)) / eps, eps = sqrt(2^-52) (1 + ||X||) / ||v||;
// the later stages use R_i = (X_i - S_i) / (dt gamma). The vector algebra runs in the kernels
// below (dot products in a fixed order: deterministic), with the scales, the projection
// coefficients, the Hessenberg matrix, the Givens rotations and the residual estimate kept on the
// device: the host reads one number per Arnoldi step, one step behind the GPU, and the triangular
// system once per GMRES cycle, which it solves; a residual evaluation is one stage launch of the
// context's pipeline in residual mode on the iterate.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "nsk_internal.h"
#include "nsk_nvtx.h"

namespace {

constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 152 * 8;
constexpr int kChunk = 4;  // Arnoldi steps replayed between two reads of a GMRES cycle's control block

// out = a x + b y + c z (y, z may be NULL; out may be x, y or z: each element is read before it
// is written by the same thread)
__global__ void __launch_bounds__(256) k_lincomb(const long long n, const double a, const double* x, const double b,
                                                 const double* y, const double c, const double* z, double* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = a * x[i];
    if (y) v = fma(b, y[i], v);
    if (z) v = fma(c, z[i], v);
    out[i] = v;
  }
}

// per-block partial sums of x . y (grid-stride per thread, then a shared-memory tree: the same
// order on every call)
__global__ void __launch_bounds__(kDotThreads) k_dot_part(const long long n, const double* __restrict__ x,
                                                          const double* __restrict__ y, double* __restrict__ part,
                                                          const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ double red[kDotThreads];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kDotThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kDotThreads) k_dot_final(const int nb, const double* __restrict__ part,
                                                           double* __restrict__ out, const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ double red[kDotThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kDotThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// sum over a warp by xor shuffles (a fixed pattern: the same order on every call)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial sums of V_j . w: vector j = blockIdx.y (all vectors at once), warp shuffles, then
// the warps' sums
__global__ void __launch_bounds__(kDotThreads) k_mdot_part(const long long n, const double* const* __restrict__ V,
                                                           const double* __restrict__ w, double* __restrict__ part,
                                                           const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ double red[kDotThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, j = blockIdx.y;
  const double* v = V[j];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(v[i], w[i], s);
  s = warp_sum(s);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (warp == 0) {
    double t = lane < kDotThreads / 32 ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) part[(size_t)j * gridDim.x + blockIdx.x] = t;
  }
}

// the two vector updates of the forward-difference product J z, with eps = c0 / ||z||
// (c0 = sqrt(2^-52) (1 + ||X||), from *c0p when given; ||z|| = sqrt(*zz), or 1 without zz)
// computed by every thread: which = 0: out = X + eps z (the perturbed state); which = 1:
// out = z - (dtg / eps) RW + (dtg / eps) RX
__global__ void __launch_bounds__(256) k_fd_combine(const long long n, const int which, const double* __restrict__ zz,
                                                    const double c0v, const double* __restrict__ c0p,
                                                    const double dtg, const double* __restrict__ X,
                                                    const double* __restrict__ z, const double* __restrict__ RW,
                                                    const double* __restrict__ RX, double* __restrict__ out,
                                                    const int* __restrict__ stop) {
  if (stop && *stop) return;
  const double c0 = c0p ? *c0p : c0v;
  const double eps = c0 / (zz ? sqrt(*zz) : 1.0);
  const double b = -dtg / eps, c = dtg / eps;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (which == 0) {
      out[i] = fma(eps, z[i], 1.0 * X[i]);
    } else {
      double v = 1.0 * z[i];
      v = fma(b, RW[i], v);
      out[i] = fma(c, RX[i], v);
    }
  }
}

constexpr int kMaxNv = 202;  // projections of a pass (krylov_dim + 1) plus w . w

// one Gram-Schmidt pass after k_mdot_part: every block sums the nb partials of each of the nred
// projections (one warp per projection, lanes over the partials, then a shuffle sum), then
// w -= sum_{j < nv} h_j V_j. With NORM (nred = nv + 1, entry nv = w . w before the pass) the new
// vector's norm follows by Pythagoras, ||w - sum_j h_j V_j||^2 = w . w - sum_j h_j^2 for an
// orthonormal basis, h[nv] becomes that norm and w is divided by it (left as is when zero).
// Block 0 writes the nred coefficients to hout for the host.
template <bool NORM>
__global__ void __launch_bounds__(256) k_gs_update(const long long n, const int nv, const double* const* __restrict__ V,
                                                   const double* __restrict__ part, const int nb,
                                                   double* __restrict__ w, double* __restrict__ hout,
                                                   const int* __restrict__ stop) {
  if (stop && *stop) return;  // uniform over the grid: before any barrier
  __shared__ double h[kMaxNv];
  __shared__ const double* vp[kMaxNv];
  __shared__ double inv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nred = NORM ? nv + 1 : nv;
  for (int j = warp; j < nred; j += blockDim.x / 32) {
    double t = 0.0;
    for (int i = lane; i < nb; i += 32) t += part[(size_t)j * nb + i];
    t = warp_sum(t);
    if (lane == 0) h[j] = t;
  }
  for (int j = threadIdx.x; j < nv; j += blockDim.x) vp[j] = V[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    double sc = 1.0;
    if (NORM) {
      double t = h[nv];
      for (int j = 0; j < nv; ++j) t = fma(-h[j], h[j], t);
      const double hn = t > 0.0 ? sqrt(t) : 0.0;
      h[nv] = hn;
      sc = hn > 0.0 ? 1.0 / hn : 1.0;
    }
    inv = sc;
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < nred; j += blockDim.x) hout[j] = h[j];
  const double s = inv;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = w[i];
#pragma unroll 4
    for (int j = 0; j < nv; ++j) v = fma(-h[j], vp[j][i], v);
    if (NORM) v = s * v;
    w[i] = v;
  }
}

// ---- element-block preconditioner: blocks of I - dt gamma J, J's diagonal blocks dR_e/dU_e ----
// local unknown k = v npe + node of element e sits at v nn + e npe + node
constexpr int kMaxBlock = 64;  // largest block (nvar npe) the shared-memory inversion takes (2D, N = 3)

// W = U with local unknown (v, node) of every element of colour c raised by
// eps_e = sqrt(2^-52) (1 + |U|)
__global__ void __launch_bounds__(256) k_fd_perturb(const long long E, const int npe, const long long nn,
                                                    const int* __restrict__ colour, const int c, const int v,
                                                    const int node, double* __restrict__ W) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
    if (colour[e] != c) continue;
    const size_t g = (size_t)v * nn + e * npe + node;
    W[g] += sqrt(ldexp(1.0, -52)) * (1.0 + fabs(W[g]));
  }
}

// column k of the blocks of the elements of colour c: J[e][i][k] = (R(W)_e,i - R(U)_e,i) / eps_e
__global__ void __launch_bounds__(256) k_fd_column(const long long E, const int nvar, const int npe, const long long nn,
                                                   const int* __restrict__ colour, const int c, const int k,
                                                   const double* __restrict__ U, const double* __restrict__ RW,
                                                   const double* __restrict__ R0, double* __restrict__ J) {
  const int n = nvar * npe;
  const int v = k / npe, node = k % npe;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < E * n; t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / n;
    const int i = (int)(t % n);
    if (colour[e] != c) continue;
    const double eps = sqrt(ldexp(1.0, -52)) * (1.0 + fabs(U[(size_t)v * nn + e * npe + node]));
    const size_t gi = (size_t)(i / npe) * nn + e * npe + i % npe;
    J[((size_t)e * n + i) * n + k] = (RW[gi] - R0[gi]) / eps;
  }
}

// block e: J_e <- (I - dtg J_e)^-1 by Gauss-Jordan elimination with partial pivoting in dynamic
// shared memory ([M | I], n x 2n doubles, n <= kMaxBlock: 64 KB at most); a zero pivot sets
// NSK_EBIT_NAN
__global__ void __launch_bounds__(128) k_block_invert(const int n, const double dtg, double* __restrict__ J,
                                                      int* __restrict__ err) {
  extern __shared__ double A[];  // row i at A + i * 2n
  __shared__ int piv;
  const int w = 2 * n;
  double* Je = J + (size_t)blockIdx.x * n * n;
  for (int t = threadIdx.x; t < n * w; t += blockDim.x) {
    const int i = t / w, j = t % w;
    A[t] = j < n ? (i == j ? 1.0 : 0.0) - dtg * Je[i * n + j] : (j - n == i ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (threadIdx.x == 0) {
      int p = c;
      for (int i = c + 1; i < n; ++i)
        if (fabs(A[i * w + c]) > fabs(A[p * w + c])) p = i;
      piv = A[p * w + c] == 0.0 ? -1 : p;
      if (piv < 0) atomicOr(err, NSK_EBIT_NAN);
    }
    __syncthreads();
    if (piv < 0) return;  // uniform over the block
    if (piv != c)
      for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const double t = A[c * w + j];
        A[c * w + j] = A[piv * w + j];
        A[piv * w + j] = t;
      }
    __syncthreads();
    const double d = A[c * w + c];
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) A[c * w + j] /= d;
    __syncthreads();
    for (int t = threadIdx.x; t < n * w; t += blockDim.x) {
      const int i = t / w, j = t % w;
      if (i != c && j != c) A[t] = fma(-A[i * w + c], A[c * w + j], A[t]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != c) A[i * w + c] = 0.0;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) Je[t] = A[(t / n) * w + n + t % n];
}

// y_e = Minv_e x_e
__global__ void __launch_bounds__(256) k_block_apply(const long long E, const int nvar, const int npe,
                                                     const long long nn, const double* __restrict__ Minv,
                                                     const double* __restrict__ x, double* __restrict__ y,
                                                     const int* __restrict__ stop) {
  if (stop && *stop) return;
  const int n = nvar * npe;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < E * n; t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / n;
    const int i = (int)(t % n);
    const double* row = Minv + ((size_t)e * n + i) * n;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s = fma(row[k], x[(size_t)(k / npe) * nn + e * npe + k % npe], s);
    y[(size_t)(i / npe) * nn + e * npe + i % npe] = s;
  }
}

// Control block of a GMRES cycle in device memory: the forward-difference scale c0, the cycle's
// starting residual norm beta, its absolute tolerance and step limit, set by k_cycle_init; the
// last step's residual estimate, the number of steps done, and stop, which ends the cycle's
// remaining steps (every kernel of an Arnoldi step returns at once when it is set).
struct CycleCtl {
  double c0, beta, tol, res;
  int kmax, stop, kdone, pad;
};
__global__ void k_cycle_init(CycleCtl* ctl, const double c0, const double beta, const double tol, const int kmax) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl->c0 = c0;
  ctl->beta = beta;
  ctl->tol = tol;
  ctl->res = beta;
  ctl->kmax = kmax;
  ctl->stop = 0;
  ctl->kdone = 0;
}

// Arnoldi step k of a GMRES cycle on the device (one thread): column k of the Hessenberg matrix
// H ((m + 1) x m, row-major) from the two Gram-Schmidt passes' coefficients (h1[0..k] + h2[0..k],
// and the new vector's norm h2[k + 1]), the earlier Givens rotations applied to it, the new
// rotation (cs, sn), and the rotated right-hand side gv (gv[0] = beta at k = 0); then the residual
// estimate |gv[k + 1]|, and stop once it is within the tolerance or the cycle's steps are used up.
__global__ void k_arnoldi_update(const int k, const int m, const double* __restrict__ h1,
                                 const double* __restrict__ h2, double* __restrict__ H, double* __restrict__ cs,
                                 double* __restrict__ sn, double* __restrict__ gv, CycleCtl* __restrict__ ctl) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || ctl->stop) return;
  if (k == 0) gv[0] = ctl->beta;
  for (int j = 0; j <= k; ++j) H[(size_t)j * m + k] = h1[j] + h2[j];
  H[(size_t)(k + 1) * m + k] = h2[k + 1];
  for (int j = 0; j < k; ++j) {  // earlier rotations
    const double a = H[(size_t)j * m + k], b = H[(size_t)(j + 1) * m + k];
    H[(size_t)j * m + k] = cs[j] * a + sn[j] * b;
    H[(size_t)(j + 1) * m + k] = -sn[j] * a + cs[j] * b;
  }
  const double a = H[(size_t)k * m + k], b = H[(size_t)(k + 1) * m + k];
  const double d = hypot(a, b);
  cs[k] = a / d;
  sn[k] = b / d;
  H[(size_t)k * m + k] = d;
  H[(size_t)(k + 1) * m + k] = 0.0;
  gv[k + 1] = -sn[k] * gv[k];
  gv[k] = cs[k] * gv[k];
  const double res = fabs(gv[k + 1]);
  ctl->res = res;
  ctl->kdone = k + 1;
  if (res <= ctl->tol || k + 1 >= ctl->kmax) ctl->stop = 1;
}

// ARK4(3)6L[2]SA, implicit part (Kennedy and Carpenter 2003): a_ij for j < i; gamma = 1/4
const double kGamma = 0.25;
const double kA6[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 4.0, 0, 0, 0, 0},
    {8611.0 / 62500.0, -1743.0 / 31250.0, 0, 0, 0},
    {5012029.0 / 34652500.0, -654441.0 / 2922500.0, 174375.0 / 388108.0, 0, 0},
    {15267082809.0 / 155376265600.0, -71443401.0 / 120774400.0, 730878875.0 / 902184768.0, 2285395.0 / 8070912.0, 0},
    {82889.0 / 524892.0, 0.0, 15625.0 / 83664.0, 69875.0 / 102672.0, -2260.0 / 8211.0},
};

struct Implicit {
  nsk_ctx* c;
  long long n;          // values of a state vector
  cudaStream_t s;
  unsigned grid;
  double* part;         // dot partials
  double* dotv;         // device result of a dot product
  long long launches = 0;
  long long rhs_evals = 0;
  int status = NSK_OK;
  // inside a cycle's Arnoldi steps: the cycle's stop flag and forward-difference scale on the
  // device (NULL elsewhere)
  const int* stop = nullptr;
  const double* c0p = nullptr;

  void lincomb(double a, const double* x, double b, const double* y, double cc, const double* z, double* out) {
    k_lincomb<<<grid, 256, 0, s>>>(n, a, x, b, y, cc, z, out);
    ++launches;
  }
  int nblk;             // blocks of the dot-product partial sums: up to kDotBlocks, one per 256 values
  double dot(const double* x, const double* y) {
    k_dot_part<<<nblk, kDotThreads, 0, s>>>(n, x, y, part, nullptr);
    k_dot_final<<<1, kDotThreads, 0, s>>>(nblk, part, dotv, nullptr);
    launches += 2;
    double h = 0.0;
    if (cudaMemcpyAsync(&h, dotv, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      status = NSK_ERR_CUDA;
    return h;
  }
  double norm(const double* x) { return sqrt(dot(x, x)); }
  // x . x into *dotv on the device (no synchronisation)
  void dot_dev(const double* x) {
    k_dot_part<<<nblk, kDotThreads, 0, s>>>(n, x, x, part, stop);
    k_dot_final<<<1, kDotThreads, 0, s>>>(nblk, part, dotv, stop);
    launches += 2;
  }
  // one Gram-Schmidt pass on w against V_0..V_{nv-1} (dV: device copy of the basis pointers):
  // the projections (and with norm, w . w, the Pythagorean norm and the normalisation) in two
  // kernels, the coefficients left in hout on the device
  void gs_pass(int nv, bool norm, double* const* dV, double* w, double* hout) {
    k_mdot_part<<<dim3(nblk, norm ? nv + 1 : nv), kDotThreads, 0, s>>>(n, dV, w, part, stop);
    if (norm)
      k_gs_update<true><<<grid, 256, 0, s>>>(n, nv, dV, part, nblk, w, hout, stop);
    else
      k_gs_update<false><<<grid, 256, 0, s>>>(n, nv, dV, part, nblk, w, hout, stop);
    launches += 2;
  }
  // the forward-difference combinations (k_fd_combine), zz = ||z||^2 on the device or NULL
  void fd_combine(int which, const double* zz, double c0, double dtg, const double* X, const double* z,
                  const double* RW, const double* RX, double* out) {
    k_fd_combine<<<grid, 256, 0, s>>>(n, which, zz, c0, c0p, dtg, X, z, RW, RX, out, stop);
    ++launches;
  }
  // out = R(X): one residual-mode stage of the context's pipeline on X
  void rhs(double* X, double* out) {
    void* saved = c->b.U;
    c->b.U = X;
    NskLaunch l = {NSK_MODE_RHS, out, 0.0, 0.0, nullptr, 0.0, nullptr, c->tpb, c->fused_face};
    const int r = nsk_ctx_launch_stage(c, l);
    c->b.U = saved;
    if (r) status = r;
    ++rhs_evals;
  }
};

}  // namespace

// colours per direction of the block Jacobian's forward differences: with BR1 an element's
// residual depends on the states up to two elements away, so same-coloured elements at least
// three apart (across the periodic wrap too) do not see each other's perturbation: the smallest
// divisor K >= 3 of ne, else ne
static int fd_colours(int ne) {
  for (int K = 3; K <= ne; ++K)
    if (ne % K == 0) return K;
  return ne;
}

int nsk_step_esdirk(nsk_ctx* c, double dt, int nsteps, double newton_tol, double krylov_tol, int krylov_dim,
                    int max_krylov, int block_precond, long long stats[4]) {
  const NskRange nvtx_range("nsk_step_esdirk");
  if (!c || !(dt > 0.0) || !isfinite(dt) || nsteps < 0 || !(newton_tol > 0.0) || !(krylov_tol > 0.0) ||
      krylov_dim < 1 || krylov_dim > 200 || max_krylov < 1 || (block_precond != 0 && block_precond != 1))
    return NSK_ERR_ARG;
  if (c->precision != NSK_FP64 || c->closure_mode != NSK_C_EXPLICIT || c->fv_path()) return NSK_ERR_ARG;
  const int nloc = c->nvar * c->npe;
  if (block_precond && (nloc > kMaxBlock || (double)c->E * nloc * nloc > 268435456.0)) return NSK_ERR_ARG;
  if (!c->state_set) return NSK_ERR_STATE;
  // the block inversion's shared memory: n x 2n doubles (above the 48 KB default from n = 56 on)
  const size_t inv_smem = sizeof(double) * 2 * (size_t)nloc * nloc;
  if (block_precond &&
      cudaFuncSetAttribute(k_block_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem) != cudaSuccess) {
    cudaGetLastError();
    return NSK_ERR_CUDA;
  }
  const int m = krylov_dim;
  const long long n = (long long)c->nvar * c->nn;
  // state-sized buffers: R_0..R_4, X, S, RX, D (Newton update), W (X + eps v), RW, V_0..V_m,
  // and with the preconditioner Z (M^-1 v) and T (the combination of the basis)
  const int nbuf = 5 + 6 + (m + 1) + (block_precond ? 2 : 0);
  double* pool = nullptr;
  if (cudaMalloc(&pool, sizeof(double) * (size_t)n * nbuf) != cudaSuccess) {
    cudaGetLastError();
    return NSK_ERR_NOMEM;
  }
  // dot partials ((m + 1) vectors x blocks), a dot result, the two Gram-Schmidt passes'
  // coefficients (m + 1, and m + 2 with the norm), m + 1 basis pointers, then the cycle's
  // Hessenberg matrix ((m + 1) x m), rotations (2 m) and right-hand side (m + 1)
  double* part = nullptr;
  const size_t part_n = (size_t)(m + 1) * kDotBlocks + 1 + (m + 1) + (m + 2) + (m + 1) + (size_t)(m + 1) * m +
                        2 * (size_t)m + (m + 1);
  if (cudaMalloc(&part, sizeof(double) * part_n) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(pool);
    return NSK_ERR_NOMEM;
  }
  auto buf = [&](int k) { return pool + (size_t)k * n; };
  double* Rj[5] = {buf(0), buf(1), buf(2), buf(3), buf(4)};
  double *X = buf(5), *S = buf(6), *RX = buf(7), *D = buf(8), *W = buf(9), *RW = buf(10);
  std::vector<double*> V(m + 1);
  for (int k = 0; k <= m; ++k) V[k] = buf(11 + k);
  double* Z = block_precond ? buf(12 + m) : nullptr;
  double* T = block_precond ? buf(13 + m) : nullptr;
  // the preconditioner's blocks and the element colours
  double* Jb = nullptr;
  int* colour = nullptr;
  int ncol = 1;
  if (block_precond) {
    std::vector<int> hc((size_t)c->E);
    int K[3] = {1, 1, 1};
    for (int k = 0; k < c->dim; ++k) K[k] = fd_colours(c->ne[k]);
    ncol = K[0] * K[1] * K[2];
    for (long long e = 0; e < c->E; ++e) {
      const long long c0 = e % c->ne[0], c1 = (e / c->ne[0]) % c->ne[1], c2 = e / ((long long)c->ne[0] * c->ne[1]);
      hc[(size_t)e] = (int)(c0 % K[0] + K[0] * (c1 % K[1] + K[1] * (c2 % K[2])));
    }
    if (cudaMalloc(&Jb, sizeof(double) * (size_t)c->E * nloc * nloc) != cudaSuccess ||
        cudaMalloc(&colour, sizeof(int) * (size_t)c->E) != cudaSuccess ||
        cudaMemcpy(colour, hc.data(), sizeof(int) * hc.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(Jb);
      cudaFree(colour);
      cudaFree(part);
      cudaFree(pool);
      return NSK_ERR_NOMEM;
    }
  }

  Implicit im;
  im.c = c;
  im.n = n;
  im.s = c->stream;
  const long long g = (n + 255) / 256;
  im.grid = (unsigned)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
  im.nblk = (int)(g < kDotBlocks ? (g > 0 ? g : 1) : kDotBlocks);
  im.part = part;
  im.dotv = part + (size_t)(m + 1) * kDotBlocks;
  double* hd1 = im.dotv + 1;       // first pass: h1[0..k]
  double* hd2 = hd1 + (m + 1);     // second pass: h2[0..k], then the new vector's norm at k + 1
  double** dV = (double**)(hd2 + (m + 2));
  double* Hd = (double*)(dV + (m + 1));
  double* csd = Hd + (size_t)(m + 1) * m;
  double* snd = csd + m;
  double* gvd = snd + m;
  if (cudaMemcpyAsync(dV, V.data(), sizeof(double*) * (m + 1), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    im.status = NSK_ERR_CUDA;
  // the cycle's control block on the device and its host copy (pinned); one CUDA graph per Arnoldi
  // step k, captured on first use and replayed for every cycle of the call
  CycleCtl* ctl = nullptr;
  CycleCtl* hctl = nullptr;
  std::vector<cudaGraphExec_t> gstep((size_t)m, nullptr);
  std::vector<long long> gstep_launches((size_t)m, 0);
  bool graphs = true;  // false after a failed capture: the steps are then launched directly
  if (cudaMalloc(&ctl, sizeof(CycleCtl)) != cudaSuccess || cudaMallocHost(&hctl, sizeof(CycleCtl)) != cudaSuccess) {
    cudaGetLastError();
    im.status = NSK_ERR_NOMEM;
  }
  // the call runs on a stream of its own (stream capture needs one other than the legacy default
  // stream), ordered after the context's stream by an event and before it again at the end; the
  // context's kernels (the residual evaluations) launch there for the call's duration
  cudaStream_t ctx_stream = c->stream, own = nullptr;
  cudaEvent_t order = nullptr;
  if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&order, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(order, ctx_stream) != cudaSuccess || cudaStreamWaitEvent(own, order, 0) != cudaSuccess) {
    cudaGetLastError();
    im.status = NSK_ERR_CUDA;
  } else {
    c->stream = own;
    im.s = own;
  }
  long long st_newton = 0, st_krylov = 0, st_fail = 0;
  double* U = (double*)c->b.U;  // U_n, then U_{n+1}
  const double gdt = kGamma * dt;
  std::vector<double> H((size_t)(m + 1) * m), gv(m + 1), y(m);  // host copies for the back substitution

  const unsigned eg = (unsigned)std::min<long long>((c->E * nloc + 255) / 256, 152 * 16);
  // z = M^-1 x (identity without the preconditioner)
  auto precond = [&](const double* x, double* z) {
    k_block_apply<<<eg, 256, 0, im.s>>>(c->E, c->nvar, c->npe, c->nn, Jb, x, z, im.stop);
    ++im.launches;
  };
  for (int step = 0; step < nsteps && im.status == NSK_OK; ++step) {
    im.rhs(U, Rj[0]);
    im.lincomb(1.0, U, 0.0, nullptr, 0.0, nullptr, X);
    if (block_precond) {  // blocks of I - dt gamma J(U_n), once per step
      for (int col = 0; col < ncol; ++col)
        for (int k = 0; k < nloc; ++k) {
          im.lincomb(1.0, U, 0.0, nullptr, 0.0, nullptr, W);
          k_fd_perturb<<<eg, 256, 0, im.s>>>(c->E, c->npe, c->nn, colour, col, k / c->npe, k % c->npe, W);
          im.rhs(W, RW);
          k_fd_column<<<eg, 256, 0, im.s>>>(c->E, c->nvar, c->npe, c->nn, colour, col, k, U, RW, Rj[0], Jb);
          im.launches += 2;
        }
      k_block_invert<<<(unsigned)c->E, 128, inv_smem, im.s>>>(nloc, gdt, Jb, c->b.err);
      ++im.launches;
    }
    for (int i = 1; i < 6 && im.status == NSK_OK; ++i) {
      // S_i = U_n + dt sum_{j<i} a_ij R_j
      im.lincomb(1.0, U, 0.0, nullptr, 0.0, nullptr, S);
      for (int j = 0; j < i; ++j)
        if (kA6[i][j] != 0.0) im.lincomb(1.0, S, dt * kA6[i][j], Rj[j], 0.0, nullptr, S);
      const double snorm = im.norm(S);
      for (int it = 0;; ++it) {
        im.rhs(X, RX);
        im.lincomb(1.0, X, -gdt, RX, -1.0, S, V[0]);  // G = X - dt gamma R(X) - S
        const double gnorm = im.norm(V[0]);
        if (im.status != NSK_OK || gnorm <= newton_tol * snorm) break;
        if (it == 20) {
          ++st_fail;
          break;
        }
        // GMRES for (I - dt gamma J) D = -G, from D = 0
        const double xn = im.norm(X);
        const double bn = gnorm;  // ||-G||
        if (cudaMemsetAsync(D, 0, sizeof(double) * (size_t)n, im.s) != cudaSuccess) im.status = NSK_ERR_CUDA;
        double beta = gnorm;
        im.lincomb(-1.0 / beta, V[0], 0.0, nullptr, 0.0, nullptr, V[0]);  // V_0 = -G / ||G||
        int its = 0;
        bool done = false;
        while (!done && im.status == NSK_OK) {
          // Arnoldi steps k = 0, 1, ...: V_{k+1} = (I - dt gamma J) z, z = M^-1 V_k (z = V_k, ||z|| = 1,
          // without the preconditioner), J z ~ (R(X + eps z) - R(X)) / eps, classical Gram-Schmidt
          // twice (CGS2: each pass's k + 1 projections in one kernel and the update in another, the
          // second pass's w . w giving the new vector's norm by Pythagoras), then the Hessenberg
          // column, the Givens rotations and the residual estimate on the device (k_arnoldi_update,
          // which sets the cycle's stop flag). Each step is a CUDA graph replayed from the host in
          // chunks of kChunk, the control block read after each chunk: the steps after the stop
          // return at once (only their residual evaluation still runs, on an unused vector).
          auto arnoldi = [&](int k) {
            const double* zk = V[k];
            if (block_precond) {
              precond(V[k], Z);
              zk = Z;
              im.dot_dev(Z);
            }
            const double* zz = block_precond ? im.dotv : nullptr;
            im.fd_combine(0, zz, 0.0, gdt, X, zk, nullptr, nullptr, W);  // W = X + eps z
            im.rhs(W, RW);
            im.fd_combine(1, zz, 0.0, gdt, nullptr, zk, RW, RX, V[k + 1]);
            im.gs_pass(k + 1, false, dV, V[k + 1], hd1);
            im.gs_pass(k + 1, true, dV, V[k + 1], hd2);
            k_arnoldi_update<<<1, 32, 0, im.s>>>(k, m, hd1, hd2, Hd, csd, snd, gvd, ctl);
            ++im.launches;
          };
          auto replay = [&](int k) {
            if (!graphs) {  // direct launches, predicated by the same control block
              im.stop = &ctl->stop;
              im.c0p = &ctl->c0;
              arnoldi(k);
              ++im.rhs_evals;
              im.stop = nullptr;
              im.c0p = nullptr;
              return;
            }
            if (!gstep[(size_t)k]) {  // capture step k once
              const long long l0 = im.launches, r0 = im.rhs_evals;
              im.stop = &ctl->stop;
              im.c0p = &ctl->c0;
              cudaGraph_t g = nullptr;
              if (cudaStreamBeginCapture(im.s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                im.status = NSK_ERR_CUDA;
              } else {
                arnoldi(k);
                if (cudaStreamEndCapture(im.s, &g) != cudaSuccess || !g ||
                    cudaGraphInstantiate(&gstep[(size_t)k], g, 0) != cudaSuccess)
                  im.status = NSK_ERR_CUDA;
                if (g) cudaGraphDestroy(g);
              }
              im.stop = nullptr;
              im.c0p = nullptr;
              gstep_launches[(size_t)k] = im.launches - l0;
              im.launches = l0;
              im.rhs_evals = r0;
              if (im.status != NSK_OK) {  // no graph: this and the later steps are launched directly
                cudaGetLastError();
                if (gstep[(size_t)k]) {
                  cudaGraphExecDestroy(gstep[(size_t)k]);
                  gstep[(size_t)k] = nullptr;
                }
                im.status = NSK_OK;
                graphs = false;
                im.stop = &ctl->stop;
                im.c0p = &ctl->c0;
                arnoldi(k);
                ++im.rhs_evals;
                im.stop = nullptr;
                im.c0p = nullptr;
                return;
              }
            }
            if (cudaGraphLaunch(gstep[(size_t)k], im.s) != cudaSuccess) {
              im.status = NSK_ERR_CUDA;
              return;
            }
            im.launches += gstep_launches[(size_t)k];
            ++im.rhs_evals;
          };
          const int kmax = std::min(m, max_krylov - its);
          k_cycle_init<<<1, 32, 0, im.s>>>(ctl, sqrt(ldexp(1.0, -52)) * (1.0 + xn), beta, krylov_tol * bn, kmax);
          ++im.launches;
          for (int k0 = 0; k0 < kmax && im.status == NSK_OK; k0 += kChunk) {
            for (int k = k0; k < std::min(k0 + kChunk, kmax) && im.status == NSK_OK; ++k) replay(k);
            if (cudaMemcpyAsync(hctl, ctl, sizeof(CycleCtl), cudaMemcpyDeviceToHost, im.s) != cudaSuccess ||
                cudaStreamSynchronize(im.s) != cudaSuccess)
              im.status = NSK_ERR_CUDA;
            if (hctl->stop) break;
          }
          if (im.status != NSK_OK) break;
          const int kk = hctl->kdone;   // Arnoldi steps of the cycle's least-squares problem
          const double resk = hctl->res;  // its residual estimate
          its += kk;
          if (kk == 0) break;
          // the cycle's triangular system and rotated right-hand side
          if (cudaMemcpyAsync(H.data(), Hd, sizeof(double) * (size_t)kk * m, cudaMemcpyDeviceToHost, im.s) !=
                  cudaSuccess ||
              cudaMemcpyAsync(gv.data(), gvd, sizeof(double) * (size_t)kk, cudaMemcpyDeviceToHost, im.s) !=
                  cudaSuccess ||
              cudaStreamSynchronize(im.s) != cudaSuccess) {
            im.status = NSK_ERR_CUDA;
            break;
          }
          for (int r = kk - 1; r >= 0; --r) {  // back substitution on the triangular Hessenberg
            double t = gv[r];
            for (int j = r + 1; j < kk; ++j) t -= H[(size_t)r * m + j] * y[j];
            y[r] = t / H[(size_t)r * m + r];
          }
          if (block_precond) {  // D += M^-1 sum_j y_j V_j
            if (cudaMemsetAsync(T, 0, sizeof(double) * (size_t)n, im.s) != cudaSuccess) im.status = NSK_ERR_CUDA;
            for (int j = 0; j < kk; ++j) im.lincomb(1.0, T, y[j], V[j], 0.0, nullptr, T);
            precond(T, Z);
            im.lincomb(1.0, D, 1.0, Z, 0.0, nullptr, D);
          } else {
            for (int j = 0; j < kk; ++j) im.lincomb(1.0, D, y[j], V[j], 0.0, nullptr, D);
          }
          if (resk <= krylov_tol * bn || its >= max_krylov) {
            done = true;
          } else {  // restart: r = -G - (I - dt gamma J) D
            const double dn = im.norm(D);
            if (!(dn > 0.0)) break;  // no progress in this cycle
            const double eps = sqrt(ldexp(1.0, -52)) * (1.0 + xn) / dn;
            im.lincomb(1.0, X, eps, D, 0.0, nullptr, W);
            im.rhs(W, RW);
            // V_0 = -G - D + (dt gamma / eps)(R(X + eps D) - R(X)); -G from X, RX, S
            im.lincomb(-1.0, X, gdt, RX, 1.0, S, V[0]);
            im.lincomb(1.0, V[0], -1.0, D, 0.0, nullptr, V[0]);
            im.lincomb(1.0, V[0], gdt / eps, RW, -gdt / eps, RX, V[0]);
            beta = im.norm(V[0]);
            if (!(beta > 0.0)) break;
            im.lincomb(1.0 / beta, V[0], 0.0, nullptr, 0.0, nullptr, V[0]);
          }
        }
        im.lincomb(1.0, X, 1.0, D, 0.0, nullptr, X);
        ++st_newton;
        st_krylov += its;
      }
      if (i < 5) im.lincomb(1.0 / gdt, X, -1.0 / gdt, S, 0.0, nullptr, Rj[i]);  // R_i = (X_i - S_i) / (dt gamma)
    }
    im.lincomb(1.0, X, 0.0, nullptr, 0.0, nullptr, U);  // stiffly accurate: U_{n+1} = X_6
  }
  if (own) {  // back to the context's stream, after the call's work
    if (c->stream == own &&
        (cudaEventRecord(order, own) != cudaSuccess || cudaStreamWaitEvent(ctx_stream, order, 0) != cudaSuccess) &&
        im.status == NSK_OK)
      im.status = NSK_ERR_CUDA;
    c->stream = ctx_stream;
    im.s = ctx_stream;
    cudaStreamDestroy(own);  // released once its work is done
  }
  if (order) cudaEventDestroy(order);
  int r = im.status;
  const int rs = nsk_ctx_sync_check(c);
  if (r == NSK_OK) r = rs;
  c->launches += im.launches;
  for (cudaGraphExec_t ge : gstep)
    if (ge) cudaGraphExecDestroy(ge);
  if (hctl) cudaFreeHost(hctl);
  cudaFree(ctl);
  cudaFree(Jb);
  cudaFree(colour);
  cudaFree(part);
  cudaFree(pool);
  if (stats) {
    stats[0] = st_newton;
    stats[1] = st_krylov;
    stats[2] = im.rhs_evals;
    stats[3] = st_fail;
  }
  return r;
}
