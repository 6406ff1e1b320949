// nsk_orig.cu -- the original third-order NSK equations (arXiv:1912.12059, Sec. 2.2, Eqs.
// (nsk_1), (nsk_2), (stress_nse), (stress_nsk)), FP64, with the same DGSEM building blocks as
// relaxation model II (nsk_kernels.cuh):
//
//   state U = (rho, m), F_k = (m_k, m_k v + p e_k - tau_{.k} - tau^K_{.k}) with the VdW p,
//   tau = mu (grad v + grad v^T - 2/3 div v I),
//   tau^K = kappa (rho lap rho + |grad rho|^2 / 2) I - kappa grad rho (x) grad rho,
//
// grad v and grad rho from the BR1 lifting of w = (v, rho), lap rho from a second BR1 lifting
// of grad rho (Sec. 3.1), the central flux for the convective part (Sec. 3.1 uses it for this
// system) and the BR1 mean of the viscous and Korteweg parts. One stage is five launches:
//   k_prolong (traces of rho, m)  ->  k_lift (Q = grad w; traces of (grad rho)_k)
//   ->  k_lift2 (lap rho; the viscous + Korteweg normal flux on the element's faces)
//   ->  k_face_nsk (central + BR1 mean)  ->  k_volume_nsk (volume, surface, update).
#include "nsk_kernels.cuh"

namespace nsk {
namespace orig {

// plain VdW pressure with q = 1/(3 - rho): p = 8 T rho q - 3 rho^2
__device__ __forceinline__ double pressure_q(const NskParams& p, double rho, double q) {
  return fma(p.t8 * rho, q, -3.0 * rho * rho);
}

template <int D, int NP, int G>
__host__ __device__ constexpr int lift2_work() {
  using S = Shape<D, NP>;
  return (G * D * S::NPE + G * S::NF * S::NFN) > (G * (S::NQ + 1) * S::NPE) ? (G * D * S::NPE + G * S::NF * S::NFN)
                                                                           : (G * (S::NQ + 1) * S::NPE);
}

// (tau + tau^K)_{.k}, momentum components, from rho, the gradients q (q[k*(d+1)+a] = d v_a/dx_k,
// q[k*(d+1)+d] = d rho/dx_k) and lap rho
template <int D>
__device__ __forceinline__ void visc_kort(const NskParams& p, const int k, const double rho, const double* q,
                                          const double lap, double* f) {
  constexpr int NW = D + 1;
  double div = 0.0, g2 = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    div += q[a * NW + a];
    g2 = fma(q[a * NW + D], q[a * NW + D], g2);
  }
  const double iso = p.kappa * fma(rho, lap, 0.5 * g2);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double tau = q[k * NW + a] + q[a * NW + k];
    if (a == k) tau = fma(-2.0 / 3.0, div, tau);
    double tk = -(p.kappa * q[a * NW + D]) * q[k * NW + D];
    if (a == k) tk += iso;
    f[a] = fma(p.mu, tau, tk);
  }
}

// Second lifting, lap rho = sum_k d/dx_k (grad rho)_k (weak form, central flux of the traces of
// (grad rho)_k on the faces of direction k); then, on each of the element's own faces, the
// viscous + Korteweg normal flux evaluated from the traces of rho, of the gradients and of
// lap rho (the flux is nonlinear in them, so it is formed at the face, as the interior
// fluxes are formed at the nodes): FVtr[a][slot][E][nfn], a < d.
template <int D, int NP, int G>
__device__ __forceinline__ void lift2_group(const NskParams& p, const double* __restrict__ U,
                                            const double* __restrict__ Utr, const double* __restrict__ Q,
                                            const double* __restrict__ Gtr, double* __restrict__ Q2,
                                            double* __restrict__ FVtr, const long long e0, double* sm) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NW = S::NW, NF = S::NF, NQ = S::NQ;
  double* sg = sm;                    // [G][D][NPE] grad rho at the nodes
  double* sgs = sm + G * D * NPE;     // [G][NF][NFN] central (grad rho)_k on the faces of direction k
  double* tb = sm + lift2_work<D, NP, G>();
  const auto& t = p.td;
  const int le = threadIdx.x / NPE, n = threadIdx.x % NPE;
  const int e = (int)e0 + le;
  const bool valid = le < G && e < p.E;
  const size_t nn = (size_t)p.nne;
  const int g = e * NPE + n;

  stage_tables<double, D, NP>(t, tb);
  double q[NQ], rho = 0.0;
  if (valid) {
    rho = U[g];
#pragma unroll
    for (int c = 0; c < NQ; ++c) q[c] = Q[c * nn + g];
#pragma unroll
    for (int k = 0; k < D; ++k) sg[(le * D + k) * NPE + n] = q[k * NW + D];
    const ElemIdx ex = elem_idx<D>(p, e);
    for (int it = n; it < NF * NFN; it += NPE) {
      const int slot = it / NFN, fn = it % NFN, k = slot >> 1, s = slot & 1;
      const int en = nbr_of(p, ex, k, s ? 1 : -1);
      const double go = Gtr[(size_t)slot * p.nfe + (e * NFN + fn)];
      const double gn = Gtr[(size_t)(2 * k + 1 - s) * p.nfe + (en * NFN + fn)];
      sgs[(le * NF + slot) * NFN + fn] = 0.5 * (go + gn);
    }
  }
  __syncthreads();
  double lap = 0.0;
  if (valid) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int i = coord<NP>(n, k), fn = face_node<D, NP>(n, k);
      const int n0 = line_base<D, NP>(fn, k), st = node_stride<NP>(k);
      const double* gl = sg + (le * D + k) * NPE + n0;
      double vol = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j) vol = fma(tb[(k * NP + i) * NP + j], gl[j * st], vol);
      const double gp = sgs[(le * NF + 2 * k + 1) * NFN + fn], gm = sgs[(le * NF + 2 * k) * NFN + fn];
      lap += fma(gp, tb[D * NP * NP + k * NP + i], fma(-gm, tb[D * NP * NP + D * NP + k * NP + i], -vol));
    }
    Q2[g] = lap;
  }
  __syncthreads();  // shared memory is reused below
  double* sq = sm;  // [G][NQ + 1][NPE] the gradients and lap rho at the nodes
  if (valid) {
#pragma unroll
    for (int c = 0; c < NQ; ++c) sq[(le * (NQ + 1) + c) * NPE + n] = q[c];
    sq[(le * (NQ + 1) + NQ) * NPE + n] = lap;
  }
  __syncthreads();
  if (valid) {
    const size_t pl = (size_t)NF * p.nfe;
    for (int it = n; it < NF * NFN; it += NPE) {
      const int slot = it / NFN, fn = it % NFN, k = slot >> 1;
      const double* L = (slot & 1) ? t.lp : t.lm;
      const int n0 = line_base<D, NP>(fn, k), st = node_stride<NP>(k);
      double tr[NQ + 1];
#pragma unroll
      for (int c = 0; c <= NQ; ++c) {
        const double* f = sq + (le * (NQ + 1) + c) * NPE + n0;
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) acc = fma(L[j], f[j * st], acc);
        tr[c] = acc;
      }
      const size_t off = (size_t)slot * p.nfe + (e * NFN + fn);
      double f[D];
      visc_kort<D>(p, k, Utr[off], tr, tr[NQ], f);
#pragma unroll
      for (int a = 0; a < D; ++a) FVtr[off + a * pl] = f[a];
    }
  }
  __syncthreads();
}

// central flux of the face between eL (+k side) and eR (-k side) minus the BR1 mean of the
// viscous + Korteweg normal fluxes: Fstar[v][k][E][nfn], v < d + 1
template <int D, int NP>
__device__ __forceinline__ void face_at(const NskParams& p, const double* __restrict__ Utr,
                                        const double* __restrict__ FVtr, double* __restrict__ Fstar, const int k,
                                        const int eL, const int fn, int& eflag) {
  using S = Shape<D, NP>;
  constexpr int NFN = S::NFN, NF = S::NF, NV = D + 1;
  const int eR = nbr_of(p, elem_idx<D>(p, eL), k, 1);
  const size_t ps = (size_t)NF * p.nfe;
  const double* tL = Utr + (size_t)(2 * k + 1) * p.nfe + (eL * NFN + fn);
  const double* tR = Utr + (size_t)(2 * k) * p.nfe + (eR * NFN + fn);
  const double* vL = FVtr + (size_t)(2 * k + 1) * p.nfe + (eL * NFN + fn);
  const double* vR = FVtr + (size_t)(2 * k) * p.nfe + (eR * NFN + fn);
  double UL[NV], UR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    UL[v] = tL[v * ps];
    UR[v] = tR[v * ps];
  }
  const double il = tL[NV * ps], ir = tR[NV * ps];                 // 1/rho
  const double ql = tL[(NV + 1) * ps], qr = tR[(NV + 1) * ps];     // 1/(3 - rho)
  eflag |= rho_flags(UL[0]) | rho_flags(UR[0]);
  const double pl = pressure_q(p, UL[0], ql), pr = pressure_q(p, UR[0], qr);
  double F[NV];
  // the normal momenta by selects over compile-time indices (the direction k is a runtime value),
  // the normal velocities once, the normal momentum flux m_k v_k + p once
  const double mL = comp1<D>(UL, k), mR = comp1<D>(UR, k);
  const double vl = mL * il, vr = mR * ir;
  const double fnn = fma(mL, vl, pl) + fma(mR, vr, pr);
  F[0] = 0.5 * (mL + mR);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const double sum = (a == k) ? fnn : fma(vl, UL[1 + a], vr * UR[1 + a]);
    F[1 + a] = fma(0.5, sum, -(0.5 * (vL[a * ps] + vR[a * ps])));
  }
  double* o = Fstar + (size_t)k * p.nfe + (eL * NFN + fn);
#pragma unroll
  for (int v = 0; v < NV; ++v) o[(size_t)v * D * p.nfe] = F[v];
}

template <int D, int NP, int G>
__host__ __device__ constexpr int volume_nsk_smem() {
  using S = Shape<D, NP>;
  return G * D * (D + 1) * S::NPE + G * S::NF * (D + 1) * S::NFN + tab_smem<D, NP>();
}

// weak-form volume integral and surface lifting of the original NSK equations (no sources),
// then the residual (RHS) or the LSRK update, as volume_group does for model II
template <int D, int NP, int G>
__device__ __forceinline__ void volume_group(const NskParams& p, double* __restrict__ U,
                                             const double* __restrict__ Q, const double* __restrict__ Q2,
                                             const double* __restrict__ Fstar, double* __restrict__ K,
                                             double* __restrict__ Rout, const int mode, const double A,
                                             const double B, const double dt, const long long e0, double* sm,
                                             int& eflag) {
  using S = Shape<D, NP>;
  constexpr int NPE = S::NPE, NFN = S::NFN, NF = S::NF, NQ = S::NQ, NV = D + 1;
  double* sf = sm;                       // [G][D][NV][NPE]
  double* sfs = sm + G * D * NV * NPE;   // [G][NF][NV][NFN]
  double* tb = sfs + G * NF * NV * NFN;
  const int le = threadIdx.x / NPE, n = threadIdx.x % NPE;
  const int e = (int)e0 + le;
  const bool valid = le < G && e < p.E;
  const size_t nn = (size_t)p.nne;
  const int g = e * NPE + n;

  stage_tables<double, D, NP>(p.td, tb);
  double u[NV], kin[NV];
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = U[v * nn + g];
    if (mode != NSK_MODE_RHS) {
#pragma unroll
      for (int v = 0; v < NV; ++v) kin[v] = K[v * nn + g];
    }
    double q[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c) q[c] = Q[c * nn + g];
    const double lap = Q2[g];
    eflag |= rho_flags(u[0]);
    const double dd = 1.0 / (u[0] * (3.0 - u[0]));
    const double inv = (3.0 - u[0]) * dd;
    const double pr = pressure_q(p, u[0], u[0] * dd);
    // the symmetric convective momentum flux, each pair k < a formed once
    double vel[D], off[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) vel[a] = u[1 + a] * inv;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i + 1; j < D; ++j) off[i][j] = u[1 + i] * vel[j];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double* f = sf + ((le * D + k) * NV) * NPE + n;
      f[0] = u[1 + k];
      double fv[D];
      visc_kort<D>(p, k, u[0], q, lap, fv);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const double fc = (a == k) ? fma(u[1 + k], vel[k], pr) : (k < a ? off[k][a] : off[a][k]);
        f[(1 + a) * NPE] = fc - fv[a];
      }
    }
    const ElemIdx ex = elem_idx<D>(p, e);
    for (int it = n; it < NF * NV * NFN; it += NPE) {
      const int fn = it % NFN, v = (it / NFN) % NV, slot = it / (NV * NFN), k = slot >> 1;
      const int src = (slot & 1) ? e : nbr_of(p, ex, k, -1);
      sfs[((le * NF + slot) * NV + v) * NFN + fn] = Fstar[(size_t)(v * D + k) * p.nfe + (src * NFN + fn)];
    }
  }
  __syncthreads();
  if (valid) {
    double res[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) res[v] = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int i = coord<NP>(n, k), fn = face_node<D, NP>(n, k);
      const int n0 = line_base<D, NP>(fn, k), st = node_stride<NP>(k);
      double dk[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) dk[j] = tb[(k * NP + i) * NP + j];
      const double lpk = tb[D * NP * NP + k * NP + i], lmk = tb[D * NP * NP + D * NP + k * NP + i];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double* f = sf + ((le * D + k) * NV + v) * NPE + n0;
        double acc = res[v];
#pragma unroll
        for (int j = 0; j < NP; ++j) acc = fma(dk[j], f[j * st], acc);
        const double fp = sfs[((le * NF + 2 * k + 1) * NV + v) * NFN + fn];
        const double fm = sfs[((le * NF + 2 * k) * NV + v) * NFN + fn];
        res[v] = fma(fm, lmk, fma(-fp, lpk, acc));
      }
    }
    if (mode == NSK_MODE_RHS) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Rout[v * nn + g] = res[v];
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double kv = fma(A, kin[v], dt * res[v]);
        K[v * nn + g] = kv;
        U[v * nn + g] = fma(B, kv, u[v]);
      }
    }
  }
  __syncthreads();
}

// ---- kernels -----------------------------------------------------------------
template <int D, int NP>
__global__ void __launch_bounds__(256) k_prolong_nsk(const NskParams p, const double* __restrict__ U,
                                                     double* __restrict__ Utr) {
  using S = Shape<D, NP>;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < p.nfe) {
    const int e = idx / S::NFN;
    prolong_trace<double, D, NP, D + 1>(p, U + (size_t)e * S::NPE, (size_t)p.nne, Utr, e, blockIdx.y,
                                        idx % S::NFN);
  }
}

template <int D, int NP, int G>
__global__ void __launch_bounds__(G * Shape<D, NP>::NPE)
    k_lift_nsk(const NskParams p, const double* __restrict__ U, const double* __restrict__ Utr,
               double* __restrict__ Q, double* __restrict__ Gtr, int* __restrict__ err) {
  __shared__ __align__(16) double sm[lift_smem<double, D, NP, G>()];
  int eflag = 0;
  lift_group<double, D, NP, G, 1>(p, U, Utr, Q, Gtr, (long long)blockIdx.x * G, sm, eflag);
  if (eflag) atomicOr(err, eflag);
}

template <int D, int NP, int G>
__global__ void __launch_bounds__(G * Shape<D, NP>::NPE)
    k_lift2_nsk(const NskParams p, const double* __restrict__ U, const double* __restrict__ Utr,
                const double* __restrict__ Q, const double* __restrict__ Gtr, double* __restrict__ Q2,
                double* __restrict__ FVtr) {
  __shared__ double sm[lift2_work<D, NP, G>() + tab_smem<D, NP>()];
  lift2_group<D, NP, G>(p, U, Utr, Q, Gtr, Q2, FVtr, (long long)blockIdx.x * G, sm);
}

template <int D, int NP>
__global__ void __launch_bounds__(256) k_face_nsk(const NskParams p, const double* __restrict__ Utr,
                                                  const double* __restrict__ FVtr, double* __restrict__ Fstar,
                                                  int* __restrict__ err) {
  using S = Shape<D, NP>;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int eflag = 0;
  if (idx < p.nfe) face_at<D, NP>(p, Utr, FVtr, Fstar, blockIdx.y, idx / S::NFN, idx % S::NFN, eflag);
  if (eflag) atomicOr(err, eflag);
}

template <int D, int NP, int G>
__global__ void __launch_bounds__(G * Shape<D, NP>::NPE)
    k_volume_nsk(const NskParams p, double* __restrict__ U, const double* __restrict__ Q,
                 const double* __restrict__ Q2, const double* __restrict__ Fstar, double* __restrict__ K,
                 double* __restrict__ Rout, const int mode, const double A, const double B,
                 const double* __restrict__ dtp, const double dtv, int* __restrict__ err) {
  __shared__ double sm[volume_nsk_smem<D, NP, G>()];
  const double dt = dtp ? *dtp : dtv;
  int eflag = 0;
  volume_group<D, NP, G>(p, U, Q, Q2, Fstar, K, Rout, mode, A, B, dt, (long long)blockIdx.x * G, sm, eflag);
  if (eflag) atomicOr(err, eflag);
}

// dt reductions: max over nodes of sum_k (|v_k| + sqrt(max(p', 0))) / h_k and max rho
template <int D>
__global__ void __launch_bounds__(256) k_dt_nsk(const NskParams p, const long long nn, const double* __restrict__ U,
                                                unsigned long long* __restrict__ lam, int* __restrict__ err) {
  double m = 0.0, rmax = 0.0;
  int eflag = 0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nn; g += (long long)gridDim.x * blockDim.x) {
    const double rho = U[g];
    eflag |= rho_flags(rho);
    const double q = 1.0 / (3.0 - rho);
    const double dp = fma(p.t24 * q, q, -6.0 * rho);
    const double a = sqrt(dp > 0.0 ? dp : 0.0);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) s += (fabs(U[(1 + k) * nn + g] / rho) + a) * (0.5 * p.rh[k]);
    m = s > m ? s : m;
    rmax = rho > rmax ? rho : rmax;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, m, o), z = __shfl_xor_sync(0xffffffffu, rmax, o);
    m = y > m ? y : m;
    rmax = z > rmax ? z : rmax;
  }
  __shared__ double red[2][8];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = m;
    red[1][threadIdx.x >> 5] = rmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      m = red[0][w] > m ? red[0][w] : m;
      rmax = red[1][w] > rmax ? red[1][w] : rmax;
    }
    atomicMax(lam, (unsigned long long)__double_as_longlong(m));
    atomicMax(lam + 1, (unsigned long long)__double_as_longlong(rmax));
  }
  if (eflag) atomicOr(err, eflag);
}

// dt = min(convective bound, viscous / dispersive bound), see nsk_compute_dt
__global__ void k_dt_final_nsk(const NskParams p, const int dim, const int N, const double cfl,
                               const unsigned long long* __restrict__ lam, double* __restrict__ dt) {
  const double lmax = __longlong_as_double((long long)lam[0]);
  const double rmax = __longlong_as_double((long long)lam[1]);
  const double tn = 2.0 * N + 1.0;
  double r = cfl / (tn * lmax);
  const double sk = sqrt(p.kappa * rmax);
  const double lamk = p.mu > sk ? p.mu : sk;
  double ih2 = 0.0;
  for (int k = 0; k < dim; ++k) ih2 += 0.25 * p.rh[k] * p.rh[k];
  if (lamk > 0.0) {
    const double dk = cfl / (tn * tn * lamk * ih2);
    r = dk < r ? dk : r;
  }
  *dt = r;
}

// ---- launchers -----------------------------------------------------------------
template <int D, int NP, int G>
int launch_stage_g(const NskParams& p, const NskBuffers& b, const NskLaunch& l, cudaStream_t s) {
  using S = Shape<D, NP>;
  int nl = 0;
  if (l.ev) cudaEventRecord(l.ev[0], s);
  k_prolong_nsk<D, NP><<<dim3(grid_for(p.nfe, 256), S::NF), 256, 0, s>>>(p, (const double*)b.U, (double*)b.Utr);
  ++nl;
  if (l.ev) cudaEventRecord(l.ev[1], s);
  const unsigned eb = (unsigned)((p.E + G - 1) / G);
  k_lift_nsk<D, NP, G><<<eb, G * S::NPE, 0, s>>>(p, (const double*)b.U, (const double*)b.Utr, (double*)b.Q,
                                                  (double*)b.Gtr, b.err);
  ++nl;
  if (l.mode != NSK_MODE_LIFT) {
    k_lift2_nsk<D, NP, G><<<eb, G * S::NPE, 0, s>>>(p, (const double*)b.U, (const double*)b.Utr,
                                                     (const double*)b.Q, (const double*)b.Gtr, (double*)b.Q2,
                                                     (double*)b.FVtr);
    ++nl;
  }
  if (l.ev) cudaEventRecord(l.ev[2], s);
  if (l.mode != NSK_MODE_LIFT) {
    k_face_nsk<D, NP><<<dim3(grid_for(p.nfe, 256), D), 256, 0, s>>>(p, (const double*)b.Utr, (const double*)b.FVtr,
                                                                     (double*)b.Fstar, b.err);
    ++nl;
    if (l.ev) cudaEventRecord(l.ev[3], s);
    k_volume_nsk<D, NP, G><<<eb, G * S::NPE, 0, s>>>(p, (double*)b.U, (const double*)b.Q, (const double*)b.Q2,
                                                      (const double*)b.Fstar, (double*)b.K, (double*)l.Rout, l.mode,
                                                      l.A, l.B, l.dt_dev, l.dt_val, b.err);
    ++nl;
    if (l.ev) cudaEventRecord(l.ev[4], s);
  }
  if (cudaGetLastError() != cudaSuccess) return NSK_ERR_CUDA;
  return nl;
}

template <int D, int NP>
int launch_stage_t(const NskParams& p, const NskBuffers& b, const NskLaunch& l, cudaStream_t s) {
  constexpr int G128 = group_for<D, NP>(128), G256 = group_for<D, NP>(256);
  return l.tpb == 128 ? launch_stage_g<D, NP, G128>(p, b, l, s) : launch_stage_g<D, NP, G256>(p, b, l, s);
}

template <int D>
int launch_stage_np(const NskParams& p, int np, const NskBuffers& b, const NskLaunch& l, cudaStream_t s) {
  switch (np) {
    case 2: return launch_stage_t<D, 2>(p, b, l, s);
    case 3: return launch_stage_t<D, 3>(p, b, l, s);
    case 4: return launch_stage_t<D, 4>(p, b, l, s);
    case 5: return launch_stage_t<D, 5>(p, b, l, s);
    case 6: return launch_stage_t<D, 6>(p, b, l, s);
    default: return NSK_ERR_ARG;
  }
}

}  // namespace orig
}  // namespace nsk

int nsk_launch_stage_nsk(int dim, const NskParams& p, int np, const NskBuffers& b, const NskLaunch& l,
                         cudaStream_t s) {
  if (!b.Gtr || !b.Q2) return NSK_ERR_STATE;
  switch (dim) {
    case 1: return nsk::orig::launch_stage_np<1>(p, np, b, l, s);
    case 2: return nsk::orig::launch_stage_np<2>(p, np, b, l, s);
    case 3: return nsk::orig::launch_stage_np<3>(p, np, b, l, s);
    default: return NSK_ERR_ARG;
  }
}

int nsk_launch_dt_nsk(const NskParams& p, int dim, const NskBuffers& b, double cfl, int N, cudaStream_t s) {
  const long long nn = p.nne;
  long long gb = (nn + 255) / 256;
  const unsigned grid = (unsigned)(gb < 152 * 8 ? (gb > 0 ? gb : 1) : 152 * 8);
  if (cudaMemsetAsync(b.lam, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) return NSK_ERR_CUDA;
  switch (dim) {
    case 1: nsk::orig::k_dt_nsk<1><<<grid, 256, 0, s>>>(p, nn, (const double*)b.U, b.lam, b.err); break;
    case 2: nsk::orig::k_dt_nsk<2><<<grid, 256, 0, s>>>(p, nn, (const double*)b.U, b.lam, b.err); break;
    case 3: nsk::orig::k_dt_nsk<3><<<grid, 256, 0, s>>>(p, nn, (const double*)b.U, b.lam, b.err); break;
    default: return NSK_ERR_ARG;
  }
  nsk::orig::k_dt_final_nsk<<<1, 1, 0, s>>>(p, dim, N, cfl, b.lam, b.dt);
  return cudaGetLastError() == cudaSuccess ? 2 : NSK_ERR_CUDA;
}
