// nsk_fv.cu -- finite-volume sub-cell shock capturing (Sec. 3.2, "Finite Volume Sub-Cell
// Approach") and Dirichlet boundaries (the 1D sharp-interface Riemann problem, Sec. 4), for
// relaxation model II in one space dimension, FP64.
//
// Element e is a DG element (flags[e] = 0: nodal values at the N+1 nodes) or an FV element
// (flags[e] = 1: the means of N+1 equidistant sub-cells, stored in the same slots). Per stage:
//   k_fv_faces   face states of every element (DG traces, or the MinMod-limited linear
//                reconstruction of (rho, v, c) on the sub-cells) and, for FV elements, the
//                difference quotients of (v, c) across the element faces;
//   k_fv_lift    BR1 lifting of w = (v, c) in the DG elements with the central w* against the
//                outer face state (neighbour or boundary), and the traces of the lifted gradient;
//   k_fv_flux    one thread per element face: LF or HLLC convective flux minus the mean of the
//                two sides' viscous fluxes (a Dirichlet boundary is a ghost side with the given
//                state and the interior side's gradient);
//   k_fv_update  DG weak form or FV sub-cell balance, sources, then the LSRK update (or R).
// k_fv_switch (before every step) evaluates the Persson-Peraire indicator on rho and converts
// elements between the two representations (the exact sub-cell mean matrix or its inverse).
// Readings of what the section leaves open: the indicator acts on rho; switches happen once
// per step, before its first stage; FV -> DG inverts the mean matrix; the reconstruction acts
// on (rho, v, c) with the neighbour value across an element face one sub-cell width away (FV
// neighbour) or half a width (DG trace, boundary state); diffusive fluxes use difference
// quotients, the source's c_x is the mean of a sub-cell's two face quotients.
#include <string.h>

#include <utility>

#include "nsk_kernels.cuh"

namespace nsk {
namespace fv {

struct FvParams {
  double M[NSK_MAXNP * NSK_MAXNP];     // sub-cell means of the nodal basis, [j][i]
  double Minv[NSK_MAXNP * NSK_MAXNP];  // its inverse, [i][j]
  double Vinv[NSK_MAXNP * NSK_MAXNP];  // nodal values -> orthonormal Legendre modes, [m][i]
  double Ub[2][3];                     // Dirichlet states outside x = lo (0) and x = hi (1)
  double upper, lower;                 // indicator thresholds (log10)
  double dx;                           // sub-cell width h / (N+1)
  int dirichlet;
};

// one-dimensional state helpers ----------------------------------------------------------
__device__ __forceinline__ void prim(const double* U, double* P) {
  P[0] = U[0];
  P[1] = U[1] / U[0];
  P[2] = U[2];
}
__device__ __forceinline__ void cons(const double* P, double* U) {
  U[0] = P[0];
  U[1] = P[0] * P[1];
  U[2] = P[2];
}
__device__ __forceinline__ double minmod(double a, double b) {
  return a * b <= 0.0 ? 0.0 : (a > 0.0 ? fmin(a, b) : fmax(a, b));
}
// viscous flux of model II in 1D from (v_x, c_x): (0, (4/3) mu v_x, (kappa/beta) c_x)
__device__ __forceinline__ void visc(const NskParams& p, const double* g, double* f) {
  f[0] = 0.0;
  f[1] = (4.0 / 3.0) * p.mu * g[0];
  f[2] = p.td.kb * g[1];
}
__device__ __forceinline__ bool bad(double rho) { return !rho_ok(rho); }

// Convective numerical flux between the states L and R (normal +x): local Lax-Friedrichs with
// the model II acoustic speed sqrt(p_alpha'), or HLLC of the barotropic (rho, m) system with
// p_alpha (Davis speeds); c has no convective flux (LF adds its jump only with c_diss).
__device__ void numflux(const NskParams& p, const double* L, const double* R, double* F, int& eflag) {
  double pl, dl, pr, dr;
  eos_both64(p, L[0], pl, dl);
  eos_both64(p, R[0], pr, dr);
  if (!sound_ok(dl) || !sound_ok(dr)) eflag |= NSK_EBIT_SOUND;
  if (bad(L[0]) || bad(R[0])) eflag |= NSK_EBIT_RHO;
  const double ul = L[1] / L[0], ur = R[1] / R[0];
  const double al = sqrt(dl), ar = sqrt(dr);
  const double fl[2] = {L[1], L[1] * ul + pl}, fr[2] = {R[1], R[1] * ur + pr};
  if (p.flux == NSK_FLUX_HLLC) {
    const double SL = fmin(ul - al, ur - ar), SR = fmax(ul + al, ur + ar);
    F[2] = 0.0;
    if (SL >= 0.0) {
      F[0] = fl[0];
      F[1] = fl[1];
      return;
    }
    if (SR <= 0.0) {
      F[0] = fr[0];
      F[1] = fr[1];
      return;
    }
    const double wl = L[0] * (SL - ul), wr = R[0] * (SR - ur);
    const double Ss = (pr - pl + wl * ul - wr * ur) / (wl - wr);
    const bool left = Ss >= 0.0;
    const double SK = left ? SL : SR, rk = left ? L[0] : R[0], mk = left ? L[1] : R[1];
    const double coef = (left ? wl : wr) / (SK - Ss);
    F[0] = (left ? fl[0] : fr[0]) + SK * (coef - rk);
    F[1] = (left ? fl[1] : fr[1]) + SK * (coef * Ss - mk);
    return;
  }
  const double lam = fmax(fabs(ul) + al, fabs(ur) + ar);
  F[0] = 0.5 * (fl[0] + fr[0]) - 0.5 * lam * (R[0] - L[0]);
  F[1] = 0.5 * (fl[1] + fr[1]) - 0.5 * lam * (R[1] - L[1]);
  F[2] = p.c_diss ? -0.5 * lam * (R[2] - L[2]) : 0.0;
}

// periodic neighbour or -1 at a Dirichlet boundary
__device__ __forceinline__ long long nbr(const NskParams& p, const FvParams& f, long long e, int side) {
  if (side == 0) return e > 0 ? e - 1 : (f.dirichlet ? -1 : p.E - 1);
  return e < p.E - 1 ? e + 1 : (f.dirichlet ? -1 : 0);
}

// value of element e's nodal polynomial of variable v at xi = -1 (side 0) or +1 (side 1)
template <int NP>
__device__ __forceinline__ double dg_trace(const NskParams& p, const double* U, long long e, int v, int side) {
  const double* L = side ? p.td.lp : p.td.lm;
  const double* u = U + (size_t)v * p.nne + e * NP;
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < NP; ++j) s = fma(L[j], u[j], s);
  return s;
}

// ---- indicator and switching --------------------------------------------------------------
template <int NP>
__device__ __forceinline__ void fv_switch_body(const NskParams& p, const FvParams& f, double* __restrict__ U,
                                               int* __restrict__ flags, double* __restrict__ ind, const long long e) {
  if (e >= p.E) return;
  const int fl = flags[e];
  double u[3][NP];
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int i = 0; i < NP; ++i) u[v][i] = U[(size_t)v * p.nne + e * NP + i];
  double rho[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    if (fl) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j) s = fma(f.Minv[i * NP + j], u[0][j], s);
      rho[i] = s;
    } else {
      rho[i] = u[0][i];
    }
  }
  double tot = 0.0, top = 0.0;
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) s = fma(f.Vinv[m * NP + i], rho[i], s);
    tot = fma(s, s, tot);
    if (m == NP - 1) top = s * s;
  }
  const double x = log10(top / tot);
  ind[e] = x;
  const bool to_fv = !fl && x > f.upper, to_dg = fl && x < f.lower;
  if (!to_fv && !to_dg) return;
  const double* T = to_fv ? f.M : f.Minv;
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j) s = fma(T[i * NP + j], u[v][j], s);
      U[(size_t)v * p.nne + e * NP + i] = s;
    }
  flags[e] = to_fv ? 1 : 0;
}

// ---- stage kernels ------------------------------------------------------------------------
// Uf[e][side][3]: face states; Gf[e][side][2]: (v_x, c_x) of the element's side of each face;
// SL[e][j][3]: MinMod slopes of (rho, v, c) per unit length in the FV elements.
template <int NP>
__device__ __forceinline__ void fv_faces_body(const NskParams& p, const FvParams& f, const double* __restrict__ U,
                                              const int* __restrict__ flags, double* __restrict__ Uf,
                                              double* __restrict__ Gf, double* __restrict__ SL,
                                              int* __restrict__ err, const long long e, const int role) {
  // role 0 handles the DG elements, role 1 the FV elements (separate warps: no divergence), -1 both
  if (e >= p.E || (role >= 0 && flags[e] != role)) return;
  int eflag = 0;
  if (!flags[e]) {
#pragma unroll
    for (int sd = 0; sd < 2; ++sd)
#pragma unroll
      for (int v = 0; v < 3; ++v) Uf[(e * 2 + sd) * 3 + v] = dg_trace<NP>(p, U, e, v, sd);
    return;
  }
  double P[NP][3];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const double c[3] = {U[e * NP + j], U[(size_t)p.nne + e * NP + j], U[2 * (size_t)p.nne + e * NP + j]};
    if (bad(c[0])) eflag |= NSK_EBIT_RHO;
    prim(c, P[j]);
  }
  double Pn[2][3], dn[2];  // the value beyond each element face, and its distance from the end cell's centre
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const long long en = nbr(p, f, e, sd);
    if (en < 0) {
      prim(f.Ub[sd], Pn[sd]);
      dn[sd] = 0.5 * f.dx;
    } else if (flags[en]) {
      const int jn = sd ? 0 : NP - 1;
      const double c[3] = {U[en * NP + jn], U[(size_t)p.nne + en * NP + jn], U[2 * (size_t)p.nne + en * NP + jn]};
      prim(c, Pn[sd]);
      dn[sd] = f.dx;
    } else {
      double c[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) c[v] = dg_trace<NP>(p, U, en, v, sd ? 0 : 1);
      prim(c, Pn[sd]);
      dn[sd] = 0.5 * f.dx;
    }
  }
  const double idx = 1.0 / f.dx;
#pragma unroll
  for (int j = 0; j < NP; ++j)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double lq = j > 0 ? (P[j][q] - P[j - 1][q]) * idx : (P[0][q] - Pn[0][q]) / dn[0];
      const double rq = j < NP - 1 ? (P[j + 1][q] - P[j][q]) * idx : (Pn[1][q] - P[NP - 1][q]) / dn[1];
      SL[(e * NP + j) * 3 + q] = minmod(lq, rq);
    }
  double Pl[3], Pr[3], Ul[3], Ur[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    Pl[q] = P[0][q] - 0.5 * f.dx * SL[(e * NP) * 3 + q];
    Pr[q] = P[NP - 1][q] + 0.5 * f.dx * SL[(e * NP + NP - 1) * 3 + q];
  }
  cons(Pl, Ul);
  cons(Pr, Ur);
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    Uf[(e * 2 + 0) * 3 + v] = Ul[v];
    Uf[(e * 2 + 1) * 3 + v] = Ur[v];
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    Gf[(e * 2 + 0) * 2 + q] = (P[0][1 + q] - Pn[0][1 + q]) / dn[0];
    Gf[(e * 2 + 1) * 2 + q] = (Pn[1][1 + q] - P[NP - 1][1 + q]) / dn[1];
  }
  if (eflag) atomicOr(err, eflag);
}

// the state beyond side sd of element e: the neighbour's facing face state or the boundary state
__device__ __forceinline__ const double* outer(const NskParams& p, const FvParams& f, const double* Uf, long long e,
                                               int sd) {
  const long long en = nbr(p, f, e, sd);
  return en < 0 ? f.Ub[sd] : Uf + (en * 2 + (sd ? 0 : 1)) * 3;
}

template <int NP>
__device__ __forceinline__ void fv_lift_body(const NskParams& p, const FvParams& f, const double* __restrict__ U,
                                             const int* __restrict__ flags, const double* __restrict__ Uf,
                                             double* __restrict__ Q, double* __restrict__ Gf, const long long e) {
  if (e >= p.E || flags[e]) return;
  const auto& t = p.td;
  double ws[2][2];  // central w* = (v, c) on the two faces
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const double* Ui = Uf + (e * 2 + sd) * 3;
    const double* Uo = outer(p, f, Uf, e, sd);
    ws[sd][0] = 0.5 * (Ui[1] / Ui[0] + Uo[1] / Uo[0]);
    ws[sd][1] = 0.5 * (Ui[2] + Uo[2]);
  }
  double w[2][NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const double rho = U[e * NP + j];
    w[0][j] = U[(size_t)p.nne + e * NP + j] / rho;
    w[1][j] = U[2 * (size_t)p.nne + e * NP + j];
  }
  double q[2][NP];
#pragma unroll
  for (int i = 0; i < NP; ++i)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      // Q_i = w*_+ lpk_i - w*_- lmk_i - sum_j dk[i][j] w_j   (2/h folded into the tables)
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j) s = fma(t.dk[0][i * NSK_MAXNP + j], w[c][j], s);
      q[c][i] = fma(ws[1][c], t.lpk[0][i], fma(-ws[0][c], t.lmk[0][i], -s));
      Q[(size_t)c * p.nne + e * NP + i] = q[c][i];
    }
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const double* L = sd ? t.lp : t.lm;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j) s = fma(L[j], q[c][j], s);
      Gf[(e * 2 + sd) * 2 + c] = s;
    }
  }
}

// face fc between elements fc - 1 and fc (face 0 and, with Dirichlet boundaries, face E are
// the boundary faces); Fh[fc][3] = convective flux - mean viscous flux
// the flux Fo on face fc (0 <= fc < number of faces)
__device__ __forceinline__ void fv_face_flux(const NskParams& p, const FvParams& f, const double* __restrict__ Uf,
                                             const double* __restrict__ Gf, const long long fc, double* Fo,
                                             int& eflag) {
  const long long eR = fc < p.E ? fc : -1;
  const long long eL = fc > 0 ? fc - 1 : (f.dirichlet ? -1 : p.E - 1);
  const double* L = eL >= 0 ? Uf + (eL * 2 + 1) * 3 : f.Ub[0];
  const double* R = eR >= 0 ? Uf + (eR * 2 + 0) * 3 : f.Ub[1];
  const double* gL = eL >= 0 ? Gf + (eL * 2 + 1) * 2 : Gf + (eR * 2 + 0) * 2;
  const double* gR = eR >= 0 ? Gf + (eR * 2 + 0) * 2 : Gf + (eL * 2 + 1) * 2;
  double F[3], vl[3], vr[3];
  numflux(p, L, R, F, eflag);
  visc(p, gL, vl);
  visc(p, gR, vr);
#pragma unroll
  for (int v = 0; v < 3; ++v) Fo[v] = F[v] - 0.5 * (vl[v] + vr[v]);
}
// the face of element e on side sd (periodic: the right face of element E - 1 is face 0)
__device__ __forceinline__ long long fv_face_of(const NskParams& p, const FvParams& f, long long e, int sd) {
  return sd == 0 ? e : ((e + 1 < p.E || f.dirichlet) ? e + 1 : 0);
}

__device__ __forceinline__ void fv_flux_body(const NskParams& p, const FvParams& f, const double* __restrict__ Uf,
                                             const double* __restrict__ Gf, double* __restrict__ Fh,
                                             int* __restrict__ err, const long long fc) {
  const long long nfaces = f.dirichlet ? p.E + 1 : p.E;
  if (fc >= nfaces) return;
  int eflag = 0;
  double F[3];
  fv_face_flux(p, f, Uf, Gf, fc, F, eflag);
#pragma unroll
  for (int v = 0; v < 3; ++v) Fh[fc * 3 + v] = F[v];
  if (!f.dirichlet && fc == 0) {  // periodic: face 0 is also the right face of element E - 1
#pragma unroll
    for (int v = 0; v < 3; ++v) Fh[p.E * 3 + v] = F[v];
  }
  if (eflag) atomicOr(err, eflag);
}

// residual of element e (DG weak form or FV sub-cell balance) and the update
template <int NP>
__device__ __forceinline__ void fv_update_body(const NskParams& p, const FvParams& f, double* __restrict__ U,
                                               double* __restrict__ K, double* __restrict__ Rout,
                                               const int* __restrict__ flags, const double* __restrict__ Gf,
                                               const double* __restrict__ SL, const double* __restrict__ Q,
                                               const double* __restrict__ Fh, const int mode, const double A,
                                               const double B, const double dt, int* __restrict__ err,
                                               const long long e, const int role) {
  if (e >= p.E || (role >= 0 && flags[e] != role)) return;  // role 0: DG elements, 1: FV elements, -1: both
  const auto& t = p.td;
  int eflag = 0;
  double u[3][NP], r[3][NP];
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int j = 0; j < NP; ++j) u[v][j] = U[(size_t)v * p.nne + e * NP + j];
  const double* Fl = Fh + e * 3;
  const double* Fr = Fh + (e + 1) * 3;
  if (!flags[e]) {
    double F[3][NP], qc[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const double rho = u[0][j], vel = u[1][j] / rho;
      if (bad(rho)) eflag |= NSK_EBIT_RHO;
      const double qv = Q[e * NP + j];
      qc[j] = Q[(size_t)p.nne + e * NP + j];
      F[0][j] = u[1][j];
      F[1][j] = fma(u[1][j], vel, eos_pa64(p, rho)) - (4.0 / 3.0) * t.mu * qv;
      F[2][j] = -t.kb * qc[j];
    }
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) s = fma(t.dk[0][i * NSK_MAXNP + j], F[v][j], s);
        r[v][i] = fma(Fl[v], t.lmk[0][i], fma(-Fr[v], t.lpk[0][i], s));
      }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      r[1][i] = fma(t.alpha * u[0][i], qc[i], r[1][i]);
      r[2][i] = fma(t.ab, u[0][i] - u[2][i], r[2][i]);
    }
  } else {
    double P[NP][3], s[NP][3];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const double c[3] = {u[0][j], u[1][j], u[2][j]};
      prim(c, P[j]);
#pragma unroll
      for (int q = 0; q < 3; ++q) s[j][q] = SL[(e * NP + j) * 3 + q];
    }
    const double idx = 1.0 / f.dx;
    double Fs[NP + 1][3], gc[NP + 1];  // sub-cell face fluxes, c_x on the sub-cell faces
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      Fs[0][v] = Fl[v];
      Fs[NP][v] = Fr[v];
    }
    gc[0] = Gf[(e * 2 + 0) * 2 + 1];
    gc[NP] = Gf[(e * 2 + 1) * 2 + 1];
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) {
      double PL[3], PR[3], UL[3], UR[3], g[2], fvv[3], F[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        PL[q] = P[j][q] + 0.5 * f.dx * s[j][q];
        PR[q] = P[j + 1][q] - 0.5 * f.dx * s[j + 1][q];
      }
      cons(PL, UL);
      cons(PR, UR);
      g[0] = (P[j + 1][1] - P[j][1]) * idx;
      g[1] = (P[j + 1][2] - P[j][2]) * idx;
      gc[j + 1] = g[1];
      numflux(p, UL, UR, F, eflag);
      visc(p, g, fvv);
#pragma unroll
      for (int v = 0; v < 3; ++v) Fs[j + 1][v] = F[v] - fvv[v];
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
#pragma unroll
      for (int v = 0; v < 3; ++v) r[v][j] = -(Fs[j + 1][v] - Fs[j][v]) * idx;
      r[1][j] = fma(t.alpha * u[0][j], 0.5 * (gc[j] + gc[j + 1]), r[1][j]);
      r[2][j] = fma(t.ab, u[0][j] - u[2][j], r[2][j]);
    }
  }
  if (mode == NSK_MODE_RHS) {
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int j = 0; j < NP; ++j) Rout[(size_t)v * p.nne + e * NP + j] = r[v][j];
  } else {
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const size_t g = (size_t)v * p.nne + e * NP + j;
        const double kv = fma(A, K[g], dt * r[v][j]);
        K[g] = kv;
        U[g] = fma(B, kv, u[v][j]);
      }
  }
  if (eflag) atomicOr(err, eflag);
}

// ---- lane groups: W lanes per element (lane j = node or sub-cell j), for the cooperative kernel ----
// The same values as the bodies above, with the same operations in the same order; what one
// thread did for every node or sub-cell of an element in turn, lane j does for its own, and the
// values of other nodes arrive by width-W shuffles. Every lane of a warp runs the same number of
// iterations (the caller's loops are warp-uniform), so the shuffles always see the whole warp;
// lanes of inactive groups (past the mesh, or elements of the other role) compute on zeros and
// store nothing.
template <int NP>
__host__ __device__ constexpr int fv_w() {
  return 8;  // > NP: a lane for each of an element's NP + 1 sub-cell faces
}
__device__ __forceinline__ double grp_get(double x, int lane, int W) { return __shfl_sync(0xffffffffu, x, lane, W); }

template <int NP>
__device__ __forceinline__ void fv_faces_group(const NskParams& p, const FvParams& f, const double* __restrict__ U,
                                               const int* __restrict__ flags, double* __restrict__ Uf,
                                               double* __restrict__ Gf, double* __restrict__ SL,
                                               int* __restrict__ err, const long long e, const int j,
                                               const int role) {
  constexpr int W = fv_w<NP>();
  const bool active = e < p.E && flags[e] == role;
  const bool mine = active && j < NP;
  int eflag = 0;
  if (role == 0) {  // DG elements: the six face traces, one per lane in turn
    if (active)
      for (int k = j; k < 6; k += W) Uf[(e * 2 + k / 3) * 3 + k % 3] = dg_trace<NP>(p, U, e, k % 3, k / 3);
    return;
  }
  double P[3] = {0.0, 0.0, 0.0};
  if (mine) {
    const double c[3] = {U[e * NP + j], U[(size_t)p.nne + e * NP + j], U[2 * (size_t)p.nne + e * NP + j]};
    if (bad(c[0])) eflag |= NSK_EBIT_RHO;
    prim(c, P);
  }
  // the value beyond the element's face on the lane's side (lane 0: side 0, lane NP - 1: side 1)
  double Pn[3] = {0.0, 0.0, 0.0}, dn = 1.0;
  const int sd = j == 0 ? 0 : 1;
  if (active && (j == 0 || j == NP - 1)) {
    const long long en = nbr(p, f, e, sd);
    if (en < 0) {
      prim(f.Ub[sd], Pn);
      dn = 0.5 * f.dx;
    } else if (flags[en]) {
      const int jn = sd ? 0 : NP - 1;
      const double c[3] = {U[en * NP + jn], U[(size_t)p.nne + en * NP + jn], U[2 * (size_t)p.nne + en * NP + jn]};
      prim(c, Pn);
      dn = f.dx;
    } else {
      double c[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) c[v] = dg_trace<NP>(p, U, en, v, sd ? 0 : 1);
      prim(c, Pn);
      dn = 0.5 * f.dx;
    }
  }
  const int base = (threadIdx.x & 31) & ~(W - 1);
  const double idx = 1.0 / f.dx;
  double slope[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double Pm = grp_get(P[q], base + (j > 0 ? j - 1 : 0), W);  // P[j - 1]
    const double Pp = grp_get(P[q], base + (j < NP - 1 ? j + 1 : j), W);  // P[j + 1]
    const double lq = j > 0 ? (P[q] - Pm) * idx : (P[q] - Pn[q]) / dn;
    const double rq = j < NP - 1 ? (Pp - P[q]) * idx : (Pn[q] - P[q]) / dn;
    slope[q] = minmod(lq, rq);
    if (mine) SL[(e * NP + j) * 3 + q] = slope[q];
  }
  if (active && (j == 0 || j == NP - 1)) {  // NP >= 2: lanes 0 and NP - 1 are different
    double Pf[3], Uo[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) Pf[q] = j == 0 ? P[q] - 0.5 * f.dx * slope[q] : P[q] + 0.5 * f.dx * slope[q];
    cons(Pf, Uo);
#pragma unroll
    for (int v = 0; v < 3; ++v) Uf[(e * 2 + sd) * 3 + v] = Uo[v];
#pragma unroll
    for (int q = 0; q < 2; ++q)
      Gf[(e * 2 + sd) * 2 + q] = j == 0 ? (P[1 + q] - Pn[1 + q]) / dn : (Pn[1 + q] - P[1 + q]) / dn;
  }
  if (eflag) atomicOr(err, eflag);
}

template <int NP>
__device__ __forceinline__ void fv_lift_group(const NskParams& p, const FvParams& f, const double* __restrict__ U,
                                              const int* __restrict__ flags, const double* __restrict__ Uf,
                                              double* __restrict__ Q, double* __restrict__ Gf, const long long e,
                                              const int j) {
  constexpr int W = fv_w<NP>();
  const bool active = e < p.E && !flags[e];
  const bool mine = active && j < NP;
  const auto& t = p.td;
  const int base = (threadIdx.x & 31) & ~(W - 1);
  double ws[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, w[2] = {0.0, 0.0};
  if (active) {
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const double* Ui = Uf + (e * 2 + sd) * 3;
      const double* Uo = outer(p, f, Uf, e, sd);
      ws[sd][0] = 0.5 * (Ui[1] / Ui[0] + Uo[1] / Uo[0]);
      ws[sd][1] = 0.5 * (Ui[2] + Uo[2]);
    }
  }
  if (mine) {
    const double rho = U[e * NP + j];
    w[0] = U[(size_t)p.nne + e * NP + j] / rho;
    w[1] = U[2 * (size_t)p.nne + e * NP + j];
  }
  double q[2];
  const int i = j < NP ? j : 0;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    double s = 0.0;
#pragma unroll
    for (int jj = 0; jj < NP; ++jj) s = fma(t.dk[0][i * NSK_MAXNP + jj], grp_get(w[c], base + jj, W), s);
    q[c] = fma(ws[1][c], t.lpk[0][i], fma(-ws[0][c], t.lmk[0][i], -s));
    if (mine) Q[(size_t)c * p.nne + e * NP + j] = q[c];
  }
  // traces of the lifted gradient: lane k < 4 sums (side k / 2, component k % 2) over the nodes
  const int ksd = (j >> 1) & 1, kc = j & 1;
  const double* L = ksd ? t.lp : t.lm;
  double s = 0.0;
#pragma unroll
  for (int jj = 0; jj < NP; ++jj) {
    const double q0 = grp_get(q[0], base + jj, W), q1 = grp_get(q[1], base + jj, W);
    s = fma(L[jj], kc ? q1 : q0, s);
  }
  if (active && j < 4) Gf[(e * 2 + ksd) * 2 + kc] = s;
}

// The update phase with the element-face fluxes evaluated in the element's own lane group (each
// face by both its elements, with the same function and inputs as the face pass: the same bits),
// so the cooperative kernel needs no face phase: lane j in [0, NP] takes face j of the element's
// NP + 1 sub-cell faces (0 and NP are the element's faces; DG elements need only those), lane
// j < NP the residual and update of node or sub-cell j.
template <int NP>
__device__ __forceinline__ void fv_update_group(const NskParams& p, const FvParams& f, double* __restrict__ U,
                                                double* __restrict__ K, const int* __restrict__ flags,
                                                const double* __restrict__ Uf, const double* __restrict__ Gf,
                                                const double* __restrict__ SL, const double* __restrict__ Q,
                                                const double A, const double B, const double dt,
                                                int* __restrict__ err, const long long e, const int j,
                                                const int role) {
  constexpr int W = fv_w<NP>();
  static_assert(NP < W, "a lane for each of the NP + 1 sub-cell faces");
  const bool active = e < p.E && flags[e] == role;
  const bool mine = active && j < NP;
  const auto& t = p.td;
  const int base = (threadIdx.x & 31) & ~(W - 1);
  const int i = j < NP ? j : 0;
  int eflag = 0;
  double u[3] = {1.0, 0.0, 0.0}, r[3];
  if (mine)
#pragma unroll
    for (int v = 0; v < 3; ++v) u[v] = U[(size_t)v * p.nne + e * NP + j];
  // the element's faces: lane 0 the left one, lane NP the right one
  double Fe[3] = {0.0, 0.0, 0.0};
  if (active && (j == 0 || j == NP)) fv_face_flux(p, f, Uf, Gf, fv_face_of(p, f, e, j == 0 ? 0 : 1), Fe, eflag);
  if (role == 0) {  // DG weak form: lane j the nodal fluxes of node j and the residual of node j
    double Fl[3], Fr[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      Fl[v] = grp_get(Fe[v], base, W);
      Fr[v] = grp_get(Fe[v], base + NP, W);
    }
    double F[3], qc;
    {
      const double rho = u[0], vel = u[1] / rho;
      if (mine && bad(rho)) eflag |= NSK_EBIT_RHO;
      const double qv = mine ? Q[e * NP + j] : 0.0;
      qc = mine ? Q[(size_t)p.nne + e * NP + j] : 0.0;
      F[0] = u[1];
      F[1] = fma(u[1], vel, eos_pa64(p, rho)) - (4.0 / 3.0) * t.mu * qv;
      F[2] = -t.kb * qc;
    }
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      double s = 0.0;
#pragma unroll
      for (int jj = 0; jj < NP; ++jj) s = fma(t.dk[0][i * NSK_MAXNP + jj], grp_get(F[v], base + jj, W), s);
      r[v] = fma(Fl[v], t.lmk[0][i], fma(-Fr[v], t.lpk[0][i], s));
    }
    r[1] = fma(t.alpha * u[0], qc, r[1]);
    r[2] = fma(t.ab, u[0] - u[2], r[2]);
  } else {  // FV sub-cell balance: lane j (0 < j < NP) the flux on the face between sub-cells j - 1, j
    double P[3], s[3] = {0.0, 0.0, 0.0};
    prim(u, P);
    if (mine)
#pragma unroll
      for (int q = 0; q < 3; ++q) s[q] = SL[(e * NP + j) * 3 + q];
    const double idx = 1.0 / f.dx;
    double Pm[3], sm[3];  // sub-cell j - 1
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      Pm[q] = grp_get(P[q], base + (j > 0 ? j - 1 : 0), W);
      sm[q] = grp_get(s[q], base + (j > 0 ? j - 1 : 0), W);
    }
    double Fs[3] = {Fe[0], Fe[1], Fe[2]}, gf = 0.0;  // the flux and c_x on sub-cell face j
    if (active && j > 0 && j < NP) {
      double PL[3], PR[3], UL[3], UR[3], g[2], fvv[3], F[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        PL[q] = Pm[q] + 0.5 * f.dx * sm[q];
        PR[q] = P[q] - 0.5 * f.dx * s[q];
      }
      cons(PL, UL);
      cons(PR, UR);
      g[0] = (P[1] - Pm[1]) * idx;
      g[1] = (P[2] - Pm[2]) * idx;
      gf = g[1];
      numflux(p, UL, UR, F, eflag);
      visc(p, g, fvv);
#pragma unroll
      for (int v = 0; v < 3; ++v) Fs[v] = F[v] - fvv[v];
    } else if (active && (j == 0 || j == NP)) {
      gf = Gf[(e * 2 + (j == 0 ? 0 : 1)) * 2 + 1];
    }
    // sub-cell j: faces j (own) and j + 1 (lane j + 1)
    double Fp[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) Fp[v] = grp_get(Fs[v], base + (j + 1 < W ? j + 1 : j), W);
    const double gp = grp_get(gf, base + (j + 1 < W ? j + 1 : j), W);
#pragma unroll
    for (int v = 0; v < 3; ++v) r[v] = -(Fp[v] - Fs[v]) * idx;
    r[1] = fma(t.alpha * u[0], 0.5 * (gf + gp), r[1]);
    r[2] = fma(t.ab, u[0] - u[2], r[2]);
  }
  if (mine)
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const size_t g = (size_t)v * p.nne + e * NP + j;
      const double kv = fma(A, K[g], dt * r[v]);
      K[g] = kv;
      U[g] = fma(B, kv, u[v]);
    }
  if (eflag) atomicOr(err, eflag);
}

// ---- one launch per kernel (any mesh size) ----------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(128) k_fv_switch(const NskParams p, const FvParams f, double* __restrict__ U,
                                                   int* __restrict__ flags, double* __restrict__ ind) {
  fv_switch_body<NP>(p, f, U, flags, ind, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}
template <int NP>
__global__ void __launch_bounds__(128) k_fv_faces(const NskParams p, const FvParams f, const double* __restrict__ U,
                                                  const int* __restrict__ flags, double* __restrict__ Uf,
                                                  double* __restrict__ Gf, double* __restrict__ SL,
                                                  int* __restrict__ err, const int split) {
  // split: blocks [0, half) take the DG elements, [half, 2 half) the FV elements
  const unsigned half = split ? gridDim.x / 2 : gridDim.x;
  const int role = split ? (int)(blockIdx.x >= half) : -1;
  const unsigned b = role > 0 ? blockIdx.x - half : blockIdx.x;
  fv_faces_body<NP>(p, f, U, flags, Uf, Gf, SL, err, (long long)b * blockDim.x + threadIdx.x, role);
}
template <int NP>
__global__ void __launch_bounds__(128) k_fv_lift(const NskParams p, const FvParams f, const double* __restrict__ U,
                                                 const int* __restrict__ flags, const double* __restrict__ Uf,
                                                 double* __restrict__ Q, double* __restrict__ Gf) {
  fv_lift_body<NP>(p, f, U, flags, Uf, Q, Gf, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}
__global__ void __launch_bounds__(128) k_fv_flux(const NskParams p, const FvParams f, const double* __restrict__ Uf,
                                                 const double* __restrict__ Gf, double* __restrict__ Fh,
                                                 int* __restrict__ err) {
  fv_flux_body(p, f, Uf, Gf, Fh, err, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}
template <int NP>
__global__ void __launch_bounds__(128)
    k_fv_update(const NskParams p, const FvParams f, double* __restrict__ U, double* __restrict__ K,
                double* __restrict__ Rout, const int* __restrict__ flags, const double* __restrict__ Gf,
                const double* __restrict__ SL, const double* __restrict__ Q, const double* __restrict__ Fh,
                const int mode, const double A, const double B, const double* __restrict__ dtp, const double dtv,
                int* __restrict__ err, const int split) {
  const double dt = dtp ? *dtp : dtv;
  const unsigned half = split ? gridDim.x / 2 : gridDim.x;
  const int role = split ? (int)(blockIdx.x >= half) : -1;
  const unsigned b = role > 0 ? blockIdx.x - half : blockIdx.x;
  fv_update_body<NP>(p, f, U, K, Rout, flags, Gf, SL, Q, Fh, mode, A, B, dt, err, (long long)b * blockDim.x + threadIdx.x,
                     role);
}

// ---- small meshes: all steps of one call in one cooperative launch ---------------------------
// An FP64 warp instruction occupies the SM's FP64 pipe for the same time whether 4 or 32 lanes
// are active, so a small mesh runs fastest spread thinly, one warp per SM, and its time is the
// length of one element's serial chain. For E <= kCoopMaxE the switch pass and the four phases of
// each stage run in one cooperative launch of one-warp blocks (the face-state and update phases
// give DG and FV elements to separate halves of the grid), separated by the bounded grid barrier;
// nsteps steps then cost one launch instead of 21 per step. Fixed dt only. The element phases run
// in lane groups (one lane per node or sub-cell face), which splits each element's chain: a
// sub-cell element's internal HLLC solves run side by side instead of one after another, and the
// update's groups evaluate the element-face fluxes themselves, so a stage has three phases.
constexpr int kCoopMaxE = 4096;
struct LsrkCoef {
  double A[5], B[5];
};

template <int NP>
__global__ void __launch_bounds__(32) k_fv_coop(const NskParams p, const FvParams f, double* __restrict__ U,
                                                double* __restrict__ K, int* __restrict__ flags,
                                                double* __restrict__ ind, double* __restrict__ Uf,
                                                double* __restrict__ Gf, double* __restrict__ SL,
                                                double* __restrict__ Q, const int nsteps,
                                                const int switching, const double dt, const LsrkCoef rk,
                                                unsigned* __restrict__ bar, int* __restrict__ err,
                                                const unsigned long long timeout_ns) {
  const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  // faces and update: the first half of the blocks takes the DG elements, the second the FV ones
  const unsigned half = gridDim.x / 2;
  const int role = blockIdx.x >= half;
  // the element phases in lane groups (W lanes per element, 32 / W elements per one-warp block
  // and iteration; the loop bounds are uniform over the warp)
  constexpr int W = fv_w<NP>(), EPW = 32 / W;
  const int j = threadIdx.x % W, grp = threadIdx.x / W;
  const long long gfirst = (long long)blockIdx.x * EPW, gstride = (long long)gridDim.x * EPW;
  const long long rgfirst = (long long)(blockIdx.x - role * half) * EPW, rgstride = (long long)half * EPW;
  for (int step = 0; step < nsteps; ++step) {
    if (switching) {
      for (long long e = first; e < p.E; e += stride) fv_switch_body<NP>(p, f, U, flags, ind, e);
      if (!grid_barrier(bar, err, timeout_ns)) return;
    }
    for (int st = 0; st < 5; ++st) {
      for (long long eb = rgfirst; eb < p.E; eb += rgstride)
        fv_faces_group<NP>(p, f, U, flags, Uf, Gf, SL, err, eb + grp, j, role);
      if (!grid_barrier(bar, err, timeout_ns)) return;
      for (long long eb = gfirst; eb < p.E; eb += gstride) fv_lift_group<NP>(p, f, U, flags, Uf, Q, Gf, eb + grp, j);
      if (!grid_barrier(bar, err, timeout_ns)) return;
      // (the element-face fluxes are evaluated by the update's lane groups: no face phase)
      for (long long eb = rgfirst; eb < p.E; eb += rgstride)
        fv_update_group<NP>(p, f, U, K, flags, Uf, Gf, SL, Q, rk.A[st], rk.B[st], dt, err, eb + grp, j, role);
      if (!grid_barrier(bar, err, timeout_ns)) return;
    }
  }
}

unsigned grid_of(long long n) { return (unsigned)((n + 127) / 128); }
constexpr long long kSplitMaxE = 65536;  // largest mesh whose per-kernel launches split DG and FV work

template <int NP>
int launch_stage_t(const NskParams& p, const FvParams& f, const FvBuffers& fb, const NskBuffers& b, int mode,
                   double* Rout, double A, double B, const double* dtp, double dtv, cudaStream_t s) {
  const long long E = p.E;
  const unsigned ge = grid_of(E);
  // small meshes: DG and FV elements in separate halves of a doubled grid (the slowest thread of
  // a kernel otherwise runs both code paths); large meshes fill the GPU without it
  const int split = E <= kSplitMaxE;
  k_fv_faces<NP><<<(split ? 2 : 1) * ge, 128, 0, s>>>(p, f, (const double*)b.U, fb.flags, fb.Uf, fb.Gf, fb.SL, b.err,
                                                     split);
  k_fv_lift<NP><<<ge, 128, 0, s>>>(p, f, (const double*)b.U, fb.flags, fb.Uf, (double*)b.Q, fb.Gf);
  k_fv_flux<<<grid_of(E + 1), 128, 0, s>>>(p, f, fb.Uf, fb.Gf, fb.Fh, b.err);
  k_fv_update<NP><<<(split ? 2 : 1) * ge, 128, 0, s>>>(p, f, (double*)b.U, (double*)b.K, Rout, fb.flags, fb.Gf, fb.SL,
                                     (const double*)b.Q, fb.Fh, mode, A, B, dtp, dtv, b.err, split);
  return cudaGetLastError() == cudaSuccess ? 4 : NSK_ERR_CUDA;
}

template <int NP>
int launch_coop_t(const NskParams& p, const FvParams& f, const FvBuffers& fb, const NskBuffers& b, int nsteps,
                  int switching, double dt, const double* A, const double* B, cudaStream_t s) {
  auto kern = k_fv_coop<NP>;
  // one element group per warp in each role half (and every face covered by the one-thread loops)
  constexpr int EPW = 32 / fv_w<NP>();
  const long long ng = (p.E + EPW - 1) / EPW, nf = (p.E + 1 + 31) / 32;
  const int grid = 2 * (int)(ng > nf ? ng : nf);
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, 0) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NSK_ERR_CUDA;
  if ((long long)per_sm * sms < grid) return 0;  // not co-resident: the caller launches per kernel
  LsrkCoef rk;
  for (int i = 0; i < 5; ++i) {
    rk.A[i] = A[i];
    rk.B[i] = B[i];
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const unsigned long long timeout_ns = 1000000000ull;  // one second per barrier wait
  // a barrier that timed out in an earlier launch may have left its arrival count behind
  if (cudaMemsetAsync(fb.bar, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return NSK_ERR_CUDA;
  if (cudaLaunchKernelEx(&cfg, kern, p, f, (double*)b.U, (double*)b.K, fb.flags, fb.ind, fb.Uf, fb.Gf, fb.SL,
                         (double*)b.Q, nsteps, switching, dt, rk, fb.bar, b.err, timeout_ns) != cudaSuccess)
    return NSK_ERR_CUDA;
  return 1;
}

}  // namespace fv
}  // namespace nsk

int nsk_fv_coop_max_elements() { return nsk::fv::kCoopMaxE; }

// 1: launched; 0: the grid would not be co-resident (nothing launched); < 0: error
int nsk_fv_launch_coop(const NskParams& p, const void* fvp, int np, const FvBuffers& fb, const NskBuffers& b,
                       int nsteps, int switching, double dt, const double* A, const double* B, cudaStream_t s) {
  const auto& f = *(const nsk::fv::FvParams*)fvp;
  if (p.E > nsk::fv::kCoopMaxE) return NSK_ERR_ARG;
  switch (np) {
    case 2: return nsk::fv::launch_coop_t<2>(p, f, fb, b, nsteps, switching, dt, A, B, s);
    case 3: return nsk::fv::launch_coop_t<3>(p, f, fb, b, nsteps, switching, dt, A, B, s);
    case 4: return nsk::fv::launch_coop_t<4>(p, f, fb, b, nsteps, switching, dt, A, B, s);
    case 5: return nsk::fv::launch_coop_t<5>(p, f, fb, b, nsteps, switching, dt, A, B, s);
    case 6: return nsk::fv::launch_coop_t<6>(p, f, fb, b, nsteps, switching, dt, A, B, s);
    default: return NSK_ERR_ARG;
  }
}

int nsk_fv_launch_stage(const NskParams& p, const void* fvp, int np, const FvBuffers& fb, const NskBuffers& b,
                        int mode, double* Rout, double A, double B, const double* dtp, double dtv, cudaStream_t s) {
  const auto& f = *(const nsk::fv::FvParams*)fvp;
  switch (np) {
    case 2: return nsk::fv::launch_stage_t<2>(p, f, fb, b, mode, Rout, A, B, dtp, dtv, s);
    case 3: return nsk::fv::launch_stage_t<3>(p, f, fb, b, mode, Rout, A, B, dtp, dtv, s);
    case 4: return nsk::fv::launch_stage_t<4>(p, f, fb, b, mode, Rout, A, B, dtp, dtv, s);
    case 5: return nsk::fv::launch_stage_t<5>(p, f, fb, b, mode, Rout, A, B, dtp, dtv, s);
    case 6: return nsk::fv::launch_stage_t<6>(p, f, fb, b, mode, Rout, A, B, dtp, dtv, s);
    default: return NSK_ERR_ARG;
  }
}

int nsk_fv_launch_switch(const NskParams& p, const void* fvp, int np, const FvBuffers& fb, double* U,
                         cudaStream_t s) {
  const auto& f = *(const nsk::fv::FvParams*)fvp;
  const unsigned ge = nsk::fv::grid_of(p.E);
  switch (np) {
    case 2: nsk::fv::k_fv_switch<2><<<ge, 128, 0, s>>>(p, f, U, fb.flags, fb.ind); break;
    case 3: nsk::fv::k_fv_switch<3><<<ge, 128, 0, s>>>(p, f, U, fb.flags, fb.ind); break;
    case 4: nsk::fv::k_fv_switch<4><<<ge, 128, 0, s>>>(p, f, U, fb.flags, fb.ind); break;
    case 5: nsk::fv::k_fv_switch<5><<<ge, 128, 0, s>>>(p, f, U, fb.flags, fb.ind); break;
    case 6: nsk::fv::k_fv_switch<6><<<ge, 128, 0, s>>>(p, f, U, fb.flags, fb.ind); break;
    default: return NSK_ERR_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? 1 : NSK_ERR_CUDA;
}

size_t nsk_fv_params_size() { return sizeof(nsk::fv::FvParams); }

// host: the tables of FvParams for N+1 nodes xi (Gauss sub-cell rule from gauss_x, gauss_w)
int nsk_fv_fill_params(void* fvp, int np, const double* xi, const double* gauss_x, const double* gauss_w, double h,
                       int dirichlet, const double* Ub_lo, const double* Ub_hi, double upper, double lower) {
  auto& f = *(nsk::fv::FvParams*)fvp;
  memset(&f, 0, sizeof(f));
  auto lag = [&](int i, double x) {
    double l = 1.0;
    for (int k = 0; k < np; ++k)
      if (k != i) l *= (x - xi[k]) / (xi[i] - xi[k]);
    return l;
  };
  for (int j = 0; j < np; ++j) {
    const double a = -1.0 + 2.0 * j / np;
    for (int i = 0; i < np; ++i) {
      double s = 0.0;
      for (int q = 0; q < np; ++q) s += gauss_w[q] * lag(i, a + (gauss_x[q] + 1.0) / np);
      f.M[j * np + i] = 0.5 * s;
    }
  }
  // inverses by Gauss-Jordan elimination with partial pivoting on [A | I]
  auto invert = [&](const double* A, double* Ainv) -> bool {
    double W[NSK_MAXNP][2 * NSK_MAXNP];
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < 2 * np; ++j) W[i][j] = j < np ? A[i * np + j] : (j - np == i ? 1.0 : 0.0);
    for (int c = 0; c < np; ++c) {
      int pr = c;
      for (int i = c + 1; i < np; ++i)
        if (fabs(W[i][c]) > fabs(W[pr][c])) pr = i;
      if (W[pr][c] == 0.0) return false;
      for (int j = 0; j < 2 * np; ++j) std::swap(W[c][j], W[pr][j]);
      const double d = W[c][c];
      for (int j = 0; j < 2 * np; ++j) W[c][j] /= d;
      for (int i = 0; i < np; ++i)
        if (i != c) {
          const double m = W[i][c];
          for (int j = 0; j < 2 * np; ++j) W[i][j] -= m * W[c][j];
        }
    }
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) Ainv[i * np + j] = W[i][np + j];
    return true;
  };
  if (!invert(f.M, f.Minv)) return NSK_ERR_ARG;
  // V[i][m] = phi_m(xi_i), phi_m = sqrt((2m+1)/2) P_m (Legendre three-term recurrence)
  double V[NSK_MAXNP * NSK_MAXNP];
  for (int i = 0; i < np; ++i) {
    double p0 = 1.0, p1 = xi[i];
    for (int m = 0; m < np; ++m) {
      double pm;
      if (m == 0) {
        pm = 1.0;
      } else if (m == 1) {
        pm = xi[i];
      } else {
        pm = ((2.0 * m - 1.0) * xi[i] * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = pm;
      }
      V[i * np + m] = sqrt((2.0 * m + 1.0) / 2.0) * pm;
    }
  }
  if (!invert(V, f.Vinv)) return NSK_ERR_ARG;
  for (int v = 0; v < 3; ++v) {
    f.Ub[0][v] = Ub_lo ? Ub_lo[v] : 1.0;
    f.Ub[1][v] = Ub_hi ? Ub_hi[v] : 1.0;
  }
  f.dirichlet = dirichlet;
  f.upper = upper;
  f.lower = lower;
  f.dx = h / np;
  return NSK_OK;
}
