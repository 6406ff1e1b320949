/*
 * nsk_oracle.c -- TEST INFRASTRUCTURE ONLY: plain FP64 CPU reference of the
 * DGSEM discretisation of relaxation model II (arXiv:1912.12059), and of the original
 * third-order NSK equations it approximates (Sec. 2.2, second BR1 lifting of Sec. 3.1).
 *
 * Written for a reader checking it against the paper by eye: element by
 * element, face by face, line by line, with the weak form of Sec. 3.1
 * (Eq. weakformulation) evaluated by Gauss quadrature, no tensor-product
 * tricks, no fusion. Build with -ffp-contract=off.
 *
 * Only the test suite, the package's smoke check and the benchmark's CPU
 * baseline may use this file. It shares no code with the CUDA library.
 */
#include "nsk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXNP 16
#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NONPHYSICAL (-3)
#define ORC_ERR_NOCONV (-6)

/* ------------------------------------------------------------------------ */
/* Van-der-Waals thermodynamics, Sec. 2.1                                    */
/* ------------------------------------------------------------------------ */

/* Reduced VdW parameters, Eq. (vdw_parameters): a = 3, b = 1/3, R = 8/3. */
static const double VDW_A = 3.0;
static const double VDW_B = 1.0 / 3.0;
static const double VDW_R = 8.0 / 3.0;

/* Eq. (vdw_freeenergy): W = rho R T ln(rho / (1 - b rho)) - a rho^2. */
double orc_free_energy(double T, double rho) {
  return rho * VDW_R * T * log(rho / (1.0 - VDW_B * rho)) - VDW_A * rho * rho;
}

/* Eq. (vdw_p): p = rho R T / (1 - b rho) - a rho^2. */
double orc_pressure(double T, double rho) {
  return rho * VDW_R * T / (1.0 - VDW_B * rho) - VDW_A * rho * rho;
}

/* dp/drho = R T / (1 - b rho)^2 - 2 a rho (derivative of Eq. vdw_p). */
double orc_dpressure(double T, double rho) {
  double q = 1.0 - VDW_B * rho;
  return VDW_R * T / (q * q) - 2.0 * VDW_A * rho;
}

/* Chemical potential W'(rho) = (W + p) / rho, from Eq. (vdw_p_as_derivative). */
double orc_chem_potential(double T, double rho) {
  return (orc_free_energy(T, rho) + orc_pressure(T, rho)) / rho;
}

/* W''(rho) = p'(rho) / rho (Sec. 2.1, p' = rho W''). */
static double second_deriv_W(double T, double rho) { return orc_dpressure(T, rho) / rho; }

/* Saturated states (Sec. 2.1): equal pressure and equal chemical potential,
 * solved by Newton's method in the two unknowns (rho_vap, rho_liq). */
int orc_maxwell(double T, double* rho_vap, double* rho_liq, double* p_sat) {
  double v = 0.3, l = 1.8;
  for (int it = 0; it < 200; ++it) {
    double F1 = orc_pressure(T, l) - orc_pressure(T, v);
    double F2 = orc_chem_potential(T, l) - orc_chem_potential(T, v);
    double J11 = -orc_dpressure(T, v), J12 = orc_dpressure(T, l);
    double J21 = -second_deriv_W(T, v), J22 = second_deriv_W(T, l);
    double det = J11 * J22 - J12 * J21;
    if (det == 0.0 || !isfinite(det)) return ORC_ERR_NOCONV;
    double dv = (F1 * J22 - F2 * J12) / det;
    double dl = (J11 * F2 - J21 * F1) / det;
    v -= dv;
    l -= dl;
    if (fabs(dv) < 1e-15 && fabs(dl) < 1e-15) break;
  }
  if (!(v > 0.0 && l > v && l < 1.0 / VDW_B)) return ORC_ERR_NOCONV;
  *rho_vap = v;
  *rho_liq = l;
  if (p_sat) *p_sat = orc_pressure(T, v);
  return ORC_OK;
}

/* Spinodal densities: the two roots of p'(rho) = 0 on (0, 1/b), by bisection.
 * alpha_* = |min W''| / 2 on (rho_sv, rho_sl), Eq. (alpha_fullyhyperbolic_limit),
 * the minimum located by golden-section search. */
int orc_spinodal(double T, double* rho_sv, double* rho_sl, double* alpha_star) {
  /* p' > 0 near rho = 0 and near rho = 1/b; p' < 0 in between for T below critical.
   * The reduced critical density is 1, so one root lies in (0,1), the other in (1,3). */
  if (!(orc_dpressure(T, 1.0) < 0.0)) return ORC_ERR_ARG;
  double a = 1e-9, b = 1.0;
  for (int it = 0; it < 200; ++it) {
    double m = 0.5 * (a + b);
    if (orc_dpressure(T, m) > 0.0) a = m; else b = m;
  }
  double sv = 0.5 * (a + b);
  a = 1.0;
  b = 1.0 / VDW_B - 1e-9;
  for (int it = 0; it < 200; ++it) {
    double m = 0.5 * (a + b);
    if (orc_dpressure(T, m) < 0.0) a = m; else b = m;
  }
  double sl = 0.5 * (a + b);
  const double g = 0.5 * (sqrt(5.0) - 1.0);
  double x0 = sv, x1 = sl;
  for (int it = 0; it < 300; ++it) {
    double c = x1 - g * (x1 - x0), d = x0 + g * (x1 - x0);
    if (second_deriv_W(T, c) < second_deriv_W(T, d)) x1 = d; else x0 = c;
  }
  *rho_sv = sv;
  *rho_sl = sl;
  *alpha_star = fabs(second_deriv_W(T, 0.5 * (x0 + x1))) / 2.0;
  return ORC_OK;
}

/* Sec. 4.3, Eq. (hoc_initialpressures): Young-Laplace pressures of the liquid and
 * vapour phases of a spherical droplet, then the densities on the liquid and vapour
 * branches of the isotherm with those pressures (Newton from the saturated states). */
int orc_young_laplace(double T, double sigma, double r, double* rho_liq, double* rho_vap) {
  double rv, rl, ps;
  int st = orc_maxwell(T, &rv, &rl, &ps);
  if (st) return st;
  double pl = ps + rl / (rl - rv) * 2.0 * sigma / r;
  double pv = ps + rv / (rl - rv) * 2.0 * sigma / r;
  double x = rl, y = rv;
  for (int it = 0; it < 100; ++it) x -= (orc_pressure(T, x) - pl) / orc_dpressure(T, x);
  for (int it = 0; it < 100; ++it) y -= (orc_pressure(T, y) - pv) / orc_dpressure(T, y);
  *rho_liq = x;
  *rho_vap = y;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Nodal basis, Sec. 3.1, Eqs. (solutionpolynomial)-(polynomialsbasis)        */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial P_n(x) and its derivative, by the three-term recurrence. */
static void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  /* P_n' = n (x P_n - P_{n-1}) / (x^2 - 1), valid away from x = +-1. */
  *dP = n * (x * p1 - p0) / (x * x - 1.0);
}

/* Gauss-Legendre nodes are the roots of P_{N+1}, weights 2 / ((1 - x^2) P'_{N+1}(x)^2).
 * Gauss-Lobatto nodes are +-1 and the roots of P'_N, weights 2 / (N (N+1) P_N(x)^2).
 * Both found by Newton's method from Chebyshev-type guesses; output ascending. */
int orc_nodes(int N, int node_type, double* xi, double* w) {
  if (N < 1 || N >= ORC_MAXNP) return ORC_ERR_ARG;
  const double pi = 3.14159265358979323846;
  int n = N + 1;
  if (node_type == 0) {
    for (int i = 0; i < n; ++i) {
      double x = -cos(pi * (i + 0.75) / (n + 0.5));
      for (int it = 0; it < 100; ++it) {
        double P, dP;
        legendre(n, x, &P, &dP);
        double dx = P / dP;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
      }
      double P, dP;
      legendre(n, x, &P, &dP);
      xi[i] = x;
      w[i] = 2.0 / ((1.0 - x * x) * dP * dP);
    }
  } else if (node_type == 1) {
    xi[0] = -1.0;
    xi[N] = 1.0;
    for (int i = 1; i < N; ++i) {
      double x = -cos(pi * i / N);
      for (int it = 0; it < 100; ++it) {
        double P, dP;
        legendre(N, x, &P, &dP);
        /* Legendre's equation: (1 - x^2) P'' = 2 x P' - N (N+1) P. */
        double d2P = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
        double dx = dP / d2P;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
      }
      xi[i] = x;
    }
    for (int i = 0; i <= N; ++i) {
      double P, dP;
      if (i == 0 || i == N) {
        P = (i == 0 && (N % 2)) ? -1.0 : 1.0; /* P_N(+-1) = (+-1)^N */
      } else {
        legendre(N, xi[i], &P, &dP);
      }
      w[i] = 2.0 / (N * (N + 1.0) * P * P);
    }
  } else {
    return ORC_ERR_ARG;
  }
  /* ascending order (the guesses already are; sort defensively) */
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && xi[j] < xi[j - 1]; --j) {
      double t = xi[j]; xi[j] = xi[j - 1]; xi[j - 1] = t;
      t = w[j]; w[j] = w[j - 1]; w[j - 1] = t;
    }
  return ORC_OK;
}

/* Lagrange polynomial l_j(x) = prod_{m != j} (x - xi_m) / (xi_j - xi_m), Eq. (polynomialsbasis). */
double orc_lagrange_eval(int N, const double* xi, int j, double x) {
  double l = 1.0;
  for (int m = 0; m <= N; ++m)
    if (m != j) l *= (x - xi[m]) / (xi[j] - xi[m]);
  return l;
}

/* l_j'(x) by the product rule applied to the product above. */
static double lagrange_deriv(int N, const double* xi, int j, double x) {
  double s = 0.0;
  for (int k = 0; k <= N; ++k) {
    if (k == j) continue;
    double t = 1.0 / (xi[j] - xi[k]);
    for (int m = 0; m <= N; ++m)
      if (m != j && m != k) t *= (x - xi[m]) / (xi[j] - xi[m]);
    s += t;
  }
  return s;
}

/* Sec. 3.1 operators of the nodal Lagrange basis: D[i][j] = l_j'(xi_i), Lm[j] = l_j(-1), Lp[j] = l_j(+1). */
void orc_lagrange_tables(int N, const double* xi, double* D, double* Lm, double* Lp) {
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N; ++j) D[i * (N + 1) + j] = lagrange_deriv(N, xi, j, xi[i]);
  for (int j = 0; j <= N; ++j) {
    Lm[j] = orc_lagrange_eval(N, xi, j, -1.0);
    Lp[j] = orc_lagrange_eval(N, xi, j, 1.0);
  }
}

/* Carpenter & Kennedy (1994) fourth-order, five-stage, 2N-storage RK, the
 * low-storage family the paper cites in Sec. 3.1. */
void orc_lsrk4_coeffs(double* A, double* B, double* C) {
  A[0] = 0.0;
  A[1] = -567301805773.0 / 1357537059087.0;
  A[2] = -2404267990393.0 / 2016746695238.0;
  A[3] = -3550918686646.0 / 2091501179385.0;
  A[4] = -1275806237668.0 / 842570457699.0;
  B[0] = 1432997174477.0 / 9575080441755.0;
  B[1] = 5161836677717.0 / 13612068292357.0;
  B[2] = 1720146321549.0 / 2090206949498.0;
  B[3] = 3134564353537.0 / 4481467310338.0;
  B[4] = 2277821191437.0 / 14882151754819.0;
  C[0] = 0.0;
  C[1] = 1432997174477.0 / 9575080441755.0;
  C[2] = 2526269341429.0 / 6820363962896.0;
  C[3] = 2006345519317.0 / 3224310063776.0;
  C[4] = 2802321613138.0 / 2924317926251.0;
}

/* ------------------------------------------------------------------------ */
/* Mesh: uniform Cartesian periodic box, affine element maps (Sec. 3.1 with   */
/* J a^k = J (2/h_k) e_k, J = prod h_k / 2).                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
  int d, np, npe, nvar, nq, model;
  long E;
  int ne[3];
  long se[3]; /* element strides */
  int sn[3];  /* node strides */
  double h[3];
  double xi[ORC_MAXNP], w[ORC_MAXNP], D[ORC_MAXNP * ORC_MAXNP], Lm[ORC_MAXNP], Lp[ORC_MAXNP];
} mesh_t;

/* the mesh of a setup: element and node strides, spacings, nodes, weights and Lagrange tables */
static int make_mesh(const orc_setup* s, mesh_t* m) {
  if (s->dim < 1 || s->dim > 3) return ORC_ERR_ARG;
  if (s->N < 1 || s->N >= ORC_MAXNP) return ORC_ERR_ARG;
  memset(m, 0, sizeof(*m));
  if (s->model != 0 && s->model != 1) return ORC_ERR_ARG;
  m->d = s->dim;
  m->model = s->model;
  m->np = s->N + 1;
  m->nvar = s->model == 1 ? s->dim + 1 : s->dim + 2;
  m->nq = s->dim * (s->dim + 1);
  m->npe = 1;
  m->E = 1;
  for (int k = 0; k < 3; ++k) {
    if (k < s->dim) {
      if (s->nelem[k] < 1 || !(s->hi[k] > s->lo[k])) return ORC_ERR_ARG;
      m->ne[k] = s->nelem[k];
      m->h[k] = (s->hi[k] - s->lo[k]) / s->nelem[k];
    } else {
      m->ne[k] = 1;
      m->h[k] = 1.0;
    }
  }
  m->se[0] = 1;
  m->se[1] = m->ne[0];
  m->se[2] = (long)m->ne[0] * m->ne[1];
  m->E = (long)m->ne[0] * m->ne[1] * m->ne[2];
  for (int k = 0; k < 3; ++k) {
    m->sn[k] = m->npe;
    if (k < s->dim) m->npe *= m->np;
  }
  if (orc_nodes(s->N, s->node_type, m->xi, m->w)) return ORC_ERR_ARG;
  orc_lagrange_tables(s->N, m->xi, m->D, m->Lm, m->Lp);
  return ORC_OK;
}

/* neighbour of element e in direction k on side dir (-1 or +1), periodic */
static long neighbour(const mesh_t* m, long e, int k, int dir) {
  int c = (int)((e / m->se[k]) % m->ne[k]);
  int cn = (c + dir + m->ne[k]) % m->ne[k];
  return e + (long)(cn - c) * m->se[k];
}

/* index of node n along direction k: i_k */
static int node_coord(const mesh_t* m, int n, int k) { return (n / m->sn[k]) % m->np; }

/* value of the element polynomial of a nodal field f (one variable, [E][npe])
 * at the face xi_k = side (-1 or +1), at the face node whose line in direction k
 * starts at base node n0: sum_j l_j(side) f_j. */
static double trace(const mesh_t* m, const double* f, long e, int k, int n0, int side) {
  const double* L = side < 0 ? m->Lm : m->Lp;
  double s = 0.0;
  for (int j = 0; j < m->np; ++j) s += L[j] * f[e * m->npe + n0 + j * m->sn[k]];
  return s;
}

/* the Van-der-Waals state space of Sec. 2.1: 0 < rho < 1/b (finite) */
static int admissible(double rho) { return rho > 0.0 && rho < 1.0 / VDW_B && isfinite(rho); }

/* lifted primitive variables: w = (v_1..v_d, c) of a model II state U = (rho, m, c);
 * w = (v_1..v_d, rho) of an original NSK state U = (rho, m) */
static void cons_to_prim(const mesh_t* m, const double* U, double* w) {
  const int d = m->d;
  for (int a = 0; a < d; ++a) w[a] = U[1 + a] / U[0];
  w[d] = m->model == 1 ? U[0] : U[d + 1];
}

/* ------------------------------------------------------------------------ */
/* Model II fluxes, Eq. (fluxes_sources_model2)                               */
/* ------------------------------------------------------------------------ */

/* modified pressure p_alpha = p + alpha rho^2 / 2, Eq. (modified_pressure) */
static double p_alpha(const orc_setup* s, double rho) {
  return orc_pressure(s->T, rho) + s->alpha * rho * rho / 2.0;
}

/* sqrt(p_alpha'(rho)), the acoustic speed of Eq. (parabolic_eigenvalues_model2) */
static double sound_speed(const orc_setup* s, double rho) {
  return sqrt(orc_dpressure(s->T, rho) + s->alpha * rho);
}

/* convective flux in direction k: (rho v_k, rho v_k v + p_alpha e_k, 0) */
static void conv_flux(const orc_setup* s, int d, int k, const double* U, double* f) {
  double rho = U[0];
  f[0] = U[1 + k];
  for (int a = 0; a < d; ++a) f[1 + a] = U[1 + k] * (U[1 + a] / rho);
  f[1 + k] += p_alpha(s, rho);
  f[d + 1] = 0.0;
}

/* viscous flux in direction k: (0, tau_{.k}, (kappa/beta) c_{x_k}),
 * tau = mu (grad v + grad v^T - 2/3 div v I), Eq. (stress_nse).
 * Q[k*(d+1) + a] = d v_a / d x_k, Q[k*(d+1) + d] = d c / d x_k. */
static void visc_flux(const orc_setup* s, int d, int k, const double* Q, double* f) {
  double div = 0.0;
  for (int a = 0; a < d; ++a) div += Q[a * (d + 1) + a];
  f[0] = 0.0;
  for (int a = 0; a < d; ++a) {
    double t = Q[k * (d + 1) + a] + Q[a * (d + 1) + k];
    if (a == k) t -= 2.0 / 3.0 * div;
    f[1 + a] = s->mu * t;
  }
  f[d + 1] = s->kappa / s->beta * Q[k * (d + 1) + d];
}

/* Convective numerical flux of one face, normal +e_k, left state UL, right state UR.
 *
 * Local Lax-Friedrichs (Sec. 3.1 names LF and HLLC): the central flux minus half the largest
 * |lambda| of Eq. (parabolic_eigenvalues_model2) times the jump, on rho and momentum (on c
 * too when c_dissipation is set; c has no convective flux).
 *
 * HLLC (Sec. 3.1 refers to Toro's textbook for it): the three-wave solver applied to the
 * barotropic system (rho, m) with the modified pressure p_alpha. Outer wave speeds after
 * Davis, S_L = min(u_L - a_L, u_R - a_R), S_R = max(u_L + a_L, u_R + a_R), a = sqrt(p_alpha'),
 * u the normal velocity; contact speed
 *   S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R)) / (rho_L (S_L - u_L) - rho_R (S_R - u_R));
 * star states U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, v with its normal component replaced by S*);
 * flux F_L if S_L >= 0, F_R if S_R <= 0, else F_K + S_K (U*_K - U_K) with K = L for S* >= 0 and
 * K = R otherwise. c is not transported: its convective numerical flux is zero. */
static void numflux(const orc_setup* s, int d, int k, const double* UL, const double* UR, double* F) {
  double fL[5], fR[5];
  conv_flux(s, d, k, UL, fL);
  conv_flux(s, d, k, UR, fR);
  const int nv = d + 2;
  const double aL = sound_speed(s, UL[0]), aR = sound_speed(s, UR[0]);
  const double uL = UL[1 + k] / UL[0], uR = UR[1 + k] / UR[0];
  if (s->flux == 1) {
    const double SL = fmin(uL - aL, uR - aR), SR = fmax(uL + aL, uR + aR);
    if (SL >= 0.0) {
      for (int v = 0; v < nv; ++v) F[v] = fL[v];
    } else if (SR <= 0.0) {
      for (int v = 0; v < nv; ++v) F[v] = fR[v];
    } else {
      const double pL = p_alpha(s, UL[0]), pR = p_alpha(s, UR[0]);
      const double Ss = (pR - pL + UL[0] * uL * (SL - uL) - UR[0] * uR * (SR - uR)) /
                        (UL[0] * (SL - uL) - UR[0] * (SR - uR));
      const int left = Ss >= 0.0;
      const double* UK = left ? UL : UR;
      const double* fK = left ? fL : fR;
      const double SK = left ? SL : SR, uK = left ? uL : uR;
      const double coef = UK[0] * (SK - uK) / (SK - Ss);
      double Us[5];
      Us[0] = coef;
      for (int a = 0; a < d; ++a) Us[1 + a] = coef * (a == k ? Ss : UK[1 + a] / UK[0]);
      Us[d + 1] = UK[d + 1];
      for (int v = 0; v < nv; ++v) F[v] = fK[v] + SK * (Us[v] - UK[v]);
    }
    F[d + 1] = 0.0;
    return;
  }
  const double lamL = fabs(uL) + aL, lamR = fabs(uR) + aR;
  const double lam = lamL > lamR ? lamL : lamR;
  for (int v = 0; v < nv; ++v) {
    F[v] = 0.5 * (fL[v] + fR[v]);
    if (v < d + 1 || s->c_dissipation) F[v] -= 0.5 * lam * (UR[v] - UL[v]);
  }
}

/* public entry of the convective numerical flux above (model II), with its argument checks */
int orc_numflux(const orc_setup* s, int k, const double* UL, const double* UR, double* F) {
  if (!s || k < 0 || k >= s->dim || !UL || !UR || !F) return ORC_ERR_ARG;
  if (!admissible(UL[0]) || !admissible(UR[0])) return ORC_ERR_NONPHYSICAL;
  numflux(s, s->dim, k, UL, UR, F);
  for (int v = 0; v < s->dim + 2; ++v)
    if (!isfinite(F[v])) return ORC_ERR_NONPHYSICAL;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* BR1 lifting, Sec. 3.1: Q - (1/J) div_xi (J a^k w) = 0 in weak form with the */
/* central flux w* = (w^- + w^+)/2, w = primitive variables (v, c).           */
/* ------------------------------------------------------------------------ */

static int lift(const orc_setup* s, const mesh_t* m, const double* U, double* Q) {
  (void)s; /* the lifting needs no physical parameter */
  const int d = m->d, np = m->np, npe = m->npe, nw = d + 1;
  const long E = m->E, nn = E * npe;
  double* W = (double*)malloc(sizeof(double) * nw * nn);
  if (!W) return ORC_ERR_ARG;
  int status = ORC_OK;
  /* primitive variables at the volume nodes (elements are independent: the OpenMP build of the
   * timed CPU baseline shares them among threads; every result is written by one iteration, so
   * both builds give the same bits) */
#pragma omp parallel for reduction(min : status) schedule(static)
  for (long e = 0; e < E; ++e)
    for (int n = 0; n < npe; ++n) {
      double Un[5], wn[4];
      for (int v = 0; v < m->nvar; ++v) Un[v] = U[v * nn + e * npe + n];
      if (!admissible(Un[0])) status = ORC_ERR_NONPHYSICAL;
      cons_to_prim(m, Un, wn);
      for (int q = 0; q < nw; ++q) W[q * nn + e * npe + n] = wn[q];
    }
#pragma omp parallel for reduction(min : status) schedule(static)
  for (long e = 0; e < E; ++e) {
    for (int k = 0; k < d; ++k) {
      const long eL = neighbour(m, e, k, -1), eR = neighbour(m, e, k, +1);
      for (int n0 = 0; n0 < npe; ++n0) {
        if (node_coord(m, n0, k) != 0) continue; /* one line per base node */
        /* conservative traces on both sides of both faces of this line */
        double Um[5], Up[5], UnbM[5], UnbP[5];
        for (int v = 0; v < m->nvar; ++v) {
          const double* f = U + v * nn;
          Um[v] = trace(m, f, e, k, n0, -1);
          Up[v] = trace(m, f, e, k, n0, +1);
          UnbM[v] = trace(m, f, eL, k, n0, +1); /* left neighbour's +1 face */
          UnbP[v] = trace(m, f, eR, k, n0, -1); /* right neighbour's -1 face */
        }
        if (!admissible(Um[0]) || !admissible(Up[0]) || !admissible(UnbM[0]) || !admissible(UnbP[0]))
          status = ORC_ERR_NONPHYSICAL;
        double wm[4], wp[4], wnm[4], wnp[4], wsm[4], wsp[4];
        cons_to_prim(m, Um, wm);
        cons_to_prim(m, Up, wp);
        cons_to_prim(m, UnbM, wnm);
        cons_to_prim(m, UnbP, wnp);
        for (int q = 0; q < nw; ++q) {
          wsm[q] = 0.5 * (wm[q] + wnm[q]);
          wsp[q] = 0.5 * (wp[q] + wnp[q]);
        }
        for (int i = 0; i < np; ++i) {
          const int node = n0 + i * m->sn[k];
          for (int q = 0; q < nw; ++q) {
            const double* f = W + q * nn + e * npe;
            /* volume term: - sum_j w_j w_q(xi_j) l_i'(xi_j) / w_i */
            double vol = 0.0;
            for (int j = 0; j < np; ++j) vol += m->w[j] * f[n0 + j * m->sn[k]] * m->D[j * np + i];
            vol /= m->w[i];
            /* surface term: (w*_+ l_i(1) - w*_- l_i(-1)) / w_i */
            double surf = (wsp[q] * m->Lp[i] - wsm[q] * m->Lm[i]) / m->w[i];
            Q[(long)(k * nw + q) * nn + e * npe + node] = (2.0 / m->h[k]) * (surf - vol);
          }
        }
      }
    }
  }
  free(W);
  return status;
}

/* public entry of the BR1 lifting above */
int orc_lift(const orc_setup* s, const double* U, double* Q) {
  mesh_t m;
  int st = make_mesh(s, &m);
  if (st) return st;
  return lift(s, &m, U, Q);
}

/* ------------------------------------------------------------------------ */
/* Residual, Eq. (weakformulation):                                          */
/*   R_i = sum_k (2/h_k) [ sum_j (w_j/w_i) l_i'(xi_j) f_k(U_j, Q_j)          */
/*                        - (f*_{k,+} l_i(1) - f*_{k,-} l_i(-1)) / w_i ] + S_i */
/* with f = f^c - f^v, f* the local Lax-Friedrichs convective flux minus the  */
/* BR1 mean of the viscous fluxes, S the model II source.                    */
/* ------------------------------------------------------------------------ */

static int residual(const orc_setup* s, const mesh_t* m, const double* U, double* R) {
  const int d = m->d, np = m->np, npe = m->npe, nv = m->nvar, nw = d + 1, nq = m->nq;
  const long E = m->E, nn = E * npe;
  double* Q = (double*)malloc(sizeof(double) * nq * nn);
  if (!Q) return ORC_ERR_ARG;
  int status = lift(s, m, U, Q);
  for (long i = 0; i < nv * nn; ++i) R[i] = 0.0;

  /* volume integral (each iteration writes its own element only) */
#pragma omp parallel for schedule(static)
  for (long e = 0; e < E; ++e) {
    for (int k = 0; k < d; ++k) {
      for (int n0 = 0; n0 < npe; ++n0) {
        if (node_coord(m, n0, k) != 0) continue;
        double F[ORC_MAXNP][5];
        for (int j = 0; j < np; ++j) {
          const int node = n0 + j * m->sn[k];
          double Un[5], Qn[12], fc[5], fv[5];
          for (int v = 0; v < nv; ++v) Un[v] = U[v * nn + e * npe + node];
          for (int q = 0; q < nq; ++q) Qn[q] = Q[q * nn + e * npe + node];
          conv_flux(s, d, k, Un, fc);
          visc_flux(s, d, k, Qn, fv);
          for (int v = 0; v < nv; ++v) F[j][v] = fc[v] - fv[v];
        }
        for (int i = 0; i < np; ++i) {
          const int node = n0 + i * m->sn[k];
          for (int v = 0; v < nv; ++v) {
            double vol = 0.0;
            for (int j = 0; j < np; ++j) vol += m->w[j] * F[j][v] * m->D[j * np + i];
            R[v * nn + e * npe + node] += (2.0 / m->h[k]) * vol / m->w[i];
          }
        }
      }
    }
  }

  /* surface integral: every face once, between element e (its +1 side) and
   * its right neighbour eR (its -1 side), outward normal of e is +e_k. First the
   * numerical flux f* of every face line (faces are independent), then its
   * lifting onto both elements, face after face in the same order, so every
   * node receives its surface terms in one fixed order. */
  const int nl = npe / np; /* face lines per element and direction */
  double* Fsall = (double*)malloc(sizeof(double) * nv * E * d * nl);
  char* skip = (char*)calloc((size_t)E * d * nl, 1);
  if (!Fsall || !skip) {
    free(Fsall);
    free(skip);
    free(Q);
    return ORC_ERR_ARG;
  }
#pragma omp parallel for reduction(min : status) schedule(static)
  for (long e = 0; e < E; ++e) {
    for (int k = 0; k < d; ++k) {
      const long eR = neighbour(m, e, k, +1);
      int line = 0;
      for (int n0 = 0; n0 < npe; ++n0) {
        if (node_coord(m, n0, k) != 0) continue;
        const long fl = (e * d + k) * nl + line++;
        double UL[5], UR[5], QL[12], QR[12];
        for (int v = 0; v < nv; ++v) {
          UL[v] = trace(m, U + v * nn, e, k, n0, +1);
          UR[v] = trace(m, U + v * nn, eR, k, n0, -1);
        }
        for (int q = 0; q < nq; ++q) {
          QL[q] = trace(m, Q + q * nn, e, k, n0, +1);
          QR[q] = trace(m, Q + q * nn, eR, k, n0, -1);
        }
        if (!admissible(UL[0]) || !admissible(UR[0])) {
          status = ORC_ERR_NONPHYSICAL;
          skip[fl] = 1;
          continue;
        }
        double fvL[5], fvR[5], Fs[5];
        visc_flux(s, d, k, QL, fvL);
        visc_flux(s, d, k, QR, fvR);
        if (!isfinite(sound_speed(s, UL[0])) || !isfinite(sound_speed(s, UR[0]))) status = ORC_ERR_NONPHYSICAL;
        /* convective numerical flux (LF or HLLC) minus the BR1 mean of the viscous fluxes */
        numflux(s, d, k, UL, UR, Fs);
        for (int v = 0; v < nv; ++v) Fs[v] -= 0.5 * (fvL[v] + fvR[v]);
        for (int v = 0; v < nv; ++v) Fsall[fl * nv + v] = Fs[v];
      }
    }
  }
  for (long e = 0; e < E; ++e) {
    for (int k = 0; k < d; ++k) {
      const long eR = neighbour(m, e, k, +1);
      int line = 0;
      for (int n0 = 0; n0 < npe; ++n0) {
        if (node_coord(m, n0, k) != 0) continue;
        const long fl = (e * d + k) * nl + line++;
        if (skip[fl]) continue;
        const double* Fs = Fsall + fl * nv;
        for (int i = 0; i < np; ++i) {
          const int node = n0 + i * m->sn[k];
          for (int v = 0; v < nv; ++v) {
            /* +1 face of e: -(2/h) f* l_i(1) / w_i ; -1 face of eR: +(2/h) f* l_i(-1) / w_i */
            R[v * nn + e * npe + node] -= (2.0 / m->h[k]) * Fs[v] * m->Lp[i] / m->w[i];
            R[v * nn + eR * npe + node] += (2.0 / m->h[k]) * Fs[v] * m->Lm[i] / m->w[i];
          }
        }
      }
    }
  }

  free(Fsall);
  free(skip);

  /* pointwise sources (0, alpha rho grad c, (alpha/beta)(rho - c)), evaluated
   * with the lifted gradient of c (Sec. 3.1, last paragraph) */
#pragma omp parallel for schedule(static)
  for (long e = 0; e < E; ++e)
    for (int n = 0; n < npe; ++n) {
      const long p = e * npe + n;
      double rho = U[p], c = U[(d + 1) * nn + p];
      for (int a = 0; a < d; ++a) R[(1 + a) * nn + p] += s->alpha * rho * Q[(a * nw + d) * nn + p];
      R[(d + 1) * nn + p] += s->alpha / s->beta * (rho - c);
    }
  (void)nw;
  free(Q);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Original NSK equations, Sec. 2.2: state (rho, m), Eqs. (nsk_1), (nsk_2),    */
/*   F_k = (m_k, m_k v + p e_k - tau_{.k} - tau^K_{.k}),                       */
/*   tau = mu (grad v + grad v^T - 2/3 div v I)           Eq. (stress_nse)     */
/*   tau^K = kappa (rho lap rho + |grad rho|^2 / 2) I - kappa grad rho (x) grad rho, Eq. (stress_nsk) */
/* with grad v and grad rho from the BR1 lifting of w = (v, rho) and lap rho  */
/* from the second BR1 lifting of grad rho (Sec. 3.1); central numerical flux */
/* for the convective part (Sec. 3.1: the central flux is used for the       */
/* original NSK equations) and the BR1 mean of the viscous and Korteweg parts. */
/* ------------------------------------------------------------------------ */

/* second lifting: Q2 = sum_k d/dx_k (grad rho)_k in weak form with the central flux of the
 * traces of (grad rho)_k on the faces of direction k */
static void lift2(const mesh_t* m, const double* Q, double* Q2) {
  const int d = m->d, np = m->np, npe = m->npe, nw = d + 1;
  const long E = m->E, nn = E * npe;
  for (long i = 0; i < nn; ++i) Q2[i] = 0.0;
  for (long e = 0; e < E; ++e) {
    for (int k = 0; k < d; ++k) {
      const double* g = Q + (long)(k * nw + d) * nn; /* (grad rho)_k */
      const long eL = neighbour(m, e, k, -1), eR = neighbour(m, e, k, +1);
      for (int n0 = 0; n0 < npe; ++n0) {
        if (node_coord(m, n0, k) != 0) continue;
        const double gsm = 0.5 * (trace(m, g, e, k, n0, -1) + trace(m, g, eL, k, n0, +1));
        const double gsp = 0.5 * (trace(m, g, e, k, n0, +1) + trace(m, g, eR, k, n0, -1));
        for (int i = 0; i < np; ++i) {
          const int node = n0 + i * m->sn[k];
          double vol = 0.0;
          for (int j = 0; j < np; ++j) vol += m->w[j] * g[e * npe + n0 + j * m->sn[k]] * m->D[j * np + i];
          vol /= m->w[i];
          const double surf = (gsp * m->Lp[i] - gsm * m->Lm[i]) / m->w[i];
          Q2[e * npe + node] += (2.0 / m->h[k]) * (surf - vol);
        }
      }
    }
  }
}

/* viscous plus Korteweg flux in direction k, (0, tau_{.k} + tau^K_{.k}), from rho, the lifted
 * gradients Q (Q[k*(d+1)+a] = d v_a/dx_k, Q[k*(d+1)+d] = d rho/dx_k) and lap rho */
static void visc_kort_flux(const orc_setup* s, int d, int k, double rho, const double* Q, double lap, double* f) {
  double div = 0.0, g2 = 0.0;
  for (int a = 0; a < d; ++a) {
    div += Q[a * (d + 1) + a];
    g2 += Q[a * (d + 1) + d] * Q[a * (d + 1) + d];
  }
  f[0] = 0.0;
  for (int a = 0; a < d; ++a) {
    double t = Q[k * (d + 1) + a] + Q[a * (d + 1) + k];
    if (a == k) t -= 2.0 / 3.0 * div;
    double tk = -s->kappa * Q[a * (d + 1) + d] * Q[k * (d + 1) + d];
    if (a == k) tk += s->kappa * (rho * lap + 0.5 * g2);
    f[1 + a] = s->mu * t + tk;
  }
}

/* convective flux of the original NSK equations: (m_k, m_k v + p e_k) with the VdW pressure */
static void conv_flux_nsk(const orc_setup* s, int d, int k, const double* U, double* f) {
  f[0] = U[1 + k];
  for (int a = 0; a < d; ++a) f[1 + a] = U[1 + k] * (U[1 + a] / U[0]);
  f[1 + k] += orc_pressure(s->T, U[0]);
}

/* residual of the original NSK equations (Sec. 2.2, Eqs. nsk_1 and nsk_2) in the weak form of
 * Eq. (weakformulation), the fluxes above, the central convective flux on the faces */
static int residual_nsk(const orc_setup* s, const mesh_t* m, const double* U, double* R) {
  const int d = m->d, np = m->np, npe = m->npe, nv = m->nvar, nq = m->nq;
  const long E = m->E, nn = E * npe;
  double* Q = (double*)malloc(sizeof(double) * (nq + 1) * nn);
  if (!Q) return ORC_ERR_ARG;
  double* Q2 = Q + (long)nq * nn;
  int status = lift(s, m, U, Q);
  lift2(m, Q, Q2);
  for (long i = 0; i < nv * nn; ++i) R[i] = 0.0;

  /* volume integral */
  for (long e = 0; e < E; ++e) {
    for (int k = 0; k < d; ++k) {
      for (int n0 = 0; n0 < npe; ++n0) {
        if (node_coord(m, n0, k) != 0) continue;
        double F[ORC_MAXNP][4];
        for (int j = 0; j < np; ++j) {
          const int node = n0 + j * m->sn[k];
          double Un[4], Qn[12], fc[4], fv[4];
          for (int v = 0; v < nv; ++v) Un[v] = U[v * nn + e * npe + node];
          for (int q = 0; q < nq; ++q) Qn[q] = Q[q * nn + e * npe + node];
          conv_flux_nsk(s, d, k, Un, fc);
          visc_kort_flux(s, d, k, Un[0], Qn, Q2[e * npe + node], fv);
          for (int v = 0; v < nv; ++v) F[j][v] = fc[v] - fv[v];
        }
        for (int i = 0; i < np; ++i) {
          const int node = n0 + i * m->sn[k];
          for (int v = 0; v < nv; ++v) {
            double vol = 0.0;
            for (int j = 0; j < np; ++j) vol += m->w[j] * F[j][v] * m->D[j * np + i];
            R[v * nn + e * npe + node] += (2.0 / m->h[k]) * vol / m->w[i];
          }
        }
      }
    }
  }

  /* surface integral, every face once (outward normal +e_k of element e) */
  for (long e = 0; e < E; ++e) {
    for (int k = 0; k < d; ++k) {
      const long eR = neighbour(m, e, k, +1);
      for (int n0 = 0; n0 < npe; ++n0) {
        if (node_coord(m, n0, k) != 0) continue;
        double UL[4], UR[4], QL[12], QR[12];
        for (int v = 0; v < nv; ++v) {
          UL[v] = trace(m, U + v * nn, e, k, n0, +1);
          UR[v] = trace(m, U + v * nn, eR, k, n0, -1);
        }
        for (int q = 0; q < nq; ++q) {
          QL[q] = trace(m, Q + q * nn, e, k, n0, +1);
          QR[q] = trace(m, Q + q * nn, eR, k, n0, -1);
        }
        const double lapL = trace(m, Q2, e, k, n0, +1), lapR = trace(m, Q2, eR, k, n0, -1);
        if (!admissible(UL[0]) || !admissible(UR[0])) {
          status = ORC_ERR_NONPHYSICAL;
          continue;
        }
        double fcL[4], fcR[4], fvL[4], fvR[4], Fs[4];
        conv_flux_nsk(s, d, k, UL, fcL);
        conv_flux_nsk(s, d, k, UR, fcR);
        visc_kort_flux(s, d, k, UL[0], QL, lapL, fvL);
        visc_kort_flux(s, d, k, UR[0], QR, lapR, fvR);
        for (int v = 0; v < nv; ++v) Fs[v] = 0.5 * (fcL[v] + fcR[v]) - 0.5 * (fvL[v] + fvR[v]);
        for (int i = 0; i < np; ++i) {
          const int node = n0 + i * m->sn[k];
          for (int v = 0; v < nv; ++v) {
            R[v * nn + e * npe + node] -= (2.0 / m->h[k]) * Fs[v] * m->Lp[i] / m->w[i];
            R[v * nn + eR * npe + node] += (2.0 / m->h[k]) * Fs[v] * m->Lm[i] / m->w[i];
          }
        }
      }
    }
  }
  free(Q);
  return status;
}

int orc_lift2(const orc_setup* s, const double* U, double* Q2) {
  mesh_t m;
  int st = make_mesh(s, &m);
  if (st) return st;
  if (s->model != 1) return ORC_ERR_ARG;
  double* Q = (double*)malloc(sizeof(double) * m.nq * m.E * m.npe);
  if (!Q) return ORC_ERR_ARG;
  st = lift(s, &m, U, Q);
  lift2(&m, Q, Q2);
  free(Q);
  return st;
}

/* the residual of the setup's model: relaxation model II or the original NSK equations */
static int rhs_any(const orc_setup* s, const mesh_t* m, const double* U, double* R) {
  return s->model == 1 ? residual_nsk(s, m, U, R) : residual(s, m, U, R);
}

/* public entry of the semi-discrete residual R(U) */
int orc_rhs(const orc_setup* s, const double* U, double* R) {
  mesh_t m;
  int st = make_mesh(s, &m);
  if (st) return st;
  if (!(s->kappa >= 0.0) || !(s->mu >= 0.0) || (s->model == 0 && !(s->beta > 0.0))) return ORC_ERR_ARG;
  return rhs_any(s, &m, U, R);
}

/* Threads the loops above run on: 1 in the plain build, the OpenMP team size in
 * the build for the timed CPU baseline (the same source compiled with -fopenmp). */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* 2N-storage update: K <- A_s K + dt R(U); U <- U + B_s K, s = 1..5. */
int orc_lsrk4(const orc_setup* s, double* U, double dt, int nsteps) {
  mesh_t m;
  int st = make_mesh(s, &m);
  if (st) return st;
  const long len = (long)m.nvar * m.E * m.npe;
  double* K = (double*)calloc(len, sizeof(double));
  double* R = (double*)malloc(sizeof(double) * len);
  if (!K || !R) { free(K); free(R); return ORC_ERR_ARG; }
  double A[5], B[5], C[5];
  orc_lsrk4_coeffs(A, B, C);
  for (int step = 0; step < nsteps && st == ORC_OK; ++step) {
    for (int stage = 0; stage < 5; ++stage) {
      st = rhs_any(s, &m, U, R);
      if (st) break;
#pragma omp parallel for schedule(static)
      for (long i = 0; i < len; ++i) {
        K[i] = A[stage] * K[i] + dt * R[i];
        U[i] = U[i] + B[stage] * K[i];
      }
    }
  }
  free(K);
  free(R);
  return st;
}

/* Time step. Eq. (numerics_dfl) gives only the parabolic bound; the convective
 * bound and the bound of the stiff relaxation source are added (the paper is
 * silent on both):
 *   dt_conv = cfl / ((2N+1) max_nodes sum_k (|v_k| + sqrt(p_alpha')) / h_k)
 *   dt_visc = cfl / ((2N+1)^2 lambda_v sum_k 1/h_k^2), lambda_v = max(mu, kappa/beta)
 *             (Eq. visc_eigenvalues; beta_RK folded into cfl)
 *   dt_src  = cfl * 4.6 * beta / alpha (4.6 just inside the real-axis stability
 *             limit of the five-stage scheme)                                   */
int orc_timestep(const orc_setup* s, const double* U, double cfl, double* dt) {
  mesh_t m;
  int st = make_mesh(s, &m);
  if (st) return st;
  const int d = m.d;
  const long nn = m.E * m.npe;
  double lam_max = 0.0, rho_max = 0.0;
  for (long p = 0; p < nn; ++p) {
    double rho = U[p];
    if (!admissible(rho)) return ORC_ERR_NONPHYSICAL;
    if (rho > rho_max) rho_max = rho;
    /* original NSK: p' < 0 in the spinodal interval, where the first-order part has no real
     * sound speed (Eq. nsk_eigenvalues); only the flow speed bounds the step there */
    double a = s->model == 1 ? sqrt(fmax(orc_dpressure(s->T, rho), 0.0)) : sound_speed(s, rho);
    if (!isfinite(a)) return ORC_ERR_NONPHYSICAL;
    double sum = 0.0;
    for (int k = 0; k < d; ++k) sum += (fabs(U[(1 + k) * nn + p] / rho) + a) / m.h[k];
    if (sum > lam_max) lam_max = sum;
  }
  const double twoNp1 = 2.0 * s->N + 1.0;
  double dt_conv = cfl / (twoNp1 * lam_max);
  double inv_h2 = 0.0;
  for (int k = 0; k < d; ++k) inv_h2 += 1.0 / (m.h[k] * m.h[k]);
  if (s->model == 1) {
    /* viscous bound with mu, and the dispersive Korteweg term: linearised about rho_0 the
     * waves obey omega^2 = p' k^2 + kappa rho_0 k^4, i.e. |omega| ~ sqrt(kappa rho_0) k^2 like
     * a diffusion with coefficient sqrt(kappa rho_max) (on the imaginary axis) */
    const double lamk = s->mu > sqrt(s->kappa * rho_max) ? s->mu : sqrt(s->kappa * rho_max);
    const double dt_k = lamk > 0.0 ? cfl / (twoNp1 * twoNp1 * lamk * inv_h2) : INFINITY;
    *dt = dt_conv < dt_k ? dt_conv : dt_k;
    return ORC_OK;
  }
  double lamv = s->mu > s->kappa / s->beta ? s->mu : s->kappa / s->beta;
  double dt_visc = lamv > 0.0 ? cfl / (twoNp1 * twoNp1 * lamv * inv_h2) : INFINITY;
  double dt_src = cfl * 4.6 * s->beta / s->alpha;
  double r = dt_conv;
  if (dt_visc < r) r = dt_visc;
  if (dt_src < r) r = dt_src;
  *dt = r;
  return ORC_OK;
}

/* Quadrature sums over the mesh with weights w_n J, J = prod_k h_k / 2:
 *   mass = sum rho;
 *   energy = sum (|m|^2/(2 rho) + W(rho) + alpha/2 (rho-c)^2 + kappa/2 |Q_c|^2),
 *            Eq. (pararelax_elliptical_energy_dynamic) with the BR1 gradient of c;
 *   l2 = sqrt(sum (rho - c)^2). */
int orc_diagnostics(const orc_setup* s, const double* U, double* mass, double* energy, double* l2_rho_c) {
  mesh_t m;
  int st = make_mesh(s, &m);
  if (st) return st;
  const int d = m.d, nw = d + 1;
  const long nn = m.E * m.npe;
  double* Q = (double*)malloc(sizeof(double) * m.nq * nn);
  if (!Q) return ORC_ERR_ARG;
  st = lift(s, &m, U, Q);
  double J = 1.0;
  for (int k = 0; k < d; ++k) J *= m.h[k] / 2.0;
  double sm = 0.0, se = 0.0, sl = 0.0;
  for (long e = 0; e < m.E; ++e)
    for (int n = 0; n < m.npe; ++n) {
      double wq = J;
      for (int k = 0; k < d; ++k) wq *= m.w[node_coord(&m, n, k)];
      const long p = e * m.npe + n;
      /* original NSK: Eq. (original_energy_dynamic), capillary energy kappa/2 |grad rho|^2 with
       * the lifted density gradient (the same slot of Q as grad c of model II) and no rho - c */
      double rho = U[p], c = s->model == 1 ? rho : U[(d + 1) * nn + p];
      double m2 = 0.0, g2 = 0.0;
      for (int a = 0; a < d; ++a) {
        m2 += U[(1 + a) * nn + p] * U[(1 + a) * nn + p];
        double gc = Q[(a * nw + d) * nn + p];
        g2 += gc * gc;
      }
      sm += wq * rho;
      se += wq * (m2 / (2.0 * rho) + orc_free_energy(s->T, rho) + s->alpha / 2.0 * (rho - c) * (rho - c) +
                  s->kappa / 2.0 * g2);
      sl += wq * (rho - c) * (rho - c);
    }
  free(Q);
  *mass = sm;
  *energy = se;
  *l2_rho_c = sqrt(sl);
  return st;
}

/* ======================================================================== */
/* Finite-volume sub-cell shock capturing, Sec. 3.2 (the section "Finite    */
/* Volume Sub-Cell Approach"), and Dirichlet boundaries, for the 1D sharp-   */
/* interface Riemann problem of Sec. 4 (model II, one space dimension).      */
/*                                                                           */
/* An element is either a DG element (nodal values) or an FV element: N+1    */
/* equidistant sub-cells holding integral means. The section fixes the       */
/* sub-cell count, the exact Gauss conversion DG -> means, the FV weak form   */
/* (phi = 1, midpoint rule on the faces, LF or HLLC), the second-order TVD    */
/* reconstruction with MinMod, the gradient from a continuous reconstruction  */
/* for the diffusive fluxes, and the Persson-Peraire indicator with two       */
/* thresholds. Where it is silent this code takes these readings:             */
/*   - the indicator acts on rho, as log10 of the energy of the highest       */
/*     orthonormal Legendre mode over the total energy;                       */
/*   - DG -> FV when Ind > upper, FV -> DG when Ind < lower (Ind of an FV     */
/*     element from the degree-N polynomial with its sub-cell means), once    */
/*     per time step, before the first stage (A_1 = 0 empties the RK          */
/*     register, so only U is converted);                                     */
/*   - FV -> DG by the inverse of the mean matrix (the unique polynomial of   */
/*     degree N with those means);                                            */
/*   - the reconstruction acts on (rho, v, c); across an element face the     */
/*     neighbour value is the adjacent sub-cell mean of an FV element (one    */
/*     sub-cell width away) or the face value of a DG element or boundary     */
/*     state (half a width away);                                             */
/*   - diffusive fluxes on FV faces use the difference quotient of the two    */
/*     neighbouring values (the 1D form of Green's identity on the continuous */
/*     piecewise-linear reconstruction); the source gradient of c in a        */
/*     sub-cell is the mean of its two face quotients;                        */
/*   - a face between a DG and an FV element pairs the DG trace (and its      */
/*     lifted gradient) with the FV side's reconstructed face value (and its  */
/*     difference quotient); the DG lifting takes the central w* of the two;  */
/*   - a Dirichlet boundary is a ghost neighbour whose face state is the      */
/*     given boundary state and whose gradient equals the interior side's.    */
/* ======================================================================== */

/* orthonormal Legendre polynomial phi_m = sqrt((2m+1)/2) P_m on [-1, 1] */
static double legendre_on(int m, double x) {
  double P, dP;
  legendre(m, x, &P, &dP);  /* dP is not used (and not defined at x = +-1) */
  return sqrt((2.0 * m + 1.0) / 2.0) * P;
}

/* solve A x = b (n x n, row-major, copied) by Gaussian elimination with partial pivoting */
static int solve_dense(int n, const double* A_in, const double* b, double* x) {
  double A[ORC_MAXNP * ORC_MAXNP], r[ORC_MAXNP];
  memcpy(A, A_in, sizeof(double) * n * n);
  memcpy(r, b, sizeof(double) * n);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (fabs(A[i * n + c]) > fabs(A[p * n + c])) p = i;
    if (A[p * n + c] == 0.0) return ORC_ERR_NOCONV;
    if (p != c) {
      for (int j = 0; j < n; ++j) {
        double t = A[c * n + j];
        A[c * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
      double t = r[c];
      r[c] = r[p];
      r[p] = t;
    }
    for (int i = c + 1; i < n; ++i) {
      const double f = A[i * n + c] / A[c * n + c];
      for (int j = c; j < n; ++j) A[i * n + j] -= f * A[c * n + j];
      r[i] -= f * r[c];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = r[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
    x[i] = s / A[i * n + i];
  }
  return ORC_OK;
}

/* Sub-cell means of the nodal basis: sub-cell j of N+1 covers xi in [a_j, a_j + 2/(N+1)],
 * a_j = -1 + 2j/(N+1); its mean of u is (1/2) sum_q w_q u(a_j + (xi_q + 1)/(N+1)) with the
 * (N+1)-point Gauss rule (xi_q, w_q) on [-1, 1], exact for degree N.
 * M[j][i] = mean of l_i over sub-cell j; Minv its inverse (means -> nodal values). */
int orc_fv_tables(int N, int node_type, double* M, double* Minv) {
  const int np = N + 1;
  double xi[ORC_MAXNP], w[ORC_MAXNP], xg[ORC_MAXNP], wg[ORC_MAXNP];
  if (N < 1 || N >= ORC_MAXNP || orc_nodes(N, node_type, xi, w) || orc_nodes(N, 0, xg, wg)) return ORC_ERR_ARG;
  for (int j = 0; j < np; ++j) {
    const double a = -1.0 + 2.0 * j / np;
    for (int i = 0; i < np; ++i) {
      double s = 0.0;
      for (int q = 0; q < np; ++q) s += wg[q] * orc_lagrange_eval(N, xi, i, a + (xg[q] + 1.0) / np);
      M[j * np + i] = 0.5 * s;
    }
  }
  if (Minv) {
    for (int c = 0; c < np; ++c) {  /* column c of the inverse: M x = e_c */
      double e[ORC_MAXNP] = {0}, x[ORC_MAXNP];
      e[c] = 1.0;
      if (solve_dense(np, M, e, x)) return ORC_ERR_NOCONV;
      for (int i = 0; i < np; ++i) Minv[i * np + c] = x[i];
    }
  }
  return ORC_OK;
}

/* Persson-Peraire indicator of nodal values u (N+1 nodes of the given type): the modal
 * coefficients uh in the orthonormal Legendre basis solve V uh = u, V[i][m] = phi_m(xi_i);
 * Ind = log10(uh_N^2 / sum_m uh_m^2). */
double orc_persson(int N, int node_type, const double* u) {
  const int np = N + 1;
  double xi[ORC_MAXNP], w[ORC_MAXNP], V[ORC_MAXNP * ORC_MAXNP], uh[ORC_MAXNP];
  if (N < 1 || N >= ORC_MAXNP || orc_nodes(N, node_type, xi, w)) return NAN;
  for (int i = 0; i < np; ++i)
    for (int m = 0; m < np; ++m) V[i * np + m] = legendre_on(m, xi[i]);
  if (solve_dense(np, V, u, uh)) return NAN;
  double tot = 0.0;
  for (int m = 0; m < np; ++m) tot += uh[m] * uh[m];
  return log10(uh[N] * uh[N] / tot);
}

/* the MinMod limiter of the second-order TVD reconstruction (Sec. 3.2): the smaller slope in
 * magnitude when both have the same sign, else zero */
static double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return a > 0.0 ? fmin(a, b) : fmax(a, b);
}

/* (rho, m, c) <-> (rho, v, c) */
static void fv_prim(const double* U, double* P) {
  P[0] = U[0];
  P[1] = U[1] / U[0];
  P[2] = U[2];
}
static void fv_cons(const double* P, double* U) {
  U[0] = P[0];
  U[1] = P[0] * P[1];
  U[2] = P[2];
}

/* Per-element face data of the 1D operator: the state on each side's face (ξ = -1: 0, +1: 1),
 * and for FV elements the reconstruction (cell primitives and MinMod slopes) and the
 * difference quotients of (v, c) across the element's two faces. */
typedef struct {
  double Uf[2][3];      /* face states */
  double gf[2][2];      /* FV: (v_x, c_x) across the face; DG: the lifted gradient trace */
  double P[ORC_MAXNP][3], sl[ORC_MAXNP][3];  /* FV: cell primitives, slopes (per unit length) */
} fv_elem_t;

/* the sub-cell scheme's scope: one space dimension, relaxation model II, a valid mesh, beta > 0 */
static int fv_check(const orc_setup* s, const orc_fv_setup* f) {
  if (!s || !f || s->dim != 1 || s->model != 0 || s->N < 1 || s->N >= ORC_MAXNP) return ORC_ERR_ARG;
  if (s->nelem[0] < 1 || !(s->hi[0] > s->lo[0]) || !(s->beta > 0.0)) return ORC_ERR_ARG;
  return ORC_OK;
}

/* DG trace of element e (nodal U[v][E][np]) at side (0: xi = -1, 1: xi = +1) */
static void fv_dg_trace(const mesh_t* m, const double* U, long e, int side, double* Uf) {
  const long nn = m->E * m->np;
  for (int v = 0; v < 3; ++v) Uf[v] = trace(m, U + v * nn, e, 0, 0, side ? +1 : -1);
}

/* The semi-discrete residual of the mixed DG/FV mesh (see the readings above). */
int orc_fv_rhs(const orc_setup* s, const orc_fv_setup* f, const int* fv, const double* U, double* R) {
  int st = fv_check(s, f);
  if (st) return st;
  mesh_t m;
  if ((st = make_mesh(s, &m))) return st;
  const int np = m.np, N = np - 1;
  const long E = m.E, nn = E * np;
  const double h = m.h[0], dx = h / np;
  fv_elem_t* el = (fv_elem_t*)calloc(E, sizeof(fv_elem_t));
  double* Q = (double*)calloc(2 * nn, sizeof(double));  /* DG elements: (v_x, c_x) at the nodes */
  if (!el || !Q) { free(el); free(Q); return ORC_ERR_ARG; }
  for (long i = 0; i < 3 * nn; ++i) {
    R[i] = 0.0;
    if (i < nn && !admissible(U[i])) st = ORC_ERR_NONPHYSICAL;
  }
  const int per = !f->dirichlet;
  /* 1. DG face traces */
  for (long e = 0; e < E; ++e)
    if (!fv[e])
      for (int sd = 0; sd < 2; ++sd) fv_dg_trace(&m, U, e, sd, el[e].Uf[sd]);
  /* 2. FV reconstruction: cell primitives, neighbour values across the element faces, slopes */
  for (long e = 0; e < E; ++e) {
    if (!fv[e]) continue;
    fv_elem_t* x = &el[e];
    for (int j = 0; j < np; ++j) {
      double Uc[3] = {U[e * np + j], U[nn + e * np + j], U[2 * nn + e * np + j]};
      fv_prim(Uc, x->P[j]);
    }
    double Pn[2][3], dn[2];  /* the value beyond each element face and its distance */
    for (int sd = 0; sd < 2; ++sd) {
      const int dir = sd ? +1 : -1;
      const int boundary = !per && ((sd == 0 && e == 0) || (sd == 1 && e == E - 1));
      if (boundary) {
        fv_prim(sd ? f->Ub_hi : f->Ub_lo, Pn[sd]);
        dn[sd] = 0.5 * dx;
        continue;
      }
      const long en = neighbour(&m, e, 0, dir);
      if (fv[en]) {
        const int jn = sd ? 0 : N;
        double Uc[3] = {U[en * np + jn], U[nn + en * np + jn], U[2 * nn + en * np + jn]};
        fv_prim(Uc, Pn[sd]);
        dn[sd] = dx;
      } else {
        double Ut[3];
        fv_dg_trace(&m, U, en, sd ? 0 : 1, Ut);
        fv_prim(Ut, Pn[sd]);
        dn[sd] = 0.5 * dx;
      }
    }
    for (int j = 0; j < np; ++j)
      for (int q = 0; q < 3; ++q) {
        const double left = j > 0 ? (x->P[j][q] - x->P[j - 1][q]) / dx : (x->P[0][q] - Pn[0][q]) / dn[0];
        const double right = j < N ? (x->P[j + 1][q] - x->P[j][q]) / dx : (Pn[1][q] - x->P[N][q]) / dn[1];
        x->sl[j][q] = minmod(left, right);
      }
    double Pl[3], Pr[3];
    for (int q = 0; q < 3; ++q) {
      Pl[q] = x->P[0][q] - 0.5 * dx * x->sl[0][q];
      Pr[q] = x->P[N][q] + 0.5 * dx * x->sl[N][q];
    }
    fv_cons(Pl, x->Uf[0]);
    fv_cons(Pr, x->Uf[1]);
    for (int q = 0; q < 2; ++q) {
      x->gf[0][q] = (x->P[0][1 + q] - Pn[0][1 + q]) / dn[0];
      x->gf[1][q] = (Pn[1][1 + q] - x->P[N][1 + q]) / dn[1];
    }
  }
  /* the state beyond face side sd of element e: the neighbour's face state or the boundary state */
#define FV_OUTER(e, sd)                                                                          \
  ((!per && (sd) == 0 && (e) == 0)       ? f->Ub_lo                                              \
   : (!per && (sd) == 1 && (e) == E - 1) ? f->Ub_hi                                              \
                                         : el[neighbour(&m, (e), 0, (sd) ? +1 : -1)].Uf[(sd) ? 0 : 1])
  /* 3. BR1 lifting of w = (v, c) in the DG elements, central w* with the outer face state */
  for (long e = 0; e < E; ++e) {
    if (fv[e]) continue;
    double ws[2][2];
    for (int sd = 0; sd < 2; ++sd) {
      const double* Uo = FV_OUTER(e, sd);
      const double* Ui = el[e].Uf[sd];
      ws[sd][0] = 0.5 * (Ui[1] / Ui[0] + Uo[1] / Uo[0]);
      ws[sd][1] = 0.5 * (Ui[2] + Uo[2]);
    }
    for (int i = 0; i < np; ++i)
      for (int q = 0; q < 2; ++q) {
        double vol = 0.0;
        for (int j = 0; j < np; ++j) {
          const long p = e * np + j;
          const double wj = q == 0 ? U[nn + p] / U[p] : U[2 * nn + p];
          vol += m.w[j] * wj * m.D[j * np + i];
        }
        const double surf = (ws[1][q] * m.Lp[i] - ws[0][q] * m.Lm[i]) / m.w[i];
        Q[q * nn + e * np + i] = (2.0 / h) * (surf - vol / m.w[i]);
      }
    for (int sd = 0; sd < 2; ++sd)
      for (int q = 0; q < 2; ++q) el[e].gf[sd][q] = trace(&m, Q + q * nn, e, 0, 0, sd ? +1 : -1);
  }
  /* 4. numerical flux (convective minus the mean of the viscous fluxes) on the element faces;
   *    face e sits between elements e - 1 and e (face E: the right boundary, Dirichlet only) */
  const long nfaces = per ? E : E + 1;
  double(*Fh)[3] = (double(*)[3])calloc(nfaces + 1, sizeof(double[3]));
  if (!Fh) { free(el); free(Q); return ORC_ERR_ARG; }
  for (long fc = 0; fc < nfaces; ++fc) {
    const long eR = fc < E ? fc : -1, eL = fc > 0 ? fc - 1 : (per ? E - 1 : -1);
    const double* UL = eL >= 0 ? el[eL].Uf[1] : f->Ub_lo;
    const double* UR = eR >= 0 ? el[eR].Uf[0] : f->Ub_hi;
    const double* gL = eL >= 0 ? el[eL].gf[1] : el[eR].gf[0];
    const double* gR = eR >= 0 ? el[eR].gf[0] : el[eL].gf[1];
    if (!admissible(UL[0]) || !admissible(UR[0])) st = ORC_ERR_NONPHYSICAL;
    double QL[2] = {gL[0], gL[1]}, QR[2] = {gR[0], gR[1]}, fvL[3], fvR[3];
    visc_flux(s, 1, 0, QL, fvL);
    visc_flux(s, 1, 0, QR, fvR);
    numflux(s, 1, 0, UL, UR, Fh[fc]);
    for (int v = 0; v < 3; ++v) Fh[fc][v] -= 0.5 * (fvL[v] + fvR[v]);
  }
  if (per) memcpy(Fh[E], Fh[0], sizeof(double[3]));  /* the right face of element E-1 */
  /* 5. residuals */
  for (long e = 0; e < E; ++e) {
    const double* Fl = Fh[e];
    const double* Fr = Fh[e + 1];
    if (!fv[e]) {
      /* DG: the weak form of Eq. (weakformulation), as in residual() above */
      double F[ORC_MAXNP][3];
      for (int j = 0; j < np; ++j) {
        const long p = e * np + j;
        double Un[3] = {U[p], U[nn + p], U[2 * nn + p]}, Qn[2] = {Q[p], Q[nn + p]}, fc[3], fvv[3];
        conv_flux(s, 1, 0, Un, fc);
        visc_flux(s, 1, 0, Qn, fvv);
        for (int v = 0; v < 3; ++v) F[j][v] = fc[v] - fvv[v];
      }
      for (int i = 0; i < np; ++i) {
        const long p = e * np + i;
        for (int v = 0; v < 3; ++v) {
          double vol = 0.0;
          for (int j = 0; j < np; ++j) vol += m.w[j] * F[j][v] * m.D[j * np + i];
          R[v * nn + p] = (2.0 / h) * (vol / m.w[i] - (Fr[v] * m.Lp[i] - Fl[v] * m.Lm[i]) / m.w[i]);
        }
        R[nn + p] += s->alpha * U[p] * Q[nn + p];
        R[2 * nn + p] += s->alpha / s->beta * (U[p] - U[2 * nn + p]);
      }
    } else {
      /* FV: dU_j/dt = -(F_{j+1/2} - F_{j-1/2}) / dx + S_j over the sub-cells */
      const fv_elem_t* x = &el[e];
      double Fs[ORC_MAXNP + 1][3], gc[ORC_MAXNP + 1];  /* sub-cell face fluxes, c_x on them */
      memcpy(Fs[0], Fl, sizeof(double[3]));
      memcpy(Fs[np], Fr, sizeof(double[3]));
      gc[0] = x->gf[0][1];
      gc[np] = x->gf[1][1];
      for (int j = 0; j < N; ++j) {
        double PL[3], PR[3], UL[3], UR[3], g[2], fvv[3];
        for (int q = 0; q < 3; ++q) {
          PL[q] = x->P[j][q] + 0.5 * dx * x->sl[j][q];
          PR[q] = x->P[j + 1][q] - 0.5 * dx * x->sl[j + 1][q];
        }
        fv_cons(PL, UL);
        fv_cons(PR, UR);
        if (!admissible(UL[0]) || !admissible(UR[0])) st = ORC_ERR_NONPHYSICAL;
        g[0] = (x->P[j + 1][1] - x->P[j][1]) / dx;
        g[1] = (x->P[j + 1][2] - x->P[j][2]) / dx;
        gc[j + 1] = g[1];
        numflux(s, 1, 0, UL, UR, Fs[j + 1]);
        visc_flux(s, 1, 0, g, fvv);
        for (int v = 0; v < 3; ++v) Fs[j + 1][v] -= fvv[v];
      }
      for (int j = 0; j < np; ++j) {
        const long p = e * np + j;
        for (int v = 0; v < 3; ++v) R[v * nn + p] = -(Fs[j + 1][v] - Fs[j][v]) / dx;
        R[nn + p] += s->alpha * U[p] * 0.5 * (gc[j] + gc[j + 1]);
        R[2 * nn + p] += s->alpha / s->beta * (U[p] - U[2 * nn + p]);
      }
    }
  }
#undef FV_OUTER
  free(Fh);
  free(el);
  free(Q);
  return st;
}

/* Indicator of every element (on rho, through the inverse mean matrix for FV elements) and the
 * switches it triggers: DG -> FV above ind_upper, FV -> DG below ind_lower; U converted in place. */
int orc_fv_switch(const orc_setup* s, const orc_fv_setup* f, int* fv, double* U, double* ind) {
  int st = fv_check(s, f);
  if (st) return st;
  const int N = s->N, np = N + 1;
  const long E = s->nelem[0], nn = E * np;
  double M[ORC_MAXNP * ORC_MAXNP], Minv[ORC_MAXNP * ORC_MAXNP];
  if ((st = orc_fv_tables(N, s->node_type, M, Minv))) return st;
  for (long e = 0; e < E; ++e) {
    double rho[ORC_MAXNP];
    for (int i = 0; i < np; ++i) {
      rho[i] = 0.0;
      if (fv[e]) {
        for (int j = 0; j < np; ++j) rho[i] += Minv[i * np + j] * U[e * np + j];
      } else {
        rho[i] = U[e * np + i];
      }
    }
    const double x = orc_persson(N, s->node_type, rho);
    if (ind) ind[e] = x;
    const int to_fv = !fv[e] && x > f->ind_upper, to_dg = fv[e] && x < f->ind_lower;
    if (!to_fv && !to_dg) continue;
    const double* T = to_fv ? M : Minv;
    for (int v = 0; v < 3; ++v) {
      double u[ORC_MAXNP], out[ORC_MAXNP];
      for (int i = 0; i < np; ++i) u[i] = U[v * nn + e * np + i];
      for (int i = 0; i < np; ++i) {
        out[i] = 0.0;
        for (int j = 0; j < np; ++j) out[i] += T[i * np + j] * u[j];
      }
      for (int i = 0; i < np; ++i) U[v * nn + e * np + i] = out[i];
    }
    fv[e] = to_fv;
  }
  return ORC_OK;
}

/* nsteps LSRK4 steps of size dt with the sub-cell scheme: the switches before every step. */
int orc_fv_lsrk4(const orc_setup* s, const orc_fv_setup* f, int* fv, double* U, double dt, int nsteps) {
  int st = fv_check(s, f);
  if (st) return st;
  const long len = 3L * s->nelem[0] * (s->N + 1);
  double* K = (double*)calloc(len, sizeof(double));
  double* R = (double*)malloc(sizeof(double) * len);
  if (!K || !R) { free(K); free(R); return ORC_ERR_ARG; }
  double A[5], B[5], C[5];
  orc_lsrk4_coeffs(A, B, C);
  for (int step = 0; step < nsteps && st == ORC_OK; ++step) {
    st = orc_fv_switch(s, f, fv, U, NULL);
    for (int stage = 0; stage < 5 && st == ORC_OK; ++stage) {
      st = orc_fv_rhs(s, f, fv, U, R);
      if (st) break;
      for (long i = 0; i < len; ++i) {
        K[i] = A[stage] * K[i] + dt * R[i];
        U[i] = U[i] + B[stage] * K[i];
      }
    }
  }
  free(K);
  free(R);
  return st;
}
