/*
 * nsk_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU reference of the explicit DGSEM discretisation of the
 * isothermal parabolic relaxation model ("relaxation model II") of the
 * Navier-Stokes-Korteweg equations (Hitz, Keim, Munz, Rohde, arXiv:1912.12059):
 *   - Sec. 2.1, Eqs. (vdw_freeenergy), (vdw_p), (vdw_parameters): Van-der-Waals EoS;
 *   - Sec. 2.3, Eqs. (modified_pressure), (fluxes_sources_model2),
 *     (parabolic_eigenvalues_model2), (alpha_fullyhyperbolic_limit): model II;
 *   - Sec. 3.1, Eqs. (solutionpolynomial)-(weakformulation): weak-form DGSEM on
 *     Gauss-Legendre (or Gauss-Lobatto) nodes, BR1 lifting of the primitive
 *     variables with the central flux, local Lax-Friedrichs (Rusanov) flux;
 *   - Sec. 3.1, Eq. (numerics_dfl): the parabolic time-step restriction;
 *   - Sec. 3.1: explicit fourth-order five-stage low-storage Runge-Kutta.
 *
 * Only the test suite, the package's smoke check and the CPU-baseline leg of
 * the benchmark may load this library. The product (the CUDA library) never
 * includes this header and shares no code with it.
 *
 * Layout of every nodal array (the same canonical layout the product uses at
 * its boundary, defined independently there): variable-major, then element
 * (lexicographic, x fastest), then node within the element (lexicographic,
 * index along x fastest). nVar = dim + 2: (rho, rho*v_1..rho*v_dim, c).
 * Lifted gradients Q: component (k*(dim+1) + w) holds d/dx_k of primitive
 * variable w, w = 0..dim-1 the velocity components, w = dim the variable c.
 */
#ifndef NSK_ORACLE_H
#define NSK_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dim;            /* 1, 2 or 3 */
  int nelem[3];       /* elements per direction; unused directions must be 1 */
  double lo[3], hi[3];/* periodic box */
  int N;              /* polynomial degree, 1..15 */
  int node_type;      /* 0 = Gauss-Legendre (the paper's nodes), 1 = Gauss-Lobatto */
  double T;           /* reduced temperature */
  double kappa;       /* capillarity eps^2*gamma of the c equation */
  double alpha;       /* Korteweg (relaxation) parameter */
  double beta;        /* parabolic relaxation parameter */
  double mu;          /* viscosity eps = 1/Re */
  int c_dissipation;  /* 0: Lax-Friedrichs jump acts on rho and momentum only; 1: on c too */
  int flux;           /* convective numerical flux: 0 = local Lax-Friedrichs, 1 = HLLC */
  int model;          /* 0 = relaxation model II (state rho, m, c); 1 = original NSK, Sec. 2.2
                         Eqs. (nsk_1), (nsk_2), (stress_nse), (stress_nsk) (state rho, m; kappa is
                         the capillarity of the Korteweg stress; alpha, beta, flux unused) */
} orc_setup;

/* Van-der-Waals EoS with the reduced parameters a=3, b=1/3, R=8/3. */
double orc_pressure(double T, double rho);
double orc_dpressure(double T, double rho);
double orc_free_energy(double T, double rho);
double orc_chem_potential(double T, double rho);
/* Saturation (Maxwell) densities; returns 0 on convergence. */
int orc_maxwell(double T, double* rho_vap, double* rho_liq, double* p_sat);
/* Spinodal densities (roots of p') and alpha_* = |min W''|/2 on the spinodal interval. */
int orc_spinodal(double T, double* rho_sv, double* rho_sl, double* alpha_star);
/* Young-Laplace-adjusted phase densities of a spherical droplet of radius r. */
int orc_young_laplace(double T, double sigma, double r, double* rho_liq, double* rho_vap);

/* 1D nodal tables: nodes xi[N+1], weights w[N+1], derivative matrix D[i*(N+1)+j] = l_j'(xi_i),
 * boundary values Lm[j] = l_j(-1), Lp[j] = l_j(+1). */
int orc_nodes(int N, int node_type, double* xi, double* w);
void orc_lagrange_tables(int N, const double* xi, double* D, double* Lm, double* Lp);
double orc_lagrange_eval(int N, const double* xi, int j, double x);

/* Carpenter-Kennedy RK4(3)5[2N] coefficients A[5], B[5], C[5]. */
void orc_lsrk4_coeffs(double* A, double* B, double* C);

/* Lifted gradients (BR1) of the primitive variables: Q[dim*(dim+1)][E][npe]. */
int orc_lift(const orc_setup* s, const double* U, double* Q);
/* Original NSK only: the second BR1 lifting (Sec. 3.1, the Q_2 equation), Q2 = div(grad rho)
 * from the lifted density gradient, [E][npe]. */
int orc_lift2(const orc_setup* s, const double* U, double* Q2);
/* Semi-discrete residual R = dU/dt (same layout as U). */
int orc_rhs(const orc_setup* s, const double* U, double* R);
/* Convective numerical flux (LF or HLLC per s->flux) of one face with normal +e_k between the
 * states UL (left) and UR (right), each (rho, m_1..m_dim, c); F has dim + 2 entries. */
int orc_numflux(const orc_setup* s, int k, const double* UL, const double* UR, double* F);
/* Advance U by nsteps explicit LSRK4 steps of size dt (in place). */
int orc_lsrk4(const orc_setup* s, double* U, double dt, int nsteps);
/* Admissible explicit time step (convective, viscous and source limits). */
int orc_timestep(const orc_setup* s, const double* U, double cfl, double* dt);
/* Quadrature sums: mass, total energy of the relaxation model, ||rho-c||_L2. */
int orc_diagnostics(const orc_setup* s, const double* U, double* mass, double* energy, double* l2_rho_c);

/* Finite-volume sub-cell shock capturing and Dirichlet boundaries (Sec. 3.2, the sub-cell
 * section; the 1D sharp-interface Riemann problem of Sec. 4), model II, dim = 1 only.
 * fv[e] = 1 marks an element holding N+1 equidistant sub-cell means instead of nodal values. */
typedef struct {
  int dirichlet;                /* 0: periodic; 1: the boundary states below outside lo and hi */
  double Ub_lo[3], Ub_hi[3];    /* (rho, m, c) */
  double ind_upper, ind_lower;  /* Persson indicator thresholds (log10): DG -> FV, FV -> DG */
} orc_fv_setup;
/* M[j][i]: mean of the nodal basis function l_i over sub-cell j; Minv = M^-1 (may be NULL). */
int orc_fv_tables(int N, int node_type, double* M, double* Minv);
/* log10 of the highest orthonormal-Legendre mode's share of the energy of nodal values u. */
double orc_persson(int N, int node_type, const double* u);
/* Residual of the mixed DG/FV mesh (same layout as U; FV elements hold means). */
int orc_fv_rhs(const orc_setup* s, const orc_fv_setup* f, const int* fv, const double* U, double* R);
/* Indicator per element (ind may be NULL) and the DG <-> FV switches it triggers, in place. */
int orc_fv_switch(const orc_setup* s, const orc_fv_setup* f, int* fv, double* U, double* ind);
/* nsteps LSRK4 steps with the switches before each step. */
int orc_fv_lsrk4(const orc_setup* s, const orc_fv_setup* f, int* fv, double* U, double dt, int nsteps);

/* Threads of this build: 1 for the plain library, the OpenMP team size for the
 * OpenMP build of the timed CPU baseline (same source, same results bit for bit). */
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
