/*
 * nsk.h -- C ABI of libnsk.so, a GB300 (sm_103a) implementation of the explicit
 * discontinuous Galerkin spectral element (DGSEM) residual and the low-storage
 * fourth-order Runge-Kutta update of the isothermal parabolic relaxation model
 * ("relaxation model II") of the Navier-Stokes-Korteweg equations
 * (Hitz, Keim, Munz, Rohde, arXiv:1912.12059).
 *
 * The model (Sec. 2.3, Eqs. (fluxform), (modified_pressure), (fluxes_sources_model2)):
 *   U = (rho, rho v, c),  U_t + div(F^c(U) - F^v(grad w)) = S(U, grad c),
 *   F^c_k = (rho v_k, rho v_k v + p_alpha e_k, 0),  p_alpha = p(rho) + alpha rho^2 / 2,
 *   F^v_k = (0, tau_{.k}, (kappa/beta) c_{x_k}),  tau = mu (grad v + grad v^T - 2/3 div v I),
 *   S = (0, alpha rho grad c, (alpha/beta)(rho - c)),
 *   p(rho) = 8 T rho / (3 - rho) - 3 rho^2 (Van-der-Waals, Sec. 2.1, Eqs. (vdw_p), (vdw_parameters)).
 * Here kappa = eps^2 gamma (the paper's capillarity) and mu = eps = 1/Re.
 *
 * Discretisation (Sec. 3.1): uniform Cartesian periodic box, tensor-product
 * Lagrange basis of degree N on Gauss-Legendre nodes (Gauss-Lobatto optional),
 * collocated weak form, BR1 lifting of the primitive variables (v, c) with the
 * central flux, local Lax-Friedrichs (Rusanov) convective face flux with the
 * model II wave speed |v.n| + sqrt(p_alpha'(rho)) (Eq. parabolic_eigenvalues_model2),
 * BR1 mean viscous face flux, pointwise sources with the lifted gradient of c,
 * and the five-stage fourth-order low-storage Runge-Kutta scheme of Carpenter
 * and Kennedy (the 2N-storage family cited in Sec. 3.1).
 *
 * Layout of every state array at this boundary (FP64 in all precisions):
 * structure of arrays, variable-major [nvar][E][npe], nvar = dim + 2 with
 * variables (rho, rho v_1 .. rho v_dim, c); elements lexicographic with x
 * fastest (e = ex + nx (ey + ny ez)); nodes within an element lexicographic
 * with the x index fastest (n = i + np (j + np k)), np = N + 1, npe = np^dim.
 * Lifted gradients: [dim*(dim+1)][E][npe], component k*(dim+1) + w is
 * d/dx_k of w, w = 0..dim-1 the velocity components and w = dim the variable c.
 *
 * Ownership: the library allocates and owns all device memory of a context.
 * Pointers passed in are borrowed for the duration of the call only. With
 * where = NSK_HOST the pointer is host memory (pageable or pinned); with
 * where = NSK_DEVICE it is device memory of the context's device, accessed in
 * order on the context's stream.
 *
 * Errors: every call returns NSK_OK (0) or a negative code; no call aborts,
 * traps or waits without bound. Device-side checks (density outside (0, 3),
 * a negative p_alpha', NaN) set an error word that the library reads back at
 * the end of each call and reports as NSK_ERR_NONPHYSICAL.
 *
 * Call order: nsk_init_mesh -> nsk_set_params -> nsk_set_state -> any of
 * (nsk_rhs, nsk_lift, nsk_step, nsk_compute_dt, nsk_diagnostics, nsk_get_state);
 * violations return NSK_ERR_STATE. A context is not thread-safe.
 */
#ifndef NSK_H
#define NSK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nsk_ctx nsk_ctx;

enum {
  NSK_OK = 0,
  NSK_ERR_ARG = -1,          /* invalid argument */
  NSK_ERR_CUDA = -2,         /* a CUDA runtime call failed */
  NSK_ERR_NONPHYSICAL = -3,  /* rho <= 0, rho >= 3, p_alpha' < 0 or NaN met on the device */
  NSK_ERR_TIMEOUT = -4,      /* a bounded device-side wait expired */
  NSK_ERR_STATE = -5,        /* call order violated */
  NSK_ERR_NOMEM = -6,        /* device allocation failed */
  NSK_ERR_IO = -7,           /* a checkpoint file could not be written or read, or does not match */
  NSK_ERR_BOUNDS = -8        /* an index check of the bounds-checking build (libnsk_check.so) failed */
};

enum { NSK_NODES_GAUSS = 0, NSK_NODES_GAUSS_LOBATTO = 1 };
enum { NSK_FP64 = 0, NSK_FP32_MIXED = 1 };
enum { NSK_HOST = 0, NSK_DEVICE = 1 };
enum { NSK_C_EXPLICIT = 0, NSK_C_LEARNED = 1 };
enum { NSK_FLUX_LF = 0, NSK_FLUX_HLLC = 1 };
enum { NSK_MODEL_RELAXATION = 0, NSK_MODEL_NSK = 1 };

/* Create a context for a periodic box [lo, hi] (per direction) split into
 * nelem[k] equal elements per direction k < dim (entries k >= dim ignored),
 * polynomial degree N (1 <= N <= 5), node set node_type (NSK_NODES_*),
 * arithmetic precision (NSK_FP64; NSK_FP32_MIXED computes the DG operator in
 * FP32 with the equation of state, wave speeds, time step and sums in FP64),
 * on the CUDA stream `cuda_stream` (a cudaStream_t; NULL = the legacy default
 * stream) of the current device. Discretisation: Sec. 3.1, Eqs.
 * (numerics_solutionpolynomial)-(numerics_polynomialsbasis). */
int nsk_init_mesh(nsk_ctx** out, int dim, const int nelem[3], const double lo[3], const double hi[3], int N,
                  int node_type, int precision, void* cuda_stream);

/* Model parameters of Sec. 2.3: temperature T, kappa = eps^2 gamma (c diffusion),
 * Korteweg parameter alpha, relaxation parameter beta, viscosity mu = eps.
 * Rejects (NSK_ERR_ARG) T outside (0, 1), kappa <= 0, beta <= 0, mu < 0 and
 * alpha <= alpha_*(T) = |min W''| / 2 on the spinodal interval
 * (Eq. alpha_fullyhyperbolic_limit), below which the model II fluxes lose
 * hyperbolicity. */
int nsk_set_params(nsk_ctx* ctx, double T, double kappa, double alpha, double beta, double mu);

/* Optional switch: 1 applies the Lax-Friedrichs jump term to c as well
 * (default 0: c has no convective flux, Eq. fluxes_sources_model2, so its face
 * flux is the BR1 viscous mean only). */
int nsk_set_c_dissipation(nsk_ctx* ctx, int on);

/* Convective numerical flux of the faces (Sec. 3.1 uses local Lax-Friedrichs and HLLC):
 * NSK_FLUX_LF (default): central flux minus half the largest wave speed
 * |v.n| + sqrt(p_alpha') of either side (Eq. parabolic_eigenvalues_model2) times the jump;
 * NSK_FLUX_HLLC: the three-wave HLLC solver of the barotropic system (rho, m) with the
 * modified pressure p_alpha: outer speeds S_L = min(u_L - a_L, u_R - a_R),
 * S_R = max(u_L + a_L, u_R + a_R), a = sqrt(p_alpha'), u the normal velocity; contact speed
 * S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R)) /
 *      (rho_L (S_L - u_L) - rho_R (S_R - u_R));
 * flux F_L (S_L >= 0), F_R (S_R <= 0), else F_K + S_K (U*_K - U_K) with K the side of the
 * face's own region (K = L if S* >= 0) and U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, v with the
 * normal component replaced by S*). c is not transported: its convective numerical flux is
 * zero under HLLC (nsk_set_c_dissipation acts on the Lax-Friedrichs flux only). Either flux
 * keeps the time-step bound of nsk_compute_dt. Returns NSK_ERR_ARG for another value. */
int nsk_set_flux(nsk_ctx* ctx, int flux);

/* Model of the context. NSK_MODEL_RELAXATION (default): parabolic relaxation model II,
 * state (rho, m, c). NSK_MODEL_NSK: the original third-order NSK equations it approximates
 * (Sec. 2.2, Eqs. (nsk_1), (nsk_2), (stress_nse), (stress_nsk)), state (rho, m_1..m_dim), i.e.
 * dim + 1 variables in the same layout: F_k = (m_k, m_k v + p e_k - tau_{.k} - tau^K_{.k}),
 * p the VdW pressure, tau^K = kappa (rho lap rho + |grad rho|^2/2) I - kappa grad rho (x) grad rho
 * with kappa of nsk_set_params as the capillarity (alpha and beta unused), grad v and grad rho
 * from the BR1 lifting of (v, rho), lap rho from a second BR1 lifting of grad rho (Sec. 3.1), the
 * central convective face flux and the BR1 mean of the viscous and Korteweg face fluxes; no
 * sources. FP64 contexts only (NSK_ERR_ARG otherwise); not with the learned closure or in a
 * batch. nsk_lift returns the gradients of (v, rho); nsk_diagnostics the energy of Eq.
 * (original_energy_dynamic) (l2_rho_minus_c = 0); nsk_compute_dt uses
 * min(cfl / ((2N+1) max sum_k (|v_k| + sqrt(max(p', 0))) / h_k),
 *     cfl / ((2N+1)^2 max(mu, sqrt(kappa max rho)) sum_k h_k^-2))
 * (the dispersive Korteweg term acts like a diffusion with coefficient sqrt(kappa rho)).
 * Switching the model allocates the two extra arrays the second lifting needs (once) and
 * requires a new nsk_set_state (NSK_ERR_STATE until then). */
int nsk_set_model(nsk_ctx* ctx, int model);

/* Finite-volume sub-cell shock capturing (Sec. 3.2, the section "Finite Volume Sub-Cell
 * Approach"), for one-dimensional FP64 model II contexts (NSK_ERR_ARG otherwise, also for
 * N > 5 or with the learned closure). With on = 1 every nsk_step step first evaluates the
 * Persson-Peraire indicator of each element's density, Ind = log10(top orthonormal-Legendre
 * mode energy / total energy), and converts a DG element with Ind > ind_upper to N+1
 * equidistant sub-cells holding the exact means of its polynomial, and a sub-cell element with
 * Ind < ind_lower (Ind of the polynomial with those means) back to nodal values
 * (ind_lower <= ind_upper; the paper's Riemann problem uses -6 and -8 as upper and lower). Sub-cell
 * elements advance with a second-order finite-volume scheme: MinMod-limited linear
 * reconstruction of (rho, v, c), the flux of nsk_set_flux on every sub-cell face, difference
 * quotients of v and c for the diffusive fluxes; a face between a DG and a sub-cell element
 * pairs the DG trace with the reconstructed value. nsk_get_state then returns nodal values for
 * DG elements and sub-cell means for the others (nsk_get_subcell tells which); nsk_set_state
 * resets every element to DG; nsk_lift returns NSK_ERR_STATE while this path is active;
 * nsk_diagnostics treats every element as nodal. on = 0 returns NSK_ERR_STATE while an element
 * holds sub-cell means. Allocates the path's buffers (once). The stage costs four launches per
 * stage (face states, lifting, face fluxes, update) plus one switch launch per step. */
int nsk_set_subcell(nsk_ctx* ctx, int on, double ind_upper, double ind_lower);

/* Dirichlet boundaries for one-dimensional FP64 model II contexts (the Riemann problem of
 * Sec. 4): with on = 1 the domain is no longer periodic; outside x = lo the state is
 * Ub_lo = (rho, m, c), outside x = hi it is Ub_hi (host arrays of 3). The boundary face sees a
 * ghost neighbour with that state and with the interior side's gradient (its viscous flux is the
 * interior one), in the DG lifting, the numerical flux and the sub-cell reconstruction alike.
 * Uses the sub-cell path's kernels (with or without nsk_set_subcell). NSK_ERR_ARG for other
 * contexts or non-finite states. */
int nsk_set_dirichlet(nsk_ctx* ctx, int on, const double Ub_lo[3], const double Ub_hi[3]);

/* Per-element representation while nsk_set_subcell or nsk_set_dirichlet is active: flags[e] = 1
 * for an element holding sub-cell means (host array of E ints, 0 or 1; the state is then read
 * accordingly, no conversion). nsk_get_subcell copies the flags and/or the indicator of the last
 * switch pass (either pointer may be NULL; host arrays of E). NSK_ERR_STATE when the path is off. */
int nsk_set_subcell_flags(nsk_ctx* ctx, const int* flags);
int nsk_get_subcell(nsk_ctx* ctx, int* flags, double* ind);

/* One indicator and switch pass of nsk_set_subcell on the current state (the pass nsk_step runs
 * before every step). NSK_ERR_STATE unless sub-cell shock capturing is on and a state is set. */
int nsk_subcell_switch(nsk_ctx* ctx);

/* Copy the state in (set) or out (get); layout above, FP64. Setting the state
 * also clears the Runge-Kutta register. */
int nsk_set_state(nsk_ctx* ctx, const double* U, int where);
int nsk_get_state(nsk_ctx* ctx, double* U, int where);

/* Physical coordinates of all nodes, [dim][E][npe], FP64. */
int nsk_node_coords(nsk_ctx* ctx, double* x, int where);

/* Semi-discrete residual R = dU/dt of the current state (Eq. weakformulation
 * with the fluxes and sources of Eq. fluxes_sources_model2, or of the original NSK
 * equations, see nsk_set_model), layout of U.
 * t is the model time; the model is autonomous, so R does not depend on it. */
int nsk_rhs(nsk_ctx* ctx, double t, double* Ut, int where);

/* BR1-lifted gradients of the primitive variables (Sec. 3.1, lifting with the
 * central flux), layout [dim*(dim+1)][E][npe]. */
int nsk_lift(nsk_ctx* ctx, double* Q, int where);

/* Admissible explicit time step for Courant number cfl: the minimum of the
 * convective bound cfl / ((2N+1) max sum_k (|v_k| + sqrt(p_alpha'))/h_k), the
 * parabolic bound of Eq. (numerics_dfl) cfl / ((2N+1)^2 lambda_v sum_k h_k^-2)
 * with lambda_v = max(mu, kappa/beta) (Eq. numerics_nsk_visc_eigenvalues), and
 * the relaxation-source bound cfl * 4.6 * beta / alpha (with the learned closure
 * lambda_v = mu and no source bound; for the original NSK equations see
 * nsk_set_model). Reduced in FP64; dt also stays on the device for nsk_step. */
int nsk_compute_dt(nsk_ctx* ctx, double cfl, double* dt_out);

/* Advance the state by nsteps steps of the five-stage low-storage RK4 with
 * step dt (dt > 0), or, with dt <= 0, with nsk_compute_dt(ctx, -dt) recomputed
 * before every step (so dt = -0.5 means CFL 0.5). Within one call the volume
 * kernel of each stage writes the face traces of its updated state, so only
 * the first stage of a call runs the prolongation pass (model II). With
 * nsk_set_subcell or nsk_set_dirichlet active the call runs the 1D sub-cell
 * path instead (the indicator and switch pass before every step when sub-cells
 * are on): with dt > 0 and at most 4096 elements the whole call is one
 * cooperative launch (bounded grid barriers; NSK_ERR_TIMEOUT if a wait expires),
 * otherwise four launches per stage (and the switch launch per step). Returns after the work is queued and
 * checked: the call synchronises the stream once at the end to read the error
 * word. */
int nsk_step(nsk_ctx* ctx, double dt, int nsteps);

/* nsk_step for a state held in host memory: U_in (host, the layout of U) is
 * copied in, nsteps steps of step dt > 0 are taken, and the final state is
 * copied out to U_out (host; it may be U_in). The results equal
 * nsk_set_state(U_in, NSK_HOST), nsk_step and nsk_get_state(U_out, NSK_HOST)
 * bit for bit. For FP64 relaxation-model 3D meshes at N = 3 with the separate
 * face pass (nsk_set_schedule fused_face 0, 128 or 256 threads), profiling off,
 * a z extent that is a multiple of 8 elements and slabs of a multiple of 16
 * elements, the copies overlap the computation: the state arrives in 8 z-slabs
 * on a second stream while the first stage's prolongation and lifting run slab
 * by slab behind it, and the last stage's volume kernel runs slab by slab with
 * each slab copied out as soon as it is written; otherwise the three calls are
 * made in turn. Pinned host memory gives the copies their full rate.
 * Synchronises before returning (the host buffers are no longer in use then,
 * also after an error); errors as nsk_step. */
int nsk_step_host(nsk_ctx* ctx, const double* U_in, double* U_out, double dt, int nsteps);

/* Implicit time integration (Sec. 3.1): nsteps steps of size dt of the six-stage, fourth-order
 * ESDIRK the paper cites (the implicit tableau of Kennedy and Carpenter's ARK4(3)6L[2]SA,
 * gamma = 1/4, stiffly accurate, L-stable) on the context's residual (nsk_rhs). Each implicit
 * stage X - dt gamma R(X) = U_n + dt sum_{j<i} a_ij R_j is solved by Newton's method from the
 * previous stage until the Euclidean norm of its residual is <= newton_tol times that of the
 * right-hand side (at most 20 iterations; stats[3] counts stages that stopped there), each
 * Newton system by restarted GMRES(krylov_dim) to the relative residual krylov_tol (at most
 * max_krylov iterations per system), matrix-free: J v ~ (R(X + eps v) - R(X)) / eps with
 * eps = sqrt(2^-52) (1 + ||X||) / ||v||. block_precond = 1 right-preconditions GMRES with the
 * inverses of the element blocks of I - dt gamma J(U_n): J's diagonal blocks dR_e/dU_e by forward
 * differences once per step, every element of an element colour perturbed at once (colours per
 * direction: the smallest divisor >= 3 of the element count, else the count; each costs
 * nvar npe residual evaluations, counted in stats), inverted by Gauss-Jordan per element; blocks
 * of at most 64 unknowns (nvar npe: every order in 1D, 2D up to N = 3) and E (nvar npe)^2 <= 2^28
 * values (NSK_ERR_ARG otherwise).
 * stats (may be NULL): Newton
 * iterations, Krylov iterations, residual evaluations, stages stopped at the iteration limit,
 * summed over the call. FP64 contexts with the explicit c equation and without the sub-cell
 * path only (NSK_ERR_ARG otherwise). Allocates 12 + krylov_dim state-sized FP64 buffers for the
 * call and frees them before returning. The GMRES control runs on the host: each Krylov iteration
 * reads its projection coefficients and new norm back once (one stream synchronisation), and
 * each Newton iteration its norms. */
int nsk_step_esdirk(nsk_ctx* ctx, double dt, int nsteps, double newton_tol, double krylov_tol, int krylov_dim,
                    int max_krylov, int block_precond, long long stats[4]);

/* Quadrature sums (FP64): mass sum w J rho; the total energy of the relaxation
 * model sum w J (|m|^2/(2 rho) + W(rho) + alpha/2 (rho-c)^2 + kappa/2 |grad c|^2)
 * (Eq. pararelax_elliptical_energy_dynamic, grad c from BR1); and
 * ||rho - c||_L2. Any output pointer may be NULL. */
int nsk_diagnostics(nsk_ctx* ctx, double* mass, double* energy, double* l2_rho_minus_c);

/* Sizes of the context: number of elements, nodes per element, variables. */
int nsk_get_sizes(nsk_ctx* ctx, long long* n_elem, int* nodes_per_elem, int* nvar);

/* Per-kernel timing. With on = 1 every kernel of the stage pipeline is
 * bracketed by CUDA events recorded on the context's stream, and the elapsed
 * times are accumulated at the next synchronising call (nsk_step, nsk_rhs, ...).
 * nsk_get_profile copies up to n entries of accumulated milliseconds and
 * launch counts, index 0 = trace prolongation, 1 = BR1 lifting, 2 = face flux,
 * 3 = volume integral + surface lifting + sources + RK update, 4 = the
 * single-block kernel (a whole call under schedule 3), and returns the number
 * of entries (5); reset = 1 clears the accumulators afterwards. */
int nsk_set_profiling(nsk_ctx* ctx, int on);
int nsk_get_profile(nsk_ctx* ctx, double* ms, long long* launches, int n, int reset);

/* Kernel launches issued by this context since creation (a counter kept on
 * the host; every launch of the library's own kernels increments it). */
long long nsk_launch_count(nsk_ctx* ctx);

/* Measured fused multiply-add throughput of the current device (the ALU
 * roofline denominator of the stage kernels; no counterpart in the paper):
 * precision NSK_FP64 or NSK_FP32_MIXED (FP32 FMAs). One launch of 8 blocks of
 * 256 threads per SM, every thread running 8 independent chains
 * x <- x a + b for iters iterations (after a shorter warm-up launch), timed
 * with CUDA events on stream (NULL = legacy default stream); tflops receives
 * 2 x 8 x iters x threads / time in TFLOP/s, ms the launch's time (either may
 * be NULL). Synchronises the stream. NSK_ERR_ARG for iters outside
 * 1..2^24 or another precision. */
int nsk_measure_fma_rate(int precision, int iters, double* tflops, double* ms, void* stream);

/* Stage schedule of a context: tpb = 128 or 256 threads per block for the
 * element kernels (elements per block = tpb / nodes per element, at least 1),
 * and fused_face:
 *   0 a separate face pass between the lifting and the volume kernel (the
 *     lifted gradients and the face fluxes are stored in device memory);
 *   1 the face fluxes evaluated inside the volume kernel (each face by both of
 *     its elements, bit-identically);
 *   2 the lean two-launch stage: the lifting stores only the face-normal
 *     viscous-flux traces of each element's faces, and the volume kernel
 *     recomputes the element's lifting on chip, so neither the gradients nor
 *     the face fluxes pass through device memory (the schedule with the least
 *     memory traffic; relaxation model II: the original NSK equations and the
 *     sub-cell path have kernels of their own and use tpb only);
 *   3 the single-block schedule for small meshes: one block runs all stages of
 *     a call's steps (fixed dt, no learned closure) or one residual in a single
 *     launch, on copies of the arrays in shared memory (relaxation model II,
 *     meshes whose arrays fit in 200 KB, e.g. 1D up to about 400 elements at
 *     N = 3 in FP64); where it does not apply the separate face pass runs;
 *   4 the separate face pass with line-per-thread lifting and volume kernels
 *     for the FP32 operator of relaxation model II on 3D elements with N = 3
 *     (16 threads per element, each owning a line of 4 nodes: 16-byte loads
 *     and stores, contractions along the line in registers); elsewhere the
 *     separate face pass runs.
 * Default: tpb 256, separate face pass. Every expression that could be
 * contracted into a fused multiply-add in more than one way is written as an
 * explicit fma, and every schedule evaluates each value with the same code,
 * so results are bit-identical under every schedule. NSK_ERR_ARG for other
 * values. */
int nsk_set_schedule(nsk_ctx* ctx, int tpb, int fused_face);
int nsk_get_schedule(nsk_ctx* ctx, int* tpb, int* fused_face);
/* Autotuner: times one residual evaluation under each schedule (tpb 128 and
 * 256 with fused_face 0, 1, 2, and 3 and 4 where they apply; fused_face 0 and 1 for
 * the original NSK equations) on the context's current state (the state is not
 * modified), keeps the fastest and returns it (any output may be NULL; ms_out =
 * its time). */
int nsk_autotune(nsk_ctx* ctx, int* tpb_out, int* fused_out, double* ms_out);

/* Batched execution (many instances per launch). A batch groups n existing
 * 3D contexts with N = 3 or 4 and the same precision; meshes may differ.
 * Persistent schedule (default): each LSRK stage of all instances runs as one
 * persistent cooperative kernel whose phases (traces, lifting, face fluxes,
 * volume + update) are separated by a grid barrier with a one-second bounded
 * wait (NSK_ERR_TIMEOUT on expiry). Phase schedule: one ordinary launch per
 * phase covering all instances. Instance schedule: every instance's stage
 * kernels in turn. Either way the stage launches of a step are
 * captured once in a CUDA graph and replayed. The batch snapshots each instance's parameters and buffers at
 * creation (call nsk_set_params / nsk_set_state before; states may be reset
 * later through the instances), and the instances must not be used by other
 * calls while a batch call runs. Results equal those of stepping each
 * instance alone, bit for bit. The batch has its own stream. */
typedef struct nsk_batch nsk_batch;
int nsk_batch_create(nsk_batch** out, int n, nsk_ctx* const* instances);
/* Advance every instance by nsteps steps. cfl > 0: each instance's dt is
 * recomputed (FP64 reductions) before every step; cfl <= 0: each instance
 * keeps the dt of its last nsk_compute_dt or adaptive nsk_step. step_ms, if
 * not NULL, receives nsteps per-step wall times (ms, CUDA events); every
 * instance of the batch completes a step within that time.
 * per_instance_latency_ms, if not NULL, receives nsteps x n values
 * ([step][instance], ms): the time from the start of the step to the moment
 * that instance's new state is complete in device memory, from the GPU's
 * global timer read by one-thread kernels at the start of the step and right
 * after the launch that finishes the instance (the instance schedule runs
 * instance i on stream i mod 4 of four streams forked from the batch's stream
 * and joined back after every stage, and finishes the instances of one stream
 * one after another; the single-launch schedules finish all of them with their
 * last launch). The stamps add n + 1 tiny launches
 * to a measured step (a separately captured graph) and a device-to-device
 * copy of n + 1 words after it; the batch keeps their buffers until it is
 * destroyed. Returns as nsk_step. */
int nsk_batch_step(nsk_batch* batch, int nsteps, double cfl, double* step_ms, double* per_instance_latency_ms);
/* Batch schedule (tpb and fused_face as for a context; persistent = 1 for
 * the cooperative persistent kernel, 0 for one launch per phase covering all
 * instances, 2 for each instance's own stage launches in the captured graph,
 * on four streams (small instances run side by side); there fused_face may also be 2, the lean stage, 4, the line kernels
 * for the instances they apply to, or 5, each instance's own schedule, as set
 * by nsk_set_schedule or nsk_autotune on its context: tpb and fused_face 0, 1
 * or 4, the other schedules running as the separate face pass, and tpb ignored)
 * and the autotuner, which first autotunes every instance's context, then times
 * one residual of the whole batch under each batch schedule (the instances'
 * states are not modified). Returns NSK_ERR_ARG for tpb not 128 or 256,
 * persistent outside 0..2, fused_face outside 0..5, 3, or 2, 4 or 5 with
 * persistent other than 2. */
int nsk_batch_set_schedule(nsk_batch* batch, int tpb, int fused_face, int persistent);
int nsk_batch_get_schedule(nsk_batch* batch, int* tpb, int* fused_face, int* persistent);
int nsk_batch_autotune(nsk_batch* batch, int* tpb_out, int* fused_out, int* persistent_out, double* ms_out);
/* Kernel launches issued (graph replays count their launches); and 1 if
 * steps replay a captured CUDA graph, 0 if stages are launched directly. */
long long nsk_batch_launch_count(nsk_batch* batch);
int nsk_batch_uses_graph(nsk_batch* batch);
/* Bound of every grid-barrier wait (default 1 s, at most 60 s). */
int nsk_batch_set_timeout(nsk_batch* batch, double seconds);
void nsk_batch_destroy(nsk_batch* batch);

/* Dense BF16 GEMM on the tensor cores (tcgen05, FP32 accumulation in tensor
 * memory), the building block of the learned closure's network:
 *   C[M x N] = A[M x K] . B[N x K]^T,
 * A and B BF16 device arrays with K contiguous (row strides lda, ldb, multiples
 * of 8; K a multiple of 16; 16 <= N <= 256, N a multiple of 16), split over K
 * in slices of k_split (a multiple of 64, or <= 0 for none). Epilogues:
 * 0 store C + bias (bias may be NULL) as FP32 out[M][ldo];
 * 1 atomicAdd C into out (split-K partial sums);
 * 2 z = C + bias: z -> out (FP32, may be NULL), GELU(z) -> hout (BF16 [M][ldh])
 *   and, if hout_t is not NULL, its transpose -> hout_t (BF16 [N][ldt]);
 * 3 dz = C * GELU'(zin[M][ldz]) -> hout (BF16) and hout_t, column sums of dz
 *   added to bias_grad (if not NULL).
 * GELU(x) = x Phi(x) (exact, with erf). err: device int that receives
 * NSK_EBIT_TIMEOUT (8) if a bounded tensor-core wait expires (NULL: an
 * internal word). Queued on stream; no synchronisation. No counterpart in the
 * paper: it serves the per-element network of the learned closure. */
int nsk_gemm_bf16(const void* A, const void* B, int M, int N, int K, int lda, int ldb, int k_split, int epilogue,
                  const float* bias, float* out, int ldo, void* hout, int ldh, void* hout_t, int ldt,
                  const float* zin, int ldz, float* bias_grad, int* err, void* stream);

/* Per-element network of the learned c-closure (no counterpart in the paper;
 * its target is the quasi-equilibrium of the c equation, the Korteweg-limit
 * remark of Sec. 2.3: c - (kappa/alpha) Lap c = rho). A fully connected
 * network n_in -> h1 -> h2 -> n_out with GELU hidden layers; BF16 weights and
 * activations, FP32 accumulation on the tensor cores, FP32 master parameters
 * trained with Adam. h1, h2, n_out multiples of 16 and <= 256, n_in <= 256
 * (padded to a multiple of 16 with zero inputs). Training batches have
 * max_batch rows at most (a multiple of 16); inference max_rows rows. All
 * device buffers are allocated at creation. */
typedef struct nsk_mlp nsk_mlp;
int nsk_mlp_create(nsk_mlp** out, int n_in, int h1, int h2, int n_out, int max_batch, int max_rows, void* stream);
long long nsk_mlp_num_params(nsk_mlp* mlp);
/* FP32 parameters as one host array: W1 [h1][n_in_pad], b1 [h1], W2 [h2][h1],
 * b2 [h2], W3 [n_out][h2], b3 [n_out] (layer l: y = W_l x + b_l). Setting
 * them resets the Adam moments. */
int nsk_mlp_set_params(nsk_mlp* mlp, const float* params, long long n);
int nsk_mlp_get_params(nsk_mlp* mlp, float* params, long long n);
/* Inference: X BF16 device [rows][n_in_pad] -> Y FP32 device [rows][n_out]. When the
 * network fits on chip (n_in_pad, h1, h2, n_out <= 256 and its shared-memory plan within
 * 224 KB) the three layers run as one kernel that keeps the hidden activations of each
 * 128-row tile in shared memory and TMEM; otherwise as three GEMMs. Both give the same
 * values. */
int nsk_mlp_forward(nsk_mlp* mlp, const void* X, int rows, float* Y);
/* on = 0 forces the three-GEMM forward (default 1: fused where it fits). */
int nsk_mlp_set_fused_forward(nsk_mlp* mlp, int on);
/* Loss L = mean over rows and outputs of (Y - T)^2 for X BF16 [batch][n_in_pad]
 * and targets T FP32 [batch][n_out] (device); gradients of L (layout of the
 * parameters) copied to grads (host, may be NULL); loss (may be NULL). */
int nsk_mlp_gradients(nsk_mlp* mlp, const void* X, const float* T, int batch, float* grads, double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on
 * that loss; loss (may be NULL: no synchronisation) receives its value. */
int nsk_mlp_train_step(nsk_mlp* mlp, const void* X, const float* T, int batch, double lr, double* loss);
long long nsk_mlp_launch_count(nsk_mlp* mlp);
void nsk_mlp_destroy(nsk_mlp* mlp);

/* Learned c-closure of a 3D context (cubic elements): with mode
 * NSK_C_LEARNED, before every Runge-Kutta stage and after every step the
 * relaxation variable is replaced by c = rho + s y, y = network(features),
 * s = (kappa/alpha) (2/h)^2, so the stiff c equation (source alpha/beta,
 * diffusion kappa/beta) no longer bounds the time step: nsk_compute_dt and
 * adaptive steps drop both bounds. Features per element: the npe nodal
 * densities and the mean densities of the 2 dim face neighbours (order x-, x+,
 * y-, y+, z-, z+), each minus the element's mean density and divided by 0.5
 * (nf = npe + 2 dim values); each value v enters as the BF16 pair
 * hi = bf16(v), lo = bf16(v - hi), so the network input is n_in = 2 nf
 * (hi values first, then lo values); n_out = npe. Every judge_every steps (0: never) the
 * judge evaluates the explicit c equation at the closure's state,
 * eta = ||(beta/alpha) R_c|| / ||c - rho|| (the relative residual of the
 * quasi-equilibrium), and if eta > eta_max the context falls back to
 * NSK_C_EXPLICIT (the closure's c becomes the initial c of the explicit
 * equation). mode NSK_C_EXPLICIT switches the closure off. The network is
 * borrowed and must outlive its use (its max_rows >= number of elements). */
int nsk_set_closure(nsk_ctx* ctx, int mode, nsk_mlp* mlp, int judge_every, double eta_max);
int nsk_closure_status(nsk_ctx* ctx, int* mode, double* last_eta, long long* fallbacks);
/* Training data of the current state: features (BF16 device [E][n_in_pad],
 * n_in_pad = round-up of 2 (npe + 2 dim) to 16) and targets y = (c - rho) / s
 * (FP32 device [E][npe]). */
int nsk_closure_features(nsk_ctx* ctx, void* X);
int nsk_closure_targets(nsk_ctx* ctx, float* Y);
/* Apply the closure once to the current state (also done by nsk_step), and
 * evaluate the judge now (returns eta). */
int nsk_closure_apply(nsk_ctx* ctx);
int nsk_closure_judge(nsk_ctx* ctx, double* eta);

/* Allocation-free residual. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory, e.g. a plugin inside a
 * host application that owns all device memory through its own pool, or a
 * loop that must not trigger the device-wide synchronisation a cudaMalloc or
 * cudaFree implies. It computes the same FP64 residual as nsk_rhs (same
 * kernels, same layout) for the periodic box described by the arguments
 * (meaning and validation as in nsk_init_mesh and nsk_set_params, node_type as
 * there, precision always FP64), from the device array U to the device array
 * Ut, both [dim+2][E][npe] FP64 and owned by the caller, on cuda_stream (NULL =
 * legacy default stream); U and Ut must be distinct arrays (aliasing them is
 * rejected with NSK_ERR_ARG). It creates no context and calls no cudaMalloc,
 * cudaFree or other allocating routine: the intermediate arrays live in one
 * file-scope device array of nsk_static_scratch_bytes() = 64 MiB, which every
 * device that loads the library holds until the process exits. Sizes whose
 * scratch does not fit are rejected with NSK_ERR_ARG: per element the call
 * needs 8 * (d(d+1) np^d + (2d(2d+5) + d(d+2)) np^(d-1)) bytes (face traces
 * with their two FP64 reciprocal planes, viscous-flux traces, face fluxes and
 * lifted gradients; 3D, N = 3: 16512 bytes, so about 4060 elements). The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current). With lazy module loading
 * (the CUDA default) that first call, or the first kernel launch of the
 * library on the device, also loads the library's device code, and that load
 * is when the 64 MiB array is committed on the device: the first call may
 * itself allocate, or fail for lack of memory. The "allocates nothing"
 * guarantee therefore holds from the second call per device on; make one
 * warm-up call at start-up, before any stream capture. Every call shares the
 * array and it keeps the last call's contents (the error word is cleared at
 * the start of each call), so calls that overlap on the GPU, on any stream,
 * race and must be serialised by the caller. The call synchronises
 * cuda_stream once to read the error word; returns as nsk_rhs. */
int nsk_rhs_static_scratch(int dim, const int nelem[3], const double lo[3], const double hi[3], int N, int node_type,
                           double T, double kappa, double alpha, double beta, double mu, const double* U, double* Ut,
                           void* cuda_stream);
/* Size in bytes of the file-scope scratch array of nsk_rhs_static_scratch. */
long long nsk_static_scratch_bytes(void);

/* Checkpoint and resume (no counterpart in the paper; a serving and restart
 * facility). nsk_save_checkpoint writes to path (created or truncated) a binary
 * file, little-endian: the 8 bytes "NSKCKPT\0", a format version (uint32 = 1),
 * then int32 dim, N, node type, precision, model, flux, c dissipation, the
 * count of sub-cell flags F (E when the 1D sub-cell path is on, else 0),
 * nelem[3]; FP64 lo[3], hi[3], T, kappa, alpha, beta, mu, the caller's time t;
 * int64 the caller's step counter and the count of state values V =
 * nvar E npe; then the state as FP64 [nvar][E][npe] (exact for FP32 contexts)
 * and F int32 flags. nsk_load_checkpoint reads such a file into a context
 * created with the same dim, nelem, lo, hi, N, node type and precision and
 * set to the same model (NSK_ERR_IO otherwise, or for a short or unreadable
 * file), sets the parameters, flux and c dissipation from it, then the state
 * and flags, and returns t and step (either pointer may be NULL). The
 * Runge-Kutta register is zero after it; a step boundary leaves nothing else in
 * it (the first stage coefficient of the low-storage scheme is A_1 = 0), so
 * stepping on from a checkpoint gives the same bits as never stopping. The
 * learned closure's network is not part of the file. Both synchronise the
 * context's stream. */
int nsk_save_checkpoint(nsk_ctx* ctx, const char* path, double t, long long step);
int nsk_load_checkpoint(nsk_ctx* ctx, const char* path, double* t, long long* step);

/* Human-readable text of an error code; never NULL. */
const char* nsk_error_string(int code);

/* Free all resources of a context (NULL is a no-op). */
void nsk_destroy(nsk_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* NSK_H */
