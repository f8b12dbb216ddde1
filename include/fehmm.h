/*
 * fehmm.h -- C ABI of the GB300 batched FE-HMM / FE^2 periodic-RVE engine.
 *
 * Method: Eidel, Fischer, Gote, "A Nonlinear Finite Element Heterogeneous Multiscale
 * Method for the Homogenization of Hyperelastic Solids and a Novel Staggered Two-Scale
 * Solution Algorithm" (arXiv:1908.08292).  At every macro quadrature point a periodic
 * representative volume element (RVE) is solved by Newton's method; it returns the
 * homogenised first Piola-Kirchhoff stress Pbar = <P> (Eq. Average-of-P-and-F) and the
 * homogenised tangent Abar = dPbar/dFbar, which the macro problem assembles into its
 * residual and tangent (Sec. 3.1-3.3).
 *
 * Conventions
 *  - Every function returns an int status: FEHMM_OK (0), a negative FEHMM_ERR_* code on an
 *    API error, or (fehmm_rve_solve only) a positive count of quadrature points whose RVE
 *    did not converge.  No exception crosses this boundary.  fehmm_status_str() names codes.
 *  - Tensors are row-major: a d x d tensor T_iJ is stored at [i*d + J]; a fourth-order
 *    tangent A_iJkL at [(i*d + J)*d*d + (k*d + L)].  Floating point data are FP64.
 *  - "device" pointers are CUDA device (or managed) memory owned by the CALLER; "host"
 *    pointers are ordinary host memory.  The library copies what it needs from host
 *    arrays during the call and keeps no caller pointer after it returns.
 *  - The context owns its device state: microstructures, the per-qp fluctuation fields
 *    (current and committed), the macro mesh tables and scratch.  One context may be used
 *    from one host thread at a time.
 *  - Calls taking a stream enqueue asynchronous work on it (a cudaStream_t passed as
 *    void*; NULL = legacy default stream); their outputs are valid once the stream has
 *    been synchronised.  Argument errors are reported synchronously; CUDA launch errors
 *    are reported as FEHMM_ERR_CUDA.
 *  - Micro RVE: the periodic unit cell [0,1]^dim split into n^dim Q1 (dim = 2, plane
 *    strain) or Hex8 (dim = 3) elements; element (i,j[,k]) has index i + n*j (+ n*n*k);
 *    node (i,j[,k]) likewise; the fluctuation of node 0 is pinned to zero.
 *  - Macro mesh: [0,1]^dim split into nx x ny (x nz) Q1/Hex8 elements with 2^dim Gauss
 *    points; node (i,j[,k]) has index i + (nx+1)*j (+ (nx+1)*(ny+1)*k), dof = node*dim + c;
 *    quadrature point q = element*2^dim + g with Gauss points ordered xi_1 fastest.
 */
#ifndef FEHMM_H
#define FEHMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fehmm_ctx fehmm_ctx;

enum {
  FEHMM_OK = 0,
  FEHMM_ERR_ARG = -1,          /* invalid argument (null pointer, size out of range) */
  FEHMM_ERR_CUDA = -2,         /* a CUDA runtime call or kernel launch failed */
  FEHMM_ERR_OOM = -3,          /* device allocation failed */
  FEHMM_ERR_STATE = -4,        /* call out of order (e.g. solve before bind_qps) */
  FEHMM_ERR_UNSUPPORTED = -5,  /* valid but unsupported configuration (e.g. odd 2D grid) */
  FEHMM_ERR_TOO_LARGE = -6     /* size beyond the fixed static scratch of the no-allocation entry */
};

enum { FEHMM_PREC_FP64 = 0, FEHMM_PREC_MIXED = 1 };

/* Preconditioner of the RVE PCG solves (fehmm_options.precond). */
enum { FEHMM_PRECOND_BLOCK_JACOBI = 0, FEHMM_PRECOND_MULTIGRID = 1 };

/* Coupling of the RVE to the macro deformation (fehmm_options.bc), Sec. 3.2: periodic
 * fluctuations (the paper's choice; the fluctuation of node 0 is pinned), or kinematically
 * uniform boundary conditions (KUBC: u = (Fbar - I) X on the whole cell boundary, i.e. zero
 * fluctuation on every node of the planes x_c = 0 of the node lattice, which the periodic
 * lattice shares with x_c = 1; the modelling error of this coupling is the boundary-layer term
 * of Eq. ModelingError). */
enum { FEHMM_BC_PERIODIC = 0, FEHMM_BC_KUBC = 1 };

/* Constitutive law of every phase (fehmm_options.law): the compressible neo-Hookean law of the
 * paper's Sec. 6 (Eq. NH-free-energy), or the St. Venant-Kirchhoff law (linear elasticity with
 * geometric nonlinearity, the paper's second material case in Sec. 6): psi = lam/2 (tr E)^2 +
 * mu E:E, S = lam tr(E) I + 2 mu E, E = (F^T F - I)/2. */
enum { FEHMM_LAW_NEO_HOOKE = 0, FEHMM_LAW_SVK = 1 };

/* Per-quadrature-point RVE status written by fehmm_rve_solve. */
enum {
  FEHMM_RVE_OK = 0,            /* Newton converged */
  FEHMM_RVE_NEWTON_CAP = 1,    /* iteration cap reached before the tolerance */
  FEHMM_RVE_J_NONPOS = 2,      /* det F <= 0 at some Gauss point (ln J undefined) */
  FEHMM_RVE_PCG_BREAKDOWN = 3, /* p^T K p <= 0 in the linear solver (tangent not SPD) */
  FEHMM_RVE_NONFINITE = 4,     /* NaN/Inf in the residual */
  FEHMM_RVE_PCG_CAP = 5,       /* the tangent-transfer solve hit its iteration cap */
  FEHMM_RVE_BAD_PHASE = 7      /* a phase id >= 4 in a device-supplied phase map (no-allocation
                                  entry point): nothing is solved, P/A/w are left unchanged */
};

/* fehmm_rve_solve flags */
enum {
  FEHMM_SOLVE_NO_TANGENT = 1,     /* skip the condensation: A is not written */
  FEHMM_SOLVE_FROM_COMMITTED = 2, /* start from the committed fluctuations (first macro
                                     iteration of a load step, Sec. 5.1 warm start) instead
                                     of the current ones */
  FEHMM_SOLVE_ENERGY = 4          /* also write Wbar = <psi> (needs W != NULL) */
};

typedef struct {
  int dim;              /* 2 or 3 */
  int precision;        /* FEHMM_PREC_FP64: every step in FP64.  FEHMM_PREC_MIXED: FP64
                           residual, Newton test, fluctuation update and homogenised sums;
                           FP32 tangent and PCG. */
  double newton_rtol;   /* stop when |R|_2 <= max(newton_rtol*|R_0|_2, newton_atol); R_0 is
                           the residual at the start of the call */
  double newton_atol;
  int max_newton;       /* Newton iterations per call; 1 gives the alternating scheme of
                           Algorithm 2 (one micro iteration per macro iteration) */
  double cg_rtol;       /* relative tolerance of the PCG for each Newton correction */
  int max_cg;
  double cond_rtol;     /* relative tolerance of the PCG solves of the tangent transfer */
  int max_cond_cg;
  int retry_stages;     /* 0..64, default 4: a point whose Newton solve ends in
                           FEHMM_RVE_J_NONPOS, FEHMM_RVE_NONFINITE or FEHMM_RVE_PCG_BREAKDOWN is
                           solved again from zero fluctuations, reaching Fbar in retry_stages
                           equal increments of Fbar - I (load continuation, each increment
                           warm-started from the last, each allowed max(max_newton, 25)
                           Newton iterations); 0 or 1 turns the retry off.  The status is that
                           of the retried solve; the Newton count adds up all stages. */
  int precond;          /* FEHMM_PRECOND_MULTIGRID (default): grids whose halving ends at
                           m nodes per axis (2D: n = 2^k m, m <= 4, n >= 6; 3D: m <= 3,
                           n >= 4) use a geometric V(1,1)-cycle with Galerkin coarse levels,
                           damped block-Jacobi smoothing and an exact coarsest solve; other
                           grids and FEHMM_PRECOND_BLOCK_JACOBI use block-Jacobi (inverted
                           nodal d x d blocks).  The choice changes iteration counts, not the
                           tolerances the solves meet. */
  int bc;               /* FEHMM_BC_PERIODIC (default) or FEHMM_BC_KUBC */
  int law;              /* FEHMM_LAW_NEO_HOOKE (default) or FEHMM_LAW_SVK */
  double mg_omega;      /* damping of the multigrid's block-Jacobi smoother, in (0, 1); the
                           V-cycle is a positive definite preconditioner only while omega <
                           2 / lambda_max(D^-1 K) (about 0.86 for Q1, 0.67 for Hex8 elasticity).
                           Default 0.7 (2D), 0.6 (3D).  A PCG that breaks down (negative
                           r^T M^-1 r: the V-cycle is not positive definite at that tangent) or
                           hits its cap is rerun with half the damping, down to omega / 8. */
  int mg_reuse;         /* 3D multigrid: 1 (default) builds the coarse levels at the first Newton
                           iteration of a solve and reuses them in the later ones; 0 rebuilds
                           them at every Newton iteration */
  int transfer_warm;    /* 1 (default): each point keeps the solutions X_c of its tangent-transfer
                           solves (d^2 fields, in the solve's arithmetic type) as load-step state
                           beside its fluctuation, and the next solve of that point starts its
                           transfer PCG from them (the residual b - K X_0, stopped at the same
                           cond_rtol relative to the right-hand side as from zero); 0: every
                           transfer PCG starts from zero */
} fehmm_options;

/* Fill `opt` with defaults for dim (2|3) and precision. */
int fehmm_default_options(fehmm_options* opt, int dim, int precision);

/* Create a context on the current CUDA device.  opt: host, copied. */
int fehmm_create(fehmm_ctx** out, const fehmm_options* opt);
int fehmm_destroy(fehmm_ctx* ctx);
int fehmm_get_options(const fehmm_ctx* ctx, fehmm_options* opt);
/* Change tolerances/caps of an existing context (dim and precision must not change). */
int fehmm_set_options(fehmm_ctx* ctx, const fehmm_options* opt);

/*
 * Add n_rve microstructures (host arrays, copied).  grid_n[r]: elements per axis of RVE r
 * (2D: even, 2..32; 3D: 2..16).  phase: concatenation of the uint8 phase maps, RVE r
 * holding grid_n[r]^dim entries in element order.  E, nu: [n_rve][n_phase] per-RVE
 * material table (Young's modulus, Poisson ratio; Lame constants are derived as in the
 * paper's Table of material parameters, Sec. 6), n_phase <= 4.  first_id (optional)
 * receives the id of the first new RVE.  Must precede fehmm_bind_qps.
 */
int fehmm_add_rves(fehmm_ctx* ctx, int n_rve, const int32_t* grid_n, const uint8_t* phase,
                   const double* E, const double* nu, int n_phase, int* first_id);

/*
 * Bind n_qp macro quadrature points to microstructures (rve_of_qp: host, [n_qp]) and
 * allocate their fluctuation state (current and committed, both zero).  Replaces any
 * previous binding.
 */
int fehmm_bind_qps(fehmm_ctx* ctx, int n_qp, const int32_t* rve_of_qp);

/*
 * One batched RVE solve (Sec. 3.3 micro Newton, Eq. Average-of-P-and-F averages and the
 * tangent transfer of Eq. k-mac-element-6) for every bound quadrature point.
 *   F      device [n_qp][d*d]   macro deformation gradient Fbar at each point (input)
 *   P      device [n_qp][d*d]   homogenised Pbar (output)
 *   A      device [n_qp][d^4]   homogenised tangent dPbar/dFbar (output; may be NULL
 *                               with FEHMM_SOLVE_NO_TANGENT)
 *   W      device [n_qp]        <psi> (output, only with FEHMM_SOLVE_ENERGY; else NULL ok)
 *   status device [n_qp] int32  FEHMM_RVE_* per point (output)
 *   iters  device [n_qp][4] int32: Newton iterations, PCG iterations of the Newton
 *          corrections, PCG iterations of the tangent transfer (sum over d*d right-hand
 *          sides), largest single tangent-transfer PCG count (output; may be NULL)
 * The fluctuation of each point starts from its current (or, with
 * FEHMM_SOLVE_FROM_COMMITTED, committed) state and the result becomes the current state.
 * Returns FEHMM_OK once enqueued; per-point failures are reported through `status`.
 */
int fehmm_rve_solve(fehmm_ctx* ctx, const double* F, double* P, double* A, double* W,
                    int32_t* status, int32_t* iters, int flags, void* stream);

/*
 * Same as fehmm_rve_solve for the quadrature points list[0 .. *count-1] only (device arrays;
 * *count is read on the device, so the list can come from fehmm_select without a host
 * round trip).  Outputs of the other points are left unchanged.  Used for the fallback of the
 * surrogate path and for its audit sample.
 */
int fehmm_rve_solve_list(fehmm_ctx* ctx, const double* F, double* P, double* A, double* W,
                         int32_t* status, int32_t* iters, int flags, const int32_t* list,
                         const int32_t* count, void* stream);

/* list <- indices q (ascending) with mask[q] == value and q % stride == 0, *count <- their
 * number (device arrays, list of n entries; stride >= 1, e.g. > 1 for an audit sample).  The
 * paper has no counterpart: it picks the points of the surrogate path (the learned part of the
 * workload) that fall back to full RVE solves, or its audit sample. */
int fehmm_select(const int32_t* mask, int n, int value, int stride, int32_t* list, int32_t* count,
                 void* stream);

/* Load-step state (Sec. 5.1: the converged micro state of a load step is the start value of the
 * next one, the warm start; Sec. 5.2: the alternating scheme carries the last micro iterate).
 * commit copies current -> committed fluctuations (and kept transfer solutions); rollback the
 * reverse (e.g. to repeat a load step after a failed macro iteration). */
int fehmm_commit(fehmm_ctx* ctx, void* stream);
int fehmm_rollback(fehmm_ctx* ctx, void* stream);

/*
 * Access to the fluctuation of quadrature point q: the periodic micro field w of the kinematics
 * u = (Fbar - I) X + w (Eq. linearization-uH with the constraints of Eq. ConstraintCondition-
 * phi_h-phi_H; device pointer to n_node*dim doubles, node-major, owned by the context, valid
 * until the next bind).  which = 0 current, 1 committed.  n_values (optional) receives the length.
 */
int fehmm_fluctuation(fehmm_ctx* ctx, int q, int which, double** dev_ptr, int* n_values);

/* The fluctuations of all bound points as one device array (the per-point fields of
 * fehmm_fluctuation concatenated in point order; owned by the context, valid until the next
 * bind): which = 0 current, 1 committed.  Lets a caller save and restore the load-step state
 * of Sec. 5.1 (e.g. to repeat a load step from the same converged state). */
int fehmm_fluctuation_all(fehmm_ctx* ctx, int which, double** dev_ptr, long long* n_values);

/* The kept tangent-transfer solutions of all bound points (see fehmm_options.transfer_warm) as
 * one device array of n_bytes bytes (owned by the context; which = 0 current, 1 committed;
 * committed and rolled back together with the fluctuations).  NULL and 0 when transfer_warm was
 * off at fehmm_bind_qps. */
int fehmm_transfer_state_all(fehmm_ctx* ctx, int which, void** dev_ptr, long long* n_bytes);

/*
 * Structured macro mesh on [0,1]^dim with n_el[c] elements along axis c (host array of
 * dim ints).  Builds the CSR pattern of the macro tangent and the colouring of the
 * assembly.  The number of macro quadrature points is n_el product * 2^dim.
 */
int fehmm_macro_create(fehmm_ctx* ctx, const int32_t* n_el);

/* Fbar = I + sum_I u_I (x) Grad N_I at every macro quadrature point (the gradient of
 * Eq. linearization-uH).  u: device [n_node*dim]; F: device [n_qp][d*d]. */
int fehmm_macro_qp_F(fehmm_ctx* ctx, const double* u, double* F, void* stream);

/*
 * Macro residual and tangent (Eq. f_I^int with S^H = <F>^-1<P>, Eq. ModifiedBilinearForm-3,
 * Eq. Assem_k_T_IK_mac):  f_I = sum_q omega_q Pbar_q Grad N_I,
 * K_IJ = sum_q omega_q Grad N_I . Abar_q . Grad N_J, omega = Gauss weight * det J.
 *   P device [n_qp][d*d], A device [n_qp][d^4] (may be NULL: K not assembled),
 *   f device [n_node*dim] (overwritten), K_vals device [nnz] (overwritten, CSR order of
 *   fehmm_macro_csr).  No boundary conditions are applied.
 */
int fehmm_macro_assemble(fehmm_ctx* ctx, const double* P, const double* A, double* f,
                         double* K_vals, void* stream);

/* Dirichlet data of the macro problem (Eq. BCs, u = u_hat on the Dirichlet boundary): host
 * arrays of n_fixed dof indices and their values at the end of the loading, copied.  Their
 * rows and columns are removed from the macro solve (du = 0 there).  Default: none. */
int fehmm_macro_set_dirichlet(fehmm_ctx* ctx, int n_fixed, const int32_t* dofs, const double* values);

/* Start of a load step: u[dof] = scale * value on every Dirichlet dof (scale = load factor of
 * the step) and, if du != NULL, du = 0.  u, du: device [n_rows]. */
int fehmm_macro_apply_dirichlet(fehmm_ctx* ctx, double* u, double* du, double scale, void* stream);

/* Load of a prescribed Dirichlet increment on the linearised macro problem (Eq. L(GH)):
 * g = K d, with d = dscale * (the Dirichlet end values of fehmm_macro_set_dirichlet) on the
 * Dirichlet dofs and zero elsewhere.  K_vals device [nnz] (CSR order of fehmm_macro_csr), g device
 * [n_rows] (output, every row).  With the tangent of the last converged state, solving
 * K_ff delta = -g_f (fehmm_macro_solve with f = g) gives the tangent predictor of the next load
 * step, u <- u + d + delta, which keeps the first macro iterate of a fine macro mesh from
 * concentrating the whole increment in the boundary elements. */
int fehmm_macro_dirichlet_load(fehmm_ctx* ctx, const double* K_vals, double dscale, double* g, void* stream);

/* Macro Newton update u += du (device [n_rows] each; du is zero on Dirichlet dofs). */
int fehmm_macro_update(fehmm_ctx* ctx, double* u, const double* du, void* stream);

/*
 * Macro Newton correction (the linearised HMM problem, Eq. L(GH)): solves K_ff du_f = -f_f
 * with du = 0 on the Dirichlet dofs, by Jacobi-preconditioned CG in FP64 on the GPU
 * (one cooperative launch; stops when the preconditioned residual norm falls below
 * rtol times its initial value, or after max_it iterations).
 *   K_vals device [nnz] (CSR order of fehmm_macro_csr), f device [n_rows], du device
 *   [n_rows] (output), info device double[3] (output): |f_free|_2 (the macro convergence
 *   measure, taken before the solve), CG iterations, status (0 converged, 1 cap,
 *   2 non-positive curvature).
 */
int fehmm_macro_solve(fehmm_ctx* ctx, const double* K_vals, const double* f, double* du, double* info,
                      double rtol, int max_it, void* stream);

/* CSR pattern of the assembled macro tangent of Eq. Assem_k_T_IK_mac (one d x d block per pair of
 * nodes sharing an element; device pointers owned by the context). */
int fehmm_macro_csr(fehmm_ctx* ctx, const int32_t** rowptr, const int32_t** col, int* n_rows,
                    int* nnz);

/*
 * Energy surrogate (the learned part of the workload; the paper has no counterpart).
 * An MLP y(x), x in R^6 -> 4 x 128 SiLU -> 1, with BF16 weights and activations and FP32
 * accumulation on tensor cores (the 128 x 128 layer products on tcgen05 with the accumulator in
 * tensor memory, the 8-wide input-layer products on mma.sync).  Parameters are packed FP32 (fehmm_mlp_num_params floats):
 * W1 [128][8] (input columns 6, 7 unused), b1 [128], W2, W3, W4 [128][128] row-major
 * ([out][in]), b2..b4 [128], w5 [128], b5 [1], padding [3].  The context holds FP32 master
 * weights, BF16 copies, AdamW moments and a workspace for up to max_batch samples.
 */
typedef struct fehmm_mlp fehmm_mlp;
int fehmm_mlp_num_params(void);
int fehmm_mlp_create(fehmm_mlp** out, int max_batch);
int fehmm_mlp_destroy(fehmm_mlp* mlp);
/* host_params: packed FP32 parameters (copied); resets the optimiser state. */
int fehmm_mlp_set_params(fehmm_mlp* mlp, const float* host_params);
/* host copies of the parameters and/or of the last computed gradient (either may be NULL). */
int fehmm_mlp_get_params(fehmm_mlp* mlp, float* host_params, float* host_grad);
/* y [B], g = dy/dx [B][6], H = d2y/dx2 [B][6][6] (device; g, H may be NULL) for x [B][6]. */
int fehmm_mlp_eval(fehmm_mlp* mlp, const float* x, int B, float* y, float* g, float* H, void* stream);
/* Training loss L = 1/2 sum_b [cy (y_b - ty_b)^2 + cg |g_b - tg_b|^2] (device x [B][6],
 * ty [B], tg [B][6]); writes L to loss (device float, may be NULL) and its exact gradient
 * with respect to the parameters to the context (read with fehmm_mlp_get_params). */
int fehmm_mlp_loss_grad(fehmm_mlp* mlp, const float* x, const float* ty, const float* tg, int B, float cy,
                        float cg, float* loss, void* stream);
/* AdamW step on the FP32 masters with the last gradient (weight decay on weights only). */
int fehmm_mlp_adamw(fehmm_mlp* mlp, float lr, float beta1, float beta2, float eps, float weight_decay,
                    void* stream);
long long fehmm_mlp_launch_count(const fehmm_mlp* mlp);
/* Synchronises the device and reports in *flag whether a tensor-core product of this MLP gave up
 * waiting for its MMAs since the last check (1: its outputs are invalid; the flag is cleared). */
int fehmm_mlp_check(fehmm_mlp* mlp, int* flag);
/* Device view of the gradient that fehmm_mlp_loss_grad wrote and fehmm_mlp_adamw reads (FP32,
 * packed like the parameters; owned by the MLP).  Data-parallel training over ranks sums it over
 * the ranks between the two calls (each rank's loss weighted by 1/(global batch)). */
int fehmm_mlp_grad_buffer(fehmm_mlp* mlp, float** dev_ptr, int* n_params);

#define FEHMM_POLY_TERMS 896 /* monomials of degree 3 to 6 in 6 variables */

typedef struct {
  double lam0, mu0;  /* Lame constants of the neo-Hookean base energy */
  double sx, sg;     /* input scale (x = Mandel(E)/sx) and output scale (W = W_base + sg y) */
  double radius;     /* trust region |U - I|_F <= radius, U = (F^T F)^(1/2) */
  double Ca[36];     /* anisotropic small-strain part of the base energy, 1/2 m(E).Ca.m(E) with
                        m(E) the Mandel vector of E (order 11,22,33,23,13,12, sqrt 2 on shears) */
  double y0, g0[6], H0[36]; /* network value, gradient and Hessian at x = 0, subtracted so that the
                        learned correction y(x) - y0 - g0.x - 1/2 x.H0.x vanishes to third order at
                        E = 0, where the base energy is exact to second order (zeros: no shift) */
  double poly[FEHMM_POLY_TERMS]; /* fitted polynomial part of the correction, in network units:
                        y_poly(x) = sum_a poly[a] x_{i1} x_{i2} ... x_{id} over the monomials of
                        degree d = 3, 4, 5, 6 in the 6 features, each degree's index tuples
                        i1 <= i2 <= ... <= id in lexicographic order (56 + 126 + 252 + 462 terms);
                        W = W_base + sg (y_poly(x) + shifted network); zeros: no polynomial */
} fehmm_surrogate_params;

/*
 * Surrogate constitutive evaluation at n macro points: F device [n][9] in; P [n][9],
 * A [n][81] (may be NULL), W [n] (may be NULL), inside [n] (1 inside the trust region,
 * else 0) out; work: device floats, fehmm_surrogate_work_floats(n) of them; n <= the MLP's
 * max_batch.  P and A are written for every point; the caller replaces the points outside
 * the trust region by full RVE solves (fehmm_select + fehmm_rve_solve_list).
 */
int fehmm_surrogate_eval(fehmm_mlp* mlp, const fehmm_surrogate_params* sp, const double* F, int n,
                         double* P, double* A, double* W, int32_t* inside, float* work, void* stream);
size_t fehmm_surrogate_work_floats(int n);

/* Base energy of the surrogate from the RVE's small-strain homogenised tangent A0 (host [81],
 * iJkL row-major, e.g. from fehmm_rve_solve at F = I): its minor-symmetric part is projected on
 * isotropy (3K = A_iijj / 3, mu0 = (A_ijij - A_iijj / 3) / 10, lam0 = K - 2 mu0 / 3) and the
 * remainder A0 - (lam0 1(x)1 + 2 mu0 I^sym) goes to sp->Ca in Mandel form.  Sets sp->lam0, mu0,
 * Ca only.  FEHMM_ERR_ARG if the projection is not positive definite. */
int fehmm_surrogate_base_law(const double* A0, fehmm_surrogate_params* sp);

/* Persistence of a trained surrogate (host file path): the packed FP32 network parameters and
 * every field of fehmm_surrogate_params, in a small binary file with a magic and a format
 * version.  load sets the network's parameters (resetting its optimiser state) and *sp.  An
 * unreadable, foreign or truncated file returns FEHMM_ERR_ARG and changes nothing. */
int fehmm_surrogate_save(fehmm_mlp* mlp, const fehmm_surrogate_params* sp, const char* path);
int fehmm_surrogate_load(fehmm_mlp* mlp, fehmm_surrogate_params* sp, const char* path);

/* Training data of the surrogate from n full RVE solves at F = U (device F [n][9], their
 * homogenised P [n][9] and W [n]): features x [n][6], value targets ty [n] and input-gradient
 * targets tg [n][6] (device floats) of the Sobolev loss of fehmm_mlp_loss_grad. */
int fehmm_surrogate_targets(const fehmm_surrogate_params* sp, const double* F, const double* P, const double* W,
                            int n, float* x, float* ty, float* tg, void* stream);

/* Polynomial part of the learned correction, fitted before the network (set-up; the paper has no
 * counterpart).  Weighted linear least squares over the first min(n, 65536) samples of the
 * training targets (device x [n][6], ty [n], tg [n][6] from fehmm_surrogate_targets): minimise
 * sum_b [ (y_poly(x_b) - ty_b)^2 / <ty^2> + |grad y_poly(x_b) - tg_b|^2 / <|tg|^2> ] over the
 * coefficients of the monomials of degree 3 to max_degree (3..6; the Sobolev loss of the network,
 * normalised the same way), normal equations accumulated in FP64 on the device and solved by
 * Cholesky on the host with a 1e-12 relative ridge.  Writes sp->poly (zero above max_degree) and
 * replaces ty, tg of all n samples by their remainders (ty - y_poly, tg - grad y_poly), which the
 * network then learns.  The polynomial has no terms below degree 3, so the third-order origin
 * condition of the correction still holds.  FEHMM_ERR_ARG on bad arguments or a normal matrix
 * that is not positive definite. */
int fehmm_surrogate_fit_poly(fehmm_surrogate_params* sp, const float* x, float* ty, float* tg, int n,
                             int max_degree, void* stream);

/*
 * Autotuner of the solver settings (project-written; the paper has no counterpart).  Times the
 * batched RVE solve (fehmm_rve_solve_list from the committed fluctuations, at the deformation
 * gradients F, device [n_qp][d*d]) on an evenly strided sample of n_sample bound points (<= 0:
 * two per SM) for every candidate setting -- preconditioner (multigrid | block-Jacobi), smoother
 * damping mg_omega (four values below the element type's positive-definiteness bound), 3D
 * coarse-level reuse, and the Newton-correction PCG tolerance (cg_rtol x {1, 10, 0.1}) -- and
 * keeps the fastest whose sample solves all converge; the tolerances the solves meet do not
 * change.  The choice is written into the context's options and, when cache_path (host text
 * file, may be NULL) is given, appended to it under a key of dimension, precision, law,
 * coupling, the grid sizes bound and the device name; a later call with a matching key applies
 * the cached choice without timing.  The current fluctuations and kept transfer solutions are
 * restored after the trials.
 * best (host, may be NULL) receives the choice.  Allocates temporary device memory; returns
 * FEHMM_ERR_UNSUPPORTED (options unchanged) if no candidate converges on the sample.
 */
typedef struct {
  int precond;              /* FEHMM_PRECOND_* */
  double mg_omega;
  double cg_rtol;
  int mg_reuse;
  double seconds_per_solve; /* measured: batch time / sample points, of the chosen setting */
  int from_cache;           /* 1: taken from the cache file, nothing timed */
  int candidates;           /* settings timed */
} fehmm_tune_result;
int fehmm_autotune(fehmm_ctx* ctx, const double* F, int n_sample, const char* cache_path, fehmm_tune_result* best,
                   void* stream);

/* Number of kernel launches this context has issued since creation (for accounting). */
long long fehmm_launch_count(const fehmm_ctx* ctx);

const char* fehmm_status_str(int code);

/*
 * No-allocation batched RVE solve, 2D, FP64 mode.  The paper has no counterpart: this is a
 * deployment variant of fehmm_rve_solve for callers that cannot call cudaMalloc (runtimes
 * that hand the library only pre-registered buffers, code running while a memory pool is
 * torn down or resized, callers that need a footprint fixed at load time).  It allocates
 * no device memory: the kernel's scratch (staged element tangents and the assembled
 * stencil, 72*n*n doubles per block) and its work counter live in a file-scope static
 * device array of fixed size (152 blocks x 72 x 256 doubles, about 22 MB), which every
 * GPU that loads the library holds until the process exits.  It takes no context: the
 * caller passes every input and output.
 *   n_qp          number of quadrature points (RVE solves)
 *   grid_n        elements per axis of every RVE: even, 2..16; larger -> FEHMM_ERR_TOO_LARGE
 *   phase_per_qp  1: phase holds one map per qp; 0: one map shared by all
 *   phase   device uint8 [phase_per_qp ? n_qp : 1][grid_n*grid_n], phase ids < 4 (a point
 *           whose map holds a larger id gets status FEHMM_RVE_BAD_PHASE and is not solved)
 *   lame    device double [phase_per_qp ? n_qp : 1][4][2]: (lambda, mu) of each phase
 *   w       device double [n_qp][grid_n*grid_n][2]: fluctuation start values in, results
 *           out (the value at node 0 is taken as zero)
 *   F, P, A, status, iters: as in fehmm_rve_solve (A may be NULL: no tangent)
 *   opt     host; dim must be 2 and precision FEHMM_PREC_FP64; tolerances, caps and bc used;
 *           law must be FEHMM_LAW_NEO_HOOKE (else FEHMM_ERR_UNSUPPORTED)
 * The first call on a device looks up the device address of the static array (with that
 * device current); make that first call before any stream capture.  All calls share the
 * array and the counter, which keep the last call's contents (the counter is cleared by
 * each call on its stream): calls that overlap on the GPU (different streams, or another
 * host thread) race and must be serialised by the caller.  Returns FEHMM_OK once enqueued.
 */
int fehmm_rve2d_solve_fp64_noalloc(int n_qp, int grid_n, int phase_per_qp, const uint8_t* phase,
                                   const double* lame, double* w, const double* F, double* P,
                                   double* A, int32_t* status, int32_t* iters,
                                   const fehmm_options* opt, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FEHMM_H */
