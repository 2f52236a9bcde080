/*
 * irk.h -- C ABI of the GB300 stage-coupled implicit Runge-Kutta solver.
 *
 * The library advances the Q1 finite-element heat equation
 *     M u' + K(kappa) u = F(t)          (Kirby & MacLachlan, "Extending Irksome",
 *                                        Sec. 2, eq. heat / rkheat)
 * on a uniform mesh of the unit square (dim = 2, per-cell kappa) or the unit cube
 * (dim = 3, 27-point Q1 stencils, kappa = 1) with homogeneous Dirichlet data (or
 * DAE-type boundary data, irk_step_dirichlet) by one s-stage Runge-Kutta step at a
 * time.  Each step solves the
 * stage-coupled system of Sec. 3, eq. block_struct_AI,
 *     (I (x) M + dt A (x) K) k = r,   r_i = F(t_n + c_i dt) - K u_n,
 * with FP64 flexible GMRES preconditioned by the block-diagonal (P_D, eq.
 * pcbjac) or block-triangular (P_L, eq. pcbgs; P_U, Sec. 3.1) stage
 * preconditioner, whose diagonal blocks M + dt a_ii K are each approximated by
 * one geometric-multigrid V-cycle (Sec. 3.1), then sets
 *     u_{n+1} = u_n + dt sum_i b_i k_i     (Sec. 2, RK update).
 *
 * Data layout (all vectors, device or host):
 *   * nodes of the full (N+1)^dim grid, x fastest (node id = ix + (N+1) iy);
 *   * a "nodal" vector holds one double per node;
 *   * a "stage" vector holds s doubles per node, node-major: v[node*s + i];
 *   * boundary entries of inputs are ignored (read as 0); boundary entries of
 *     outputs are written as 0 (homogeneous Dirichlet: by the DAE-type
 *     conditions of Sec. 2.1 the stage values vanish there);
 *   * per-cell data (kappa) is N^dim doubles, cells x fastest.
 *
 * Pointers: vector arguments may be device pointers or host pointers; the
 * library asks the CUDA runtime which one it got and, for host memory, copies
 * through its own device buffers inside the call.  All device work is
 * enqueued on the stream given to irk_create (NULL = the legacy default
 * stream).  The caller keeps ownership of every pointer it passes; the handle
 * owns all scratch memory (Krylov basis, multigrid level vectors).
 *
 * Errors: every entry point returns IRK_OK (0) or a negative IRK_E* code and
 * records a message that irk_last_error() returns (per thread).  No C++
 * exception crosses this boundary.
 */
#ifndef IRK_H
#define IRK_H

#ifdef __cplusplus
extern "C" {
#endif

#define IRK_OK 0
#define IRK_EINVAL (-1)     /* bad argument, tableau, mesh or option */
#define IRK_ENOMEM (-2)     /* device or host allocation failed (for tests, IRK_FAIL_DEVICE_ALLOC=n in the
                               environment makes every n-th device allocation of the process fail) */
#define IRK_ECUDA (-3)      /* a CUDA runtime call failed */
#define IRK_ENOCONV (-4)    /* FGMRES reached maxit; outputs hold the last iterate */
#define IRK_ENONFINITE (-5) /* NaN or Inf in the residual */

/* block stage preconditioners (Sec. 3.1) */
#define IRK_PC_DIAG 0  /* P_D = I (x) M + dt D (x) K          (eq. pcbjac, AI form)   */
#define IRK_PC_LOWER 1 /* P_L = I (x) M + dt (L + D) (x) K    (eq. pcbgs, AI form)    */
#define IRK_PC_UPPER 2 /* P_U = I (x) M + dt (U + D) (x) K    (Sec. 3.1)              */
#define IRK_PC_RANA_LD 3 /* I (x) M + dt (L D) (x) K with A = L D U, L unit lower, U unit
                            upper: the Rana-type preconditioner (eq. pcranald, AI form)   */
#define IRK_PC_MONOLITHIC 4 /* monolithic multigrid (Sec. 3, monolithic multigrid): one V-cycle
                            on the whole stage system with stage-coupled point-block Jacobi
                            relaxation (additive Schwarz on Q1 vertex patches) and an exact
                            coupled coarsest solve; dim = 2, AI splitting, FGMRES; the
                            transposed preconditioner is the exactly transposed cycle     */

/* Arnoldi orthogonalisation (the paper does not fix one) */
#define IRK_ORTH_CGS2 0 /* classical Gram-Schmidt, always two passes                       */
#define IRK_ORTH_DGKS 1 /* classical Gram-Schmidt, second pass only when ||w'|| < ||w||/sqrt(2)
                           (Daniel-Gragg-Kaufman-Stewart test), norm by Pythagoras otherwise   */
#define IRK_ORTH_CGS 2  /* classical Gram-Schmidt, one pass (the GMRES default of the PETSc
                           stack the paper used); the norm of the new vector is reduced
                           directly, and at convergence the true residual ||r - S x|| is
                           recomputed and iteration continues if it misses rtol              */

/* outer solver */
#define IRK_SOLVER_FGMRES 0  /* FGMRES on the whole stage system (any tableau)                    */
#define IRK_SOLVER_DIRK_CG 1 /* lower-triangular A with a_ii > 0 (DIRK, Sec. 2.3): the stages one
                                after another, each by CG preconditioned with one V-cycle         */

/* stage formulation (Sec. 2.2, Sec. 3) */
#define IRK_SPLIT_AI 0 /* stage derivatives k: (I (x) M + dt A (x) K) k = r            (eq. block_struct_AI) */
#define IRK_SPLIT_IA 1 /* w = (A (x) I) k: (A^{-1} (x) M + dt I (x) K) w = r          (eq. block_struct_IA);
                          the preconditioners are then (T^{-1} (x) M) + dt (I (x) K) with T = D, L + D, U + D
                          or L D as printed in eq. pcbjac / pcbgs / pcranald                              */

/* storage / arithmetic of the multigrid V-cycles inside the FP64 FGMRES */
#define IRK_PREC_FP64 0 /* vectors and arithmetic in double                         */
#define IRK_PREC_FP32 1 /* vectors and arithmetic in float                          */
#define IRK_PREC_BF16 2 /* vectors stored as bfloat16, arithmetic in float          */

#define IRK_MAX_STAGES 4

typedef struct irk_handle irk_handle;

typedef struct {
  int dim;             /* 2 (quadrilaterals) or 3 (hexahedra; kappa must be NULL) */
  int n_cells;         /* N: cells per axis of the uniform mesh of [0,1]^dim */
  int levels;          /* multigrid levels >= 1; N divisible by 2^(levels-1), coarsest >= 2 cells */
  const double* kappa; /* host, N^dim per-cell diffusivities (> 0), or NULL for kappa = 1 (dim = 3: NULL
                          only); copied */
} irk_mesh;

typedef struct {
  int s;            /* stages, 1..IRK_MAX_STAGES */
  const double* A;  /* host, s*s row-major Butcher matrix; copied */
  const double* b;  /* host, s weights; copied */
  const double* c;  /* host, s abscissae; copied */
} irk_tableau;

typedef struct {
  int precond;      /* IRK_PC_* */
  int vcycle_prec;  /* IRK_PREC_* */
  int nu_pre;       /* weighted-Jacobi pre-smoothing sweeps per level (default 2) */
  int nu_post;      /* post-smoothing sweeps per level (default 2) */
  double omega;     /* Jacobi weight (default 2/3) */
  double rtol;      /* stop when ||r_j||_2 <= rtol ||r_0||_2 (default 1e-10) */
  int restart;      /* FGMRES restart length m (default 50) */
  int maxit;        /* total FGMRES iterations allowed per solve (default 500) */
  int orth;         /* IRK_ORTH_* (default IRK_ORTH_CGS2) */
  int solver;       /* IRK_SOLVER_* (default IRK_SOLVER_FGMRES) */
  int splitting;    /* IRK_SPLIT_* (default IRK_SPLIT_AI); IA needs an invertible A and FGMRES */
  int warm_start;   /* 1: irk_step starts FGMRES from the stage solution (w in the IA form) of this handle's
                       previous irk_step, unless a call since has replaced it (irk_step_dirichlet,
                       irk_step_adjoint, an IA-form irk_solve, irk_reset_initial_guess) or its residual is
                       not below ||r||_2; the stopping test stays ||r_j||_2 <= rtol ||r||_2 with r the
                       step's right-hand side, so the residual bound is that of a zero start.
                       0 (default): zero initial guess (the paper does not say which it uses).
                       Ignored by IRK_SOLVER_DIRK_CG. */
} irk_options;

typedef struct {
  int fgmres_its;   /* Krylov iterations of the last solve: FGMRES Arnoldi steps, or CG
                       iterations summed over the stages for IRK_SOLVER_DIRK_CG */
  int vcycles;      /* single-block V-cycles applied in the last solve */
  double rel_resid; /* final ||r||_2 / ||r_0||_2 estimate of the last solve */
  int converged;    /* 1 if rel_resid <= rtol */
} irk_stats;

/* Fill *opt with the defaults listed above (P_L, FP64 V-cycles, CGS2 Arnoldi). */
void irk_default_options(irk_options* opt);

/* Build a solver for one mesh, tableau and step size (Sec. 3, eq. block_struct_AI).
 * Validates the tableau (finite entries; row sums of A equal c to 1e-6, which
 * also rejects a transposed A), builds the Galerkin multigrid hierarchy of M and K(kappa) on the host, factors the
 * coarsest blocks, uploads everything and allocates the Krylov basis.
 * Device memory, with n = (N+1)^dim nodes and s stages: the Krylov basis, (2 restart + 1) vectors of 8 s n
 * bytes; four level vectors per level in the V-cycle precision; in 2D per level the stencil records (5 planes,
 * FP64 and FP32) and the records of each diagonal block; FP64 V-cycles add nine planes of 8 bytes per node and
 * stage on coarse levels of at least 513 nodes per axis, and with triangular sweeps on the finest level; the IA
 * form adds five planes per stage on the finest level; monolithic multigrid adds s^2 values per node and level.
 * stream: a cudaStream_t (NULL = legacy default stream).  *out is set on success. */
int irk_create(irk_handle** out, const irk_mesh* mesh, const irk_tableau* tab, double dt,
               const irk_options* opt, void* stream);

/* Release every resource of the handle (NULL is accepted). */
int irk_destroy(irk_handle* h);

/* Replace the per-cell diffusivity (host, N^dim doubles) and rebuild the
 * operators, the hierarchy and the coarse factors; the step size is kept. */
int irk_set_kappa(irk_handle* h, const double* kappa_host);

/* With irk_options.warm_start = 1: make the next irk_step start FGMRES from zero (as the first step of a
 * handle does), e.g. before a new trajectory from other initial data.  A no-op otherwise.  Returns IRK_OK,
 * or IRK_EINVAL for a NULL handle. */
int irk_reset_initial_guess(irk_handle* h);

/* One RK step (Sec. 2): solve for the stages k and set
 * u_np1 = u_n + dt sum_i b_i k_i.
 *   u_n        nodal, input.
 *   f_space    nodal, optional (NULL = 0): spatial load vector F^ (integrals of f against the hats).
 *   f_coef     host, s doubles, optional (NULL = all 1): F_i += f_coef[i] * F^.
 *   f_stages   stage vector, optional (NULL = 0): F_i += f_stages[:, i].
 *   u_np1      nodal, output (may alias u_n).
 *   stages_out stage vector, optional output of k.
 *   stats      optional.
 * With irk_options.warm_start = 1 FGMRES starts from the previous step's stages (see there).
 * Returns IRK_ENOCONV if FGMRES did not reach rtol within maxit (outputs still written). */
int irk_step(irk_handle* h, const double* u_n, const double* f_space, const double* f_coef,
             const double* f_stages, double* u_np1, double* stages_out, irk_stats* stats);

/* One RK step with non-homogeneous Dirichlet data imposed the DAE way (Sec. 2.1): on every
 * boundary node the stage values satisfy u_n + dt sum_j a_ij k_j = g(t_n + c_i dt), so there
 * k = A^{-1} (g - u_n) / dt, and the interior rows of the stage equations take those boundary
 * stages to the right-hand side.  u_np1 = u_n + dt sum_i b_i k_i on all nodes (for stiffly
 * accurate tableaux u_np1 = g(t_{n+1}) on the boundary).
 *   u_n        nodal, input; its boundary entries are the current boundary values.
 *   g_stages   stage vector: g(t_n + c_i dt) at node p in g_stages[p * s + i] (boundary entries
 *              are read, interior entries ignored).
 *   f_space, f_coef, f_stages, u_np1, stages_out, stats: as in irk_step; F holds the loads of
 *              the interior test functions (boundary entries ignored).  stages_out returns k on
 *              all nodes.
 * Needs an invertible Butcher matrix (IRK_EINVAL otherwise).  With IRK_SPLIT_IA the boundary
 * values of w = (A (x) I) k are (g - u_n) / dt directly.  Returns IRK_ENOCONV as irk_step. */
int irk_step_dirichlet(irk_handle* h, const double* u_n, const double* g_stages, const double* f_space,
                       const double* f_coef, const double* f_stages, double* u_np1, double* stages_out,
                       irk_stats* stats);

/* Solve (I (x) M + dt A (x) K) k = r for a given stage vector r (no RK update); with IRK_SPLIT_IA
 * the IA system is solved for w and k = (A^{-1} (x) I) w is returned. */
int irk_solve(irk_handle* h, const double* r, double* k, irk_stats* stats);

/* y = (I (x) M + dt A (x) K) x for stage vectors (transpose != 0: A^T instead of A);
 * with IRK_SPLIT_IA: y = (A^{-1} (x) M + dt I (x) K) x (A^{-T} for transpose). */
int irk_apply_operator(irk_handle* h, const double* x, double* y, int transpose);

/* y = M x for nodal vectors (the Q1 mass matrix; boundary entries of x read as 0,
 * of y written as 0).  Used for M-weighted objectives such as 1/2 ||u - u*||_M^2.
 * dim = 2 only (IRK_EINVAL for dim = 3). */
int irk_apply_mass(irk_handle* h, const double* x, double* y);

/* z = P^{-1} v: one application of the configured block preconditioner, each
 * block approximated by one V-cycle (transpose != 0: the transposed
 * preconditioner P^T, used by the adjoint). */
int irk_apply_preconditioner(irk_handle* h, const double* v, double* z, int transpose);

/* Discrete adjoint of irk_step (not in the paper).  With S = I (x) M + dt A (x) K:
 *   solve S^T mu = dt (b (x) lam_np1) by FGMRES with the transposed preconditioner,
 *   lam_n = lam_np1 - K sum_i mu_i,
 *   grad[c] += -kappa_c sum_i mu_i|_c^T K_e U_i|_c,  U_i = u_n + dt sum_j a_ij k_j,
 * where K_e is the unit-diffusivity element matrix, so grad accumulates dJ/d(log kappa).
 *   u_n, stages   the forward step's input state and stages (nodal / stage vectors).
 *   lam_np1       nodal adjoint state after the step (input); lam_n nodal output (may alias).
 *   grad_accum    per-cell, N^dim doubles, accumulated (+=); may be NULL.
 * dim = 2 and IRK_SPLIT_AI only (IRK_EINVAL otherwise); FGMRES or IRK_SOLVER_DIRK_CG. */
int irk_step_adjoint(irk_handle* h, const double* u_n, const double* stages, const double* lam_np1,
                     double* lam_n, double* grad_accum, irk_stats* stats);

/* z = P^{-1} v like irk_apply_preconditioner, for callers that cannot allocate
 * device memory when they apply it: host threads that must not enter the
 * allocator (real-time loops, where a cudaMalloc or an allocator lock would
 * break the latency budget) and embeddings in a framework that owns all device
 * memory and gives the library a fixed budget.  The paper has no counterpart;
 * it is an interface convenience.
 *   v, z       device pointers (host pointers are rejected: staging would allocate).
 *   transpose  as irk_apply_preconditioner (needs IRK_SPLIT_AI, else IRK_EINVAL).
 * The V-cycle level vectors live in one static device array of 16 MiB shared by
 * every call in the process (each GPU that loads the library holds it until exit);
 * handles whose V-cycle needs more scratch than that are rejected with IRK_EINVAL.
 * The first call on a device looks up the array's device address (no allocation);
 * make that first call before any stream capture.  Each call clears the part of
 * the array it uses, so results never depend on earlier calls, but calls that
 * overlap on the GPU (other streams, other threads, other handles) race on the
 * shared array and must be serialised by the caller.  The triangular sweeps also
 * write two buffers the handle allocated at irk_create (the FP64 first-sweep
 * buffer and the FP32 / BF16 stage copies), so calls on one handle race there too.
 * Returns after the work has finished on the handle's stream.  Allocates no device
 * memory: calls no cudaMalloc, cudaFree or other allocating CUDA or torch routine. */
int irk_apply_preconditioner_noalloc(irk_handle* h, const double* v, double* z, int transpose);

/* Kernel classes counted by the built-in instrumentation. */
#define IRK_K_STAGE_APPLY 0 /* stage operator (FP64)                        */
#define IRK_K_JACOBI 1      /* weighted-Jacobi sweep, finest level           */
#define IRK_K_RESIDUAL 2    /* multigrid residual, finest level              */
#define IRK_K_RESTRICT 3    /* restriction from the finest level             */
#define IRK_K_PROLONG 4     /* prolongation + correction into the finest level */
#define IRK_K_COARSE 5      /* coarsest-level dense solve                    */
#define IRK_K_MULTIDOT 6    /* Arnoldi multi-dot partial sums                */
#define IRK_K_AXPY 7        /* Arnoldi / solution multi-axpy                 */
#define IRK_K_BLOCK_RHS 8   /* triangular-preconditioner block right side    */
#define IRK_K_OTHER 9       /* reductions, scaling, Givens, casts, RHS, update */
#define IRK_K_MG_COARSE 10  /* V-cycle work on coarse levels whose finer grid has >= 513 nodes
                               per axis (large-tile fused legs)                          */
#define IRK_K_MG_TAIL 11    /* V-cycle work on the smaller coarse levels (small-tile legs)   */
#define IRK_K_COUNT 12

typedef struct {
  long long launches;                   /* kernels launched since the last irk_perf_select */
  long long class_launches[IRK_K_COUNT];
  double class_bytes[IRK_K_COUNT];      /* algorithmic DRAM bytes (each operand moved once) */
  double class_flops[IRK_K_COUNT];      /* algorithmic floating-point operations */
  long long timed_launches[IRK_K_COUNT];/* launches bracketed by CUDA events */
  double timed_ms[IRK_K_COUNT];         /* their summed device time */
  double timed_bytes[IRK_K_COUNT];
  double timed_flops[IRK_K_COUNT];
} irk_perf;

/* Reset the counters; time every launch of the classes in class_mask (bit k =
 * IRK_K_k) with a pair of CUDA events on the handle's stream (0 = no timing). */
int irk_perf_select(irk_handle* h, unsigned class_mask);

/* Copy the counters (synchronises the handle's stream to read the events). */
int irk_perf_read(irk_handle* h, irk_perf* out);

/* The message recorded by the last failing call on this thread ("" if none). */
const char* irk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IRK_H */
