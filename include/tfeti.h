/*
 * tfeti.h -- C ABI of the GB300 TFETI solver for one-time-step von Mises
 * elastoplasticity with linear isotropic hardening.
 *
 * Method: Cermak, Kozubek, Sysala, Valdman, "A TFETI Domain Decomposition
 * Solver for Elastoplastic Problems".  Section, equation and algorithm
 * numbers below refer to that paper.
 *
 * General conventions
 * -------------------
 * - Every call returns an int status (TFETI_OK = 0 on success); no C++
 *   exception crosses this boundary.  tfeti_last_error(ctx) returns a message
 *   for the last failing call on that context.
 * - "device" pointers are CUDA global-memory pointers on the context's device;
 *   "host" pointers are ordinary CPU memory.  The caller owns every buffer it
 *   passes; the context owns everything it allocates and frees it in
 *   tfeti_destroy.  Null is accepted only where a parameter says "nullable".
 * - All device work of a context is enqueued on the CUDA stream given to
 *   tfeti_setup (or tfeti_setup_case); the context also owns internal streams
 *   that it joins to that stream before a call returns.  Calls that return
 *   host data synchronise that stream.
 * - A context is used by one host thread at a time; different contexts may be
 *   used from different threads at once (ssn_time_step_cases does so).
 * - Floating point is IEEE binary64 throughout unless stated.
 *
 * Discretisation and layouts (all shared with the documentation of the CPU
 * oracle, which implements them independently)
 * ------------------------------------------------------------------------
 * - Box [0,Lx]x[0,Ly]x[0,Lz] of nx*ny*nz trilinear 8-node bricks with 2x2x2
 *   Gauss points (the paper uses P1 tetrahedra, Sec. 3.1; |T| of eqs. (F_def)
 *   and (K_def) becomes the Gauss weight times det J = hx hy hz / 8).
 * - Global node (i,j,k) has id i + (nx+1)(j + (ny+1) k).
 * - Subdomains are a tensor product of per-axis cuts; box (I,J,K) has id
 *   p = I + sx (J + sy K).  Local node (li,lj,lk) of a box with (ax,ay,az)
 *   elements has id li + (ax+1)(lj + (ay+1) lk); local dof = 3 lnode + c.
 * - Decomposed vectors (u, f, du) concatenate the subdomain vectors in
 *   subdomain order: length n_dof = sum_p 3 (ax+1)(ay+1)(az+1).
 * - Element local nodes: bottom face counter-clockwise then top face,
 *   offsets (0,0,0)(1,0,0)(1,1,0)(0,1,0)(0,0,1)(1,0,1)(1,1,1)(0,1,1).
 *   Elements of a box are numbered x-fastest; Gauss point g = gx + 2 gy + 4 gz
 *   at reference coordinates (2 g_d - 1)/sqrt(3).  The Gauss-point index is
 *   gp = 8 (elem_off[p] + local element) + g, n_gp = 8 * n_elements.
 * - Stress vectors (s11,s22,s33,s12,s23,s13); strain vectors with engineering
 *   shears (e11,e22,e33,2e12,2e23,2e13) (eq. (stress_strain_vector)).
 *   Gauss-point arrays are structure-of-arrays: a [6][n_gp] stress array
 *   holds component c of point gp at c*n_gp + gp.
 * - Multipliers (rows of the orthonormal B of eq. (equ.set.matrix.B)) come in
 *   (global node, component) order.  The copies of a node are ordered by
 *   subdomain id.  A component fixed by a Dirichlet mask gives one identity
 *   row per copy; a free component with k >= 2 copies gives the k-1 Helmert
 *   rows (e_1 + ... + e_j - j e_{j+1}) / sqrt(j (j+1)), j = 1..k-1, i.e. the
 *   orthonormalised redundant gluing rows of Sec. 4.1.
 * - The generalised inverse K_p^+ is the fixing-node one of Remark 1: the
 *   rows/columns of the dofs {x,y,z of local node (0,0,0); y,z of (ax,0,0);
 *   z of (0,ay,0)} are removed and the rest is banded-Cholesky factorised.
 *   u and lambda do not depend on this choice; alpha and d do.
 */
#ifndef TFETI_H
#define TFETI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define TFETI_OK                 0
#define TFETI_ERR_ARG            1  /* invalid argument, size or pointer              */
#define TFETI_ERR_CUDA           2  /* a CUDA runtime call failed                     */
#define TFETI_ERR_OOM            3  /* device or host allocation failed               */
#define TFETI_ERR_NUMERIC        4  /* non-positive pivot in a subdomain factorisation */
#define TFETI_ERR_SINGULAR       5  /* coarse matrix G G^T not SPD (Ker K ∩ Ker B ≠ 0) */
#define TFETI_ERR_NOT_CONVERGED  6  /* iteration limit reached (last iterate written)  */
#define TFETI_ERR_BREAKDOWN      7  /* p^T F p <= 0 in PCGP                           */
#define TFETI_ERR_NONFINITE      8  /* NaN or Inf met in a residual or scalar         */
#define TFETI_ERR_TIMEOUT        9  /* a bounded device wait (bulk copy, MMA) gave up */

/* ---- problem description (host struct, copied by tfeti_setup) ------------ */
#define TFETI_PRECOND_NONE   0
#define TFETI_PRECOND_LUMPED 1      /* F^-1 ~ B K B^T (Sec. 4.2) */
/* F^-1 ~ Bbar Sbar Bbar^T (Sec. 4.2): Sbar_p the Schur complement of K_p onto the
 * nodes that carry Dirichlet or gluing rows (all components of such a node), the
 * other nodes eliminated; Bbar the columns of B there.  Applied without forming
 * Sbar: Sbar x_b = (K_p [x_b; -K_ii^-1 (K_p [x_b; 0])_i])_b with a banded Cholesky
 * of K_ii (shared by elastic subdomains of one shape and constrained-dof pattern,
 * refactorised for subdomains with plastic points). */
#define TFETI_PRECOND_DIRICHLET 2

typedef struct tfeti_problem {
    int32_t nel[3];            /* elements per axis, each >= 1                         */
    double  length[3];         /* box edge lengths, > 0                                */
    int32_t nsub[3];           /* subdomains per axis, each >= 1                       */
    const int32_t* cuts[3];    /* host, nullable: per axis nsub[a]+1 increasing cut
                                  positions from 0 to nel[a]; NULL = equal split
                                  (nel[a] must then be divisible by nsub[a])           */
    double  young, poisson;    /* E > 0, 0 < nu < 0.5                                  */
    double  sigma_y, hardening;/* initial yield stress > 0, hardening modulus H_m > 0 */
    int32_t dirichlet[6];      /* per face x0,x1,y0,y1,z0,z1: bit c = component c fixed */
    int32_t traction_face;     /* 0..5 in the same face order: the loaded face          */
    int32_t precond;           /* TFETI_PRECOND_*                                      */
    int32_t coarse;            /* TFETI_COARSE_*: how H = (G G^T)^-1 is applied         */
} tfeti_problem;

/* The coarse solve of the projector P_N (Sec. 4.2): AUTO (0) picks DENSE for
 * n_coarse <= 6144 and PLANES above.  DENSE: the explicit inverse H (n_coarse^2
 * doubles, 4.8 GB at 4096 subdomains) applied by one GEMV.  PLANES: G G^T is block
 * tridiagonal over the planes of subdomains with equal z index (a subdomain couples
 * only to the boxes around it); its block LDL^T with explicit inverses of the pivot
 * blocks is applied by 2 nz - 1 dependent GEMVs of (6 nx ny)^2, nz planes of nx x ny
 * subdomains (3 x 16 x 1536^2 doubles = 0.9 GB at 16^3 subdomains).  Both give H g to
 * rounding. */
#define TFETI_COARSE_AUTO   0
#define TFETI_COARSE_DENSE  1
#define TFETI_COARSE_PLANES 2

typedef struct tfeti_sizes {
    int64_t n_sub;             /* s                                                     */
    int64_t n_dof;             /* decomposed dofs                                       */
    int64_t n_elements;
    int64_t n_gp;              /* 8 n_elements                                          */
    int64_t n_mult;            /* m, number of rows of B                                */
    int64_t n_coarse;          /* l = 6 s                                               */
    int64_t n_nodes;           /* global nodes                                          */
    int64_t n_copy;            /* interface copy slots (3 per interface node copy)      */
    int64_t max_band;          /* largest subdomain half bandwidth (dofs)               */
    int64_t device_bytes;      /* device memory the context holds (0 for a plan)        */
} tfeti_sizes;

/* ---- host-only plan: mesh, partition and index maps, no GPU needed -------- */
typedef struct tfeti_plan tfeti_plan;

/* Builds the mesh numbering, subdomains, B (Sec. 4.1) and fixing dofs on the
 * host.  Errors: TFETI_ERR_ARG (bad sizes/cuts/material), TFETI_ERR_OOM. */
int tfeti_plan_create(const tfeti_problem* prob, tfeti_plan** out);
int tfeti_plan_destroy(tfeti_plan* plan);
int tfeti_plan_sizes(const tfeti_plan* plan, tfeti_sizes* out);
/* B as COO in row order (copies in subdomain order within a row); each array
 * holds plan nnz(B) entries, host memory, caller-allocated.  *nnz receives the
 * count; pass null arrays to query it. */
int tfeti_plan_export_B(const tfeti_plan* plan, int64_t* rows, int64_t* cols, double* vals, int64_t* nnz);
/* Per subdomain: origin[3], dims[3] (elements), dof offset, element offset,
 * half bandwidth: 9 int64 per subdomain, host memory [n_sub][9]. */
int tfeti_plan_export_subdomains(const tfeti_plan* plan, int64_t* out);
/* Fixing dofs: 6 local dof indices per subdomain, host [n_sub][6]. */
int tfeti_plan_export_fixing(const tfeti_plan* plan, int32_t* out);

/* ---- device context -------------------------------------------------------- */
typedef struct tfeti_ctx tfeti_ctx;

/* Sec. 4.1-4.2, Algorithm 3 line 1 set-up: builds the plan, uploads the index
 * maps, forms the element tables, the rigid-body bases R_p, G = R^T B^T, the
 * coarse matrix G G^T and its inverse H (factorised once: G depends only on B
 * and R), and the shared elastic factors of every subdomain shape.  The state
 * (u, sigma, kappa) starts at zero (Algorithm 1 line 1).  `cuda_stream` is a
 * cudaStream_t (nullable = default stream) on the current device.
 * Errors: TFETI_ERR_ARG, TFETI_ERR_OOM, TFETI_ERR_CUDA, TFETI_ERR_SINGULAR,
 * TFETI_ERR_NUMERIC. */
int tfeti_setup(const tfeti_problem* prob, void* cuda_stream, tfeti_ctx** out);

/* Case context: another load case on the mesh, decomposition and elastic material
 * (E, nu) of `base`, with its own yield stress sigma_y and hardening modulus H_m
 * (Sec. 2's material parameters; both > 0).  Everything that depends only on the
 * mesh, B, R and the elastic stiffness is shared with base, read-only, not copied:
 * index maps, R, G, the coarse inverse H (and its FP32 copy), the shape templates'
 * elastic factors and boundary blocks, the Dirichlet templates and the dual Schur
 * blocks.  The case owns its state (zero at creation), the factors of its plastic
 * subdomains and its work vectors, and has its own settings (precision, history,
 * learned start, timing).  base must be a context made by tfeti_setup, must outlive
 * the case, and must not be modified by another thread while a case context is being
 * set up or switched to mixed precision.  cuda_stream: the case's stream (nullable: the
 * context creates and owns a non-blocking stream).
 * Errors: TFETI_ERR_ARG, TFETI_ERR_OOM, TFETI_ERR_CUDA. */
int tfeti_setup_case(tfeti_ctx* base, double sigma_y, double hardening, void* cuda_stream, tfeti_ctx** out);
int tfeti_destroy(tfeti_ctx* ctx);
int tfeti_sizes_get(const tfeti_ctx* ctx, tfeti_sizes* out);
const char* tfeti_last_error(const tfeti_ctx* ctx);
const char* tfeti_status_str(int status);

/* Decomposed load of a uniform traction t (host double[3]) on the problem's
 * traction face: each element face gives t * area / 4 to each of its four
 * nodes in the subdomain owning the element.  f_out: device [n_dof]. */
int tfeti_traction_load(tfeti_ctx* ctx, const double* t, double* f_out);

/* Return mapping at every Gauss point (Sec. 2.4 eqs. (elast_pred),
 * (plast_corr), (stress_op), (hardening_op); Algorithm 5 lines 6-7) for the
 * displacement increment du (device [n_dof]) from the committed state
 * sigma_k, kappa_k.  Outputs (device, caller-owned): dsigma [6][n_gp],
 * dkappa [n_gp], plastic [n_gp] (1 iff Phi(sigma_k + C eta, kappa_k) > 0),
 * Dtan (nullable) [21][n_gp]: the Clarke derivative T^o_k of Sec. 3.1 as the
 * upper triangle of the 6x6 matrix, row-major (00,01,..,05,11,..,55). */
int tfeti_return_map(tfeti_ctx* ctx, const double* du, double* dsigma, double* dkappa,
                     uint8_t* plastic, double* Dtan);

/* Algorithm 5 lines 8-9 for every subdomain at du (device [n_dof]):
 * f^p = df^p - sum_T |T| dsigma_T^T G_T R_T and K^p = sum_T |T| (T^o G_T R_T)^T G_T R_T,
 * then the generalised inverse of every K^p is prepared (banded Cholesky of
 * K_rr; subdomains whose Gauss points are all elastic reuse the shared factor
 * of their shape, the others are factorised into a slot of the context's pool of
 * own factor records, which grows on demand).  df: device [n_dof]; f_out: device
 * [n_dof], nullable.  The assembled operator stays in the context for
 * tfeti_dual_pcg and the operator calls below.  Errors: TFETI_ERR_NUMERIC,
 * TFETI_ERR_OOM (the pool could not grow). */
int tfeti_assemble_tangent(tfeti_ctx* ctx, const double* du, const double* df, double* f_out);

typedef struct tfeti_pcg_info {
    int32_t iterations;        /* PCGP iterations j                                     */
    int32_t converged;         /* 1 if ||w|| <= rtol ||r^0||                             */
    int32_t used_lambda0;      /* 1: caller lambda0; 2: history start; 3: with the MLP  */
    int32_t f_applies;         /* FP64 subdomain-solve passes incl. set-up and recovery */
    double  r0_norm;           /* ||r^0|| = ||d~||                                      */
    double  w_norm;            /* last ||w^{j-1}||                                      */
    double  seconds;           /* wall time of the call                                 */
    int32_t f32_applies;       /* F-applies with FP32 subdomain solves (mixed precision) */
    int32_t outer_iterations;  /* FP64 refinement steps (mixed precision), else 0        */
} tfeti_pcg_info;

/* Algorithm 3 on the operator left by tfeti_assemble_tangent, for the
 * decomposed right-hand side f (device [n_dof]): lambda_Im = N^T H e,
 * d~ = d - F lambda_Im, PCGP with the lumped preconditioner and the stopping
 * test ||w^{j-1}|| <= rtol ||r^0|| after the updates, then alpha = H N (d - F lambda)
 * and u = K^+ (f - B^T lambda) + R alpha.  By linearity d - F lambda =
 * B K^+ (f - B^T lambda), so d~ and the recovery each take one subdomain-solve pass
 * v = K^+ (f - B^T lambda) (the residual B v and u = v + R alpha share it) instead of
 * the two of d and F lambda.  u_out: device [n_dof], nullable; lambda_out:
 * device [n_mult], nullable; lambda0: device [n_mult], nullable -- if given,
 * lambda_Ker starts from P_N lambda0 instead of o.  info: host, nullable.
 * Errors: TFETI_ERR_NOT_CONVERGED (last iterate written), TFETI_ERR_BREAKDOWN,
 * TFETI_ERR_NONFINITE, TFETI_ERR_TIMEOUT (a bounded wait of the F-apply kernels on a
 * bulk copy or MMA gave up; the context stays usable). */
int tfeti_dual_pcg(tfeti_ctx* ctx, const double* f, double* u_out, double* lambda_out,
                   const double* lambda0, double rtol, int32_t maxit, tfeti_pcg_info* info);

#define TFETI_MAX_NEWTON 64
typedef struct tfeti_step_info {
    int32_t newton;                          /* Newton iterations i                       */
    int32_t converged;
    int32_t pcg[TFETI_MAX_NEWTON];           /* PCGP iterations per Newton iteration      */
    int64_t plastic[TFETI_MAX_NEWTON];       /* plastic Gauss points per Newton iteration */
    double  criterion[TFETI_MAX_NEWTON];     /* ||du_i - du_{i-1}|| / (||du_i|| + ||du_{i-1}||) */
    int32_t refactored[TFETI_MAX_NEWTON];    /* subdomains refactorised per iteration     */
    int64_t plastic_committed;               /* plastic points of the committed state     */
    double  seconds;
    int32_t outer[TFETI_MAX_NEWTON];         /* FP64 refinement steps per Newton iteration */
    int32_t history[TFETI_MAX_NEWTON];       /* 1: history start, 2: with the MLP vector  */
} tfeti_step_info;

/* Algorithm 4 for one time step: du = o; Newton iterations of Algorithm 5 +
 * Algorithm 3 with the relative-increment stop of Algorithm 2; then commits
 * u += du and sigma, kappa += T_k, T_kappa evaluated at the final du.  On any
 * error the committed state is left at step k.  df: the load increment, host
 * memory if df_on_host != 0 else device [n_dof].  info: host, nullable.
 * Errors: TFETI_ERR_NOT_CONVERGED, and those of the calls above. */
int ssn_time_step(tfeti_ctx* ctx, const double* df, int32_t df_on_host, double newton_tol,
                  double pcg_rtol, int32_t newton_maxit, int32_t pcg_maxit, tfeti_step_info* info);

/* One time step (Algorithm 4) of n_cases independent cases at once: case k runs
 * ssn_time_step(ctxs[k], df[k], ...) on a host thread of its own and on its context's
 * stream, so the GPU overlaps the cases' kernels (the cases' Newton and PCGP iteration
 * counts differ; each stops on its own test).  ctxs: n_cases distinct contexts, each
 * with its own stream (e.g. the case contexts of one base, with or without the base);
 * df[k]: case k's load increment (host if df_on_host, else device [n_dof]); info:
 * host [n_cases], nullable.  Returns when every case's step has ended: TFETI_OK, or
 * the first non-OK status in case order (each failed case keeps its state at step k
 * and its message in tfeti_last_error(ctxs[k])). */
int ssn_time_step_cases(tfeti_ctx* const* ctxs, int32_t n_cases, const double* const* df, int32_t df_on_host,
                        double newton_tol, double pcg_rtol, int32_t newton_maxit, int32_t pcg_maxit,
                        tfeti_step_info* info);

/* Arithmetic of the dual solve.  TFETI_PRECISION_FP64 (default): Algorithm 3 in
 * FP64.  TFETI_PRECISION_MIXED: the PCGP of Algorithm 3 runs as FP64 iterative
 * refinement of the dual problem -- the true residual r = d~ - F lambda_Ker is
 * formed with FP64 subdomain solves and corrected by inner PCGP solves (FP64
 * vectors and scalars) whose operators are FP32: the projector with FP32 copies
 * of R and H, the lumped preconditioner with FP32 boundary blocks, and F with
 * subdomains still on their shape's elastic tangent applying the shape's dual
 * Schur block S = (K^+)_{boundary,boundary} (formed once in FP64, stored FP32) as
 * one GEMM per shape and the others running FP32 banded solves with their factors
 * rounded to FP32.  Each correction is projected in FP64 before it is added, so
 * lambda_Ker stays in Ker N.  Each inner solve reduces its projected residual by
 * inner_rtol (0 < inner_rtol < 1, e.g. 1e-4).  The stopping test
 * ||P r|| <= rtol ||d~|| is applied to the FP64 residual, so both modes reach
 * the same dual residual.  The paper has no mixed-precision variant; this is an
 * implementation choice for GPUs whose FP64 rate is far below their FP32 rate.
 * Switching to MIXED allocates the FP32 copies (the first time) and forms S. */
#define TFETI_PRECISION_FP64  0
#define TFETI_PRECISION_MIXED 1
int tfeti_set_precision(tfeti_ctx* ctx, int32_t mode, double inner_rtol);

/* Start of the dual PCGP from the solver's history (extension; Algorithm 3 starts
 * from lambda_Ker = o, which stays the default q = 0).  With q in 1..8 the context
 * keeps the last q solutions lambda_j (in Ker N) of tfeti_dual_pcg and their
 * products F lambda_j (= d~_j - r_j).  For a new right-hand side it solves the
 * q x q Galerkin system (L^T F L) c = L^T d~ (the F-norm-optimal start in
 * span{lambda_j}; vectors found dependent are dropped) and, if the residual this
 * predicts with the stored products is below half of ||P d~||, starts from
 * lambda_Ker = P sum_j c_j lambda_j; if the true projected residual is not below
 * ||P d~|| it falls back to lambda_Ker = o.  The stopping test stays
 * ||w|| <= rtol ||d~||, so the converged solution is the same within the
 * tolerance.  Stored products of earlier tangents are used as they are (the
 * fallback covers a stale prediction).  Resets the history. */
int tfeti_set_recycling(tfeti_ctx* ctx, int32_t q);

/* Learned start (extension; needs tfeti_set_recycling with q in 1..7): for Newton
 * iteration i <= 4 of every load step a per-interface MLP predicts lambda_Ker row by
 * row from the row's values of lambda_Ker at iteration i of the previous two load
 * steps (la, lb), the current d~, the load-increment ratio rho = df.df_prev /
 * |df_prev|^2, the plastic fractions of the row's subdomains now and at iteration i
 * of the previous step, and i: features x = (la/s, (la - lb)/s, d~/s_d, rho, pf_now,
 * pf_prev, (i-1)/3, 0), s = RMS(la), s_d = RMS(d~); prediction s (x_0 + net(x)), net =
 * 8 -> 64 -> 64 -> 1 with ReLU, FP16 weights, FP32 accumulation.  Where the stored
 * solutions alone do not meet the stopping test, the projected prediction joins them
 * as one more vector of the Galerkin start (its product by one F-apply, FP32 in the
 * mixed mode; the zero start stays the fallback).  A solve where the network's vector
 * lowers the predicted residual by less than 10 % counts against it; after two such
 * solves in a row at a Newton index it is consulted there only every fourth time, and
 * trains there only after the solves that consulted it.
 * After each solve the stored solutions could not start well the network takes
 * `epochs` Adam steps (learning rate lr, FP32 master weights) on 64 x 128 rows of the
 * solve against its lambda_Ker, on a low-priority stream of its own beside the next
 * Newton iteration (the next prediction waits for it).  Weights start from a fixed
 * seed with a zero last layer (the untrained predictor is la).  enable = 0 turns it
 * off. */
#define TFETI_MLP_PARAMS 4801
int tfeti_set_learned(tfeti_ctx* ctx, int32_t enable, int32_t epochs, double lr);

/* Subdomains with few plastic points on their shape's elastic factor in the mixed mode (an
 * extension; default mode 2).  The plastic tangent of Algorithm 5 differs from the shape's
 * elastic matrix by the element corrections, K_p = K_el - U U^T with six columns per plastic
 * Gauss point (sqrt(a |T|) B^T F, F F^T = E_eps, and sqrt(b |T|) B^T n of the Clarke tangent,
 * Sec. 3.1), so by the Sherman-Morrison-Woodbury identity the fixing-dof generalised inverse
 * (Remark 1) is K_p^+ = K_el^+ + Z C^-1 Z^T with Z = K_el^+ U and C = I - U^T K_el^+ U (set up in
 * FP64 at every assembly from the shape's dense FP64 K_el^+, formed once).
 *   mode 1: the inner FP32 F-apply of such a subdomain joins its shape's tensor-core GEMM with
 *           the elastic subdomains and adds Z_b (C^-1 Z_b^T x_b) (b: its boundary dofs), instead
 *           of a banded FP32 solve; its FP64 solves still use its refactorised tangent.
 *   mode 2: as 1, and its FP64 solves (residual solves, F-applies, K^+ applies) run on the
 *           shape's elastic factor plus Z C^-1 Z^T v, so it is not refactorised at all (not with
 *           the Dirichlet preconditioner, whose K_ii factors need the refactorisation).
 *   mode 0: off.
 * Applies to shapes with a dual Schur block in use and at most 3072 dofs and to subdomains with
 * at most 96 plastic points; the others keep the refactorisation and banded solves.  Takes
 * effect at the next assembly.  A later change of the Schur blocks in use (threshold, format)
 * first refactorises the subdomains of mode 2.  Errors: TFETI_ERR_ARG (mode not 0..2).
 * Stats: subdomain set-ups so since the context was made, and set-ups that fell back to the
 * refactorisation (a C whose Cholesky failed). */
int tfeti_set_woodbury(tfeti_ctx* ctx, int32_t mode);
int tfeti_get_woodbury_stats(tfeti_ctx* ctx, int64_t* subdomains, int64_t* fallbacks);

/* The inner PCGP iteration of the mixed mode as one cooperative launch between two F-applies
 * (an extension; default off): the contraction of F p and p.Fp, the lambda and r updates, w = P r,
 * the lumped preconditioner, y = P z and the new search direction run in one kernel with one CTA
 * per SM and grid barriers between the phases (each wait bounded: one that gives up ends the
 * dual solve with TFETI_ERR_TIMEOUT).  It applies with the lumped preconditioner, the dense coarse
 * solve and no deflation, and not inside ssn_time_step_cases with several contexts; otherwise the
 * iteration runs as separate kernels.  No other cooperative launch of the whole device may run
 * concurrently with a context's dual solves while it is on.  enable = 1 turns it on (measured
 * slower than the separate kernels on GB300: every phase is a chain of dependent loads that the
 * fusion does not shorten).  tfeti_get_fused_inner: *active = 1 if the next inner solve uses it
 * (mixed mode). */
int tfeti_set_fused_inner(tfeti_ctx* ctx, int32_t enable);
int tfeti_get_fused_inner(tfeti_ctx* ctx, int32_t* active);

/* Deflation of the inner PCGP of the mixed mode (an extension; Algorithm 3's projected CG
 * with the search directions kept conjugate to a deflation space W).  Per dual solve, at its
 * first inner solve, W holds the network's prediction (when the learned start formed one)
 * and the most recent stored solutions of the history start, up to k vectors, each
 * projected by P_N; A W is taken with the inner FP32 operators (P F P) and E = W^T A W is
 * inverted over its independent columns.  Every inner solve then starts from the Galerkin
 * correction in span W and each search direction loses its A-conjugate part in span W:
 * p = y + beta p - W E^-1 (A W)^T y.  If an outer refinement pass with deflation does not
 * reduce the FP64 residual, the rest of that dual solve runs the plain inner PCGP (fallback).
 * k = 0 (default) switches it off.  Requires tfeti_set_recycling (else TFETI_ERR_ARG); costs
 * k FP32 F-applies per dual solve that reaches the inner iterations.  Errors: TFETI_ERR_ARG
 * (k outside 0..8), TFETI_ERR_OOM. */
int tfeti_set_deflation(tfeti_ctx* ctx, int32_t k);
/* Since the last tfeti_set_deflation: deflation spaces formed, their total kept vectors,
 * and dual solves that fell back to the plain inner PCGP (all nullable). */
int tfeti_get_deflation_stats(tfeti_ctx* ctx, int64_t* setups, int64_t* vectors, int64_t* fallbacks);
/* For tests and tools: the FP32 master weights (host float[TFETI_MLP_PARAMS]: W1 [64][8],
 * b1 [64], W2 [64][64], b2 [64], w3 [64], b3), the prediction y (device [n_mult]) for
 * given device inputs la, lb, d [n_mult], pf_now, pf_prev [n_sub] and host scal[4] =
 * (1/s, 1/s_d, rho, s) with the index feature 0, and `steps` Adam steps towards the
 * device target [n_mult]. */
int tfeti_mlp_weights(tfeti_ctx* ctx, float* out);
int tfeti_mlp_predict(tfeti_ctx* ctx, const double* la, const double* lb, const double* d, const float* pf_now,
                      const float* pf_prev, const float* scal, double* y);
int tfeti_mlp_train(tfeti_ctx* ctx, const double* la, const double* lb, const double* d, const float* pf_now,
                    const float* pf_prev, const float* scal, const double* target, int32_t steps);

/* How the FP64 F-apply of the PCGP iterations treats subdomains still on their
 * shape's elastic tangent (Sec. 4.2 leaves the K^+ apply open).  BANDED (default):
 * forward and backward substitution with the shape's factor.  SCHUR: one DGEMM per
 * shape with the shape's dual Schur block S = (K^+)_{boundary,boundary} (formed once
 * in FP64 from the same factor, 1158^2 doubles for an 8^3 box), which has the same
 * flop count but keeps all SMs busy; subdomains with plastic points keep their
 * banded solves (on a second stream).  The set-up and recovery solves, which need
 * the whole local vector, stay banded. */
#define TFETI_FAPPLY_BANDED 0
#define TFETI_FAPPLY_SCHUR  1
int tfeti_set_fapply(tfeti_ctx* ctx, int32_t mode);

/* Operand format of the inner (FP32) F-apply's dual Schur blocks in the mixed mode
 * (an extension; F = B K^+ B^T of eq. (equ:sps3) applied to the subdomains on their
 * shape's elastic tangent as Y = X S on the tensor cores, FP32 accumulation).
 * TF32X3 (default): S and X split into TF32 hi/lo parts, three MMAs per step (FP32
 * accuracy).  BF16: S stored once in BF16 (half the bytes of one FP32 copy), X split
 * into BF16 hi/lo, two MMAs per step; the product then carries S's BF16 rounding
 * (~4e-3 relative) and the FP64 refinement of the mixed mode takes correspondingly
 * more outer passes.  Requires TFETI_PRECISION_MIXED (else TFETI_ERR_ARG); the BF16
 * tiles are formed at the first switch (a case context shares its base's); the inner
 * F-apply's threshold is tuned again.  Errors: TFETI_ERR_ARG, TFETI_ERR_OOM. */
#define TFETI_SCHUR_TF32X3 0
#define TFETI_SCHUR_BF16   1
int tfeti_set_schur_format(tfeti_ctx* ctx, int32_t format);
/* Overrides the autotuned choice of the inner F-apply in the mixed mode: shapes with at
 * least `threshold` subdomains (and a formed dual Schur block, i.e. at least 4) apply
 * it on the tensor cores, the others run FP32 banded solves; a later change of the
 * Schur operand format keeps it.  threshold = 0 tunes again by timing (and lets the
 * format change re-tune).  Requires TFETI_PRECISION_MIXED (else TFETI_ERR_ARG). */
int tfeti_set_schur_threshold(tfeti_ctx* ctx, int32_t threshold);

/* Autotuner of the mixed mode's inner F-apply (run when the mixed mode is switched on):
 * shapes with at least kSchurMinCount = 4 subdomains form their dual Schur block; a
 * shape applies it (one tensor-core GEMM over its elastic subdomains) only if it has at
 * least T subdomains, the others take FP32 banded solves.  T is chosen among 4, 16, 64
 * and "never" by timing the FP32 F-apply once per distinct choice.  Outputs (host,
 * nullable): the chosen T (1 << 30 = never, 0 = not tuned yet), the number of shapes
 * applying their block, and the four measured times in ms (-1 if not measured). */
int tfeti_get_tuning(tfeti_ctx* ctx, int32_t* schur_threshold, int32_t* n_schur_shapes, float* tune_ms);

/* Launch mode of the mixed-precision inner PCGP.  enable != 0 (default): each
 * inner solve is one CUDA graph launch whose body is one iteration inside a
 * WHILE conditional node, the scalars staying on the device.  enable == 0: the
 * same kernels launched one by one from the host, with the same arithmetic and
 * results (profilers that do not see into conditional graph bodies need this). */
int tfeti_set_graphs(tfeti_ctx* ctx, int32_t enable);

/* Load magnitude of the workloads: t_y = sigma_y / max_g sqrt(3/2) ||dev sigma_g||
 * for the elastic response to the unit traction `dir` (host double[3]) on the
 * traction face, solved with tfeti_dual_pcg at rtol.  Requires the zero
 * state (fresh context); leaves the committed state unchanged. */
int tfeti_first_yield_traction(tfeti_ctx* ctx, const double* dir, double rtol, double* t_y);

/* ---- committed state (checkpoint / resume, Algorithm 4 line 16-17) -------- */
/* u: [n_dof], sigma: [6][n_gp], kappa: [n_gp]; device pointers, each nullable. */
int tfeti_get_state(tfeti_ctx* ctx, double* u, double* sigma, double* kappa);
int tfeti_set_state(tfeti_ctx* ctx, const double* u, const double* sigma, const double* kappa);

/* ---- dual operators on the last assembled tangent (for tests and tools) --- */
/* y = F x = B K^+ B^T x (eq. (equ:sps3)); x, y device [n_mult]. */
int tfeti_apply_F(tfeti_ctx* ctx, const double* x, double* y);
/* y = F x with the FP32 operators of the mixed mode's inner iterations (dual Schur
 * blocks on the tensor cores for subdomains on their shape's elastic tangent, FP32
 * banded solves for the others); requires TFETI_PRECISION_MIXED, else TFETI_ERR_ARG.
 * x, y device [n_mult]. */
int tfeti_apply_F32(tfeti_ctx* ctx, const double* x, double* y);
/* y = P_N x = x - N^T (N N^T)^{-1} N x (Sec. 4.2); device [n_mult]. */
int tfeti_apply_projector(tfeti_ctx* ctx, const double* x, double* y);
/* y = the problem's preconditioner applied to x (lumped B K B^T or Dirichlet
 * Bbar Sbar Bbar^T, Sec. 4.2); device [n_mult]. */
int tfeti_apply_precond(tfeti_ctx* ctx, const double* x, double* y);
/* y = N x = -R^T B^T x; x device [n_mult], y device [n_coarse]. */
int tfeti_apply_N(tfeti_ctx* ctx, const double* x, double* y);
/* y = K^+ x per subdomain; device [n_dof]. */
int tfeti_apply_kdag(tfeti_ctx* ctx, const double* x, double* y);
/* y = K x per subdomain (the assembled tangent, fixing dofs untouched); device [n_dof]. */
int tfeti_apply_K(tfeti_ctx* ctx, const double* x, double* y);

/* ---- projector without device allocation ------------------------------------ */
/* The paper has no counterpart to this call.  It is a deployment variant of
 * tfeti_apply_projector for callers that cannot call cudaMalloc when they apply
 * the operator: their device memory is owned by another allocator (a caching
 * pool sized to the whole GPU), or their policy forbids allocation after
 * start-up.  It computes the same y = P_N x (x, y: device [n_mult]) but keeps
 * its two work vectors (G x and H G x) in a static device array of
 * 2 x TFETI_NOALLOC_MAX_COARSE doubles (384 KiB) that every GPU loading the
 * library holds until the process exits; it allocates nothing.
 * - Contexts with n_coarse > TFETI_NOALLOC_MAX_COARSE (more than 4096
 *   subdomains) are rejected with TFETI_ERR_ARG.
 * - The call runs on the context's device (the device current at its set-up):
 *   it makes that device current for its duration and then restores the
 *   caller's current device.
 * - The first call for a device resolves the array's device address on that
 *   device with cudaGetSymbolAddress; make that first call before any stream
 *   capture.
 * - All calls on a device share the array: calls whose kernels overlap on the
 *   GPU race.  Both work vectors are overwritten before they are read, so no
 *   clearing is needed between calls.
 * - It waits for its kernels before it returns (it synchronises the context's
 *   stream), and reports a failed launch or an earlier asynchronous fault on
 *   that stream as TFETI_ERR_CUDA. */
#define TFETI_NOALLOC_MAX_COARSE 24576
int tfeti_apply_projector_noalloc(tfeti_ctx* ctx, const double* x, double* y);

/* ---- timing of the last calls (host) ---------------------------------------- */
typedef struct tfeti_timing {
    double f_apply_ms_total;   /* summed device time of the F-apply kernel launches     */
    int64_t f_apply_launches;
    double f_apply_bytes;      /* algorithmic bytes of one F-apply                      */
    double f_apply_flops;      /* FP64 flops of one F-apply                             */
    double factor_ms_total;
    int64_t factor_launches;
    int64_t kernel_launches;   /* library kernels launched since the last reset         */
    /* FP64 Schur F-apply (TFETI_FAPPLY_SCHUR): device time of the gather + DGEMM launches,
     * their count (one per F-apply) and their summed algorithmic flops and bytes */
    double schur_ms_total;
    int64_t schur_launches;
    double schur_flops_total;
    double schur_bytes_total;
    /* mixed mode: device time of the inner FP32 PCGP solves launched as graphs, their PCGP
     * iterations and graph body runs (each run is one iteration; the last may stop early) */
    double inner_ms_total;
    int64_t inner_iterations;
    int64_t inner_body_runs;
} tfeti_timing;
int tfeti_timing_get(tfeti_ctx* ctx, tfeti_timing* out);
int tfeti_timing_reset(tfeti_ctx* ctx, int32_t enable_events);

/* Failure detection of the bounded device waits (no context needed): one CTA waits on
 * an mbarrier phase that nothing completes, with the bounded wait of the F-apply
 * kernels limited to limit_cycles SM cycles (1 .. 2^31); the wait gives up, the kernel
 * returns normally and *gave_up (host) is set to 1 (0 would mean the wait completed).
 * Nothing faults or hangs; the device stays usable.  cuda_stream: nullable. */
int tfeti_check_bounded_wait(void* cuda_stream, int64_t limit_cycles, int32_t* gave_up);

/* FP64 FMA throughput of the current device (no context needed; the paper has no
 * counterpart: it is the roofline denominator of the FP64 kernels, whose
 * arithmetic intensity lies above the FP64 ridge on this hardware).  Every thread
 * of 4 CTAs x 256 threads per SM runs 16 independent FMA chains for `iters`
 * iterations after a short warm-up launch; *tflops (host) = 32 x threads x iters /
 * CUDA-event time of the launch, in TFLOP/s.  cuda_stream: nullable.  Errors:
 * TFETI_ERR_ARG (iters < 1, null output), TFETI_ERR_CUDA. */
int tfeti_measure_fp64_fma(void* cuda_stream, int32_t iters, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* TFETI_H */
