/*
 * igamg.h -- C ABI of the GB300 library for the structure-preserving geometric
 * multigrid V-cycle of Coley, Benzaken & Evans, "A geometric multigrid method for
 * isogeometric compatible discretizations of the generalized Stokes and Oseen
 * problems" (arXiv 1705.09282).
 *
 * Problem (Sec. 2, eqs. for the generalized Stokes / Oseen systems; weak form Sec. 3.1,
 * Nitsche no-slip Sec. 3.3):
 *     sigma u + beta.grad u - nu Lap u + grad p = f,  div u = 0  on (0,1)^2,
 *     u.n = 0 strongly, u x n = 0 weakly with penalty C_I nu / h, C_I = 4(p-1) (Sec. 6).
 * Discretization: 2D compatible B-splines (Sec. 4.3) -- streamfunction degree p,
 * velocity S^{p,p-1} x S^{p-1,p}, pressure S^{p-1,p-1}, maximal smoothness, uniform
 * knots, n_fine elements per direction; mean(p) = 0 by a Lagrange multiplier.
 *
 * Vector layout (U, F, R; device or host as stated, double, contiguous), on a level
 * with n elements per direction, q = p-1:
 *     [ u_x : (n+q) rows (y) x (n+p-2) columns (x, interior indices 1..n+p-2), x fastest
 *       u_y : (n+p-2) rows (y, interior 1..n+p-2) x (n+q) columns (x), x fastest
 *       p   : (n+q) x (n+q), x fastest
 *       lambda (the multiplier) ]
 * Levels are numbered 0 (coarsest, n_fine >> (n_levels-1) elements) .. n_levels-1 (finest).
 *
 * 3D (dim = 3, unit cube; Sec. 4.3 in three dimensions, Sec. 6.3): velocity
 * S^{p,q,q} x S^{q,p,q} x S^{q,q,p}, pressure S^{q,q,q}; with ni = n+p-2, nq = n+q:
 *     [ u_x : (z: nq) x (y: nq) x (x: ni, interior 1..ni), x fastest
 *       u_y : nq x ni x nq     u_z : ni x nq x nq      p : nq x nq x nq      lambda ]
 * f and beta are sampled at the quadrature points as (3, nG, nG, nG) [comp][z][y][x].
 * Subdomains are the supports of the vector-potential basis functions (Sec. 5.2), in
 * three families; the smoother is multiplicative (eq. MSM) only and beta must be NULL
 * (other choices return IGAMG_EUNSUPPORTED), as are igamg_streamfunction,
 * igamg_warm_start and igamg_residual_static.
 *
 * Conventions: every call enqueues its GPU work on the stream given to igamg_create
 * (a cudaStream_t passed as void*) and returns without synchronising, unless it says
 * otherwise.  The caller owns U, F, R (device memory, e.g. from PyTorch); the library
 * owns the hierarchy and every workspace, allocated in igamg_create and freed in
 * igamg_destroy; no other call allocates device memory.  A handle is not thread-safe.
 * Return value: 0 on success, a negative IGAMG_E* code on error (nothing is enqueued
 * then), IGAMG_NOT_CONVERGED (> 0) from igamg_solve when max_cycles ran out.
 */
#ifndef IGAMG_H
#define IGAMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  IGAMG_OK = 0,
  IGAMG_NOT_CONVERGED = 1,
  IGAMG_EINVAL = -1,       /* bad argument: null pointer, size, level, degree ... */
  IGAMG_EUNSUPPORTED = -2, /* valid but not built (e.g. dim = 3, p > 3) */
  IGAMG_ESINGULAR = -3,    /* a local patch or the coarsest matrix had a zero pivot */
  IGAMG_ENONFINITE = -4,   /* NaN / Inf in a residual norm */
  IGAMG_ECUDA = -5,        /* a CUDA runtime call failed */
  IGAMG_ETIMEOUT = -6
};

enum { IGAMG_MULT = 0, IGAMG_ADD = 1 };          /* eq. MSM / eq. ASM of Sec. 5.2 */
/* Precision / wrapper of the solve:
 *   IGAMG_FP64         plain FP64 V-cycles (Algorithm 1 as the solver)
 *   IGAMG_FP32_IR      FP32 V-cycles inside FP64 iterative refinement
 *   IGAMG_FGMRES_FP64  FGMRES(m) in FP64 with one FP64 V-cycle as right preconditioner
 *   IGAMG_FGMRES_FP32  FGMRES(m) in FP64 with one FP32 V-cycle as right preconditioner
 * In every mode each update of the velocity is divergence-free to FP64 round-off (the FP32
 * corrections enter through the FP64 curl of a potential, Sec. 4.3 complex). */
enum { IGAMG_FP64 = 0, IGAMG_FP32_IR = 1, IGAMG_FGMRES_FP64 = 2, IGAMG_FGMRES_FP32 = 3 };

typedef struct {
  int dim;            /* 2, or 3 (unit cube, see the 3D layout above) */
  int p;              /* streamfunction degree (Sec. 6 convention), 2 or 3 */
  int n_fine;         /* elements per direction on the finest grid */
  int n_levels;       /* number of grids; n_fine must be divisible by 2^(n_levels-1) */
  double sigma, nu;   /* reaction and viscosity, both > 0 */
  double c_penalty;   /* Nitsche constant C_I; <= 0 selects 4(p-1) (Sec. 6) */
  const double* beta_qp; /* host; advection at the quadrature points, (2, nG, nG) like f,
                            or NULL for generalized Stokes */
  int smoother;       /* IGAMG_MULT or IGAMG_ADD */
  double eta;         /* additive scaling factor (Sec. 5.2, eq. ASM); <= 0 selects 0.3 (the
                       * paper runs 0.5, under which these subdomains diverge in pressure) */
  int nu1, nu2;       /* pre- / post-smoothing sweeps (Algorithm 1) */
  int precision;      /* IGAMG_FP64, IGAMG_FP32_IR, IGAMG_FGMRES_FP64 or IGAMG_FGMRES_FP32 */
  int restart;        /* FGMRES: Krylov directions per restart cycle; <= 0 selects 20 */
  int gamma;          /* coarse cycles per level: <= 1 the V-cycle of Algorithm 1, 2 the
                         W-cycle (the second coarse cycle continues from the first); Sec. 5
                         opening paragraph.  At most 4. */
  int fmg;            /* 1: every solve's first step is one full-multigrid pass (nested
                         iteration: the residual restricted to all levels, the coarsest
                         solved exactly, one cycle per finer level from the prolongated
                         coarser solution), U += its result; it counts as one cycle.
                         Not with the FGMRES precisions (IGAMG_EUNSUPPORTED). */
  int geometry;       /* IGAMG_GEOM_SQUARE (unit square / cube); generalized Stokes only:
                         IGAMG_GEOM_QUARTER_ANNULUS (2D, Sec. 6.2's domain) or
                         IGAMG_GEOM_HOLLOW_CYLINDER (3D, Sec. 6.4: the annulus extruded by 0.1) */
  double r_inner, r_outer; /* quarter annulus radii; <= 0 selects 0.075 and 0.225 */
} igamg_problem;

/* Domains.  The quarter annulus {r_inner <= |x| <= r_outer, x, y >= 0} is the image of the
 * unit square under F(xi, eta) = (r_inner + (r_outer - r_inner) xi) C(eta), C the rational
 * quadratic Bezier quarter circle (control points (1,0), (1,1), (0,1), weights 1, 1/sqrt(2),
 * 1): xi is radial, eta angular.  The discrete spaces are the push-forwards of Sec. 4.3
 * (velocity by the contravariant Piola map, pressure by 1/det J), so U keeps the unit
 * square's layout of parametric coefficients, div u = (1/det J) div_hat u_hat stays exactly
 * zero, and the curl / streamfunction entry points act on the same coefficients.  The
 * operator has variable coefficients and couples u_x with u_y; it is assembled on the host
 * at creation (Nitsche terms on all four walls with h = the element height normal to the
 * wall), the coarse operators are Galerkin products and every patch has its own inverse. */
/* The hollow cylinder section is that map extruded: F(xi, eta, zeta) = (quarter-annulus map
 * of (xi, eta), 0.1 zeta); its operator couples u_x with u_y (an extra record box per row of
 * those two), u_z only with itself and the pressure. */
enum { IGAMG_GEOM_SQUARE = 0, IGAMG_GEOM_QUARTER_ANNULUS = 1, IGAMG_GEOM_HOLLOW_CYLINDER = 2 };

typedef struct {
  int n;              /* elements per direction on this level */
  int nx_ux, ny_ux;   /* u_x block: columns (x) and rows (y) */
  int nx_uy, ny_uy;
  int n_pdir;         /* pressure coefficients per direction, n+p-1 */
  long long n_ux, n_uy, n_p, n_total; /* n_total includes lambda */
  int n_patches;      /* interior streamfunction supports = (n+p-2)^2 (3D: vector-potential
                         supports, 3 (n+p-1)(n+p-2)^2) */
  int n_colours;      /* (p+1)^2 (3D: 3 p (p+1)^2) */
  int n_quad;         /* quadrature points per element per direction (p+2) */
  int dim;            /* 2 or 3 */
  long long n_uz;     /* 3D: size of the u_z block (0 in 2D) */
} igamg_sizes;

typedef struct {
  int cycles;            /* V-cycles done */
  double res0;           /* ||F - K U_0||_2 */
  double rel_residual;   /* ||F - K U||_2 / res0 at exit */
  double div_inf;        /* max |coefficient of div u| at exit */
  double* history;       /* optional caller buffer for relative residuals, or NULL */
  int history_cap;       /* its capacity */
} igamg_report;

typedef struct igamg_handle igamg_handle;

/* Builds the level hierarchy (Sec. 5.1): 1D factors of every level's operator, the
 * knot-insertion transfers, the patch subdomains with their bordered local inverses
 * (Sec. 5.2), the colouring and the inverse of the coarsest matrix, and uploads them.
 * Synchronous.  *out receives a new handle (free with igamg_destroy). */
int igamg_create(const igamg_problem* prob, void* cuda_stream, igamg_handle** out);
void igamg_destroy(igamg_handle* h);
const char* igamg_strerror(int code);

/* Sizes of one level (0 = coarsest). */
int igamg_get_sizes(const igamg_handle* h, int level, igamg_sizes* out);

/* Writes the n*G 1D quadrature abscissae of the finest level into x (host, capacity cap);
 * f and beta are sampled at their tensor products, layout (2, n*G, n*G) [comp][y][x]. */
int igamg_quad_points(const igamg_handle* h, double* x, size_t cap, size_t* n_out);

/* Physical coordinates of the finest level's quadrature points (host, capacity cap >= *n_out):
 * 2D (2, n*G, n*G) [x or y][eta point][xi point], 3D (3, n*G, n*G, n*G) [x, y or z][zeta][eta]
 * [xi]; on the unit square / cube the tensor products of igamg_quad_points, on a mapped
 * domain their images under the map. */
int igamg_quad_points_xy(const igamg_handle* h, double* xy, size_t cap, size_t* n_out);

/* F = (l(v), 0, 0), l(v) = int v.f (Sec. 3.1), f at the quadrature points (device), layout
 * (2, n*G, n*G) (3D: (3, n*G, n*G, n*G)).  On a mapped domain f is the physical field at the
 * points of igamg_quad_points_xy and l(v) = int (J^T f) . v_hat dxi (Sec. 4.3 push-forward). */
int igamg_load_vector(igamg_handle* h, const double* f_qp, double* F);

/* R = F - K_l U on level l (Sec. 3.4; coarse K_l = R K P, Sec. 5.1).  If norm_out is
 * not NULL the call synchronises and writes ||R||_2 there (host). */
int igamg_residual(igamg_handle* h, int level, const double* U, const double* F,
                   double* R, double* norm_out);

/* `sweeps` applications of the level's Schwarz smoother to U in place (Sec. 5.2). */
int igamg_smooth(igamg_handle* h, int level, double* U, const double* F, int sweeps);

/* The form of level `level`'s multiplicative sweep that the autotuner chose at creation (2D):
 * *lanes = lanes per local row of the 8-DOF patches (1 or 2), *threads = threads per block,
 * *tiles = 0 for one launch per colour, else the number of tiles of the pipelined sweep
 * (1: the whole level in one block).  Any output may be NULL.  Errors: IGAMG_EINVAL,
 * IGAMG_EUNSUPPORTED (3D handle). */
int igamg_level_form(const igamg_handle* h, int level, int* lanes, int* threads, int* tiles);

/* The number of independent multiply-add chains per patch row (4 or 2) of level `level`'s
 * one-lane FP64 colour kernel, as the autotuner chose it at creation (4 for the other forms;
 * the FP32 kernels always use 4): 4 shortens each lane's dependent chain, 2 spends four fewer
 * FP64 adds per lane.  Errors:
 * IGAMG_EINVAL (NULL handle or output, level out of range), IGAMG_EUNSUPPORTED (3D handle). */
int igamg_level_chains(const igamg_handle* h, int level, int* chains);

/* The same in FP32 (the inner smoother of the FP32-in-FP64 modes): U, F are FP32 device
 * vectors in the level's layout; the handle must be 2D with precision IGAMG_FP32_IR or
 * IGAMG_FGMRES_FP32 (else IGAMG_EUNSUPPORTED). */
int igamg_smooth_f32(igamg_handle* h, int level, float* U, const float* F, int sweeps);

/* R = F - K_l U in FP32 on level `level` (the inner residual of the FP32-in-FP64 modes, Sec. 5.1
 * step 2 of the V-cycle): U, F, R are FP32 device vectors in the level's layout; the lambda row
 * and the norm as in igamg_residual (the norm is accumulated in FP64).  Same handle
 * requirements and errors as igamg_smooth_f32. */
int igamg_residual_f32(igamg_handle* h, int level, const float* U, const float* F, float* R,
                       double* norm_out);

/* How the finest level's residual applies the operator, per precision (2D handles):
 * 0 = class stencils (generalized Stokes on the square, no advection), 1 = one stored record
 * per row (Stokes part plus the advection term of Sec. 3.1's generalized Oseen problem),
 * 2 = Stokes part from the class stencils plus the advection term evaluated matrix-free,
 * element by element at the (p+2)^2 Gauss points with sum factorisation.  The handle times
 * forms 1 and 2 at creation and keeps the faster (IGAMG_ADV_FORM=records or =mf pins one).
 * *form64 is the FP64 path's form; *form32 the FP32 V-cycle's, or -1 if the handle has none.
 * Either output may be NULL.  Errors: IGAMG_EINVAL (NULL handle), IGAMG_EUNSUPPORTED (3D). */
int igamg_residual_form(const igamg_handle* h, int* form64, int* form32);

/* Sets the finest residual's operator form of a generalized-Oseen handle on the square:
 * 1 = per-row records, 2 = matrix-free advection, 0 = leave that precision's form as it is;
 * form64 for the FP64 path, form32 for the FP32 V-cycle.  Synchronises the handle's streams
 * and drops its captured solve graphs (they are captured again on the next solve).  Errors:
 * IGAMG_EINVAL (NULL handle, a form outside 0..2), IGAMG_EUNSUPPORTED (3D handle, no advection
 * term, or form32 set on a handle without an FP32 V-cycle). */
int igamg_set_residual_form(igamg_handle* h, int form64, int form32);

/* G = R_l r = P_{l-1}^T r: restriction from level l to level l-1 (Sec. 5.1). */
int igamg_restrict(igamg_handle* h, int level, const double* r_fine, double* g_coarse);

/* u_fine += P_{l-1} u_coarse: prolongation from level l-1 to level l (Sec. 5.1). */
int igamg_prolong_add(igamg_handle* h, int level, const double* u_coarse, double* u_fine);

/* U = K_0^{-1} G on the coarsest level (Algorithm 1, exact solve). */
int igamg_coarse_solve(igamg_handle* h, const double* G, double* U);

/* One V-cycle MGV(n_levels-1, U, F) of Algorithm 1, in place on U (device). */
int igamg_vcycle(igamg_handle* h, double* U, const double* F);

/* V-cycles until ||F - K U||_2 <= rtol ||F - K U_0||_2 or max_cycles (Sec. 6 protocol with
 * the tolerance as a parameter).  Synchronises once per cycle to read the norm.
 * FGMRES modes: max_cycles bounds the preconditioner applications (V-cycles), the report
 * counts them, its history holds the Krylov residual estimates, and the stopping test uses
 * the true residual at the end of each restart cycle.  igamg_vcycle on such a handle runs one
 * V-cycle of the underlying precision (FP64, or one FP32 refinement step).
 * rep may be NULL.  Returns IGAMG_NOT_CONVERGED (U holds the last iterate) if the
 * tolerance was not met, IGAMG_ENONFINITE if a norm was NaN/Inf. */
int igamg_solve(igamg_handle* h, double* U, const double* F, double rtol, int max_cycles,
                igamg_report* rep);

/* End-to-end form of igamg_solve with HOST buffers: copies f (host, quadrature points)
 * and the initial U (host) to the device, builds F, solves, copies U back.  Synchronous. */
int igamg_solve_host(igamg_handle* h, const double* f_qp_host, double* U_host, double rtol,
                     int max_cycles, igamg_report* rep);

/* n independent solves at once (same contract as igamg_solve for each), e.g. a sweep of
 * sigma/nu values or of right-hand sides.  2D FP64 multiplicative V-cycle solves step in
 * lockstep in groups of 8 or more: first one group per mesh structure (same p, n_fine,
 * levels, sweeps, domain and operator form), then one group per cycle shape (p, sweeps,
 * domain, operator form) of the remaining solves, whatever their mesh sizes (their V-cycles
 * aligned from the finest grid); each
 * V-cycle step is one launch over up to 24 of them, converged solves switched off on the
 * device; the group's first call with a new list of handles and vectors allocates its small
 * workspace and captures its graphs (kept with the group's first handle and reused while the
 * list is the same).  All other solves run on their handles' own internal streams, each cycle
 * a captured graph, and each solve's next cycle is launched as soon as its own residual norm
 * is back, so latency-bound small solves overlap and none waits for another.  Work is ordered
 * after, and joined back into, the streams given to igamg_create.  U[i], F[i]:
 * device vectors of handles[i]; reports, status: NULL or arrays of n (status[i] =
 * igamg_solve's return value for solve i).  Handles must be distinct (IGAMG_EINVAL).  Returns
 * the first negative status, else IGAMG_NOT_CONVERGED if any solve ran out of cycles, else 0.
 * Synchronous.  n = 0 returns 0. */
int igamg_solve_batch(int n, igamg_handle** handles, double** U, const double** F, double rtol,
                      int max_cycles, igamg_report* reports, int* status);

/* As igamg_solve / igamg_solve_batch, but stopping at an absolute residual norm
 * ||F - K U||_2 <= atol (per solve), e.g. atol = 1e-8 ||F||_2 to compare initial guesses
 * fairly (a better guess must not be asked for a smaller residual). */
int igamg_solve_abs(igamg_handle* h, double* U, const double* F, double atol, int max_cycles,
                    igamg_report* rep);
int igamg_solve_batch_abs(int n, igamg_handle** handles, double** U, const double** F,
                          const double* atol, int max_cycles, igamg_report* reports, int* status);

/* Discrete streamfunction psi (FP64, (n+p-2)^2 interior coefficients) of a divergence-free
 * velocity in U, by integrating u_x = d psi/dy along y from the bottom wall (Sec. 4.3
 * complex: curl is onto the divergence-free velocities).  Target data for the warm start. */
int igamg_streamfunction(igamg_handle* h, const double* U, double* psi);

/* Learned warm start from a two-channel network output grid (float, (2, n+p, n+p), device):
 * U = (curl psi, p, 0) with psi = psi_scale * channel 0 on the interior (boundary ring
 * ignored) and the pressure coefficients = p_scale * channel 1 on its leading
 * (n+p-1) x (n+p-1) points.  The velocity is exactly divergence-free. */
int igamg_warm_start(igamg_handle* h, const float* grid, double psi_scale, double p_scale, double* U);

/* The same guess with its two predicted fields scaled against F (device, the load vector):
 * U = (alpha curl psi, beta p), u = curl(psi_scale * channel 0) and p = p_scale * channel 1
 * as above.  (alpha, beta) minimise ||F - K U||_2, the residual that an absolute stopping
 * test measures (Eq. (3.1)'s matrix K, Sec. 3): a 2 x 2 least-squares problem from five
 * inner products.  alpha = beta = 0 is admissible, so the first residual is never larger
 * than that of the zero guess; an exact solution direction is reproduced exactly.  The
 * velocity stays exactly divergence-free.  Synchronises; alpha, beta (host) may be NULL.
 * Uses the handle's host-solve and residual workspaces: not concurrent with its solves.
 * Errors: IGAMG_EINVAL (null pointer), IGAMG_EUNSUPPORTED (3D handle), IGAMG_ENONFINITE. */
int igamg_warm_start_minres(igamg_handle* h, const float* grid, double psi_scale, double p_scale,
                            const double* F, double* U, double* alpha, double* beta);

/* ---- the warm-start network ------------------------------------------------------------
 * 3x3 convolutions in_channels -> width -> width -> width -> 2, GELU after the first three
 * (only in_channels = 3, width = 32 are built); layer l spreads its taps by dilations[l]
 * in {1, 2, 4, 8} (NULL: all 1), which widens the receptive field without more layers.
 * Inputs x: (B, 3, H, W) float, device; outputs / targets: (B, 2, H, W) float, device
 * (channel 0: scaled streamfunction, channel 1: scaled pressure).  The loss is the sum of
 * the channels' mean squared errors, channel 0 over the interior points (the boundary
 * ring, where psi = 0, is excluded), channel 1 over the leading (H-1) x (W-1) points.
 * Weights are used in BF16 with FP32 accumulation; the optimizer (Adam) keeps an FP32
 * master copy.  Work goes on the given stream; workspaces grow on first use of a larger
 * B*H*W. */
typedef struct igamg_nn igamg_nn;
int igamg_nn_create(int in_channels, int width, const int* dilations, unsigned long long seed,
                    void* cuda_stream, igamg_nn** out);
void igamg_nn_destroy(igamg_nn* nn);
int igamg_nn_num_params(const igamg_nn* nn);
/* parameters in the order w1 (32,3,3,3), b1, w2 (32,32,3,3), b2, w3, b3, w4 (2,32,3,3), b4 */
int igamg_nn_get_params(igamg_nn* nn, float* host, size_t cap);
int igamg_nn_set_params(igamg_nn* nn, const float* host, size_t n);
int igamg_nn_forward(igamg_nn* nn, int B, int H, int W, const float* x, float* out);
/* loss (host) and, if grad_host != NULL, the gradient (host, parameter order); no update */
int igamg_nn_loss_grad(igamg_nn* nn, int B, int H, int W, const float* x, const float* target,
                       double* loss, float* grad_host);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on one minibatch; loss (host) optional */
int igamg_nn_train_step(igamg_nn* nn, int B, int H, int W, const float* x, const float* target,
                        float lr, double* loss);

/* max over pressure-space coefficients of |div u_h| (Lemma, Sec. 4.1: zero up to
 * round-off for the iterates of Sec. 5.3).  Synchronises; result on the host. */
int igamg_div_inf(igamg_handle* h, const double* U, double* out);

/* Velocity blocks of U = curl psi = (d psi/dy, -d psi/dx) for psi given on the
 * (n+p-2)^2 interior streamfunction coefficients (Sec. 4.3 complex); the pressure and
 * lambda entries of U are not touched.
 * 3D: psi is a vector potential in S^{q,p,p} x S^{p,q,p} x S^{p,p,q} with psi x n = 0,
 * given as three consecutive families of nq*ni*ni coefficients each, x fastest:
 *   psi_x: (z: ni, interior) x (y: ni, interior) x (x: nq),
 *   psi_y: (z: ni) x (y: nq) x (x: ni),   psi_z: (z: nq) x (y: ni) x (x: ni). */
int igamg_curl(igamg_handle* h, const double* psi, double* U);

/* Same result as igamg_residual on level `level` of the hierarchy that *prob describes,
 * but without a handle and without allocating device memory: for callers that cannot
 * call cudaMalloc (their device memory is owned by a pool, an arena or a host framework).
 * The paper has no counterpart; this is a deployment convenience.
 *   Scratch: a 1 MiB array that the library declares statically in device memory
 *   (each GPU that loads the library keeps it until exit) holds this level's class
 *   stencil tables (10,164 doubles for p = 2, 44,550 for p = 3) and two partial sums per
 *   256 rows.  That fits levels of up to n = 2270 elements per direction for p = 2 and
 *   n = 1919 for p = 3; a larger level is rejected before any GPU work: the call returns
 *   IGAMG_EINVAL and prints the needed and available sizes on stderr.
 *   The first call on a device looks up the array's device address (with that device
 *   current, under a lock, so first calls from several threads are safe) and keeps it
 *   for the life of the process; make that first call before any stream capture.  After
 *   cudaDeviceReset on a device the kept address is stale: do not call this entry point
 *   on that device again in the same process.
 *   Every call reuses the same array and rewrites all of it that it reads, so nothing
 *   carries over; calls whose GPU work overlaps (other streams, other threads) race on
 *   it and must be serialised by the caller.
 *   U, F, R: device, layout above, R written; norm_out: host or NULL (if given, the call
 *   synchronises the stream).  cuda_stream: a cudaStream_t as void*, or NULL.
 *   Errors: IGAMG_EINVAL (bad sizes or pointers, level too large), IGAMG_EUNSUPPORTED
 *   (not 2D Stokes on the square with p = 2 or 3, or cuda_stream in capture mode),
 *   IGAMG_ECUDA. */
int igamg_residual_static(const igamg_problem* prob, int level, const double* U,
                          const double* F, double* R, double* norm_out, void* cuda_stream);

/* ---- measurement ----------------------------------------------------------------------
 * Arithmetic peak probe, not part of the method: enqueues one kernel of `blocks` blocks of
 * 256 threads, each thread running 8 independent multiply-add chains for `iters` rounds in
 * FP64 (fp64 != 0) or FP32, and stores one value per thread into out (device, blocks * 256
 * doubles or floats).  *flops (host, may be NULL) receives the kernel's multiply-add flops
 * (2 per FMA).  Timed by the caller with events on cuda_stream, it gives the GPU's
 * measured FMA throughput, the denominator of the roofline of FMA-issue-bound kernels.
 * Errors: IGAMG_EINVAL (non-positive sizes, null out), IGAMG_ECUDA (launch failed). */
int igamg_probe_fma(int fp64, int blocks, int iters, void* out, void* cuda_stream, double* flops);

/* ---- host-only inspection of the set-up (no GPU needed; for tests) -------------------
 * Each call builds the hierarchy on the host and copies one piece out, dense, row-major.
 * They exist so that the host set-up can be checked against an independent assembly
 * without a GPU.  cap is the capacity of the output in doubles; *n_out gets the number
 * of rows (the matrix is n_out x n_out or n_out x *n_cols). */

/* K_l as the library applies it (Sec. 3.4; coarse levels = R K P of Sec. 5.1). */
int igamg_host_level_matrix(const igamg_problem* prob, int level, double* K, size_t cap,
                            long long* n_out);
/* K_l rebuilt through the row evaluation that the GPU kernels run (class stencils). */
int igamg_host_operator_rows(const igamg_problem* prob, int level, double* K, size_t cap,
                             long long* n_out);
/* KV = K_l V (V, KV: host, n = level's n_total entries) through the same row evaluation
 * the GPU kernels run: a cheap check of the row tables on large levels. */
int igamg_host_operator_apply(const igamg_problem* prob, int level, const double* V, double* KV,
                              size_t n);
/* P_{l-1} (rows: level l, columns: level l-1), block diag(P^v, P^q, 1) of Sec. 5.1. */
int igamg_host_prolongation(const igamg_problem* prob, int level, double* P, size_t cap,
                            long long* n_rows, long long* n_cols);
/* Patch tables of level l (Sec. 5.2): for patch k in colour-major order, colour[k] and
 * its DOF list dofs[k*maxl .. k*maxl+maxl) (-1 padded).  Capacities in entries. */
int igamg_host_patches(const igamg_problem* prob, int level, int* colour, int* dofs,
                       size_t cap_patches, size_t cap_dofs, int* n_patches, int* maxl);

#ifdef __cplusplus
}
#endif
#endif
