/*
 * fhs.h - C ABI of the GB300 (sm_103a) Faceted HyperSARA PDFB hot path.
 *
 * Method: Thouvenin, Abdulaziz, Dabbech, Repetti, Wiaux, "Parallel faceted
 * imaging in radio interferometry via proximal splitting (Faceted HyperSARA)",
 * arXiv 2003.07358.  One call of fhs_pdfb_iter performs iterations of
 * Algorithm 2 on every spectral sub-cube ("cube") of a context.
 *
 * General conventions
 *  - Every array argument is a DEVICE pointer owned by the caller unless the
 *    comment says "host".  The library owns only its context (geometry tables,
 *    sorted visibility coordinates, FFT and filter tables, scratch buffers).
 *  - Real arrays are float32; complex arrays are complex64 stored as
 *    interleaved (re, im) float pairs and passed as float*.
 *  - Images are [L][n1][n2] row-major (channel, row, column).
 *  - Visibility-domain arrays (y, v, u_prev, results of fhs_measure) are in the
 *    context's INTERNAL order: channel-major, each channel sorted by grid
 *    tile.  fhs_vis_to_internal / fhs_vis_to_user convert from / to the
 *    caller's order (the order of the uv array given to fhs_create).
 *  - All work is asynchronous on the stream given to fhs_create, except the
 *    calls documented as synchronising.  Calls on one context must not overlap.
 *  - Errors: every call returns an fhs_status; nothing aborts.  The message of
 *    the last error is returned by fhs_last_error.  A CUDA error that leaves
 *    the context unusable returns FHS_ERR_CUDA on every later call.
 */
#ifndef FHS_H
#define FHS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fhs_ctx fhs_ctx;
typedef int32_t fhs_status;

enum {
  FHS_OK = 0,
  FHS_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range */
  FHS_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed   */
  FHS_ERR_OOM = 3,         /* device memory for the context could not be allocated */
  FHS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up (fhs_sync) */
  FHS_ERR_NONFINITE = 5,   /* a norm reduction produced NaN or Inf          */
  FHS_ERR_UNSUPPORTED = 6  /* shape outside what this build implements      */
};

enum { FHS_WIN_TRIANGULAR = 0, FHS_WIN_SINE = 1 };

/* One spectral sub-cube (Section 2.4.1: channel-interleaved sub-problems
 * are independent).  Shapes this build supports: n1, n2 powers of two in
 * [16, 4096]; 1 <= L <= 64; 1 <= Qy <= n1/16, 1 <= Qx <= n2/16;
 * 0 <= overlap < 0.5; 1 <= B <= 16.                                         */
typedef struct {
  int32_t n1, n2;        /* image rows, columns                                 */
  int32_t L;             /* channels of this sub-cube                           */
  int32_t Qy, Qx;        /* spatial facet grid, Section 2.4.2 (nuclear facets)  */
  double overlap;        /* nuclear facet overlap, fraction of the tile side    */
  int32_t window;        /* FHS_WIN_TRIANGULAR (Fig. 2) or FHS_WIN_SINE         */
  int32_t B;             /* data blocks per channel, Eq. (2)                    */
  const int64_t* M;      /* host [L*B]: visibilities of (channel l, block b)    */
  const float* uv;       /* host [sum(M)][2]: (u, v) in rad/pixel, |u|,|v| < pi,
                            channel-major, block-contiguous; u pairs with the
                            column coordinate c - n2/2, v with the row r - n1/2 */
  double tau, zeta, kappa;   /* step sizes of Algorithm 2 (Section 3.2)         */
  const double* eta;     /* host [L]: eta_l = 1/||Phi_l||_S^2                   */
  double mu;             /* mu_c = upsilon_c, Eq. (FHS sparsity heuristic)      */
  const double* mu_bar;  /* host [Qy*Qx]: mu_bar_{c,q} = upsilon_bar_{c,q}      */
  const double* eps;     /* host [L*B]: l2-ball radii eps_{l,b}, Eq. (3)        */
} fhs_cube_desc;

/* Sizes of the caller-owned arrays of one cube. */
typedef struct {
  int64_t n_pix;         /* n1*n2                                               */
  int64_t n_vis;         /* total visibilities of the cube (all channels)       */
  int64_t n_coef;        /* I: SARA coefficients per channel (layout below)     */
  int64_t n_facet_pix;   /* sum over nuclear facets of their pixel count        */
  int32_t n_facets;      /* Qy*Qx                                               */
  int32_t n_blocks;      /* L*B                                                 */
} fhs_sizes;

/* Dual variables and weights of one cube (Algorithm 2 inputs), caller-owned:
 *  W         [L][I] float: SARA dual, coefficient layout:
 *            for basis b = db1..db8 (filter length 2b): for level j = 1..4:
 *            subbands d0 (rows: low, cols: high), d1 (rows: high, cols: low),
 *            d2 (high, high), each [r_j][c_j] row-major with
 *            r_j = floor((r_{j-1} + 2b - 1)/2), r_0 = n1 (c_j likewise);
 *            then LL4 [r_4][c_4]; after db8 the Dirac block [n1][n2].
 *  theta     [I] float: l2,1 weights (Eq. 10), shared by the channels.
 *  P         float: nuclear duals, facet q = qy*Qx + qx stored [L][h_q][w_q]
 *            at offset L * sum_{q'<q} h_q' w_q'; facet q covers rows
 *            [floor(qy n1/Qy) - o, floor((qy+1) n1/Qy)) with
 *            o = floor(overlap * tile height) for qy > 0 (0 for qy = 0);
 *            columns likewise.
 *  theta_bar [Qy*Qx][L] float: nuclear weights (Eq. 9), index j pairs with the
 *            j-th largest singular value.
 *  v         [n_vis] complex64, internal order: data duals v_{l,b}.
 *  u_prev    [n_vis] complex64, internal order: Phi x^{(p-1)} (Algorithm 2
 *            extrapolation 2 Phi x^{(p)} - Phi x^{(p-1)}); set it to Phi x^{(0)}
 *            (fhs_measure) before the first iteration.                       */
typedef struct {
  float* W;
  float* theta;
  float* P;
  float* theta_bar;
  float* v;
  float* u_prev;
} fhs_state;

/* Per-cube arguments of fhs_pdfb_iter. */
typedef struct {
  float* X;              /* [L][n1][n2] primal iterate, updated in place        */
  float* Xcheck;         /* [L][n1][n2] 2 X^{(p+1)} - X^{(p)}, updated in place */
  const float* y;        /* [n_vis] complex64 data, internal order              */
  fhs_state state;
} fhs_iterate;

/* Statistics of the last iteration of a cube (host). */
typedef struct {
  double xi;             /* ||X^{(p+1)} - X^{(p)}||_F / ||X^{(p)}||_F           */
  double res_norm;       /* ||r||_2, r_{l,b} = ||y_{l,b} - Phi_{l,b} x_l^{(p)}|| */
  double eps_norm;       /* ||eps||_2                                           */
} fhs_iter_stats;

/* ---------------------------------------------------------------- context */
/* Create a context for `ncubes` sub-cubes.  Sorts the visibilities of every
 * channel by grid tile (host counting sort), builds the FFT, Kaiser-Bessel,
 * Daubechies and facet tables, counts per grid tile the largest number of 7x7
 * footprints covering one cell (one kernel launch; it fixes the gridder's
 * fixed-point scale) and allocates scratch.  `stream` is a
 * cudaStream_t (NULL = legacy default stream).  Synchronising.
 * Errors: INVALID_ARG (shape, NULL pointer, non-finite parameter),
 * UNSUPPORTED (shape outside this build), OOM, CUDA.                       */
fhs_status fhs_create(const fhs_cube_desc* cubes, int32_t ncubes, void* stream, fhs_ctx** out);
fhs_status fhs_destroy(fhs_ctx* ctx);
fhs_status fhs_get_sizes(const fhs_ctx* ctx, int32_t cube, fhs_sizes* out);
/* Synchronise the context stream and report deferred errors. */
fhs_status fhs_sync(fhs_ctx* ctx);
/* Message of the last error of `ctx` (or of the last failed fhs_create when
 * ctx is NULL); valid until the next call on the context. */
const char* fhs_last_error(const fhs_ctx* ctx);

/* Permutation of the cube's visibilities: perm[i] = caller index (0-based,
 * within the cube's uv array) of internal visibility i.  Host [n_vis]. */
fhs_status fhs_vis_permutation(const fhs_ctx* ctx, int32_t cube, int64_t* perm_host);
/* internal[i] = user[perm[i]] and user[perm[i]] = internal[i] (complex64). */
fhs_status fhs_vis_to_internal(fhs_ctx* ctx, int32_t cube, const float* user, float* internal);
fhs_status fhs_vis_to_user(fhs_ctx* ctx, int32_t cube, const float* internal, float* user);

/* -------------------------------------------------------------- operators */
/* y = Phi x for every channel, Eq. (1): Phi_l = G_l F Z with Z the 2x
 * zero-padding and Kaiser-Bessel deapodisation s = 1/phi_hat(2 pi p / K),
 * F the 2n1 x 2n2 DFT (exp(-2 pi i k p / K), centred pixel coordinates), G
 * the 7x7 Kaiser-Bessel interpolation (beta = 2.34 * 7, taps
 * k_j = floor(t - 3.5) + 1 + j, t = omega K / 2 pi).
 * x: [L][n1][n2] float; y: [n_vis] complex64, internal order (overwritten). */
fhs_status fhs_measure(fhs_ctx* ctx, int32_t cube, const float* x, float* y);
/* x = Re Phi^dagger v (exact transpose of fhs_measure, real part; Table 2
 * last row restricts the primal to real images).  x overwritten. */
fhs_status fhs_adjoint(fhs_ctx* ctx, int32_t cube, const float* v, float* x);
/* ||Phi_l||_S^2 of every channel by the power method on Re(Phi^dagger Phi)
 * (Section 2.3.1 footnote): stop at relative variation < rel_tol or after
 * max_iter iterations; start vector all ones.  out: host [L].  Synchronising. */
fhs_status fhs_opnorm_sq(fhs_ctx* ctx, int32_t cube, int32_t max_iter, double rel_tol, double* out);

/* Psi^dagger x: SARA analysis of every channel (Section 2.3.1; layout of W).
 * x [L][n1][n2] -> coef [L][I] (overwritten). */
fhs_status fhs_sara_analysis(fhs_ctx* ctx, int32_t cube, const float* x, float* coef);
/* Psi w: exact transpose of fhs_sara_analysis, coef [L][I] -> x [L][n1][n2] (overwritten). */
fhs_status fhs_sara_synthesis(fhs_ctx* ctx, int32_t cube, const float* coef, float* x);

/* ------------------------------------------------------ dual updates (Alg. 2) */
/* Sparsity duals of every facet (Algorithm 2, W update and Table 2 row 3):
 * W <- (I - prox_{kappa^-1 mu ||.||_{2,1,theta}})(W + Psi^dagger Xcheck),
 * then A += kappa Psi W.  The faceted operators Psi_q^dagger S_q sum exactly
 * to Psi^dagger (Section 2.4.2), so facets only partition W.  W in place. */
fhs_status fhs_prox_l21_sara_facets(fhs_ctx* ctx, int32_t cube, const float* xcheck,
                                    float* W, const float* theta, float* A);
/* Low-rankness duals of every facet (Algorithm 2, P update, Table 2 row 2):
 * P_q <- (I - prox_{zeta^-1 mu_bar_q ||.||_{*,theta_bar_q}})(P_q + D_q S~_q Xcheck),
 * then A += zeta S~_q^T D_q P_q.  The prox is computed as P_q <- Z V diag(m) V^T
 * with Z^T Z = V diag(s^2) V^T (FP64 eigen-solve) and m_j = min(1, alpha_j / s_j). */
fhs_status fhs_prox_nuclear_facets(fhs_ctx* ctx, int32_t cube, const float* xcheck,
                                   float* P, const float* theta_bar, float* A);
/* Data duals with U = I (Table 2 row 4): for every (l, b),
 * v_{l,b} = (z - y)(1 - min(1, eps_{l,b} / ||z - y||)) = (I - P_B(y, eps))(z).
 * z, y, v_out: [n_vis] complex64 internal order; dnorm_out: host [L*B]
 * receives ||z_{l,b} - y_{l,b}||_2 in FP64 (may be NULL).  Synchronising
 * when dnorm_out is not NULL. */
fhs_status fhs_proj_l2ball_blocks(fhs_ctx* ctx, int32_t cube, const float* z, const float* y,
                                  float* v_out, double* dnorm_out);
/* Weights of Algorithm 1 from x: theta_i = mu / (||[Psi^dagger x]_i||_2 + mu)
 * (Eq. 10) and theta_bar_{q,j} = mu_bar_q / (s_j(D_q S~_q x) + mu_bar_q) (Eq. 9). */
fhs_status fhs_reweight(fhs_ctx* ctx, int32_t cube, const float* x, float* theta, float* theta_bar);

/* Parameters of a cube from its noise levels, computed on the device (Sections
 * 2.3-2.4): ||Phi_l||_S^2 by the power method of fhs_opnorm_sq (power_iters,
 * rel_tol), then eta_l = 1/||Phi_l||_S^2, eps_{l,b} = sqrt(sigma_l^2 (M_l + 2 sqrt(M_l))
 * M_{l,b} / M_l) (Eq. 3), and with sigma_bar_l = sigma_l / ||Phi_l||_S and sigma_bar^2
 * their mean square, mu = sigma_bar (m_chi(L) + s_chi(L)) (FHS sparsity heuristic) and
 * mu_bar_q = sigma_bar sqrt(N~_q L / min(N~_q, L)) (low-rank heuristic); m_chi, s_chi
 * are the mean and standard deviation of the chi distribution with L degrees of
 * freedom.  The values replace the cube's eta, eps, mu and mu_bar (tau, zeta, kappa
 * unchanged).  sigma: host [L], finite, >= 0.  Outputs (host, each may be NULL):
 * eta [L], eps [L*B], mu [1], mu_bar [Qy*Qx].  Synchronising.
 * Errors: INVALID_ARG, NONFINITE, UNSUPPORTED, CUDA. */
fhs_status fhs_heuristic_params(fhs_ctx* ctx, int32_t cube, const double* sigma, int32_t power_iters, double rel_tol,
                                double* eta_out, double* eps_out, double* mu_out, double* mu_bar_out);

/* Preconditioned data duals of a cube (Section 3.2; Algorithm 2 v line with
 * U_{l,b} != I): v <- U (I - prox^U_B)(U^-1 v + Phi x_check), the U-metric projection
 * onto B(y_{l,b}, eps_{l,b}) approximated by n_sub forward-backward sub-iterations
 * w <- P_B(w - gamma U (w - z)), gamma = 1 / max U over the block, started from the
 * Euclidean projection P_B(z).  U: host [n_vis] in the caller's order, finite, > 0, or
 * NULL for the inverse sampling density: U = 1 / (number of the channel's visibilities
 * whose nearest cell of the 2n1 x 2n2 grid, round(omega K / 2 pi) mod K, is the
 * visibility's own).  n_sub = 0 returns to U = I (closed-form projections).  While
 * n_sub > 0, fhs_opnorm_sq and fhs_heuristic_params return ||U^1/2 Phi_l||^2 and
 * eta_l = 1 / ||U^1/2 Phi_l||^2 (Section 3.2); set eta with one of them afterwards.
 * fhs_proj_l2ball_blocks stays the Euclidean projection.  Synchronising.
 * Errors: INVALID_ARG, OOM, CUDA. */
fhs_status fhs_set_preconditioning(fhs_ctx* ctx, int32_t cube, int32_t n_sub, const float* U);

/* DDE-extended de-gridding kernels of a cube (Section 2.1, after Eq. 1): row m of G_l
 * becomes the Kaiser-Bessel kernel convolved with the visibility's compact Fourier-
 * domain DDE kernel K_m, g_m[k] = sum_j K_m[j] phi(t_r - (k_r - j_r)) phi(t_c - (k_c -
 * j_c)) for j in [-R, R]^2, a (7 + 2R) x (7 + 2R) footprint (15 x 15 for S_d = 9).  The
 * visibilities then model the sky multiplied by the pattern a_m(p) = sum_j K_m[j]
 * exp(-2 pi i (j_r p_r / K1 + j_c p_c / K2)).  Every operator of the cube follows:
 * fhs_measure, fhs_adjoint (conjugated kernels), fhs_pdfb_iter, fhs_solve,
 * fhs_opnorm_sq and fhs_heuristic_params (set eta again afterwards).
 *  S_d    : kernel side, odd in [1, 9]; 0 returns to the plain 7 x 7 rows;
 *  n_kern : number of kernels (>= 1);
 *  kern   : host, complex64 as float pairs, [n_kern][S_d][S_d], first index along grid
 *           rows (the v axis, j_r = index - R), second along columns (u);
 *  kidx   : host [n_vis] int32 in the caller's visibility order, kernel of each
 *           visibility, in [0, n_kern).
 * The library copies both; gridding stays bitwise deterministic.  Synchronising.
 * Errors: INVALID_ARG (S_d, an index out of range, a non-finite coefficient),
 * UNSUPPORTED (footprint wider than a grid tile, K < 16), OOM, CUDA. */
fhs_status fhs_set_dde(fhs_ctx* ctx, int32_t cube, int32_t S_d, int32_t n_kern, const float* kern,
                       const int32_t* kidx);

/* Replace the algorithm parameters of a cube (same meaning and host arrays as in
 * fhs_cube_desc: eta [L], mu_bar [Qy*Qx], eps [L*B]).  Lets a caller compute
 * eta = 1/||Phi_l||^2 with fhs_opnorm_sq and the noise-based heuristics
 * (Sections 2.3-2.4) on a context before iterating.  Synchronising. */
fhs_status fhs_set_params(fhs_ctx* ctx, int32_t cube, double tau, double zeta, double kappa, const double* eta,
                          double mu, const double* mu_bar, const double* eps);
/* Kernel path used by fhs_pdfb_iter, fhs_prox_l21_sara_facets and fhs_reweight:
 * FHS_PATH_FAST (default) uses the fused kernels, the tensor-core facet Grams and one
 * CUDA graph per iteration; FHS_PATH_PLAIN the unfused one-launch-per-pass kernels,
 * the CUDA-core float-float Grams and direct launches without a graph (the FP32
 * path that the fast one is measured against).  Both compute the same operators. */
enum { FHS_PATH_FAST = 0, FHS_PATH_PLAIN = 1 };
fhs_status fhs_set_path(fhs_ctx* ctx, int32_t path);
/* Concurrent lanes of fhs_pdfb_iter on the fast path (a scheduling choice; the paper's
 * sub-cubes are independent problems, Section 2.4.1).  With lanes = 2..4 and as many
 * cubes, the cubes are dealt to the lanes (largest first, each to the lane with the
 * least work so far, work ~ L n1 n2 + visibilities) and every lane runs its cubes on
 * its own CUDA streams with its own scratch buffers inside the iteration's graph, so
 * that the launches of cubes too small to fill the GPU run side by side.  Default 1:
 * cubes whose launches fill the GPU on their own gain nothing from sharing it.  Each
 * further lane's scratch (about the size of the first: the largest cube's grids,
 * wavelet coefficients and visibility buffers) is allocated by the next fhs_pdfb_iter;
 * lanes that the device memory cannot hold are not made (no error).  Lowering the
 * count frees the lanes above it.  Results do not depend on the lane count: every
 * cube's arithmetic is the same, bit for bit.  fhs_get_lanes reports the lanes the next
 * iteration uses (1 until the further lanes exist).  Errors: INVALID_ARG (lanes not in
 * [1, 4]). */
fhs_status fhs_set_lanes(fhs_ctx* ctx, int32_t lanes);
fhs_status fhs_get_lanes(const fhs_ctx* ctx, int32_t* lanes);
/* Number of CUDA kernels this library has launched in this process so far. */
uint64_t fhs_kernel_launches(void);

/* Kernel timer (a measurement hook; the paper has no counterpart).  With
 * kernel = FHS_TIMER_GRID (the gridding kernel, G^T of Algorithm 2) or
 * FHS_TIMER_DEGRID (the degridding + l2-ball data-dual kernel), fhs_pdfb_iter
 * records a CUDA event pair around that kernel's launch for every cube, inside
 * its CUDA graph as well; FHS_TIMER_NONE (default) records nothing.  Changing
 * the selection re-captures the graph on the next call.
 * fhs_kernel_timer_read synchronises on the last recorded events and returns
 * the summed device time (ms) of the selected kernel's launches in the most
 * recent iteration and their number (the cube count); FHS_ERR_INVALID_ARG if no
 * timer is selected or no iteration has run since the selection. */
enum { FHS_TIMER_NONE = 0, FHS_TIMER_GRID = 1, FHS_TIMER_DEGRID = 2 };
fhs_status fhs_set_kernel_timer(fhs_ctx* ctx, int32_t kernel);
fhs_status fhs_kernel_timer_read(fhs_ctx* ctx, double* ms_total, int32_t* launches);

/* n_iter iterations of Algorithm 2 on every cube.  it: host [ncubes].
 * stats: host [ncubes] or NULL; when not NULL the call synchronises and
 * fills the statistics of the last iteration. */
fhs_status fhs_pdfb_iter(fhs_ctx* ctx, const fhs_iterate* it, int32_t n_iter, fhs_iter_stats* stats);

/* The same iterations with the data and the result in HOST memory: for every cube,
 * y_host[c] (complex64, [n_vis], the caller's visibility order) is copied to the
 * device and put in internal order (into it[c].y, which must be a device array of
 * n_vis complex64), n_iter iterations run as in fhs_pdfb_iter, and it[c].X is copied
 * back to X_host[c] ([L][n1][n2] float).  Host buffers may be pageable or pinned
 * (pinned ones copy faster).  Synchronising.  Errors: as fhs_pdfb_iter. */
fhs_status fhs_pdfb_iter_host(fhs_ctx* ctx, const fhs_iterate* it, const float* const* y_host, float* const* X_host,
                              int32_t n_iter, fhs_iter_stats* stats);

/* ------------------------------------------- Algorithm 1 with stopping rules */
/* Stopping rules of Algorithm 2 (PDFB runs while p < p_min, or p < p_max and
 * (xi > xi_pdfb or ||r|| > res_factor ||eps||); Section 4.1 uses res_factor = 1.01)
 * and of Algorithm 1 (reweighting cycles run while t < t_max and
 * xi_rw = ||X^(t+1) - X^(t)||_F / ||X^(t)||_F > xi_reweight). */
enum { FHS_MAX_SOLVE_CYCLES = 32 };
typedef struct {
  int32_t p_min, p_max;        /* 1 <= p_min <= p_max                                */
  double xi_pdfb;              /* >= 0                                               */
  double res_factor;           /* >= 0                                               */
  int32_t t_max;               /* 1 .. FHS_MAX_SOLVE_CYCLES                          */
  double xi_reweight;          /* >= 0                                               */
} fhs_solve_params;

/* Outcome of fhs_solve for one cube (host). */
typedef struct {
  int32_t cycles;                                      /* reweighting cycles run       */
  int32_t iterations;                                  /* PDFB iterations, all cycles  */
  int32_t iterations_per_cycle[FHS_MAX_SOLVE_CYCLES];
  double xi;                   /* last PDFB iteration's relative variation           */
  double res_norm;             /* last PDFB iteration's ||r||                        */
  double xi_reweight;          /* last cycle's relative variation of X               */
  int32_t nonfinite;           /* 1 if a statistic was NaN or Inf (the loops stopped) */
} fhs_solve_report;

/* Algorithm 1 around Algorithm 2 on every cube, entirely on the device: per cube one
 * CUDA graph with two nested WHILE nodes whose conditions are set by kernels that
 * evaluate the stopping rules; no host round trip per iteration.  Cycle t: weights
 * from X^(t) (Eqs. 9-10, into state.theta / state.theta_bar), X_check = X and
 * u_prev = Phi X (Algorithm 2 restarts from X^(t)), PDFB iterations until the rule
 * holds, then xi_rw.  The duals (W, P, v) carry over between cycles (warm start).
 * it: host [ncubes] (as fhs_pdfb_iter); prm: host; report: host [ncubes], filled on
 * return.  Synchronising.  Cubes run one after another.  Errors: INVALID_ARG,
 * NONFINITE (a statistic was NaN or Inf; the report says where it stopped), TIMEOUT,
 * CUDA.  The kernel timer (fhs_set_kernel_timer) records nothing inside fhs_solve. */
fhs_status fhs_solve(fhs_ctx* ctx, const fhs_iterate* it, const fhs_solve_params* prm, fhs_solve_report* report);

/* ----------------------------------------------------------- checkpoints */
/* Save / restore the state of Algorithms 1-2 (the warm start of Algorithm 1: X,
 * X_check, W, theta, P, theta_bar, v, u_prev of every cube, and each cube's parameters
 * tau, zeta, kappa, mu, eta, mu_bar, eps) to a file.  Loading checks the file's
 * version, a 64-bit hash of its contents and that every cube has the context's shape
 * before anything is changed; the iterations then continue exactly where they
 * stopped (the data y and the preconditioner are the caller's to set again).  The
 * arrays are copied through host memory in 64 MB pieces.  Synchronising.
 * Errors: INVALID_ARG (path, I/O, wrong or corrupt file, other shape), CUDA. */
fhs_status fhs_checkpoint_save(fhs_ctx* ctx, const fhs_iterate* it, const char* path);
fhs_status fhs_checkpoint_load(fhs_ctx* ctx, const fhs_iterate* it, const char* path);

/* ------------------------------------------------ fault-injection hooks */
/* For tests of the error paths without faulting a GPU.  fhs_set_wait_limit shortens
 * the first phase of every bounded device-side wait (TMA copies, tensor-core MMAs) to
 * `spins` polls (0 restores the default, about 4 M; -1 gives up without polling, so every
 * such wait reports a timeout); the second phase, which lets copies
 * and MMAs in flight land before a kernel moves on, keeps its full length.  A wait that
 * runs out sets the device status word: the next synchronising call returns
 * FHS_ERR_TIMEOUT and the outputs of that call are undefined; later calls work.
 * fhs_set_alloc_limit caps the device bytes the library allocates on the calling thread
 * from the start of each fhs_create (0: no cap); a request beyond it fails with
 * FHS_ERR_OOM.  Both apply process-wide. */
/* ------------------------------------------------------------- autotuner */
/* Per-shape launch choices of a cube, for the batching form (many cubes of different
 * shapes, Section 2.4.1).  Each candidate is a kernel the library also runs untuned:
 *  grid_tile        : side (cells) of the gridder / de-gridder tiles, 32 or 64; it
 *                     fixes the internal visibility order, so it is chosen inside
 *                     fhs_create from trial cubes over the first two channels;
 *  degrid_tiled     : 1 tile-staged (TMA) de-gridder, 0 direct per-visibility one;
 *  gram_tc          : 1 tcgen05 error-free facet Gram (L <= 32), 0 CUDA-core float-float;
 *  sara_fast        : 1 fused SARA tiles, 0 separate analysis / dual / synthesis passes;
 *  prox_ctas_per_sm : CTAs per SM of the fused l2,1 dual pass;
 *  source           : 0 defaults (autotuning off), 1 measured, 2 read from the cache;
 *  ms               : measured times (ms): [0] grid + de-grid with 32-cell tiles, [1] with
 *                     64, [2] tile-staged de-grid, [3] direct, [4] tcgen05 Gram, [5]
 *                     CUDA-core Gram, [6] SARA weights by separate passes, [7..9] fused
 *                     with 4, 8, 16 CTAs per SM (0 where not measured). */
typedef struct {
  int32_t grid_tile;
  int32_t degrid_tiled;
  int32_t gram_tc;
  int32_t sara_fast;
  int32_t prox_ctas_per_sm;
  int32_t source;
  double ms[10];
} fhs_tuning;

/* Process-wide switch for the contexts created afterwards.  mode 0: defaults (tile 64,
 * tile-staged de-gridder, tcgen05 Gram, fused SARA, 16 CTAs per SM); 1: read each
 * cube's choices from the cache file when it holds the cube's key (device name,
 * compute capability, n1 x n2, L, Qy x Qx, B, total visibilities), else measure them in
 * fhs_create (pattern inputs, CUDA events: one warm-up, three timed launches per
 * candidate) and write them to the file; 2: always measure, then write.  cache_path:
 * a JSON object of objects of numbers, or NULL for no file.  The file is replaced
 * atomically (write + rename).  Errors: INVALID_ARG (mode). */
fhs_status fhs_set_autotune(int32_t mode, const char* cache_path);
/* The choices of a cube.  Errors: INVALID_ARG. */
fhs_status fhs_get_tuning(const fhs_ctx* ctx, int32_t cube, fhs_tuning* out);

fhs_status fhs_set_wait_limit(int64_t spins);
fhs_status fhs_set_alloc_limit(uint64_t bytes);

/* ------------------------------------------------- allocation-free variant */
/* The paper has no counterpart of this entry point: it serves callers that may
 * not allocate device memory (a host application that owns all device memory
 * through its own pool and passes only pre-allocated buffers, or a
 * latency-critical loop that must not enter the allocator).  Such callers
 * cannot create an fhs_ctx.
 *
 * Same result as fhs_proj_l2ball_blocks, on plain arrays: for each segment s,
 * v[i] = (z[i] - y[i]) (1 - min(1, eps[s] / ||z_s - y_s||_2)) for
 * seg_off[s] <= i < seg_off[s+1]; v_s = 0 whenever ||z_s - y_s|| <= eps[s],
 * the zero-norm case included.  A segment whose norm is NaN or Inf gets
 * v_s = NaN.
 *  z, y, v_out : device, complex64 (interleaved float pairs), caller's order,
 *                at least seg_off[nseg] elements each;
 *  seg_off     : host [nseg + 1], non-decreasing, seg_off[0] >= 0;
 *  nseg        : 1..64 (the size of the static scratch; larger -> INVALID_ARG);
 *  eps         : host [nseg], finite, >= 0;
 *  dnorm_out   : host [nseg] receives ||z_s - y_s||_2 in FP64, or NULL;
 *                when not NULL the call synchronises `stream` (so it must be
 *                NULL while that stream is being captured into a graph) and
 *                returns NONFINITE if a norm is NaN or Inf;
 *  stream      : cudaStream_t (NULL = legacy default stream).
 * Never calls cudaMalloc, cudaFree or any allocating routine.  Its scratch is a
 * fixed 156 KB array in the library's device globals, held by every GPU that
 * loads the library until the process exits and shared by all calls on a
 * device: calls that overlap on the GPU race and must be serialised by the
 * caller.  The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress, device current) and keeps it for the process; make
 * that first call before any stream capture begins, and do not reset the
 * device (cudaDeviceReset) afterwards.  Three kernel launches per call.
 * Errors: INVALID_ARG, CUDA, NONFINITE; the message is returned by
 * fhs_noalloc_last_error (per host thread). */
fhs_status fhs_proj_l2ball_noalloc(const float* z, const float* y, const int64_t* seg_off, int32_t nseg,
                                   const double* eps, float* v_out, double* dnorm_out, void* stream);
const char* fhs_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FHS_H */
