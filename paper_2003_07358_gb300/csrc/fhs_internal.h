// Internal declarations of the GB300 Faceted HyperSARA library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fhs.h"

namespace fhs {

constexpr int kTaps = 7;          // Kaiser-Bessel support J
constexpr int kPolyDeg = 9;       // per-tap polynomial degree of the kernel fit (fit error
                                  // about 1e-9, below the FP32 evaluation error of 7e-8)
constexpr int kGridTile = 64;     // gridder tile side (cells)
constexpr int kDdeMaxR = 4;       // DDE kernels up to 9 x 9 (extended footprints up to 15 x 15)
constexpr int kLevels = 4;        // SARA decomposition levels
constexpr int kMaxB = 16;         // data blocks per channel
constexpr int kMaxL = 64;         // channels per cube
constexpr int kMaxLanes = 4;      // concurrent lanes of an iteration (fhs_set_lanes)
constexpr int kMaxFilt = 16;      // longest Daubechies filter (db8)
constexpr int kMaxSolveCycles = FHS_MAX_SOLVE_CYCLES;

// ------------------------------------------------------------ device tables
// Kaiser-Bessel weights: phi(f + 2.5 - j) = sum_d kb_poly[j][d] (2f - 1)^d, f in [0, 1).
struct KbPoly { float c[kTaps][kPolyDeg + 1]; };

// Daubechies filters: h (low) and g (high) of db1..db8, filter b has length 2(b+1).
struct Filters { float h[8][kMaxFilt]; float g[8][kMaxFilt]; };

// ------------------------------------------------------------------- cube
struct SaraLayout {
  int rows[8][kLevels + 1], cols[8][kLevels + 1];
  int64_t off[8][kLevels + 1][4];   // [basis][level 1..4][subband 0..2, 3 = LL4]
  int64_t dirac_off;
  int64_t I;
};

struct NucFacet {                    // one nuclear facet
  int r0, r1, c0, c1;                // covered pixels [r0, r1) x [c0, c1)
  int64_t p_off;                     // offset of its P block in units of floats (includes L)
  int wy_off, wx_off;                // offsets of its 1-D windows in the window tables
};

// Radix plan of a mixed-radix (4, 2, 3) DFT of length n = 2^a 3^b.
struct GenPlan {
  int n;
  int npass;
  int radix[24];
};

struct Cube {
  int n1, n2, L, Qy, Qx, B, window;
  bool pow2 = true;                          // n1, n2 powers of two (else 3 * 2^m: mixed-radix DFTs)
  GenPlan plan_r{}, plan_c{};                // column (length K1) and row (length K2) plans
  double rho, tau, zeta, kappa, mu;
  std::vector<double> eta, mu_bar, eps;     // host copies
  int K1, K2;
  int N1c, N2c;                              // column FFT factorisation K1 = N1c * N2c
  SaraLayout sara;
  std::vector<NucFacet> facets;
  int64_t n_facet_pix;
  int max_facet_pix;
  // visibilities
  std::vector<int64_t> M_lb;                 // [L*B]
  std::vector<int64_t> vis_off;              // [L+1] channel offsets (internal order == caller order per channel)
  int64_t n_vis;
  int64_t max_M;
  std::vector<int64_t> perm_host;            // internal -> caller index
  float2* d_uv = nullptr;                    // [n_vis] internal order
  int64_t* d_vis_off = nullptr;              // [L+1]
  uint8_t* d_blk = nullptr;                  // [n_vis] block id
  int64_t* d_perm = nullptr;                 // [n_vis]
  int32_t* d_tile_off = nullptr;             // [L][ntiles*4 + 1] per-channel tile/class offsets (relative)
  int ntile_r, ntile_c, tile;                // gridder tiles
  int* d_ncmax = nullptr;                    // [L][ntiles] most footprints covering one cell of a tile
  // device copies of per-cube parameters and tables
  NucFacet* d_facets = nullptr;
  float* d_win = nullptr;                    // window tables (y and x windows concatenated)
  int* d_tile_of = nullptr;                  // [n1 + n2]: tile index of each row, then of each column
  double* d_win64 = nullptr;                 // window tables in FP64 (reweighting Gram)
  float* d_scale_r = nullptr;                // [n1] deapodisation s_r
  float* d_scale_c = nullptr;                // [n2]
  double* d_eps = nullptr;                   // [L*B]
  int64_t* d_M_lb = nullptr;                 // [L*B] visibilities per (channel, block)
  // preconditioned data duals (Section 3.2): n_sub forward-backward sub-iterations
  // (0: U = I, Euclidean projections), U per visibility (internal order), gamma per block
  int n_sub = 0;
  float* d_U = nullptr;                      // [n_vis]
  // DDE-extended G (Section 2.1): kernel half-width R (-1: plain Kaiser-Bessel rows),
  // kernels [n_kern][2R+1][2R+1], kernel of each visibility (internal order), per kernel
  // sum of |Re| + |Im| (rounded up), per (channel, tile) largest extended-footprint count
  // launch choices of the autotuner (defaults: tile-staged de-gridder, tensor-core Gram
  // where L <= 32, fused SARA tiles, 16 CTAs per SM for the l2,1 dual pass)
  int degrid_tiled = 1;
  int gram_tc = 1;
  int sara_fast = 1;
  int prox_cps = 16;
  int tuned = 0;                             // 0 defaults, 1 measured, 2 from the cache file
  double tune_ms[10] = {0};
  int dde_R = -1;
  int dde_nkern = 0;
  float2* d_dde_kern = nullptr;
  int32_t* d_dde_idx = nullptr;
  float* d_dde_l1 = nullptr;
  int* d_dde_ncmax = nullptr;
  float* d_gamma = nullptr;                  // [L*B] 1 / max U of the block
  float* d_eta = nullptr;                    // [L]
  float* d_mubar = nullptr;                  // [Q]
  // TMA descriptors of the degridder's tile staging over a grid scratch buffer, viewed
  // as [L][N1c][N2c][K2] (rows in the column transform's digit-reversed order): the T
  // tile rows and the 6 halo rows of a grid tile.  Two slots: the grid of each lane of
  // concurrent cubes; a launch uses the slot encoded over the grid it is given, and the
  // asynchronous copies when there is none.
  CUtensorMap tm_rows[kMaxLanes], tm_halo[kMaxLanes];
  const float2* tm_grid[kMaxLanes] = {nullptr, nullptr, nullptr, nullptr};
};

struct Scratch {
  float2* grid = nullptr;    size_t grid_elems = 0;     // [L][K1][K2]
  float2* pack = nullptr;                               // [L][K1][n2/2] packed column transform
  float* coef = nullptr;     size_t coef_elems = 0;     // [L][I]
  float* t0 = nullptr;       size_t t_elems = 0;        // SARA temporaries
  float* t1 = nullptr;
  float* t2 = nullptr;
  float* t3 = nullptr;
  float* img = nullptr;      size_t img_elems = 0;      // [L][n1][n2]
  float* img2 = nullptr;
  float2* vis = nullptr;     size_t vis_elems = 0;      // [n_vis]
  float2* vis2 = nullptr;                               // [n_vis] forward-backward iterate (preconditioning)
  double* red = nullptr;     size_t red_elems = 0;      // reduction partials
  double* red_host = nullptr;                           // pinned host copy
  double* gram = nullptr;    size_t gram_elems = 0;     // nuclear Gram partials (FP64)
  float* nucM = nullptr;     size_t nucM_elems = 0;     // [Q][L][L]
  float* blk_scale = nullptr;                           // [L*B]
  double* blk_out = nullptr;                            // [2][L*B]
  float* ll1 = nullptr;                                 // LL1 band of each basis (fused SARA)
  float* ll2 = nullptr;                                 // LL2 band of each basis
  float* ll3 = nullptr;                                 // LL3 band of each basis
  double* stat = nullptr;                               // per cube: primal partials, then block norms
  size_t stat_stride = 0;
  int64_t ll1_off[8] = {0};                             // per-basis offsets into ll1
  int64_t ll2_off[8] = {0};                             // into ll2
  int64_t ll3_off[8] = {0};                             // into ll3
};

// Streams, events and scratch of one further lane of an iteration.
struct Lane {
  Scratch s;
  cudaStream_t stream = nullptr, aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;   // this lane's fork to / join from its aux stream
  cudaEvent_t ev_done = nullptr;                      // the lane's last work (joined by the first lane)
};

}  // namespace fhs

struct fhs_ctx {
  cudaStream_t stream = nullptr;
  std::vector<fhs::Cube> cubes;
  fhs::Scratch s;
  float2* d_tw = nullptr;          // twiddles exp(-2 pi i k / Kmax), k < Kmax
  int Kmax = 0;
  std::string err;
  bool broken = false;
  int path = FHS_PATH_FAST;        // FHS_PATH_FAST or FHS_PATH_PLAIN
  // CUDA graph of one PDFB iteration of every cube, replayed on gstream
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // second stream of an iteration: the facet Grams and eigen-solves of the nuclear duals
  // run beside the data term (they read Xcheck and P only) and join before the update of A
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // further lanes of an iteration (fast path, two or more cubes): cube c runs on lane
  // lane_of[c]; lane k > 0 has its own streams, events and scratch in xl[k - 1]
  int lanes = 1;                   // requested lanes (fhs_set_lanes)
  std::vector<fhs::Lane> xl;       // lanes 1.. whose resources exist
  std::vector<int> lane_of;        // [ncubes] lane of each cube
  cudaEvent_t ev_lanes_fork = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<const void*> graph_key;
  uint64_t graph_kernels = 0;
  // kernel timer: FHS_TIMER_* selection, one event pair per cube, whether an
  // iteration has recorded them since the selection
  int timer = FHS_TIMER_NONE;
  bool timer_off = false;          // true while fhs_solve captures (no event nodes in its loops)
  void* solve_dev = nullptr;       // [ncubes] device control states of fhs_solve
  uint64_t param_version = 0;      // bumped by calls that change what an iteration graph holds
  std::vector<cudaEvent_t> tev;
  bool timer_armed = false;
};

namespace fhs {

// Count of kernel launches made by this library (fhs_kernel_launches).
void note_launches(int n);

// --------------------------------------------------------- kernel launchers
// Tables (constant memory lives in the translation unit that uses it).
cudaError_t upload_kb_poly(const KbPoly& p);
cudaError_t upload_filters(const Filters& f);

// FFT / NUFFT (nufft.cu)
void launch_measure(fhs_ctx* ctx, const Cube& cb, const float* x, float2* y, cudaStream_t st);
void launch_fft_forward(fhs_ctx* ctx, const Cube& cb, const float* x, float2* grid, cudaStream_t st);
void launch_fft_adjoint(fhs_ctx* ctx, const Cube& cb, float2* grid, float* out, const float* eta,
                        bool accumulate, cudaStream_t st);
void launch_fft_forward_fast(fhs_ctx* ctx, const Cube& cb, const float* x, float2* grid, cudaStream_t st);
bool fft_forward_packed(const Cube& cb);
void launch_fft_adjoint_fast(fhs_ctx* ctx, const Cube& cb, float2* grid, float* out, const float* eta,
                             bool accumulate, cudaStream_t st);
void launch_degrid(const Cube& cb, const float2* grid, float2* out, bool tiled, cudaStream_t st);
void encode_degrid_maps(fhs_ctx* ctx);
void encode_cube_maps(Cube& cb, const float2* grid, int slot);
void launch_fill_pattern(float* p, int64_t n, uint32_t seed, cudaStream_t st);
void launch_gram(fhs_ctx* ctx, const Cube& cb, const float* xcheck, const float* P, bool tc, cudaStream_t st);
int num_sms();   // streaming multiprocessors of the current device
unsigned read_device_status(bool clear);
int degrid_tiled_parts(const Cube& cb);
void launch_degrid_pdfb_tiled(const Cube& cb, const float2* grid, const float2* y, const float2* v, float2* d_out,
                              float2* u_prev, double* partials, cudaStream_t st);
void launch_degrid_pdfb(const Cube& cb, const float2* grid, const float2* y, const float2* v, float2* d_out,
                        float2* u_prev, double* partials, int nparts, cudaStream_t st);
int degrid_parts(const Cube& cb);
void launch_block_finalize(const Cube& cb, const double* partials, int nparts, float* scale, double* out,
                           cudaStream_t st);
int host_first_tap(float om, int K);
void launch_grid(const Cube& cb, const float2* vals, const float* blk_scale, float2* v_write,
                 float2* grid, cudaStream_t st);
void launch_grid_count(const Cube& cb, cudaStream_t st);
void launch_degrid_dde(const Cube& cb, const float2* grid, float2* out, cudaStream_t st);
void launch_degrid_pdfb_dde(const Cube& cb, const float2* grid, const float2* y, const float2* v, float2* d_out,
                            float2* u_prev, double* partials, int nparts, cudaStream_t st);
void launch_grid_dde(const Cube& cb, const float2* vals, const float* blk_scale, float2* v_write, float2* grid,
                     cudaStream_t st);
void launch_grid_dde_count(const Cube& cb, cudaStream_t st);
void launch_l2ball_partials(const Cube& cb, const float2* z, const float2* y, float2* d,
                            double* partials, int nparts, cudaStream_t st);
void launch_l2ball_scale(const Cube& cb, const float2* d, const float* scale, float2* v, cudaStream_t st);
void launch_precond_duals(const Cube& cb, float2* d, float2* t, float* blk_scale, double* partials, cudaStream_t st);
void launch_vis_scale(float2* v, const float* f, int64_t n, bool divide, cudaStream_t st);
void launch_vis_gather(const int64_t* perm, int64_t n, const float2* in, float2* out, cudaStream_t st);
void launch_vis_scatter(const int64_t* perm, int64_t n, const float2* in, float2* out, cudaStream_t st);

// SARA (sara.cu)
void launch_sara_analysis(fhs_ctx* ctx, const Cube& cb, const float* x, float* coef, cudaStream_t st);
void launch_sara_synthesis(fhs_ctx* ctx, const Cube& cb, const float* coef, float* out, float scale,
                           bool accumulate, cudaStream_t st);
void launch_l21_dual(const Cube& cb, float* W, const float* coef, const float* theta, cudaStream_t st);
void launch_l21_weights(const Cube& cb, const float* coef, float* theta, cudaStream_t st);
// fused analysis + l2,1 dual (+ synthesis into A), or weights mode (theta_out)
void launch_sara_fast(fhs_ctx* ctx, const Cube& cb, const float* x, float* W, const float* theta, float* A,
                      float* theta_out, bool weights, cudaStream_t st);
bool sara_fast_supported(const Cube& cb);

// nuclear (nuclear.cu)
void launch_nuclear(fhs_ctx* ctx, const Cube& cb, const float* xcheck, float* P, const float* theta_bar,
                    float* A, bool weights_mode, float* theta_bar_out, cudaStream_t st);
// the two halves of launch_nuclear: facet Grams + eigen-solves (reads Xcheck and P only),
// then P <- Z M_q and A += zeta D_q P_q
void launch_nuclear_gram_eig(fhs_ctx* ctx, const Cube& cb, const float* xcheck, const float* P,
                             const float* theta_bar, bool weights_mode, float* theta_bar_out, cudaStream_t st);
void launch_nuclear_apply(fhs_ctx* ctx, const Cube& cb, const float* xcheck, float* P, float* A, cudaStream_t st);

// error-free facet Gram on tcgen05 tensor cores (gram_tc.cu): FP64 partials in the
// layout of k_gram; false when the cube's channel count is outside what it supports
bool launch_gram_tc(const Cube& cb, const float* xcheck, const float* P, double* part, int nchunk_max,
                    cudaStream_t st);
unsigned read_gram_status(bool clear);
cudaError_t set_gram_wait_first(long long spins);
// first phase of every bounded device-side wait (0: default); the drain waits keep
// their full length
cudaError_t set_wait_first(long long spins);

// device control of Algorithms 1-2 (solve.cu); the state is an opaque device struct
size_t solve_state_bytes();
void launch_solve_begin(void* sd, cudaStream_t st);
void launch_solve_cycle_begin(const float* X, float* Xt, float* Xc, int64_t n, void* sd,
                              cudaGraphConditionalHandle inner, cudaStream_t st);
void launch_solve_pdfb_check(const double* stat, int pp, int LB, double eps_norm, const fhs_solve_params& prm,
                             void* sd, cudaGraphConditionalHandle inner, cudaStream_t st);
void launch_solve_cycle_check(const float* X, const float* Xt, int64_t n, double* part, const fhs_solve_params& prm,
                              void* sd, cudaGraphConditionalHandle outer, cudaStream_t st);
cudaError_t read_solve_state(const void* sd_dev, fhs_solve_report* rep, cudaStream_t st);

// noise-based parameters (heuristics.cu): eta, eps, mu, mu_bar from sigma and ||Phi_l||^2
// (device [L] each); out: device FP64 [eta L][eps L*B][mu][mu_bar Q]; updates the cube's
// kernel-side parameter arrays
void launch_heuristics(const Cube& cb, const double* sigma, const double* opn, double* out, cudaStream_t st);

// primal (primal.cu)
void launch_primal(const Cube& cb, float* X, float* Xc, const float* A, double* partials, int nparts,
                   cudaStream_t st);
int primal_parts(const Cube& cb);
void launch_sumsq(const float* a, int64_t n_per_ch, int L, double* partials, int nparts, cudaStream_t st);
void launch_scale_by_channel(float* x, int64_t n_per_ch, int L, const double* inv, cudaStream_t st);

}  // namespace fhs
