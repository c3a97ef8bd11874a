// Device-side control of Algorithm 1 (reweighting) around Algorithm 2 (PDFB): the
// stopping rules are evaluated by small kernels that set the conditions of the WHILE
// nodes of a CUDA graph, so a whole solve runs without host round trips.
//
// Per cube, the graph is
//   begin  ->  WHILE(outer) { weights (Eqs. 9-10); X_t = X; X_check = X; u_prev = Phi X;
//                             p = 0;  WHILE(inner) { PDFB iteration; check }; cycle check }
// with the rules of Algorithm 2 (run while p < p_min, or p < p_max and (xi > xi_pdfb or
// ||r|| > res_factor ||eps||)) and of Algorithm 1 (run while t < t_max and
// xi_rw > xi_reweight).  A non-finite statistic stops both loops and is reported.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "fhs_internal.h"

namespace fhs {

// One cube's control state (device).
struct SolveDev {
  int p;                      // PDFB iterations of the current cycle
  int t;                      // cycles completed
  int total;                  // PDFB iterations, all cycles
  int nonfinite;              // 1 if a statistic was NaN or Inf
  int per_cycle[kMaxSolveCycles];
  double xi, res, xi_rw;
};

size_t solve_state_bytes() { return sizeof(SolveDev); }

__global__ void k_solve_begin(SolveDev* sd) {
  if (threadIdx.x != 0) return;
  sd->p = 0;
  sd->t = 0;
  sd->total = 0;
  sd->nonfinite = 0;
  for (int k = 0; k < kMaxSolveCycles; ++k) sd->per_cycle[k] = 0;
  sd->xi = sd->res = sd->xi_rw = INFINITY;
}

// Start of a cycle: X_t = X and X_check = X (Algorithm 2 restarts with
// X_check^(0) = X^(0)); thread 0 resets p and arms the inner loop.
__global__ void k_solve_cycle_begin(const float* __restrict__ X, float* __restrict__ Xt, float* __restrict__ Xc,
                                    int64_t n, SolveDev* sd, cudaGraphConditionalHandle inner) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = X[i];
    Xt[i] = v;
    Xc[i] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sd->p = 0;
    cudaGraphSetConditional(inner, 1u);
  }
}

// After a PDFB iteration: xi and ||r|| from the iteration's fixed-order partial sums
// (primal partials [pp][2] = (||dX||^2, ||X||^2), block norms after them: [2][L B] with
// ||y - Phi x|| second), then Algorithm 2's rule.
__global__ void k_solve_pdfb_check(const double* __restrict__ stat, int pp, int LB, double eps_norm, int p_min,
                                   int p_max, double xi_pdfb, double res_factor, SolveDev* sd,
                                   cudaGraphConditionalHandle inner) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double dx2 = 0.0, x2 = 0.0, r2 = 0.0;
  for (int k = 0; k < pp; ++k) {
    dx2 += stat[2 * k];
    x2 += stat[2 * k + 1];
  }
  const double* blk = stat + 2 * pp;
  for (int k = 0; k < LB; ++k) r2 += blk[LB + k] * blk[LB + k];
  const double xi = x2 > 0.0 ? sqrt(dx2 / x2) : INFINITY;
  const double res = sqrt(r2);
  const int p = sd->p + 1;
  sd->p = p;
  sd->total += 1;
  if (sd->t < kMaxSolveCycles) sd->per_cycle[sd->t] = p;
  sd->xi = xi;
  sd->res = res;
  const bool finite = isfinite(dx2) && !isnan(x2) && isfinite(r2);
  if (!finite) sd->nonfinite = 1;
  const bool more = finite && (p < p_min || (p < p_max && (xi > xi_pdfb || res > res_factor * eps_norm)));
  cudaGraphSetConditional(inner, more ? 1u : 0u);
}

// Partial sums of ||X - X_t||^2 and ||X_t||^2 (one slot pair per CTA, fixed order).
__global__ void __launch_bounds__(256) k_solve_rw_partials(const float* __restrict__ X, const float* __restrict__ Xt,
                                                           int64_t n, double* __restrict__ part) {
  double d2 = 0.0, t2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = X[i], b = Xt[i];
    d2 += (a - b) * (a - b);
    t2 += b * b;
  }
  __shared__ double s0[8], s1[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    t2 += __shfl_xor_sync(0xffffffffu, t2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s0[threadIdx.x >> 5] = d2;
    s1[threadIdx.x >> 5] = t2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += s0[w];
      b += s1[w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// End of a cycle: xi_rw and Algorithm 1's rule.
__global__ void k_solve_cycle_check(const double* __restrict__ part, int nparts, int t_max, double xi_reweight,
                                    SolveDev* sd, cudaGraphConditionalHandle outer) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double d2 = 0.0, t2 = 0.0;
  for (int k = 0; k < nparts; ++k) {
    d2 += part[2 * k];
    t2 += part[2 * k + 1];
  }
  const double xi_rw = t2 > 0.0 ? sqrt(d2 / t2) : INFINITY;
  const int t = sd->t + 1;
  sd->t = t;
  sd->xi_rw = xi_rw;
  if (isnan(d2) || isnan(t2)) sd->nonfinite = 1;
  const bool more = !sd->nonfinite && t < t_max && t < kMaxSolveCycles && xi_rw > xi_reweight;
  cudaGraphSetConditional(outer, more ? 1u : 0u);
}

void launch_solve_begin(void* sd, cudaStream_t st) {
  k_solve_begin<<<1, 32, 0, st>>>((SolveDev*)sd);
  note_launches(1);
}

void launch_solve_cycle_begin(const float* X, float* Xt, float* Xc, int64_t n, void* sd,
                              cudaGraphConditionalHandle inner, cudaStream_t st) {
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * 152, (n + 255) / 256));
  k_solve_cycle_begin<<<blocks, 256, 0, st>>>(X, Xt, Xc, n, (SolveDev*)sd, inner);
  note_launches(1);
}

void launch_solve_pdfb_check(const double* stat, int pp, int LB, double eps_norm, const fhs_solve_params& prm,
                             void* sd, cudaGraphConditionalHandle inner, cudaStream_t st) {
  k_solve_pdfb_check<<<1, 32, 0, st>>>(stat, pp, LB, eps_norm, prm.p_min, prm.p_max, prm.xi_pdfb, prm.res_factor,
                                       (SolveDev*)sd, inner);
  note_launches(1);
}

void launch_solve_cycle_check(const float* X, const float* Xt, int64_t n, double* part, const fhs_solve_params& prm,
                              void* sd, cudaGraphConditionalHandle outer, cudaStream_t st) {
  constexpr int kParts = 2 * 152;
  k_solve_rw_partials<<<kParts, 256, 0, st>>>(X, Xt, n, part);
  k_solve_cycle_check<<<1, 32, 0, st>>>(part, kParts, prm.t_max, prm.xi_reweight, (SolveDev*)sd, outer);
  note_launches(2);
}

cudaError_t read_solve_state(const void* sd_dev, fhs_solve_report* rep, cudaStream_t st) {
  SolveDev h;
  cudaError_t e = cudaMemcpyAsync(&h, sd_dev, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  rep->cycles = h.t;
  rep->iterations = h.total;
  for (int k = 0; k < kMaxSolveCycles; ++k) rep->iterations_per_cycle[k] = h.per_cycle[k];
  rep->xi = h.xi;
  rep->res_norm = h.res;
  rep->xi_reweight = h.xi_rw;
  rep->nonfinite = h.nonfinite;
  return cudaSuccess;
}

}  // namespace fhs
