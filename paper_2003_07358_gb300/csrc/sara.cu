// SARA dictionary Psi^dagger = [db1..db8, Dirac] / 3 (Section 2.3.1) and the
// reweighted l2,1 dual update of Algorithm 2 on GB300.
//
// The faceted transform of Section 2.4.2 (each facet extended by its filter
// support) sums exactly to the global transform, so the kernels compute the
// global operator level by level; facets only partition the coefficients.
// Each level is two separable passes (along columns, then rows), one thread
// per output coefficient, filters in constant memory.  Coefficient layout:
// fhs.h (basis-major, 3 detail subbands per level, LL4, then Dirac), planar
// per channel ([L][I]) so that the channel norm of a coefficient reads L
// coalesced planes.
#include <cuda_runtime.h>

#include "fhs_internal.h"

namespace fhs {

__constant__ Filters c_filt;

cudaError_t upload_filters(const Filters& f) { return cudaMemcpyToSymbol(c_filt, &f, sizeof(f)); }

// ------------------------------------------------------------ analysis
// lx/hx[l][r][k] = sum_t f[t] a[l][r][2k+1-t]  (zero outside [0, m2))
__global__ void k_ana_cols(const float* __restrict__ a, float* __restrict__ lx, float* __restrict__ hx, int L, int m1,
                           int m2, int mo2, int basis) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = (int64_t)L * m1 * mo2;
  if (idx >= total) return;
  const int F = 2 * (basis + 1);
  int k = (int)(idx % mo2);
  int64_t rl = idx / mo2;                 // l * m1 + r
  const float* row = a + rl * m2;
  float sl = 0.f, sh = 0.f;
  for (int t = 0; t < F; ++t) {
    int i = 2 * k + 1 - t;
    if (i >= 0 && i < m2) {
      float x = row[i];
      sl = fmaf(c_filt.h[basis][t], x, sl);
      sh = fmaf(c_filt.g[basis][t], x, sh);
    }
  }
  lx[idx] = sl;
  hx[idx] = sh;
}

// Filtering along rows of lx/hx [l][m1][mo2]: LL -> ll_out (or the LL4 block of
// coef), d0 = h(hx), d1 = g(lx), d2 = g(hx) -> coef at the level's offsets, /3.
__global__ void k_ana_rows(const float* __restrict__ lx, const float* __restrict__ hx, float* __restrict__ ll_out,
                           float* __restrict__ coef, int64_t I, int64_t off0, int64_t off1, int64_t off2,
                           int64_t off_ll, int L, int m1, int mo1, int mo2, int basis) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = (int64_t)L * mo1 * mo2;
  if (idx >= total) return;
  const int F = 2 * (basis + 1);
  int c = (int)(idx % mo2);
  int k = (int)((idx / mo2) % mo1);
  int l = (int)(idx / ((int64_t)mo2 * mo1));
  const float* lxl = lx + (size_t)l * m1 * mo2;
  const float* hxl = hx + (size_t)l * m1 * mo2;
  float ll = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
  for (int t = 0; t < F; ++t) {
    int i = 2 * k + 1 - t;
    if (i >= 0 && i < m1) {
      float vl = lxl[(size_t)i * mo2 + c];
      float vh = hxl[(size_t)i * mo2 + c];
      float h = c_filt.h[basis][t], g = c_filt.g[basis][t];
      ll = fmaf(h, vl, ll);
      d1 = fmaf(g, vl, d1);
      d0 = fmaf(h, vh, d0);
      d2 = fmaf(g, vh, d2);
    }
  }
  const float third = 1.f / 3.f;
  int64_t pos = (int64_t)k * mo2 + c;
  float* cl = coef + (size_t)l * I;
  cl[off0 + pos] = d0 * third;
  cl[off1 + pos] = d1 * third;
  cl[off2 + pos] = d2 * third;
  if (ll_out) ll_out[idx] = ll;
  else cl[off_ll + pos] = ll * third;
}

__global__ void k_dirac_ana(const float* __restrict__ x, float* __restrict__ coef, int64_t I, int64_t off, int64_t N,
                            int L) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)L * N) return;
  int l = (int)(idx / N);
  coef[(size_t)l * I + off + (idx % N)] = x[idx] * (1.f / 3.f);
}

// ----------------------------------------------------------- synthesis
// Transpose of k_ana_rows: lx[l][i][c] = sum_k h[2k+1-i] LL[k][c] + g[2k+1-i] d1[k][c],
// hx[l][i][c] = sum_k h[2k+1-i] d0[k][c] + g[2k+1-i] d2[k][c], i < m1.
// LL comes from ll_in (synthesised coarser level) or the LL4 block of coef (/3).
__global__ void k_syn_rows(const float* __restrict__ ll_in, const float* __restrict__ coef, int64_t I, int64_t off0,
                           int64_t off1, int64_t off2, int64_t off_ll, float* __restrict__ lx, float* __restrict__ hx,
                           int L, int m1, int mo1, int mo2, int basis) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = (int64_t)L * m1 * mo2;
  if (idx >= total) return;
  const int F = 2 * (basis + 1);
  int c = (int)(idx % mo2);
  int i = (int)((idx / mo2) % m1);
  int l = (int)(idx / ((int64_t)mo2 * m1));
  const float* cl = coef + (size_t)l * I;
  const float* lli = ll_in ? ll_in + (size_t)l * mo1 * mo2 : nullptr;
  const float third = 1.f / 3.f;
  int k_lo = (i) / 2;                     // ceil((i-1)/2) for i >= 0
  int k_hi = (i + F - 2) / 2;
  if (k_hi > mo1 - 1) k_hi = mo1 - 1;
  float sl = 0.f, sh = 0.f;
  for (int k = k_lo; k <= k_hi; ++k) {
    int t = 2 * k + 1 - i;
    if (t < 0 || t >= F) continue;
    int64_t pos = (int64_t)k * mo2 + c;
    float h = c_filt.h[basis][t], g = c_filt.g[basis][t];
    float vll = lli ? lli[pos] : cl[off_ll + pos] * third;
    sl = fmaf(h, vll, sl);
    sl = fmaf(g, cl[off1 + pos] * third, sl);
    sh = fmaf(h, cl[off0 + pos] * third, sh);
    sh = fmaf(g, cl[off2 + pos] * third, sh);
  }
  lx[idx] = sl;
  hx[idx] = sh;
}

// Transpose of k_ana_cols: a[l][r][i] = sum_k h[2k+1-i] lx[l][r][k] + g[2k+1-i] hx[l][r][k], i < m2.
// Output to a temporary (overwrite) or to the final image: out = acc ? out + s*a : s*a.
__global__ void k_syn_cols(const float* __restrict__ lx, const float* __restrict__ hx, float* __restrict__ out,
                           float s, int accumulate, int L, int m1, int m2, int mo2, int basis) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = (int64_t)L * m1 * m2;
  if (idx >= total) return;
  const int F = 2 * (basis + 1);
  int i = (int)(idx % m2);
  int64_t rl = idx / m2;
  const float* lr = lx + rl * mo2;
  const float* hr = hx + rl * mo2;
  int k_lo = i / 2;
  int k_hi = (i + F - 2) / 2;
  if (k_hi > mo2 - 1) k_hi = mo2 - 1;
  float acc = 0.f;
  for (int k = k_lo; k <= k_hi; ++k) {
    int t = 2 * k + 1 - i;
    if (t < 0 || t >= F) continue;
    acc = fmaf(c_filt.h[basis][t], lr[k], acc);
    acc = fmaf(c_filt.g[basis][t], hr[k], acc);
  }
  out[idx] = accumulate ? fmaf(s, acc, out[idx]) : s * acc;
}

__global__ void k_dirac_syn(const float* __restrict__ coef, int64_t I, int64_t off, int64_t N, int L,
                            float* __restrict__ out, float s, int accumulate) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)L * N) return;
  int l = (int)(idx / N);
  float v = coef[(size_t)l * I + off + (idx % N)] * (s / 3.f);
  out[idx] = accumulate ? out[idx] + v : v;
}

// ---------------------------------------------------- l2,1 dual / weights
// W <- Z min(1, alpha_i / ||Z_i||), Z = W + coef, alpha_i = (mu / kappa) theta_i.
__global__ void k_l21_dual(float* __restrict__ W, const float* __restrict__ coef, const float* __restrict__ theta,
                           float alpha_scale, int64_t I, int L) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  float z[kMaxL];
  float n2 = 0.f;
#pragma unroll
  for (int l = 0; l < kMaxL; ++l) {
    if (l < L) {
      float v = W[(size_t)l * I + i] + coef[(size_t)l * I + i];
      z[l] = v;
      n2 = fmaf(v, v, n2);
    }
  }
  float nrm = sqrtf(n2);
  float alpha = alpha_scale * theta[i];
  float f = nrm > alpha ? alpha / nrm : 1.f;
#pragma unroll
  for (int l = 0; l < kMaxL; ++l)
    if (l < L) W[(size_t)l * I + i] = z[l] * f;
}

// theta_i = mu / (||coef_i||_2 + mu) (Eq. 10 with upsilon = mu)
__global__ void k_l21_weights(const float* __restrict__ coef, float* __restrict__ theta, float mu, int64_t I, int L) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  float n2 = 0.f;
  for (int l = 0; l < L; ++l) {
    float v = coef[(size_t)l * I + i];
    n2 = fmaf(v, v, n2);
  }
  theta[i] = mu / (sqrtf(n2) + mu);
}

// ------------------------------------------------------------- launchers
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

void launch_sara_analysis(fhs_ctx* ctx, const Cube& cb, const float* x, float* coef, cudaStream_t st) {
  const SaraLayout& S = cb.sara;
  const int L = cb.L;
  float* lx = ctx->s.t0;
  float* hx = ctx->s.t1;
  float* llA = ctx->s.t2;
  float* llB = ctx->s.t3;
  for (int b = 0; b < 8; ++b) {
    const float* in = x;
    for (int j = 1; j <= kLevels; ++j) {
      int m1 = S.rows[b][j - 1], m2 = S.cols[b][j - 1];
      int mo1 = S.rows[b][j], mo2 = S.cols[b][j];
      int64_t n = (int64_t)L * m1 * mo2;
      k_ana_cols<<<nblk(n, 256), 256, 0, st>>>(in, lx, hx, L, m1, m2, mo2, b);
      note_launches(1);
      float* llo = (j == kLevels) ? nullptr : ((j & 1) ? llA : llB);
      int64_t n2 = (int64_t)L * mo1 * mo2;
      k_ana_rows<<<nblk(n2, 256), 256, 0, st>>>(lx, hx, llo, coef, S.I, S.off[b][j][0], S.off[b][j][1],
                                                S.off[b][j][2], S.off[b][kLevels][3], L, m1, mo1, mo2, b);
      note_launches(1);
      in = llo;
    }
  }
  int64_t N = (int64_t)cb.n1 * cb.n2;
  k_dirac_ana<<<nblk(L * N, 256), 256, 0, st>>>(x, coef, S.I, S.dirac_off, N, L);
  note_launches(1);
}

void launch_sara_synthesis(fhs_ctx* ctx, const Cube& cb, const float* coef, float* out, float scale, bool accumulate,
                           cudaStream_t st) {
  const SaraLayout& S = cb.sara;
  const int L = cb.L;
  float* lx = ctx->s.t0;
  float* hx = ctx->s.t1;
  float* llA = ctx->s.t2;
  float* llB = ctx->s.t3;
  bool acc = accumulate;
  for (int b = 0; b < 8; ++b) {
    const float* ll_in = nullptr;   // level 4 reads LL4 from coef
    for (int j = kLevels; j >= 1; --j) {
      int m1 = S.rows[b][j - 1], m2 = S.cols[b][j - 1];
      int mo1 = S.rows[b][j], mo2 = S.cols[b][j];
      int64_t n = (int64_t)L * m1 * mo2;
      k_syn_rows<<<nblk(n, 256), 256, 0, st>>>(ll_in, coef, S.I, S.off[b][j][0], S.off[b][j][1], S.off[b][j][2],
                                               S.off[b][kLevels][3], lx, hx, L, m1, mo1, mo2, b);
      note_launches(1);
      int64_t n2 = (int64_t)L * m1 * m2;
      if (j > 1) {
        float* llo = (ll_in == llA) ? llB : llA;
        k_syn_cols<<<nblk(n2, 256), 256, 0, st>>>(lx, hx, llo, 1.f, 0, L, m1, m2, mo2, b);
        note_launches(1);
        ll_in = llo;
      } else {
        k_syn_cols<<<nblk(n2, 256), 256, 0, st>>>(lx, hx, out, scale, acc ? 1 : 0, L, m1, m2, mo2, b);
        note_launches(1);
        acc = true;
      }
    }
  }
  int64_t N = (int64_t)cb.n1 * cb.n2;
  k_dirac_syn<<<nblk(L * N, 256), 256, 0, st>>>(coef, S.I, S.dirac_off, N, L, out, scale, acc ? 1 : 0);
  note_launches(1);
}

void launch_l21_dual(const Cube& cb, float* W, const float* coef, const float* theta, cudaStream_t st) {
  float alpha_scale = (float)(cb.mu / cb.kappa);
  k_l21_dual<<<nblk(cb.sara.I, 256), 256, 0, st>>>(W, coef, theta, alpha_scale, cb.sara.I, cb.L);
  note_launches(1);
}

void launch_l21_weights(const Cube& cb, const float* coef, float* theta, cudaStream_t st) {
  k_l21_weights<<<nblk(cb.sara.I, 256), 256, 0, st>>>(coef, theta, (float)cb.mu, cb.sara.I, cb.L);
  note_launches(1);
}

}  // namespace fhs

#include "sara_fast.cuh"
