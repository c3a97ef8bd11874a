// Reweighted nuclear-norm duals of the apodised facets (Algorithm 2 P update,
// Table 2 row 2) on GB300.
//
// For facet q with Z_q = P_q + D_q S~_q Xcheck (N~_q x L):
//   (I - prox_{alpha ||.||_*,theta})(Z) = U diag(min(s_j, alpha_j)) V^T = Z V diag(m) V^T,
//   m_j = min(1, alpha_j / s_j), Z^T Z = V diag(s^2) V^T.
// Three kernels:
//   k_gram   : partial Gram matrices Z^T Z of pixel chunks (FP32, staged in smem);
//   k_eig    : FP64 sum of the partials in fixed order, cyclic Jacobi
//              eigen-solve of the L x L Gram, M_q = V diag(m) V^T (or weights);
//   k_apply  : pixel-driven: for each pixel and each facet covering it,
//              P_q <- Z_q M_q and A += zeta D_q P_q (every A pixel written once).
#include <cuda_runtime.h>

#include "fhs_internal.h"

namespace fhs {

constexpr int kGramChunk = 1024;   // pixels per Gram partial
constexpr int kGramSub = 64;       // pixels staged in shared memory at a time

__device__ __forceinline__ float facet_weight(const NucFacet& f, const float* __restrict__ win, int rr, int cc) {
  return win[f.wy_off + rr] * win[f.wx_off + cc];
}

// Error-free transformation a + b = s + e (Knuth TwoSum), no contraction.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Partial Gram of chunk blockIdx.x of facet blockIdx.y, accumulated in
// float-float: each product a*b = p + e exactly (FMA), the running sum keeps a
// high part and a compensation term, so the partial equals the exact Gram of
// the FP32 matrix Z to ~1e-14 relative.  (A plain FP32 Gram has absolute
// errors ~eps * lambda_max, which wipes out singular values below
// sqrt(eps) s_max.)  Thread owns an LB x LB block of G; Lp = L rounded up to a
// multiple of LB.  Output: FP64 partials [Q][nchunk_max][L][L].
template <int LB>
__global__ void __launch_bounds__(256, LB == 4 ? 1 : 3) k_gram(const float* __restrict__ xc, const float* __restrict__ P,
                                              const NucFacet* __restrict__ facets, const float* __restrict__ win,
                                              int n1, int n2, int L, int use_P, double* __restrict__ part,
                                              int nchunk_max) {
  // the staged sub-chunk and, after the last one, the per-group partial sums
  __shared__ union {
    float z[kGramSub][kMaxL + 1];
    double red[256 * LB * LB];
  } sm;
  auto& z = sm.z;
  auto& red = sm.red;
  const int q = blockIdx.y;
  const NucFacet f = facets[q];
  const int h = f.r1 - f.r0, w = f.c1 - f.c0;
  const int Nq = h * w;
  const int p0 = blockIdx.x * kGramChunk;
  if (p0 >= Nq) return;
  const int p1 = min(Nq, p0 + kGramChunk);
  const int Lp = (L + LB - 1) / LB * LB;
  const int nb = Lp / LB;
  // thread -> (upper-triangle block pair, pixel group): npairs pairs, G groups share
  // the pixels of each staged sub-chunk; the groups are summed in a fixed order
  const int npairs = nb * (nb + 1) / 2;
  const int G = max(1, (int)blockDim.x / npairs);
  const int pair = threadIdx.x % npairs, g = threadIdx.x / npairs;
  const bool active = g < G;
  int ta = 0, rem = pair;
  while (rem >= nb - ta) { rem -= nb - ta; ++ta; }
  const int tb = ta + rem;
  float hi[LB][LB], lo[LB][LB];
#pragma unroll
  for (int i = 0; i < LB; ++i)
#pragma unroll
    for (int j = 0; j < LB; ++j) hi[i][j] = lo[i][j] = 0.f;
  const size_t N = (size_t)n1 * n2;
  // staging: thread -> pixel spix of the sub-chunk and channels sl0 + 4k; up to 16
  // channels the next sub-chunk's values are loaded into registers while the current
  // one is reduced
  constexpr int NPT = LB == 2 ? 4 : 1;      // channels per thread (Lp <= 4 NPT when prefetching)
  static_assert(kGramSub * 4 == 256, "256 threads stage 64 pixels x 4 channel lanes");
  const int spix = threadIdx.x % kGramSub, sl0 = threadIdx.x / kGramSub;
  float pre[NPT];
  auto fetch = [&](int s0) {
    const int p = s0 + spix;
    const bool okp = p < p1;
    int rr = 0, cc = 0;
    float d = 0.f;
    if (okp) {
      rr = p / w;
      cc = p - rr * w;
      d = facet_weight(f, win, rr, cc);
    }
    const size_t xo = (size_t)(f.r0 + rr) * n2 + (f.c0 + cc);
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      const int l = sl0 + 4 * k;
      float val = 0.f;
      if (okp && l < L) {
        val = d * xc[l * N + xo];
        if (use_P) val += P[f.p_off + (size_t)l * Nq + p];
      }
      pre[k] = val;
    }
  };
  constexpr bool PF = LB <= 2;         // prefetch (registers permitting)
  if (PF) fetch(p0);
  for (int s0 = p0; s0 < p1; s0 += kGramSub) {
    if constexpr (PF) {
#pragma unroll
      for (int k = 0; k < NPT; ++k)
        if (sl0 + 4 * k < Lp) z[spix][sl0 + 4 * k] = pre[k];
    } else {
#pragma unroll 4
      for (int idx = threadIdx.x; idx < kGramSub * Lp; idx += blockDim.x) {
        const int pix = idx % kGramSub, l = idx / kGramSub;
        const int p = s0 + pix;
        float val = 0.f;
        if (p < p1 && l < L) {
          const int rr = p / w, cc = p - rr * w;
          const float d = facet_weight(f, win, rr, cc);
          val = d * xc[l * N + (size_t)(f.r0 + rr) * n2 + (f.c0 + cc)];
          if (use_P) val += P[f.p_off + (size_t)l * Nq + p];
        }
        z[pix][l] = val;
      }
    }
    __syncthreads();
    if (PF && s0 + kGramSub < p1) fetch(s0 + kGramSub);
    if (active) {
      for (int pix = g; pix < kGramSub; pix += G) {
        float a[LB], b[LB];
#pragma unroll
        for (int i = 0; i < LB; ++i) a[i] = z[pix][ta * LB + i];
#pragma unroll
        for (int j = 0; j < LB; ++j) b[j] = z[pix][tb * LB + j];
#pragma unroll
        for (int i = 0; i < LB; ++i)
#pragma unroll
          for (int j = 0; j < LB; ++j) {
            float pr = __fmul_rn(a[i], b[j]);
            float pe = __fmaf_rn(a[i], b[j], -pr);
            float s, e;
            two_sum(hi[i][j], pr, s, e);
            hi[i][j] = s;
            lo[i][j] = __fadd_rn(lo[i][j], __fadd_rn(e, pe));
          }
      }
    }
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int i = 0; i < LB; ++i)
#pragma unroll
      for (int j = 0; j < LB; ++j) red[((size_t)g * npairs + pair) * LB * LB + i * LB + j] = (double)hi[i][j] + (double)lo[i][j];
  }
  __syncthreads();
  double* out = part + ((size_t)q * nchunk_max + blockIdx.x) * L * L;
  for (int k = threadIdx.x; k < npairs * LB * LB; k += blockDim.x) {
    const int pr = k / (LB * LB), ij = k - pr * LB * LB, i = ij / LB, j = ij - i * LB;
    double v = 0.0;
    for (int gg = 0; gg < G; ++gg) v += red[((size_t)gg * npairs + pr) * LB * LB + ij];
    int xa = 0, xr = pr;
    while (xr >= nb - xa) { xr -= nb - xa; ++xa; }
    const int a = xa * LB + i, b = (xa + xr) * LB + j;
    if (a < L && b < L) {
      out[a * L + b] = v;
      out[b * L + a] = v;
    }
  }
}

// FP64 partial Gram of D_q S~_q x (weights mode of Algorithm 1, once per
// reweighting cycle): z = wy * wx * x formed and multiplied in FP64 so that
// the small singular values entering theta_bar = mu_bar / (s + mu_bar) are not
// limited by rounding z to FP32.
__global__ void __launch_bounds__(256) k_gram_f64(const float* __restrict__ xc, const NucFacet* __restrict__ facets,
                                                  const double* __restrict__ win64, int n1, int n2, int L,
                                                  double* __restrict__ part, int nchunk_max) {
  __shared__ double z[kGramSub / 2][kMaxL + 1];
  constexpr int SUB = kGramSub / 2;
  const int q = blockIdx.y;
  const NucFacet f = facets[q];
  const int h = f.r1 - f.r0, w = f.c1 - f.c0;
  const int Nq = h * w;
  const int p0 = blockIdx.x * kGramChunk;
  if (p0 >= Nq) return;
  const int p1 = min(Nq, p0 + kGramChunk);
  const int LB = L <= 16 ? 1 : (L <= 32 ? 2 : 4);
  const int Lp = (L + LB - 1) / LB * LB;
  const int nb = Lp / LB;
  const int ta = threadIdx.x / nb, tb = threadIdx.x % nb;
  const bool active = ta < nb && ta <= tb;
  double acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const size_t N = (size_t)n1 * n2;
  for (int s0 = p0; s0 < p1; s0 += SUB) {
    for (int idx = threadIdx.x; idx < SUB * Lp; idx += blockDim.x) {
      int pix = idx % SUB, l = idx / SUB;
      int p = s0 + pix;
      double val = 0.0;
      if (p < p1 && l < L) {
        int rr = p / w, cc = p % w;
        val = win64[f.wy_off + rr] * win64[f.wx_off + cc] * (double)xc[l * N + (size_t)(f.r0 + rr) * n2 + (f.c0 + cc)];
      }
      z[pix][l] = val;
    }
    __syncthreads();
    if (active) {
      for (int pix = 0; pix < SUB; ++pix)
        for (int i = 0; i < LB; ++i)
          for (int j = 0; j < LB; ++j) acc[i][j] = fma(z[pix][ta * LB + i], z[pix][tb * LB + j], acc[i][j]);
    }
    __syncthreads();
  }
  if (active) {
    double* out = part + ((size_t)q * nchunk_max + blockIdx.x) * L * L;
    for (int i = 0; i < LB; ++i)
      for (int j = 0; j < LB; ++j) {
        int a = ta * LB + i, b = tb * LB + j;
        if (a < L && b < L) {
          out[a * L + b] = acc[i][j];
          out[b * L + a] = acc[i][j];
        }
      }
  }
}

// One warp per facet: G = sum of partial Grams (FP64, fixed order), cyclic
// Jacobi eigen-decomposition G = V diag(lambda) V^T, s = sqrt(max(lambda, 0))
// sorted descending, then either M = V diag(m) V^T with
// m_j = min(1, alpha_j / s_j), alpha_j = (mu_bar_q / zeta) theta_bar_q[rank j]
// (dual mode), or theta_bar_q[rank] = mu_bar_q / (s + mu_bar_q) (weights mode).
__global__ void __launch_bounds__(32) k_eig(const double* __restrict__ part, int nchunk_max,
                                            const NucFacet* __restrict__ facets, int L,
                                            const float* __restrict__ theta_bar, const float* __restrict__ mubar,
                                            float inv_zeta, float* __restrict__ Mout, float* __restrict__ tb_out,
                                            int weights_mode, int max_sweeps) {
  extern __shared__ double sh[];
  const int Ls = L + 1;
  double* G = sh;                 // [L][L+1]
  double* V = sh + L * Ls;        // [L][L+1]
  double* lam = V + L * Ls;       // [L]
  double* rc = lam + L;           // [L/2 + 1] rotation cosines of a round
  double* rs = rc + (L / 2 + 1);  // [L/2 + 1] sines
  int* rank = (int*)(rs + (L / 2 + 1));   // [L]
  int* rp = rank + L;             // [L/2 + 1] pair indices
  int* rr = rp + (L / 2 + 1);
  const int q = blockIdx.x, lane = threadIdx.x;
  const NucFacet f = facets[q];
  const int Nq = (f.r1 - f.r0) * (f.c1 - f.c0);
  const int nch = (Nq + kGramChunk - 1) / kGramChunk;
  // sum of the chunk partials, chunk 0 first: eight entries of the lane at a time, so
  // that each chunk's eight loads are in flight together (the order of the additions of
  // an entry is the chunk order either way)
  constexpr int kEigBatch = 8;
  for (int e0 = lane; e0 < L * L; e0 += 32 * kEigBatch) {
    double s[kEigBatch];
#pragma unroll
    for (int k = 0; k < kEigBatch; ++k) s[k] = 0.0;
    const double* pq = part + (size_t)q * nchunk_max * L * L;
    for (int c = 0; c < nch; ++c) {
      const double* pc = pq + (size_t)c * L * L;
#pragma unroll
      for (int k = 0; k < kEigBatch; ++k) {
        const int idx = e0 + 32 * k;
        if (idx < L * L) s[k] += pc[idx];
      }
    }
#pragma unroll
    for (int k = 0; k < kEigBatch; ++k) {
      const int idx = e0 + 32 * k;
      if (idx < L * L) {
        const int a = idx / L, b = idx % L;
        G[a * Ls + b] = s[k];
        V[a * Ls + b] = (a == b) ? 1.0 : 0.0;
      }
    }
  }
  __syncwarp();
  // symmetrise (the partial Grams are symmetric up to rounding order)
  for (int idx = lane; idx < L * L; idx += 32) {
    int a = idx / L, b = idx % L;
    if (a < b) {
      double m = 0.5 * (G[a * Ls + b] + G[b * Ls + a]);
      G[a * Ls + b] = m;
      G[b * Ls + a] = m;
    }
  }
  __syncwarp();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    __syncwarp();
    double off = 0.0, dia = 0.0;
    for (int idx = lane; idx < L * L; idx += 32) {
      int a = idx / L, b = idx % L;
      double g = G[a * Ls + b];
      if (a == b) dia += g * g; else off += g * g;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if (off <= 1e-30 * dia || off == 0.0) break;
    // one sweep = Le - 1 rounds of the round-robin tournament over Le = L rounded up to
    // even (index L is a dummy); a round rotates Le/2 disjoint pairs at once: lane j
    // computes pair j's rotation from the round's G, then rows and columns are
    // updated for all pairs (the pairs are disjoint, so this is exact)
    const int Le = (L + 1) & ~1, H = Le / 2;
    for (int rnd = 0; rnd < Le - 1; ++rnd) {
      auto player = [&](int k) { return k == 0 ? 0 : ((k - 1 + rnd) % (Le - 1)) + 1; };
      __syncwarp();
      for (int j = lane; j < H; j += 32) {
        int p = player(j), r = player(Le - 1 - j);
        if (p > r) { int t = p; p = r; r = t; }
        double c = 1.0, sn = 0.0;
        if (r < L) {
          const double gpr = G[p * Ls + r], gpp = G[p * Ls + p], grr = G[r * Ls + r];
          if (fabs(gpr) > 1e-300 && fabs(gpr) > 1e-18 * sqrt(fabs(gpp * grr))) {
            const double th = (grr - gpp) / (2.0 * gpr);
            const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
          }
        }
        rp[j] = p; rr[j] = r; rc[j] = c; rs[j] = sn;
      }
      __syncwarp();
      for (int idx = lane; idx < H * L; idx += 32) {     // rows p, r
        const int j = idx / L, k = idx - j * L;
        const int p = rp[j], r = rr[j];
        if (r >= L || rs[j] == 0.0) continue;
        const double c = rc[j], sn = rs[j];
        const double a = G[p * Ls + k], b = G[r * Ls + k];
        G[p * Ls + k] = c * a - sn * b;
        G[r * Ls + k] = sn * a + c * b;
      }
      __syncwarp();
      for (int idx = lane; idx < H * L; idx += 32) {     // columns p, r and eigenvectors
        const int j = idx / L, k = idx - j * L;
        const int p = rp[j], r = rr[j];
        if (r >= L || rs[j] == 0.0) continue;
        const double c = rc[j], sn = rs[j];
        const double a = G[k * Ls + p], b = G[k * Ls + r];
        G[k * Ls + p] = c * a - sn * b;
        G[k * Ls + r] = sn * a + c * b;
        const double va = V[k * Ls + p], vb = V[k * Ls + r];
        V[k * Ls + p] = c * va - sn * vb;
        V[k * Ls + r] = sn * va + c * vb;
      }
    }
  }
  __syncwarp();
  for (int j = lane; j < L; j += 32) lam[j] = G[j * Ls + j];
  __syncwarp();
  for (int j = lane; j < L; j += 32) {
    int rk = 0;
    for (int k = 0; k < L; ++k) rk += (lam[k] > lam[j]) || (lam[k] == lam[j] && k < j);
    rank[j] = rk;
  }
  __syncwarp();
  const float mb = mubar[q];
  if (weights_mode) {
    for (int j = lane; j < L; j += 32) {
      double s = sqrt(fmax(lam[j], 0.0));
      tb_out[(size_t)q * L + rank[j]] = (float)((double)mb / (s + (double)mb));
    }
    return;
  }
  // m_j stored in lam
  __syncwarp();
  for (int j = lane; j < L; j += 32) {
    double s = sqrt(fmax(lam[j], 0.0));
    double alpha = (double)mb * (double)inv_zeta * (double)theta_bar[(size_t)q * L + rank[j]];
    lam[j] = (s > alpha) ? alpha / s : 1.0;
  }
  __syncwarp();
  // M_q^T, rows padded to Lp = L rounded up to 4 (zeros), so that a row is read as float4
  const int Lp = (L + 3) & ~3;
  for (int idx = lane; idx < L * Lp; idx += 32) {
    int b = idx / Lp, a = idx % Lp;
    double m = 0.0;
    if (a < L)
      for (int j = 0; j < L; ++j) m += V[a * Ls + j] * lam[j] * V[b * Ls + j];
    Mout[(size_t)q * L * Lp + idx] = (float)m;
  }
}

// Pixel-driven update: each thread owns one pixel; for every facet covering it,
// z = P_q + D_q x, P_q <- z M_q, A += zeta D_q P_q.  Row b of M_q^T is read as
// float4 (one load per four FMAs, the same address across the warp).  Up to 16
// channels the A contributions of all covering facets are summed in shared memory
// (one slot per thread and channel) and A is read and written once per pixel with all
// of its loads in flight; above that, A is updated per facet.
template <int LMAX>
__global__ void __launch_bounds__(256) k_apply(const float* __restrict__ xc, float* __restrict__ P,
                                               const NucFacet* __restrict__ facets, const float* __restrict__ win,
                                               const float* __restrict__ Mt, int n1, int n2, int L, int Qy, int Qx,
                                               const int* __restrict__ ty_of, const int* __restrict__ tx_of,
                                               float zeta, float* __restrict__ A) {
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int r = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (r >= n1 || c >= n2) return;
  const size_t N = (size_t)n1 * n2;
  const size_t pix = (size_t)r * n2 + c;
  const int Lp = (L + 3) & ~3;
  const int ty = ty_of[r], tx = tx_of[c];
  if constexpr (LMAX <= 16) {
    __shared__ float sacc[LMAX][256];          // this thread's A contributions, per channel
    float* acc = &sacc[0][threadIdx.x];
#pragma unroll
    for (int b = 0; b < LMAX; ++b) acc[b * 256] = 0.f;
    for (int dy = 0; dy < 2; ++dy) {
      const int qy = ty + dy;
      if (qy >= Qy) break;
      for (int dx = 0; dx < 2; ++dx) {
        const int qx = tx + dx;
        if (qx >= Qx) break;
        const NucFacet f = facets[qy * Qx + qx];
        if (r < f.r0 || r >= f.r1 || c < f.c0 || c >= f.c1) continue;
        const int w = f.c1 - f.c0;
        const int Nq = (f.r1 - f.r0) * w;
        const int p = (r - f.r0) * w + (c - f.c0);
        const float d = facet_weight(f, win, r - f.r0, c - f.c0);
        float* Pq = P + f.p_off;
        float z[LMAX];
#pragma unroll
        for (int l = 0; l < LMAX; ++l) z[l] = (l < L) ? fmaf(d, xc[l * N + pix], Pq[(size_t)l * Nq + p]) : 0.f;
        const float4* Mq = reinterpret_cast<const float4*>(Mt + (size_t)(qy * Qx + qx) * L * Lp);
        const float zd = zeta * d;
#pragma unroll 1
        for (int b = 0; b < L; ++b) {
          const float4* row = Mq + (size_t)b * (Lp / 4);
          float s = 0.f;
#pragma unroll
          for (int a4 = 0; a4 < LMAX / 4; ++a4) {
            if (4 * a4 < L) {
              const float4 m = __ldg(row + a4);
              s = fmaf(z[4 * a4], m.x, s);
              s = fmaf(z[4 * a4 + 1], m.y, s);
              s = fmaf(z[4 * a4 + 2], m.z, s);
              s = fmaf(z[4 * a4 + 3], m.w, s);
            }
          }
          Pq[(size_t)b * Nq + p] = s;
          acc[b * 256] = fmaf(zd, s, acc[b * 256]);
        }
      }
    }
#pragma unroll
    for (int b0 = 0; b0 < LMAX; b0 += 8) {
      float a_old[8];
#pragma unroll
      for (int b = 0; b < 8; ++b) a_old[b] = (b0 + b < L) ? A[(b0 + b) * N + pix] : 0.f;
#pragma unroll
      for (int b = 0; b < 8; ++b)
        if (b0 + b < L) A[(b0 + b) * N + pix] = a_old[b] + acc[(b0 + b) * 256];
    }
    return;
  }
  for (int dy = 0; dy < 2; ++dy) {
    int qy = ty + dy;
    if (qy >= Qy) break;
    for (int dx = 0; dx < 2; ++dx) {
      int qx = tx + dx;
      if (qx >= Qx) break;
      const NucFacet f = facets[qy * Qx + qx];
      if (r < f.r0 || r >= f.r1 || c < f.c0 || c >= f.c1) continue;
      const int w = f.c1 - f.c0;
      const int Nq = (f.r1 - f.r0) * w;
      const int p = (r - f.r0) * w + (c - f.c0);
      const float d = facet_weight(f, win, r - f.r0, c - f.c0);
      float* Pq = P + f.p_off;
      float z[LMAX];
#pragma unroll
      for (int l = 0; l < LMAX; ++l) z[l] = (l < L) ? fmaf(d, xc[l * N + pix], Pq[(size_t)l * Nq + p]) : 0.f;
      const float4* Mq = reinterpret_cast<const float4*>(Mt + (size_t)(qy * Qx + qx) * L * Lp);
      const float zd = zeta * d;
#pragma unroll 1
      for (int b = 0; b < L; ++b) {
        const float4* row = Mq + (size_t)b * (Lp / 4);
        float s = 0.f;
#pragma unroll
        for (int a4 = 0; a4 < LMAX / 4; ++a4) {
          if (4 * a4 < L) {
            const float4 m = __ldg(row + a4);
            s = fmaf(z[4 * a4], m.x, s);
            s = fmaf(z[4 * a4 + 1], m.y, s);
            s = fmaf(z[4 * a4 + 2], m.z, s);
            s = fmaf(z[4 * a4 + 3], m.w, s);
          }
        }
        Pq[(size_t)b * Nq + p] = s;
        A[b * N + pix] = fmaf(zd, s, A[b * N + pix]);
      }
    }
  }
}

static int nchunk_max(const Cube& cb) { return (cb.max_facet_pix + kGramChunk - 1) / kGramChunk; }

void launch_nuclear(fhs_ctx* ctx, const Cube& cb, const float* xcheck, float* P, const float* theta_bar, float* A,
                    bool weights_mode, float* theta_bar_out, cudaStream_t st) {
  launch_nuclear_gram_eig(ctx, cb, xcheck, P, theta_bar, weights_mode, theta_bar_out, st);
  if (!weights_mode) launch_nuclear_apply(ctx, cb, xcheck, P, A, st);
}

// Per-chunk partial Grams of Z_q = D_q S~_q xcheck (+ P_q) into ctx->s.gram: the tcgen05
// kernel when tc and L <= 32, else the CUDA-core float-float kernel.
void launch_gram(fhs_ctx* ctx, const Cube& cb, const float* xcheck, const float* P, bool tc, cudaStream_t st) {
  const int L = cb.L;
  const int nch = nchunk_max(cb);
  dim3 gg(nch, cb.Qy * cb.Qx);
  const int use_P = P != nullptr ? 1 : 0;
  if (tc && launch_gram_tc(cb, xcheck, P, ctx->s.gram, nch, st)) return;   // counts its launch
  if (L <= 4) k_gram<1><<<gg, 256, 0, st>>>(xcheck, P, cb.d_facets, cb.d_win, cb.n1, cb.n2, L, use_P, ctx->s.gram, nch);
  else if (L <= 16) k_gram<2><<<gg, 256, 0, st>>>(xcheck, P, cb.d_facets, cb.d_win, cb.n1, cb.n2, L, use_P, ctx->s.gram, nch);
  else k_gram<4><<<gg, 256, 0, st>>>(xcheck, P, cb.d_facets, cb.d_win, cb.n1, cb.n2, L, use_P, ctx->s.gram, nch);
  note_launches(1);
}

void launch_nuclear_gram_eig(fhs_ctx* ctx, const Cube& cb, const float* xcheck, const float* P,
                             const float* theta_bar, bool weights_mode, float* theta_bar_out, cudaStream_t st) {
  const int L = cb.L;
  const int Q = cb.Qy * cb.Qx;
  const int nch = nchunk_max(cb);
  dim3 gg(nch, Q);
  if (weights_mode) {
    k_gram_f64<<<gg, 256, 0, st>>>(xcheck, cb.d_facets, cb.d_win64, cb.n1, cb.n2, L, ctx->s.gram, nch);
    note_launches(1);
  } else {
    launch_gram(ctx, cb, xcheck, P, ctx->path == FHS_PATH_FAST && cb.gram_tc, st);
  }
  size_t sm = (size_t)2 * L * (L + 1) * sizeof(double) + L * sizeof(double) + 2 * (L / 2 + 1) * sizeof(double) +
              (L + 2 * (L / 2 + 1)) * sizeof(int);
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024); attr = true; }
  k_eig<<<Q, 32, sm, st>>>(ctx->s.gram, nch, cb.d_facets, L, theta_bar, cb.d_mubar, (float)(1.0 / cb.zeta),
                           ctx->s.nucM, theta_bar_out, weights_mode ? 1 : 0, 40);
  note_launches(1);
}

void launch_nuclear_apply(fhs_ctx* ctx, const Cube& cb, const float* xcheck, float* P, float* A, cudaStream_t st) {
  const int L = cb.L;
  dim3 ga((cb.n2 + 31) / 32, (cb.n1 + 7) / 8);
  const int* tyo = cb.d_tile_of;
  const int* txo = cb.d_tile_of + cb.n1;
  float zeta = (float)cb.zeta;
  if (L <= 16) k_apply<16><<<ga, 256, 0, st>>>(xcheck, P, cb.d_facets, cb.d_win, ctx->s.nucM, cb.n1, cb.n2, L, cb.Qy, cb.Qx, tyo, txo, zeta, A);
  else if (L <= 32) k_apply<32><<<ga, 256, 0, st>>>(xcheck, P, cb.d_facets, cb.d_win, ctx->s.nucM, cb.n1, cb.n2, L, cb.Qy, cb.Qx, tyo, txo, zeta, A);
  else k_apply<64><<<ga, 256, 0, st>>>(xcheck, P, cb.d_facets, cb.d_win, ctx->s.nucM, cb.n1, cb.n2, L, cb.Qy, cb.Qx, tyo, txo, zeta, A);
  note_launches(1);
}

}  // namespace fhs
