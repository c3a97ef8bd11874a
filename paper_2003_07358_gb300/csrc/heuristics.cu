// Algorithm parameters from the noise level, computed on the device (Sections 2.3-2.4):
//   eta_l        = 1 / ||Phi_l||_S^2                           (step size, Section 3.2)
//   eps_{l,b}    = sqrt(sigma_l^2 (M_l + 2 sqrt(M_l)) M_{l,b} / M_l)    (Eq. 3 radii)
//   sigma_bar_l  = sigma_l / ||Phi_l||_S,  sigma_bar^2 = mean_l sigma_bar_l^2
//   mu           = sigma_bar (m_chi(L) + s_chi(L))              (FHS sparsity heuristic)
//   mu_bar_q     = sigma_bar sqrt(N~_q L / J_q),  J_q = min(N~_q, L)   (low-rank heuristic)
// with m_chi(k) = sqrt(2) Gamma((k + 1) / 2) / Gamma(k / 2) and s_chi(k) = sqrt(k - m_chi^2),
// the mean and standard deviation of the chi distribution with k degrees of freedom.
#include <cuda_runtime.h>
#include <math.h>

#include "fhs_internal.h"

namespace fhs {

// One CTA.  in: sigma [L], opnorm_sq [L] (FP64), M_lb [L*B]; out (FP64):
// [eta L][eps L*B][mu 1][mu_bar Q]; also the kernel-side copies d_eta, d_eps, d_mubar.
__global__ void k_heuristics(const double* __restrict__ sigma, const double* __restrict__ opn,
                             const int64_t* __restrict__ M_lb, const NucFacet* __restrict__ facets, int L, int B, int Q,
                             double* __restrict__ out, float* __restrict__ d_eta, double* __restrict__ d_eps,
                             float* __restrict__ d_mubar) {
  __shared__ double s_sbar2;
  double* eta = out;
  double* eps = out + L;
  double* mu = eps + L * B;
  double* mub = mu + 1;
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    eta[l] = 1.0 / opn[l];
    d_eta[l] = (float)eta[l];
    double Ml = 0.0;
    for (int b = 0; b < B; ++b) Ml += (double)M_lb[l * B + b];
    const double e2 = sigma[l] * sigma[l] * (Ml + 2.0 * sqrt(Ml));
    for (int b = 0; b < B; ++b) {
      const double v = Ml > 0.0 ? sqrt(e2 * (double)M_lb[l * B + b] / Ml) : 0.0;
      eps[l * B + b] = v;
      d_eps[l * B + b] = v;
    }
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int l = 0; l < L; ++l) s += sigma[l] * sigma[l] / opn[l];   // sigma_bar_l^2, fixed order
    s_sbar2 = s / L;
    const double k = (double)L;
    const double m = sqrt(2.0) * exp(lgamma((k + 1.0) / 2.0) - lgamma(k / 2.0));
    *mu = sqrt(s_sbar2) * (m + sqrt(fmax(k - m * m, 0.0)));
  }
  __syncthreads();
  const double sbar = sqrt(s_sbar2);
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    const NucFacet f = facets[q];
    const double Nq = (double)(f.r1 - f.r0) * (double)(f.c1 - f.c0);
    const double v = sbar * sqrt(Nq * L / fmin(Nq, (double)L));
    mub[q] = v;
    d_mubar[q] = (float)v;
  }
}

void launch_heuristics(const Cube& cb, const double* sigma, const double* opn, double* out, cudaStream_t st) {
  k_heuristics<<<1, 256, 0, st>>>(sigma, opn, cb.d_M_lb, cb.d_facets, cb.L, cb.B, cb.Qy * cb.Qx, out, cb.d_eta,
                                  cb.d_eps, cb.d_mubar);
  note_launches(1);
}

}  // namespace fhs
