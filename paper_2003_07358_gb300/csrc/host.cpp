// Host side of the GB300 Faceted HyperSARA library: context set-up (tables,
// facet geometry, visibility tile sort, scratch) and the C-ABI entry points
// declared in include/fhs.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <complex>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "fhs_internal.h"

using namespace fhs;
using cd = std::complex<double>;

namespace {
std::atomic<uint64_t> g_launches{0};
}

void fhs::note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

int fhs::num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        v <= 0)
      return 152;
    n = v;
  }
  return n;
}

namespace {

thread_local std::string g_create_err;

const double kPi = 3.14159265358979323846;

// --------------------------------------------------------------- errors
struct Fail {
  fhs_status st;
  std::string msg;
};

#define FHS_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw Fail{e_ == cudaErrorMemoryAllocation ? FHS_ERR_OOM : FHS_ERR_CUDA,            \
                 std::string(#call) + ": " + cudaGetErrorString(e_)};                     \
  } while (0)

#define FHS_REQUIRE(cond, code, text)                  \
  do {                                                 \
    if (!(cond)) throw Fail{code, std::string(text)};  \
  } while (0)

void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Fail{FHS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

template <class F>
fhs_status guarded(fhs_ctx* ctx, F&& f) {
  if (!ctx) return FHS_ERR_INVALID_ARG;
  if (ctx->broken) {
    ctx->err = "context unusable after an earlier CUDA error: " + ctx->err;
    return FHS_ERR_CUDA;
  }
  try {
    f();
    return FHS_OK;
  } catch (const Fail& e) {
    ctx->err = e.msg;
    if (e.st == FHS_ERR_CUDA) ctx->broken = true;
    return e.st;
  } catch (const std::exception& e) {
    ctx->err = e.what();
    return FHS_ERR_CUDA;
  }
}

// ------------------------------------------------- Daubechies filters
// Roots of sum_k c[k] y^k by Durand-Kerner (Weierstrass) iterations, then
// Newton polishing on the original polynomial.
std::vector<cd> poly_roots(const std::vector<double>& c) {
  const int n = (int)c.size() - 1;
  std::vector<cd> a(n + 1);
  for (int k = 0; k <= n; ++k) a[k] = c[k] / c[n];
  auto eval = [&](cd z) {
    cd p = a[n];
    for (int k = n - 1; k >= 0; --k) p = p * z + a[k];
    return p;
  };
  std::vector<cd> z(n);
  cd seed(0.4, 0.9);
  for (int k = 0; k < n; ++k) z[k] = std::pow(seed, k + 1);
  for (int it = 0; it < 2000; ++it) {
    double change = 0.0;
    for (int k = 0; k < n; ++k) {
      cd den = 1.0;
      for (int j = 0; j < n; ++j)
        if (j != k) den *= (z[k] - z[j]);
      cd dz = eval(z[k]) / den;
      z[k] -= dz;
      change = std::max(change, std::abs(dz) / (1.0 + std::abs(z[k])));
    }
    if (change < 1e-16) break;
  }
  for (int k = 0; k < n; ++k) {
    for (int it = 0; it < 5; ++it) {
      cd p = a[n], dp = 0.0;
      for (int j = n - 1; j >= 0; --j) {
        dp = dp * z[k] + p;
        p = p * z[k] + a[j];
      }
      if (std::abs(dp) == 0.0) break;
      z[k] -= p / dp;
    }
  }
  return z;
}

// Extremal-phase Daubechies scaling filter of order N (length 2N):
// |H|^2 = 2 cos^{2N}(w/2) P_N(sin^2(w/2)), P_N(y) = sum_{k<N} C(N-1+k, k) y^k;
// each root y_i of P_N contributes the root z_i of z + 1/z = 2 - 4 y_i inside
// the unit circle; H(w) = c (1 + w)^N prod (1 - z_i w), sum h = sqrt(2).
std::vector<double> daubechies(int N) {
  std::vector<cd> poly{cd(1.0)};
  auto mul = [&](cd a0, cd a1) {   // poly *= (a0 + a1 w)
    std::vector<cd> out(poly.size() + 1, cd(0.0));
    for (size_t k = 0; k < poly.size(); ++k) {
      out[k] += poly[k] * a0;
      out[k + 1] += poly[k] * a1;
    }
    poly.swap(out);
  };
  if (N > 1) {
    std::vector<double> p(N);
    for (int k = 0; k < N; ++k) {
      double binom = 1.0;   // C(N-1+k, k)
      for (int i = 1; i <= k; ++i) binom = binom * (N - 1 + i) / i;
      p[k] = binom;
    }
    for (cd y : poly_roots(p)) {
      cd b = 2.0 - 4.0 * y;
      cd disc = std::sqrt(b * b - 4.0);
      cd z1 = (b + disc) / 2.0, z2 = (b - disc) / 2.0;
      cd z = std::abs(z1) < 1.0 ? z1 : z2;
      mul(cd(1.0), -z);
    }
  }
  for (int k = 0; k < N; ++k) mul(cd(1.0), cd(1.0));
  std::vector<double> h(poly.size());
  double s = 0.0;
  for (size_t k = 0; k < poly.size(); ++k) {
    h[k] = poly[k].real();
    s += h[k];
  }
  for (double& v : h) v *= sqrt(2.0) / s;
  double e = 0.0;
  for (double v : h) e += v * v;
  FHS_REQUIRE(fabs(e - 1.0) < 1e-10, FHS_ERR_CUDA, "Daubechies construction lost orthonormality");
  return h;
}

// ----------------------------------------------------- Kaiser-Bessel
const double kBeta = 2.34 * 7.0;

double bessel_i0(double x) {   // power series sum (x^2/4)^k / (k!)^2
  double q = x * x / 4.0, t = 1.0, s = 1.0;
  for (int k = 1; k < 500; ++k) {
    t *= q / ((double)k * k);
    s += t;
    if (t < 1e-18 * s) break;
  }
  return s;
}

double kb_phi(double u) {
  double a = 1.0 - (2.0 * u / 7.0) * (2.0 * u / 7.0);
  if (a < 0.0) return 0.0;
  return bessel_i0(kBeta * sqrt(a)) / bessel_i0(kBeta);
}

// Continuous Fourier transform of phi: 7 sinh(z) / z / I0(beta), z = sqrt(beta^2 - (7 theta / 2)^2).
double kb_phi_hat(double theta) {
  double r = kBeta * kBeta - (3.5 * theta) * (3.5 * theta);
  double v;
  if (r > 0) { double z = sqrt(r); v = sinh(z) / z; }
  else if (r < 0) { double z = sqrt(-r); v = sin(z) / z; }
  else v = 1.0;
  return 7.0 * v / bessel_i0(kBeta);
}

// Chebyshev interpolation of phi(f + 2.5 - j), f = (x + 1)/2, x in [-1, 1], as
// monomials in x; the fit error is checked against phi in double.
KbPoly kb_poly() {
  const int D = kPolyDeg;
  KbPoly out;
  double worst = 0.0;
  for (int j = 0; j < kTaps; ++j) {
    std::vector<double> xs(D + 1), fs(D + 1);
    for (int k = 0; k <= D; ++k) {
      xs[k] = cos(kPi * (k + 0.5) / (D + 1));
      fs[k] = kb_phi((xs[k] + 1.0) / 2.0 + 2.5 - j);
    }
    std::vector<double> cheb(D + 1, 0.0);
    for (int m = 0; m <= D; ++m) {
      double s = 0.0;
      for (int k = 0; k <= D; ++k) s += fs[k] * cos(m * kPi * (k + 0.5) / (D + 1));
      cheb[m] = s * 2.0 / (D + 1);
    }
    cheb[0] *= 0.5;
    // Chebyshev -> monomial: T_0 = 1, T_1 = x, T_{m+1} = 2x T_m - T_{m-1}
    std::vector<double> mono(D + 1, 0.0), tm1(D + 1, 0.0), tm(D + 1, 0.0), tp(D + 1, 0.0);
    tm1[0] = 1.0;
    tm[1] = 1.0;
    mono[0] += cheb[0];
    for (int d = 0; d <= D; ++d) mono[d] += cheb[1] * tm[d];
    for (int m = 2; m <= D; ++m) {
      std::fill(tp.begin(), tp.end(), 0.0);
      for (int d = 0; d < D; ++d) tp[d + 1] += 2.0 * tm[d];
      for (int d = 0; d <= D; ++d) tp[d] -= tm1[d];
      for (int d = 0; d <= D; ++d) mono[d] += cheb[m] * tp[d];
      tm1 = tm;
      tm = tp;
    }
    for (int d = 0; d <= D; ++d) out.c[j][d] = (float)mono[d];
    for (int t = 0; t <= 200; ++t) {
      double x = -1.0 + 2.0 * t / 200.0, p = 0.0;
      for (int d = D; d >= 0; --d) p = p * x + mono[d];
      worst = std::max(worst, fabs(p - kb_phi((x + 1.0) / 2.0 + 2.5 - j)));
    }
  }
  FHS_REQUIRE(worst < 1e-8, FHS_ERR_CUDA, "Kaiser-Bessel polynomial fit is inaccurate");
  return out;
}

// ------------------------------------------------------------ geometry
std::vector<int> tile_bounds(int n, int Q) {
  std::vector<int> b(Q + 1);
  for (int i = 0; i <= Q; ++i) b[i] = (int)(((int64_t)i * n) / Q);
  return b;
}

double window_w(int i, int o, int kind) {
  if (kind == FHS_WIN_TRIANGULAR) return (i + 1.0) / (o + 1.0);
  double s = sin(kPi * (i + 1.0) / (2.0 * (o + 1.0)));
  return s * s;
}

// 1-D nuclear facets along one axis: start, end and window per tile.
void nuclear_axis(int n, int Q, double rho, int kind, std::vector<int>& start, std::vector<int>& end,
                  std::vector<std::vector<double>>& win) {
  std::vector<int> tb = tile_bounds(n, Q);
  std::vector<int> ov(Q);
  for (int i = 0; i < Q; ++i) ov[i] = i == 0 ? 0 : (int)floor(rho * (tb[i + 1] - tb[i]));
  start.resize(Q);
  end.resize(Q);
  win.resize(Q);
  for (int i = 0; i < Q; ++i) {
    start[i] = tb[i] - ov[i];
    end[i] = tb[i + 1];
    std::vector<double> w(end[i] - start[i], 1.0);
    for (int k = 0; k < ov[i]; ++k) w[k] = window_w(k, ov[i], kind);
    if (i + 1 < Q && ov[i + 1] > 0) {
      int o2 = ov[i + 1];
      for (int k = 0; k < o2; ++k) w[(end[i] - o2 - start[i]) + k] = 1.0 - window_w(k, o2, kind);
    }
    win[i].assign(w.begin(), w.end());
  }
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// n = 2^a 3^b with b >= 1 (the mixed-radix transforms' sizes)
bool pow2_times3(int n) {
  if (n <= 0 || n % 3) return false;
  while (n % 3 == 0) n /= 3;
  return pow2(n);
}

// Radix plan of a length-n DFT, n = 2^a 3^b: radix-4 passes, one radix-2 pass when a is
// odd, then the radix-3 passes.
GenPlan gen_plan(int n) {
  GenPlan p{};
  p.n = n;
  int a = 0, b = 0, m = n;
  while (m % 2 == 0) { m /= 2; ++a; }
  while (m % 3 == 0) { m /= 3; ++b; }
  for (int k = 0; k < a / 2; ++k) p.radix[p.npass++] = 4;
  if (a % 2) p.radix[p.npass++] = 2;
  for (int k = 0; k < b; ++k) p.radix[p.npass++] = 3;
  return p;
}

// Fault-injection hook: a cap on the device bytes the library allocates on this thread
// from the start of the last fhs_create (0: none); a request beyond it fails as OOM.
std::atomic<uint64_t> g_alloc_limit{0};
thread_local uint64_t g_alloc_used = 0;

template <class T>
T* dalloc(size_t n) {
  T* p = nullptr;
  if (n == 0) n = 1;
  const uint64_t lim = g_alloc_limit.load();
  if (lim && g_alloc_used + n * sizeof(T) > lim)
    throw Fail{FHS_ERR_OOM, "device allocation limit of " + std::to_string(lim) + " bytes reached"};
  FHS_CUDA(cudaMalloc((void**)&p, n * sizeof(T)));
  g_alloc_used += n * sizeof(T);
  return p;
}

template <class T>
void upload(T* dst, const T* src, size_t n, cudaStream_t st) {
  if (n) FHS_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, st));
}

void build_cube(Cube& cb, const fhs_cube_desc& d, cudaStream_t st, int tile) {
  FHS_REQUIRE(d.M && d.uv && d.eta && d.mu_bar && d.eps, FHS_ERR_INVALID_ARG, "NULL host array in cube descriptor");
  const bool p2 = pow2(d.n1) && pow2(d.n2);
  FHS_REQUIRE(d.n1 >= 16 && d.n2 >= 16 &&
                  (p2 || ((pow2(d.n1) || pow2_times3(d.n1)) && (pow2(d.n2) || pow2_times3(d.n2)) &&
                          d.n1 % 16 == 0 && d.n2 % 16 == 0 && d.n1 <= 1536 && d.n2 <= 1536)),
              FHS_ERR_UNSUPPORTED,
              "n1, n2 must be powers of two >= 16, or multiples of 16 of the form 2^a 3^b up to 1536");
  FHS_REQUIRE(d.n1 <= 4096 && d.n2 <= 4096, FHS_ERR_UNSUPPORTED, "n1, n2 must be <= 4096");
  FHS_REQUIRE(d.L >= 1 && d.L <= kMaxL, FHS_ERR_UNSUPPORTED, "L must be in [1, 64]");
  FHS_REQUIRE(d.Qy >= 1 && d.Qx >= 1 && d.Qy <= d.n1 / 16 + (d.n1 < 16) && d.Qx <= d.n2 / 16 + (d.n2 < 16),
              FHS_ERR_UNSUPPORTED, "facet grid must satisfy 1 <= Q <= n/16");
  FHS_REQUIRE(d.overlap >= 0.0 && d.overlap < 0.5, FHS_ERR_INVALID_ARG, "overlap must be in [0, 0.5)");
  FHS_REQUIRE(d.window == FHS_WIN_TRIANGULAR || d.window == FHS_WIN_SINE, FHS_ERR_INVALID_ARG, "unknown window");
  FHS_REQUIRE(d.B >= 1 && d.B <= kMaxB, FHS_ERR_UNSUPPORTED, "B must be in [1, 16]");
  FHS_REQUIRE(std::isfinite(d.tau) && std::isfinite(d.zeta) && std::isfinite(d.kappa) && std::isfinite(d.mu) &&
                  d.tau > 0 && d.zeta > 0 && d.kappa > 0 && d.mu >= 0,
              FHS_ERR_INVALID_ARG, "tau, zeta, kappa must be positive and mu non-negative");
  cb.n1 = d.n1; cb.n2 = d.n2; cb.L = d.L; cb.Qy = d.Qy; cb.Qx = d.Qx; cb.B = d.B; cb.window = d.window;
  cb.rho = d.overlap; cb.tau = d.tau; cb.zeta = d.zeta; cb.kappa = d.kappa; cb.mu = d.mu;
  cb.eta.assign(d.eta, d.eta + d.L);
  cb.mu_bar.assign(d.mu_bar, d.mu_bar + d.Qy * d.Qx);
  cb.eps.assign(d.eps, d.eps + d.L * d.B);
  for (double v : cb.eta) FHS_REQUIRE(std::isfinite(v) && v > 0, FHS_ERR_INVALID_ARG, "eta must be positive");
  for (double v : cb.mu_bar) FHS_REQUIRE(std::isfinite(v) && v >= 0, FHS_ERR_INVALID_ARG, "mu_bar must be >= 0");
  for (double v : cb.eps) FHS_REQUIRE(std::isfinite(v) && v >= 0, FHS_ERR_INVALID_ARG, "eps must be >= 0");
  cb.K1 = 2 * d.n1;
  cb.K2 = 2 * d.n2;
  cb.pow2 = p2;
  if (cb.K1 <= 1024 || !p2) { cb.N1c = cb.K1; cb.N2c = 1; }    // one-pass column transform
  else { cb.N1c = 64; cb.N2c = cb.K1 / 64; }
  cb.plan_r = gen_plan(cb.K1);
  cb.plan_c = gen_plan(cb.K2);

  // SARA layout
  SaraLayout& S = cb.sara;
  int64_t cur = 0;
  for (int b = 0; b < 8; ++b) {
    int F = 2 * (b + 1);
    S.rows[b][0] = d.n1;
    S.cols[b][0] = d.n2;
    for (int j = 1; j <= kLevels; ++j) {
      S.rows[b][j] = (S.rows[b][j - 1] + F - 1) / 2;
      S.cols[b][j] = (S.cols[b][j - 1] + F - 1) / 2;
    }
    for (int j = 1; j <= kLevels; ++j) {
      int64_t sz = (int64_t)S.rows[b][j] * S.cols[b][j];
      for (int s = 0; s < 3; ++s) { S.off[b][j][s] = cur; cur += sz; }
    }
    S.off[b][kLevels][3] = cur;
    cur += (int64_t)S.rows[b][kLevels] * S.cols[b][kLevels];
  }
  S.dirac_off = cur;
  cur += (int64_t)d.n1 * d.n2;
  S.I = cur;

  // nuclear facets
  std::vector<int> ys, ye, xs, xe;
  std::vector<std::vector<double>> wy, wx;
  nuclear_axis(d.n1, d.Qy, d.overlap, d.window, ys, ye, wy);
  nuclear_axis(d.n2, d.Qx, d.overlap, d.window, xs, xe, wx);
  std::vector<double> win64;
  std::vector<int> wy_off(d.Qy), wx_off(d.Qx);
  for (int i = 0; i < d.Qy; ++i) { wy_off[i] = (int)win64.size(); win64.insert(win64.end(), wy[i].begin(), wy[i].end()); }
  for (int i = 0; i < d.Qx; ++i) { wx_off[i] = (int)win64.size(); win64.insert(win64.end(), wx[i].begin(), wx[i].end()); }
  std::vector<float> win(win64.begin(), win64.end());
  cb.facets.clear();
  int64_t poff = 0;
  cb.max_facet_pix = 0;
  for (int qy = 0; qy < d.Qy; ++qy)
    for (int qx = 0; qx < d.Qx; ++qx) {
      NucFacet f;
      f.r0 = ys[qy]; f.r1 = ye[qy]; f.c0 = xs[qx]; f.c1 = xe[qx];
      f.p_off = poff;
      f.wy_off = wy_off[qy];
      f.wx_off = wx_off[qx];
      int np = (f.r1 - f.r0) * (f.c1 - f.c0);
      FHS_REQUIRE(np >= d.L, FHS_ERR_UNSUPPORTED, "a nuclear facet has fewer pixels than channels");
      cb.max_facet_pix = std::max(cb.max_facet_pix, np);
      poff += (int64_t)np * d.L;
      cb.facets.push_back(f);
    }
  cb.n_facet_pix = poff / d.L;
  std::vector<int> tile_of(d.n1 + d.n2);
  {
    std::vector<int> tb = tile_bounds(d.n1, d.Qy);
    for (int r = 0, t = 0; r < d.n1; ++r) { while (r >= tb[t + 1]) ++t; tile_of[r] = t; }
    std::vector<int> tc = tile_bounds(d.n2, d.Qx);
    for (int c = 0, t = 0; c < d.n2; ++c) { while (c >= tc[t + 1]) ++t; tile_of[d.n1 + c] = t; }
  }

  // deapodisation s = 1 / phi_hat(2 pi p / K), p = i - n/2
  std::vector<float> sr(d.n1), sc(d.n2);
  for (int i = 0; i < d.n1; ++i) sr[i] = (float)(1.0 / kb_phi_hat(2.0 * kPi * (i - d.n1 / 2) / cb.K1));
  for (int i = 0; i < d.n2; ++i) sc[i] = (float)(1.0 / kb_phi_hat(2.0 * kPi * (i - d.n2 / 2) / cb.K2));

  // visibilities: per-channel tile sort (counting sort, stable)
  cb.M_lb.assign(d.M, d.M + d.L * d.B);
  cb.vis_off.assign(d.L + 1, 0);
  cb.max_M = 0;
  for (int l = 0; l < d.L; ++l) {
    int64_t m = 0;
    for (int b = 0; b < d.B; ++b) {
      FHS_REQUIRE(cb.M_lb[l * d.B + b] >= 0, FHS_ERR_INVALID_ARG, "negative visibility count");
      m += cb.M_lb[l * d.B + b];
    }
    FHS_REQUIRE(m < (int64_t)1 << 31, FHS_ERR_UNSUPPORTED, "more than 2^31 visibilities in a channel");
    cb.vis_off[l + 1] = cb.vis_off[l] + m;
    cb.max_M = std::max(cb.max_M, m);
  }
  cb.n_vis = cb.vis_off[d.L];
  cb.tile = std::min(tile, std::min(cb.K1, cb.K2));
  if (cb.K1 % cb.tile || cb.K2 % cb.tile) cb.tile = 32;      // K = 2^a 3^b: a multiple of 32
  cb.ntile_r = cb.K1 / cb.tile;
  cb.ntile_c = cb.K2 / cb.tile;
  const int T = cb.tile;
  const int nkeys = cb.ntile_r * cb.ntile_c * 4;
  cb.perm_host.assign(cb.n_vis, 0);
  std::vector<int32_t> tile_off((size_t)d.L * (nkeys + 1));
  std::vector<float2> uv_int(cb.n_vis);
  std::vector<uint8_t> blk_int(cb.n_vis);
  std::vector<int32_t> key, cnt(nkeys + 1);
  std::vector<uint8_t> blk_user, res;
  std::vector<int64_t> order, slots;
  for (int l = 0; l < d.L; ++l) {
    const int64_t off = cb.vis_off[l], m = cb.vis_off[l + 1] - off;
    key.assign(m, 0);
    res.assign(m, 0);
    blk_user.assign(m, 0);
    {
      int64_t k = 0;
      for (int b = 0; b < d.B; ++b)
        for (int64_t t = 0; t < cb.M_lb[l * d.B + b]; ++t) blk_user[k++] = (uint8_t)b;
    }
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t i = 0; i < m; ++i) {
      float u = d.uv[2 * (off + i)], v = d.uv[2 * (off + i) + 1];
      FHS_REQUIRE(std::isfinite(u) && std::isfinite(v) && fabsf(u) < (float)kPi && fabsf(v) < (float)kPi,
                  FHS_ERR_INVALID_ARG, "uv coordinates must be finite and inside (-pi, pi)");
      int kr = ((host_first_tap(v, cb.K1) % cb.K1) + cb.K1) % cb.K1;
      int kc = ((host_first_tap(u, cb.K2) % cb.K2) + cb.K2) % cb.K2;
      int tr = kr / T, tc = kc / T, lr = kr % T, lc = kc % T;
      bool down = lr + kTaps - 1 >= T, right = lc + kTaps - 1 >= T;
      int cls = down ? (right ? 2 : 1) : (right ? 3 : 0);
      key[i] = (tr * cb.ntile_c + tc) * 4 + cls;
      res[i] = (uint8_t)((8 * lr + lc) & 31);
      cnt[key[i] + 1]++;
    }
    for (int k = 0; k < nkeys; ++k) cnt[k + 1] += cnt[k];
    int32_t* to = &tile_off[(size_t)l * (nkeys + 1)];
    for (int k = 0; k <= nkeys; ++k) to[k] = cnt[k];
    order.assign(m, 0);
    for (int64_t i = 0; i < m; ++i) order[cnt[key[i]]++] = i;
    // Within each (tile, class) bucket, deal the visibilities round-robin over
    // (8 row + column) mod 32 of their first tap in the tile: 32 consecutive
    // visibilities then have distinct residues, so the 32 lanes of a warp touch 32
    // different shared-memory banks at every tap in the gridder and 16 different bank
    // pairs per half-warp in the tile-staged degridder (row strides 8 mod 32 ints and
    // 8 mod 16 float2).  Unlike the column alone, whose residues 26..31 cover one
    // interior column where the others cover two, this key is close to uniform over a
    // tile, so the rounds stay full.
    for (int k = 0; k < nkeys; ++k) {
      const int64_t b0 = to[k], b1 = to[k + 1];
      if (b1 - b0 <= 1) continue;
      int64_t rc[33] = {0};
      for (int64_t j = b0; j < b1; ++j) rc[res[order[j]] + 1]++;
      int64_t maxc = 0;
      for (int r = 0; r < 32; ++r) maxc = std::max(maxc, rc[r + 1]);
      for (int r = 0; r < 32; ++r) rc[r + 1] += rc[r];
      slots.assign(b1 - b0, 0);
      int64_t fill[32];
      for (int r = 0; r < 32; ++r) fill[r] = rc[r];
      for (int64_t j = b0; j < b1; ++j) slots[fill[res[order[j]]]++] = order[j];
      int64_t o = b0;
      for (int64_t rank = 0; rank < maxc; ++rank)
        for (int r = 0; r < 32; ++r)
          if (rc[r] + rank < rc[r + 1]) order[o++] = slots[rc[r] + rank];
    }
    for (int64_t j = 0; j < m; ++j) {
      const int64_t i = order[j], pos = off + j;
      cb.perm_host[pos] = off + i;
      uv_int[pos] = make_float2(d.uv[2 * (off + i)], d.uv[2 * (off + i) + 1]);
      blk_int[pos] = blk_user[i];
    }
  }

  // device copies
  cb.d_uv = dalloc<float2>(cb.n_vis);
  cb.d_blk = dalloc<uint8_t>(cb.n_vis);
  cb.d_perm = dalloc<int64_t>(cb.n_vis);
  cb.d_vis_off = dalloc<int64_t>(d.L + 1);
  cb.d_tile_off = dalloc<int32_t>(tile_off.size());
  cb.d_facets = dalloc<NucFacet>(cb.facets.size());
  cb.d_win = dalloc<float>(win.size());
  cb.d_win64 = dalloc<double>(win64.size());
  cb.d_tile_of = dalloc<int>(tile_of.size());
  cb.d_scale_r = dalloc<float>(d.n1);
  cb.d_scale_c = dalloc<float>(d.n2);
  cb.d_eps = dalloc<double>(cb.eps.size());
  cb.d_eta = dalloc<float>(d.L);
  cb.d_mubar = dalloc<float>(cb.mu_bar.size());
  cb.d_M_lb = dalloc<int64_t>(cb.M_lb.size());
  std::vector<float> eta_f(cb.eta.begin(), cb.eta.end()), mub_f(cb.mu_bar.begin(), cb.mu_bar.end());
  upload(cb.d_uv, uv_int.data(), uv_int.size(), st);
  upload(cb.d_blk, blk_int.data(), blk_int.size(), st);
  upload(cb.d_perm, cb.perm_host.data(), cb.perm_host.size(), st);
  upload(cb.d_vis_off, cb.vis_off.data(), cb.vis_off.size(), st);
  upload(cb.d_tile_off, tile_off.data(), tile_off.size(), st);
  upload(cb.d_facets, cb.facets.data(), cb.facets.size(), st);
  upload(cb.d_win, win.data(), win.size(), st);
  upload(cb.d_win64, win64.data(), win64.size(), st);
  upload(cb.d_tile_of, tile_of.data(), tile_of.size(), st);
  upload(cb.d_scale_r, sr.data(), sr.size(), st);
  upload(cb.d_scale_c, sc.data(), sc.size(), st);
  upload(cb.d_eps, cb.eps.data(), cb.eps.size(), st);
  upload(cb.d_eta, eta_f.data(), eta_f.size(), st);
  upload(cb.d_mubar, mub_f.data(), mub_f.size(), st);
  upload(cb.d_M_lb, cb.M_lb.data(), cb.M_lb.size(), st);
  // per grid tile, the most footprints that cover one of its cells (fixes the
  // gridder's fixed-point scale; depends on the uv coverage only)
  cb.d_ncmax = dalloc<int>((size_t)d.L * cb.ntile_r * cb.ntile_c);
  launch_grid_count(cb, st);
  FHS_CUDA(cudaGetLastError());
  FHS_CUDA(cudaStreamSynchronize(st));
}

void free_cube(Cube& cb) {
  void* ps[] = {cb.d_uv, cb.d_blk, cb.d_perm, cb.d_vis_off, cb.d_tile_off, cb.d_facets, cb.d_win, cb.d_win64, cb.d_tile_of,
                cb.d_scale_r, cb.d_scale_c, cb.d_eps, cb.d_eta, cb.d_mubar, cb.d_ncmax, cb.d_M_lb, cb.d_U, cb.d_gamma,
                cb.d_dde_kern, cb.d_dde_idx, cb.d_dde_l1, cb.d_dde_ncmax};
  for (void* p : ps)
    if (p) cudaFree(p);
}

void alloc_scratch(fhs_ctx* ctx) {
  Scratch& s = ctx->s;
  size_t grid = 0, coef = 0, tlx = 0, tll = 0, img = 0, vis = 0, red = 2 * 1216 + 16, gram = 0, nm = 0, lb = 0;
  for (const Cube& cb : ctx->cubes) {
    const size_t L = cb.L;
    grid = std::max(grid, L * cb.K1 * cb.K2);
    coef = std::max(coef, L * (size_t)cb.sara.I);
    for (int b = 0; b < 8; ++b)
      for (int j = 1; j <= kLevels; ++j) {
        tlx = std::max(tlx, L * cb.sara.rows[b][j - 1] * cb.sara.cols[b][j]);
        tll = std::max(tll, L * cb.sara.rows[b][j] * cb.sara.cols[b][j]);
      }
    img = std::max(img, L * cb.n1 * cb.n2);
    vis = std::max(vis, (size_t)cb.n_vis);
    red = std::max(red, L * (size_t)degrid_parts(cb) * 2 * cb.B);
    red = std::max(red, L * (size_t)degrid_tiled_parts(cb) * 2 * cb.B);
    red = std::max(red, L * 64 * 2);
    int nch = (cb.max_facet_pix + 1023) / 1024;
    gram = std::max(gram, (size_t)cb.facets.size() * nch * L * L);
    nm = std::max(nm, (size_t)cb.facets.size() * L * ((L + 3) & ~3));   // M_q^T rows padded to 16 B
    lb = std::max(lb, L * cb.B);
  }
  size_t ll1 = 0, ll2 = 0, ll3 = 0;
  for (const Cube& cb : ctx->cubes) {
    size_t t1 = 0, t2 = 0, t3 = 0;
    for (int b = 0; b < 8; ++b) {
      t1 += (size_t)cb.L * cb.sara.rows[b][1] * cb.sara.cols[b][1];
      t2 += (size_t)cb.L * cb.sara.rows[b][2] * cb.sara.cols[b][2];
      t3 += (size_t)cb.L * cb.sara.rows[b][3] * cb.sara.cols[b][3];
    }
    ll1 = std::max(ll1, t1);
    ll2 = std::max(ll2, t2);
    ll3 = std::max(ll3, t3);
  }
  s.grid = dalloc<float2>(grid); s.grid_elems = grid;
  size_t pack = 0;
  for (const Cube& cb : ctx->cubes)
    if (fft_forward_packed(cb)) pack = std::max(pack, (size_t)cb.L * cb.K1 * (cb.n2 / 2));
  if (pack) s.pack = dalloc<float2>(pack);
  s.coef_elems = coef;          // allocated on first use of the plain path (ensure_coef)
  s.ll1 = dalloc<float>(ll1);
  s.ll2 = dalloc<float>(ll2);
  s.ll3 = dalloc<float>(ll3);
  s.t0 = dalloc<float>(tlx); s.t1 = dalloc<float>(tlx);
  s.t2 = dalloc<float>(tll); s.t3 = dalloc<float>(tll);
  s.t_elems = tlx;
  s.img = dalloc<float>(img); s.img2 = dalloc<float>(img); s.img_elems = img;
  s.vis = dalloc<float2>(vis); s.vis_elems = vis;
  s.red = dalloc<double>(red); s.red_elems = red;
  FHS_CUDA(cudaMallocHost((void**)&s.red_host, red * sizeof(double)));
  s.gram = dalloc<double>(gram); s.gram_elems = gram;
  s.nucM = dalloc<float>(nm); s.nucM_elems = nm;
  s.blk_scale = dalloc<float>(lb);
  s.blk_out = dalloc<double>(2 * lb + 2 * kMaxL);
  s.stat_stride = 2 * 1216 + 2 * lb;
  s.stat = dalloc<double>(s.stat_stride * ctx->cubes.size());
}

void free_scratch(Scratch& s) {
  void* ps[] = {s.grid, s.pack, s.coef, s.t0, s.t1, s.t2, s.t3, s.img, s.img2, s.vis, s.vis2, s.red, s.gram, s.nucM,
                s.blk_scale,
                s.blk_out, s.ll1, s.ll2, s.ll3, s.stat};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (s.red_host) cudaFreeHost(s.red_host);
}

// Further lanes: each has its own streams, events and a scratch set like the first
// lane's (the plain path's coefficient buffer excepted); all share the statistics
// region.  Allocated by fhs_pdfb_iter before it captures; lanes that the device memory
// cannot hold are not made (the context keeps the lanes it has).
void free_lane(fhs_ctx* ctx, Lane& x, int slot) {
  if (x.stream) cudaStreamSynchronize(x.stream);
  if (x.aux) cudaStreamSynchronize(x.aux);
  Scratch& s = x.s;
  void* ps[] = {s.grid, s.pack, s.coef, s.t0, s.t1, s.t2, s.t3, s.img, s.vis, s.vis2, s.red, s.gram, s.nucM,
                s.blk_scale, s.blk_out, s.ll1, s.ll2, s.ll3};
  for (void* p : ps)
    if (p) cudaFree(p);
  s = Scratch();
  if (x.stream) cudaStreamDestroy(x.stream);
  if (x.aux) cudaStreamDestroy(x.aux);
  for (cudaEvent_t e : {x.ev_fork, x.ev_join, x.ev_done})
    if (e) cudaEventDestroy(e);
  x = Lane();
  for (Cube& cb : ctx->cubes) cb.tm_grid[slot] = nullptr;
}

// Frees the lanes from index `keep` on (lane 0 is the context's own).
void free_lanes(fhs_ctx* ctx, int keep) {
  while ((int)ctx->xl.size() + 1 > std::max(keep, 1)) {
    const int k = (int)ctx->xl.size();
    free_lane(ctx, ctx->xl.back(), k);
    ctx->xl.pop_back();
  }
}

// Makes one more lane like the first; false (nothing kept) when memory is short.
bool make_lane(fhs_ctx* ctx) {
  const Scratch& a = ctx->s;
  Lane x;
  Scratch& b = x.s;
  bool ok = true;
  auto get = [&](auto*& p, size_t n, size_t elem) {
    using T = std::remove_reference_t<decltype(*p)>;
    if (!ok || n == 0) return;
    const uint64_t lim = g_alloc_limit.load();
    void* q = nullptr;
    if ((lim && g_alloc_used + n * elem > lim) || cudaMalloc(&q, n * elem) != cudaSuccess) {
      cudaGetLastError();          // an allocation failure leaves no sticky error
      ok = false;
      return;
    }
    g_alloc_used += n * elem;
    p = (T*)q;
  };
  size_t ll1 = 0, ll2 = 0, ll3 = 0, tll = 0;
  for (const Cube& cb : ctx->cubes) {
    size_t t1 = 0, t2 = 0, t3 = 0;
    for (int k = 0; k < 8; ++k) {
      t1 += (size_t)cb.L * cb.sara.rows[k][1] * cb.sara.cols[k][1];
      t2 += (size_t)cb.L * cb.sara.rows[k][2] * cb.sara.cols[k][2];
      t3 += (size_t)cb.L * cb.sara.rows[k][3] * cb.sara.cols[k][3];
      for (int j = 1; j <= kLevels; ++j) tll = std::max(tll, (size_t)cb.L * cb.sara.rows[k][j] * cb.sara.cols[k][j]);
    }
    ll1 = std::max(ll1, t1);
    ll2 = std::max(ll2, t2);
    ll3 = std::max(ll3, t3);
  }
  size_t pack = 0;
  for (const Cube& cb : ctx->cubes)
    if (fft_forward_packed(cb)) pack = std::max(pack, (size_t)cb.L * cb.K1 * (cb.n2 / 2));
  get(b.grid, a.grid_elems, sizeof(float2));
  get(b.pack, pack, sizeof(float2));
  get(b.coef, a.coef_elems, sizeof(float));
  get(b.t0, a.t_elems, sizeof(float));     // separate SARA passes (an autotuner choice)
  get(b.t1, a.t_elems, sizeof(float));
  get(b.t2, tll, sizeof(float));
  get(b.t3, tll, sizeof(float));
  get(b.img, a.img_elems, sizeof(float));
  get(b.vis, a.vis_elems, sizeof(float2));
  if (a.vis2) get(b.vis2, a.vis_elems, sizeof(float2));
  get(b.red, a.red_elems, sizeof(double));
  get(b.gram, a.gram_elems, sizeof(double));
  get(b.nucM, a.nucM_elems, sizeof(float));
  size_t lb = 0;
  for (const Cube& cb : ctx->cubes) lb = std::max(lb, (size_t)cb.L * cb.B);
  get(b.blk_scale, lb, sizeof(float));
  get(b.blk_out, 2 * lb + 2 * kMaxL, sizeof(double));
  get(b.ll1, ll1, sizeof(float));
  get(b.ll2, ll2, sizeof(float));
  get(b.ll3, ll3, sizeof(float));
  b.grid_elems = a.grid_elems;
  b.coef_elems = a.coef_elems;
  b.img_elems = a.img_elems;
  b.vis_elems = a.vis_elems;
  b.red_elems = a.red_elems;
  b.gram_elems = a.gram_elems;
  b.nucM_elems = a.nucM_elems;
  b.t_elems = a.t_elems;
  b.stat_stride = a.stat_stride;
  if (ok) {
    ok = cudaStreamCreateWithFlags(&x.stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&x.aux, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&x.ev_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&x.ev_join, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&x.ev_done, cudaEventDisableTiming) == cudaSuccess;
  }
  const int slot = (int)ctx->xl.size() + 1;
  if (!ok) {
    free_lane(ctx, x, slot);
    cudaGetLastError();
    return false;
  }
  b.stat = a.stat;                 // shared: each cube writes its own part
  for (Cube& cb : ctx->cubes) encode_cube_maps(cb, b.grid, slot);
  ctx->xl.push_back(x);
  return true;
}

// Lanes the next iteration uses: the requested count, at most one per cube, on the fast
// path (the plain comparison path stays a single stream of direct launches).
int lanes_in_use(const fhs_ctx* ctx) {
  if (ctx->path != FHS_PATH_FAST) return 1;
  return std::max(1, std::min({ctx->lanes, (int)ctx->cubes.size(), (int)ctx->xl.size() + 1}));
}

// Makes the requested lanes (outside any capture) and deals the cubes to them: largest
// first, each to the lane with the least work so far (work ~ pixel-channels plus
// visibilities).
void ensure_lanes(fhs_ctx* ctx) {
  const int nc = (int)ctx->cubes.size();
  if (ctx->path != FHS_PATH_FAST) return;
  const int want = std::min(ctx->lanes, nc);
  while ((int)ctx->xl.size() + 1 < want)
    if (!make_lane(ctx)) {
      ctx->lanes = (int)ctx->xl.size() + 1;    // not enough device memory for more lanes
      break;
    }
  if (!ctx->ev_lanes_fork && !ctx->xl.empty())
    FHS_CUDA(cudaEventCreateWithFlags(&ctx->ev_lanes_fork, cudaEventDisableTiming));
  const int nl = lanes_in_use(ctx);
  std::vector<int> order(nc);
  for (int c = 0; c < nc; ++c) order[c] = c;
  auto work = [&](int c) {
    const Cube& cb = ctx->cubes[c];
    return (double)cb.L * cb.n1 * cb.n2 + (double)cb.n_vis;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
  std::vector<double> load(nl, 0.0);
  ctx->lane_of.assign(nc, 0);
  for (int c : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    ctx->lane_of[c] = k;
    load[k] += work(c);
  }
}

const Cube& get_cube(fhs_ctx* ctx, int32_t c) {
  FHS_REQUIRE(c >= 0 && c < (int32_t)ctx->cubes.size(), FHS_ERR_INVALID_ARG, "cube index out of range");
  return ctx->cubes[c];
}

// ------------------------------------------------------ composite steps
// Per-basis offsets of the synthesised LL1 bands used by the fused SARA path.
void set_ll1_offsets(fhs_ctx* ctx, const Cube& cb) {
  int64_t off = 0;
  for (int b = 0; b < 8; ++b) {
    ctx->s.ll1_off[b] = off;
    off += (int64_t)cb.L * cb.sara.rows[b][1] * cb.sara.cols[b][1];
  }
}

// The plain path's [L][I] coefficient buffer, allocated on first use.
void ensure_coef(fhs_ctx* ctx) {
  if (!ctx->s.coef) ctx->s.coef = dalloc<float>(ctx->s.coef_elems);
}

bool use_fast(fhs_ctx* ctx, const Cube& cb) { return ctx->path == FHS_PATH_FAST && sara_fast_supported(cb); }

void sara_dual(fhs_ctx* ctx, const Cube& cb, const float* xcheck, float* W, const float* theta, float* A) {
  cudaStream_t st = ctx->stream;
  if (use_fast(ctx, cb) && cb.sara_fast) {
    ensure_coef(ctx);
    set_ll1_offsets(ctx, cb);
    launch_sara_fast(ctx, cb, xcheck, W, theta, A, nullptr, false, st);
  } else {
    ensure_coef(ctx);
    launch_sara_analysis(ctx, cb, xcheck, ctx->s.coef, st);
    launch_l21_dual(cb, W, ctx->s.coef, theta, st);
    launch_sara_synthesis(ctx, cb, W, A, (float)cb.kappa, true, st);
  }
  check_launch("sara dual");
}

void adjoint_into(fhs_ctx* ctx, const Cube& cb, const float2* vals, const float* blk_scale, float2* v_write,
                  float* out, const float* eta, bool accumulate) {
  cudaStream_t st = ctx->stream;
  launch_grid(cb, vals, blk_scale, v_write, ctx->s.grid, st);
  launch_fft_adjoint(ctx, cb, ctx->s.grid, out, eta, accumulate, st);
  check_launch("adjoint");
}

// Event k of the kernel timer when `which` is the selected kernel.
// (External record: inside a stream capture it becomes an event-record node of the
// graph, so every replay records the event.)
void timer_mark(fhs_ctx* ctx, int which, int k) {
  if (ctx->timer != which || ctx->timer_off) return;
  FHS_CUDA(cudaEventRecordWithFlags(ctx->tev[k], ctx->stream, cudaEventRecordExternal));
}

// One iteration of Algorithm 2 on cube c, on ctx->stream; the primal partial sums and
// the block norms land in the cube's statistics region.
void pdfb_iteration_cube(fhs_ctx* ctx, int c, const fhs_iterate& a) {
  cudaStream_t st = ctx->stream;
  {
    const Cube& cb = ctx->cubes[c];
    float* A = ctx->s.img;
    double* stat = ctx->s.stat + ctx->s.stat_stride * c;
    const int pp = primal_parts(cb);
    // data fidelity first: x_hat = F Z x, degrid + l2-ball duals, grid; its adjoint
    // writes every pixel of A, and the nuclear and SARA duals then add to it (no
    // clearing pass, no read of A in the adjoint)
    // fork: the facet Grams and eigen-solves of the nuclear duals (they read Xcheck and P
    // only) run on the second stream beside the data term
    FHS_CUDA(cudaEventRecord(ctx->ev_fork, st));
    FHS_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
    launch_nuclear_gram_eig(ctx, cb, a.Xcheck, a.state.P, a.state.theta_bar, false, nullptr, ctx->aux);
    check_launch("nuclear Gram");
    FHS_CUDA(cudaEventRecord(ctx->ev_join, ctx->aux));
    launch_fft_forward(ctx, cb, a.X, ctx->s.grid, st);
    // preconditioned duals (Section 3.2): the degridder forms d = U^-1 v + Phi x_check - y
    if (cb.n_sub > 0) launch_vis_scale((float2*)a.state.v, cb.d_U, cb.n_vis, true, st);
    int np;
    if (cb.dde_R >= 0) {
      // DDE-extended rows (Section 2.1): the warp-per-visibility de-gridder
      np = degrid_parts(cb);
      timer_mark(ctx, FHS_TIMER_DEGRID, 2 * c);
      launch_degrid_pdfb_dde(cb, ctx->s.grid, (const float2*)a.y, (const float2*)a.state.v, ctx->s.vis,
                             (float2*)a.state.u_prev, ctx->s.red, np, st);
      timer_mark(ctx, FHS_TIMER_DEGRID, 2 * c + 1);
    } else if (use_fast(ctx, cb) && cb.degrid_tiled) {
      np = degrid_tiled_parts(cb);
      timer_mark(ctx, FHS_TIMER_DEGRID, 2 * c);
      launch_degrid_pdfb_tiled(cb, ctx->s.grid, (const float2*)a.y, (const float2*)a.state.v, ctx->s.vis,
                               (float2*)a.state.u_prev, ctx->s.red, st);
      timer_mark(ctx, FHS_TIMER_DEGRID, 2 * c + 1);
    } else {
      np = degrid_parts(cb);
      launch_degrid_pdfb(cb, ctx->s.grid, (const float2*)a.y, (const float2*)a.state.v, ctx->s.vis,
                         (float2*)a.state.u_prev, ctx->s.red, np, st);
    }
    launch_block_finalize(cb, ctx->s.red, np, ctx->s.blk_scale, stat + 2 * pp, st);
    const float* gscale = ctx->s.blk_scale;
    if (cb.n_sub > 0) {
      // U-metric projections by forward-backward sub-iterations; s.vis <- v = U (d - w)
      launch_precond_duals(cb, ctx->s.vis, ctx->s.vis2, ctx->s.blk_scale, ctx->s.red, st);
      check_launch("preconditioned duals");
      gscale = nullptr;
    }
    timer_mark(ctx, FHS_TIMER_GRID, 2 * c);
    launch_grid(cb, ctx->s.vis, gscale, (float2*)a.state.v, ctx->s.grid, st);
    timer_mark(ctx, FHS_TIMER_GRID, 2 * c + 1);
    launch_fft_adjoint(ctx, cb, ctx->s.grid, A, cb.d_eta, false, st);
    check_launch("adjoint");
    FHS_CUDA(cudaStreamWaitEvent(st, ctx->ev_join, 0));          // join
    launch_nuclear_apply(ctx, cb, a.Xcheck, a.state.P, A, st);
    check_launch("nuclear dual");
    sara_dual(ctx, cb, a.Xcheck, a.state.W, a.state.theta, A);
    launch_primal(cb, a.X, a.Xcheck, A, stat, pp, st);
    check_launch("primal");
  }
}

// Exchanges the first lane's streams, events and scratch with lane x's: the launchers
// use ctx->stream, ctx->aux and ctx->s, so a cube issued between two swaps runs on
// lane x.  All lanes share the statistics region.
void swap_lane(fhs_ctx* ctx, Lane& x) {
  std::swap(ctx->s, x.s);
  std::swap(ctx->stream, x.stream);
  std::swap(ctx->aux, x.aux);
  std::swap(ctx->ev_fork, x.ev_fork);
  std::swap(ctx->ev_join, x.ev_join);
}

// One iteration of Algorithm 2 on every cube.  The sub-cubes are independent problems
// (Section 2.4.1): with several lanes, cube c runs on lane lane_of[c], so that the
// launches of cubes too small to fill the GPU run side by side.
void pdfb_iteration(fhs_ctx* ctx, const fhs_iterate* it) {
  const int nc = (int)ctx->cubes.size();
  const int nl = lanes_in_use(ctx);
  if (nl == 1 || (int)ctx->lane_of.size() != nc) {
    for (int c = 0; c < nc; ++c) pdfb_iteration_cube(ctx, c, it[c]);
    return;
  }
  FHS_CUDA(cudaEventRecord(ctx->ev_lanes_fork, ctx->stream));
  for (int k = 1; k < nl; ++k) FHS_CUDA(cudaStreamWaitEvent(ctx->xl[k - 1].stream, ctx->ev_lanes_fork, 0));
  for (int c = 0; c < nc; ++c) {
    const int k = ctx->lane_of[c] < nl ? ctx->lane_of[c] : 0;
    if (k > 0) swap_lane(ctx, ctx->xl[k - 1]);
    try {
      pdfb_iteration_cube(ctx, c, it[c]);
    } catch (...) {
      if (k > 0) swap_lane(ctx, ctx->xl[k - 1]);
      throw;
    }
    if (k > 0) swap_lane(ctx, ctx->xl[k - 1]);
  }
  for (int k = 1; k < nl; ++k) {
    Lane& x = ctx->xl[k - 1];
    FHS_CUDA(cudaEventRecord(x.ev_done, x.stream));
    FHS_CUDA(cudaStreamWaitEvent(ctx->stream, x.ev_done, 0));
  }
}

// Weights of Algorithm 1 (Eqs. 9-10) of cube c from x, on ctx->stream.
void reweight_cube(fhs_ctx* ctx, const Cube& cb, const float* x, float* theta, float* theta_bar) {
  cudaStream_t st = ctx->stream;
  ensure_coef(ctx);
  if (use_fast(ctx, cb) && cb.sara_fast) {
    launch_sara_fast(ctx, cb, x, nullptr, nullptr, nullptr, theta, true, st);
  } else {
    launch_sara_analysis(ctx, cb, x, ctx->s.coef, st);
    launch_l21_weights(cb, ctx->s.coef, theta, st);
  }
  launch_nuclear(ctx, cb, x, nullptr, nullptr, nullptr, true, theta_bar, st);
  check_launch("reweight");
}

// Adds a WHILE node at the current capture position of `st` and returns its body.
cudaGraph_t capture_while_node(cudaStream_t st, cudaGraphConditionalHandle h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  FHS_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
  FHS_REQUIRE(cs == cudaStreamCaptureStatusActive, FHS_ERR_CUDA, "stream is not capturing");
  cudaGraphNodeParams prm = {cudaGraphNodeTypeConditional};
  prm.conditional.handle = h;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  FHS_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &prm));
  FHS_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return prm.conditional.phGraph_out[0];
}

// The graph of Algorithm 1 around Algorithm 2 for cube c (see solve.cu):
//   begin -> WHILE(outer) { weights; X_t = X, X_check = X; u_prev = Phi X;
//                           WHILE(inner) { PDFB iteration; rule of Algorithm 2 };
//                           xi_rw, rule of Algorithm 1 }
// Captured on `cs` with ctx->stream redirected there.
// Kernels captured in each part of the solve graph (for the launch counter).
struct SolveCounts {
  uint64_t top = 0, cycle = 0, iteration = 0;
};

cudaGraph_t build_solve_graph(fhs_ctx* ctx, int c, const fhs_iterate& a, const fhs_solve_params& prm, cudaStream_t cs,
                              SolveCounts& cnt) {
  const Cube& cb = ctx->cubes[c];
  const int64_t n = (int64_t)cb.L * cb.n1 * cb.n2;
  void* sd = (char*)ctx->solve_dev + (size_t)c * solve_state_bytes();
  double eps2 = 0.0;
  for (double e : cb.eps) eps2 += e * e;
  const double eps_norm = sqrt(eps2);
  const double* stat = ctx->s.stat + ctx->s.stat_stride * c;
  float* Xt = ctx->s.img2;
  cudaGraph_t top = nullptr;
  FHS_CUDA(cudaGraphCreate(&top, 0));
  try {
    cudaGraphConditionalHandle h_out, h_in;
    FHS_CUDA(cudaGraphConditionalHandleCreate(&h_out, top, 1, cudaGraphCondAssignDefault));
    // top level: reset the control state, then the outer loop
    FHS_CUDA(cudaStreamBeginCaptureToGraph(cs, top, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ctx->stream = cs;
    uint64_t l0 = g_launches.load();
    launch_solve_begin(sd, cs);
    check_launch("solve begin");
    cudaGraph_t body_out = capture_while_node(cs, h_out);
    FHS_CUDA(cudaStreamEndCapture(cs, &top));
    cnt.top = g_launches.load() - l0;
    l0 = g_launches.load();
    // outer body: one reweighting cycle
    FHS_CUDA(cudaGraphConditionalHandleCreate(&h_in, body_out, 1, 0));
    FHS_CUDA(cudaStreamBeginCaptureToGraph(cs, body_out, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    reweight_cube(ctx, cb, a.X, a.state.theta, a.state.theta_bar);
    launch_solve_cycle_begin(a.X, Xt, a.Xcheck, n, sd, h_in, cs);
    launch_measure(ctx, cb, a.X, (float2*)a.state.u_prev, cs);
    check_launch("solve cycle begin");
    cudaGraph_t body_in = capture_while_node(cs, h_in);
    launch_solve_cycle_check(a.X, Xt, n, ctx->s.red, prm, sd, h_out, cs);
    check_launch("solve cycle check");
    FHS_CUDA(cudaStreamEndCapture(cs, &body_out));
    cnt.cycle = g_launches.load() - l0;
    l0 = g_launches.load();
    // inner body: one PDFB iteration and the rule of Algorithm 2
    FHS_CUDA(cudaStreamBeginCaptureToGraph(cs, body_in, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    pdfb_iteration_cube(ctx, c, a);
    launch_solve_pdfb_check(stat, primal_parts(cb), cb.L * cb.B, eps_norm, prm, sd, h_in, cs);
    check_launch("solve check");
    FHS_CUDA(cudaStreamEndCapture(cs, &body_in));
    cnt.iteration = g_launches.load() - l0;
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamCaptureStatus st_;
    if (cudaStreamIsCapturing(cs, &st_) == cudaSuccess && st_ != cudaStreamCaptureStatusNone)
      cudaStreamEndCapture(cs, &g);
    cudaGraphDestroy(top);
    throw;
  }
  return top;
}

}  // namespace

namespace {
// ||Phi_l||_S^2 of every channel of cube `cb` by the power method (Section 2.3.1
// footnote); out: host [L].  Synchronising.
void opnorm_sq(fhs_ctx* ctx, const Cube& cb, int32_t max_iter, double rel_tol, double* out) {
  cudaStream_t st = ctx->stream;
  const int L = cb.L;
  const int64_t N = (int64_t)cb.n1 * cb.n2;
  const int np = 64;
  // deterministic pseudo-random start (xorshift64), unit norm per channel: a
  // constant start is an even image and stays in the even eigenspace of the
  // point-symmetric operator Re(Phi^dagger Phi)
  std::vector<float> x0(N);
  uint64_t state = 0x9E3779B97F4A7C15ull;
  double nrm = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    state ^= state << 13; state ^= state >> 7; state ^= state << 17;
    x0[i] = (float)((double)(state >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    nrm += (double)x0[i] * x0[i];
  }
  for (int64_t i = 0; i < N; ++i) x0[i] = (float)(x0[i] / sqrt(nrm));
  for (int l = 0; l < L; ++l) upload(ctx->s.img2 + l * N, x0.data(), N, st);
  std::vector<double> val(L, 0.0), inv(L);
  std::vector<char> done(L, 0);
  double* dinv = ctx->s.blk_out;   // L doubles of scratch
  for (int it = 0; it < max_iter; ++it) {
    launch_measure(ctx, cb, ctx->s.img2, ctx->s.vis, st);
    if (cb.n_sub > 0) launch_vis_scale(ctx->s.vis, cb.d_U, cb.n_vis, false, st);   // ||U^1/2 Phi||^2
    adjoint_into(ctx, cb, ctx->s.vis, nullptr, nullptr, ctx->s.img, nullptr, false);
    launch_sumsq(ctx->s.img, N, L, ctx->s.red, np, st);
    check_launch("power method");
    FHS_CUDA(cudaMemcpyAsync(ctx->s.red_host, ctx->s.red, (size_t)L * np * 2 * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    FHS_CUDA(cudaStreamSynchronize(st));
    bool all = true;
    for (int l = 0; l < L; ++l) {
      double s = 0.0;
      for (int p = 0; p < np; ++p) s += ctx->s.red_host[2 * ((size_t)l * np + p)];
      double nv = sqrt(s);
      FHS_REQUIRE(std::isfinite(nv) && nv > 0, FHS_ERR_NONFINITE, "power method norm is not finite/positive");
      if (!done[l] && val[l] > 0 && fabs(nv - val[l]) / nv < rel_tol) done[l] = 1;
      val[l] = nv;
      inv[l] = 1.0 / nv;
      all = all && done[l];
    }
    if (all) break;
    upload(dinv, inv.data(), L, st);
    launch_scale_by_channel(ctx->s.img, N, L, dinv, st);
    FHS_CUDA(cudaMemcpyAsync(ctx->s.img2, ctx->s.img, (size_t)L * N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    check_launch("power method scale");
  }
  FHS_CUDA(cudaStreamSynchronize(st));
  for (int l = 0; l < L; ++l) out[l] = val[l];
}

}  // namespace

namespace {
// ------------------------------------------------------------ checkpoints
// File: "FHSCKPT1", ncubes (int64), per cube its shape (n1, n2, L, B, Qy, Qx, n_vis, I,
// facet pixels, n_sub: int64) and parameters (tau, zeta, kappa, mu, eta[L], mu_bar[Q],
// eps[L B]: double), then the arrays X, Xcheck, W, theta, P, theta_bar, v, u_prev of every
// cube, then the FNV-1a 64 hash of everything after the magic.
constexpr char kCkptMagic[8] = {'F', 'H', 'S', 'C', 'K', 'P', 'T', '1'};
constexpr size_t kCkptChunk = (size_t)64 << 20;

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
  }
};

struct CkptArray {
  void* dev;
  size_t bytes;
};

std::vector<CkptArray> ckpt_arrays(const Cube& cb, const fhs_iterate& a) {
  const size_t img = (size_t)cb.L * cb.n1 * cb.n2 * 4, Q = (size_t)cb.Qy * cb.Qx;
  return {{a.X, img}, {a.Xcheck, img}, {a.state.W, (size_t)cb.L * cb.sara.I * 4}, {a.state.theta, (size_t)cb.sara.I * 4},
          {a.state.P, (size_t)cb.L * cb.n_facet_pix * 4}, {a.state.theta_bar, Q * cb.L * 4},
          {a.state.v, (size_t)cb.n_vis * 8}, {a.state.u_prev, (size_t)cb.n_vis * 8}};
}

std::vector<int64_t> ckpt_shape(const Cube& cb) {
  return {cb.n1, cb.n2, cb.L, cb.B, cb.Qy, cb.Qx, cb.n_vis, cb.sara.I, cb.n_facet_pix, cb.n_sub};
}

std::vector<double> ckpt_params(const Cube& cb) {
  std::vector<double> p{cb.tau, cb.zeta, cb.kappa, cb.mu};
  p.insert(p.end(), cb.eta.begin(), cb.eta.end());
  p.insert(p.end(), cb.mu_bar.begin(), cb.mu_bar.end());
  p.insert(p.end(), cb.eps.begin(), cb.eps.end());
  return p;
}

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) fclose(f);
  }
};

void check_iterates(fhs_ctx* ctx, const fhs_iterate* it) {
  FHS_REQUIRE(it, FHS_ERR_INVALID_ARG, "NULL iterates");
  for (int c = 0; c < (int)ctx->cubes.size(); ++c) {
    const fhs_iterate& a = it[c];
    FHS_REQUIRE(a.X && a.Xcheck && a.state.W && a.state.theta && a.state.P && a.state.theta_bar && a.state.v &&
                    a.state.u_prev,
                FHS_ERR_INVALID_ARG, "NULL array in fhs_iterate");
  }
}

// ================================================================ autotuner
// Per-shape launch choices (the batching form runs many cubes of different shapes,
// Section 2.4.1): the gridder tile side (32 or 64 cells; it fixes the visibility order,
// so it is chosen before the cube is built, from trial cubes over the first two
// channels), then, once the context's scratch exists, the de-gridder (tile-staged or
// direct), the facet Gram (tcgen05 or CUDA-core float-float), and the SARA pass (fused
// tiles with 4, 8 or 16 CTAs per SM for the l2,1 pass, or the per-pass kernels).  Every
// candidate is a kernel the library also runs untuned; each is timed with CUDA events
// (one warm-up, three timed launches) on pattern inputs.  Choices are kept in a JSON
// file keyed by device and shape, read back instead of measuring.
struct TuneChoice {
  int grid_tile = kGridTile, degrid_tiled = 1, gram_tc = 1, sara_fast = 1, prox_cps = 16, source = 0;
  double ms[10] = {0};
};

std::atomic<int> g_tune_mode{0};
std::mutex g_tune_mu;
std::string g_tune_path;
using TuneFile = std::map<std::string, std::map<std::string, double>>;

std::string tune_key(const fhs_cube_desc& d) {
  int dev = 0;
  cudaDeviceProp p;
  FHS_CUDA(cudaGetDevice(&dev));
  FHS_CUDA(cudaGetDeviceProperties(&p, dev));
  int64_t m = 0;
  for (int k = 0; k < d.L * d.B; ++k) m += d.M[k];
  std::string name = p.name;
  for (char& ch : name)
    if (ch == '"' || ch == '\\' || (unsigned char)ch < 32) ch = '_';
  char buf[320];
  snprintf(buf, sizeof(buf), "%s|sm_%d%d|n=%dx%d|L=%d|Q=%dx%d|B=%d|M=%lld", name.c_str(), p.major, p.minor, d.n1,
           d.n2, d.L, d.Qy, d.Qx, d.B, (long long)m);
  return buf;
}

// The cache file: one JSON object whose members are objects of numbers.  A missing or
// unreadable file reads as empty.
struct JsonScan {
  const std::string& s;
  size_t i = 0;
  void ws() { while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) ++i; }
  bool eat(char c) {
    ws();
    if (i < s.size() && s[i] == c) { ++i; return true; }
    return false;
  }
  bool str(std::string& out) {
    ws();
    if (i >= s.size() || s[i] != '"') return false;
    out.clear();
    for (++i; i < s.size() && s[i] != '"'; ++i) {
      if (s[i] == '\\' && i + 1 < s.size()) ++i;
      out.push_back(s[i]);
    }
    return i++ < s.size();
  }
  bool num(double& v) {
    ws();
    const char* b = s.c_str() + i;
    char* e = nullptr;
    v = strtod(b, &e);
    if (e == b) return false;
    i += (size_t)(e - b);
    return true;
  }
};

TuneFile read_tune_file(const std::string& path) {
  TuneFile f;
  FILE* fp = fopen(path.c_str(), "rb");
  if (!fp) return f;
  std::string s;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof(buf), fp)) > 0) s.append(buf, n);
  fclose(fp);
  JsonScan js{s};
  TuneFile out;
  if (!js.eat('{')) return f;
  if (js.eat('}')) return out;
  for (;;) {
    std::string key, name;
    if (!js.str(key) || !js.eat(':') || !js.eat('{')) return f;
    std::map<std::string, double>& m = out[key];
    if (!js.eat('}')) {
      for (;;) {
        double v;
        if (!js.str(name) || !js.eat(':') || !js.num(v)) return f;
        m[name] = v;
        if (js.eat('}')) break;
        if (!js.eat(',')) return f;
      }
    }
    if (js.eat('}')) return out;
    if (!js.eat(',')) return f;
  }
}

void write_tune_file(const std::string& path, const TuneFile& f) {
  const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
  FILE* fp = fopen(tmp.c_str(), "wb");
  FHS_REQUIRE(fp, FHS_ERR_INVALID_ARG, "cannot write the tuning cache " + tmp);
  fprintf(fp, "{\n");
  size_t k = 0;
  for (const auto& e : f) {
    fprintf(fp, "  \"%s\": {", e.first.c_str());
    size_t j = 0;
    for (const auto& kv : e.second) fprintf(fp, "%s\"%s\": %.17g", j++ ? ", " : "", kv.first.c_str(), kv.second);
    fprintf(fp, "}%s\n", ++k < f.size() ? "," : "");
  }
  fprintf(fp, "}\n");
  const bool ok = fclose(fp) == 0;
  FHS_REQUIRE(ok && rename(tmp.c_str(), path.c_str()) == 0, FHS_ERR_INVALID_ARG,
              "cannot write the tuning cache " + path);
}

bool tune_lookup(const std::string& key, TuneChoice& ch) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune_path.empty() || g_tune_mode.load() == 2) return false;
  TuneFile f = read_tune_file(g_tune_path);
  auto it = f.find(key);
  if (it == f.end()) return false;
  auto get = [&](const char* n, int dflt) {
    auto v = it->second.find(n);
    return v == it->second.end() ? dflt : (int)v->second;
  };
  ch.grid_tile = get("grid_tile", kGridTile);
  ch.degrid_tiled = get("degrid_tiled", 1);
  ch.gram_tc = get("gram_tc", 1);
  ch.sara_fast = get("sara_fast", 1);
  ch.prox_cps = get("prox_ctas_per_sm", 16);
  FHS_REQUIRE((ch.grid_tile == 32 || ch.grid_tile == 64) && ch.prox_cps >= 1 && ch.prox_cps <= 64,
              FHS_ERR_INVALID_ARG, "tuning cache entry out of range: " + key);
  for (int k = 0; k < 10; ++k) {
    auto v = it->second.find("ms_" + std::to_string(k));
    ch.ms[k] = v == it->second.end() ? 0.0 : v->second;
  }
  ch.source = 2;
  return true;
}

void tune_store(const std::string& key, const TuneChoice& ch) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune_path.empty()) return;
  TuneFile f = read_tune_file(g_tune_path);
  std::map<std::string, double>& m = f[key];
  m.clear();
  m["grid_tile"] = ch.grid_tile;
  m["degrid_tiled"] = ch.degrid_tiled;
  m["gram_tc"] = ch.gram_tc;
  m["sara_fast"] = ch.sara_fast;
  m["prox_ctas_per_sm"] = ch.prox_cps;
  for (int k = 0; k < 10; ++k) m["ms_" + std::to_string(k)] = ch.ms[k];
  write_tune_file(g_tune_path, f);
}

// Mean time of fn over three launches after one warm-up, in ms.
template <class F>
double time_ms(cudaStream_t st, F&& fn) {
  fn();
  cudaEvent_t a = nullptr, b = nullptr;
  FHS_CUDA(cudaEventCreate(&a));
  FHS_CUDA(cudaEventCreate(&b));
  float ms = 0.f;
  cudaError_t e = cudaEventRecord(a, st);
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) fn();
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  FHS_CUDA(e);
  check_launch("autotune");
  return ms / 3.0;
}

// Gridding + tile-staged de-gridding of a trial cube over the first two channels of d
// with tile side T.
double trial_tile_ms(const fhs_cube_desc& d, int T, cudaStream_t st) {
  fhs_cube_desc t = d;
  t.L = std::min(d.L, 2);
  Cube cb;
  float2 *grid = nullptr, *vals = nullptr, *out = nullptr;
  auto release = [&] {
    for (void* p : {(void*)grid, (void*)vals, (void*)out})
      if (p) cudaFree(p);
    free_cube(cb);
  };
  try {
    build_cube(cb, t, st, T);
    const size_t ng = (size_t)cb.L * cb.K1 * cb.K2;
    grid = dalloc<float2>(ng);
    vals = dalloc<float2>(cb.n_vis);
    out = dalloc<float2>(cb.n_vis);
    launch_fill_pattern((float*)vals, 2 * cb.n_vis, 3, st);
    launch_fill_pattern((float*)grid, 2 * (int64_t)ng, 4, st);
    encode_cube_maps(cb, grid, 0);
    const double ms = time_ms(st, [&] {
      launch_grid(cb, vals, nullptr, nullptr, grid, st);
      launch_degrid(cb, grid, out, true, st);
    });
    FHS_CUDA(cudaStreamSynchronize(st));
    release();
    return ms;
  } catch (...) {
    cudaStreamSynchronize(st);
    release();
    throw;
  }
}

// Grid tile of cube d (cache, else trial cubes); the other fields of ch are set from the
// cache or left for tune_runtime.
TuneChoice tune_before_build(const fhs_cube_desc& d, cudaStream_t st) {
  TuneChoice ch;
  if (tune_lookup(tune_key(d), ch)) return ch;
  const int kmin = std::min(2 * d.n1, 2 * d.n2);
  ch.source = 1;
  if (kmin > 32) {
    ch.ms[0] = trial_tile_ms(d, 32, st);
    ch.ms[1] = trial_tile_ms(d, 64, st);
    ch.grid_tile = ch.ms[0] < ch.ms[1] ? 32 : 64;
  } else {
    ch.grid_tile = 32;
  }
  return ch;
}

// Runtime choices of cube c on the context's scratch (pattern inputs), then the cache.
void tune_after_build(fhs_ctx* ctx, int c, TuneChoice& ch, const std::string& key) {
  Cube& cb = ctx->cubes[c];
  if (ch.source == 1) {
    cudaStream_t st = ctx->stream;
    const int64_t npix = (int64_t)cb.L * cb.n1 * cb.n2;
    launch_fill_pattern(ctx->s.img, npix, 5, st);
    launch_fill_pattern((float*)ctx->s.grid, 2 * (int64_t)cb.L * cb.K1 * cb.K2, 6, st);
    ch.ms[2] = time_ms(st, [&] { launch_degrid(cb, ctx->s.grid, ctx->s.vis, true, st); });
    ch.ms[3] = time_ms(st, [&] { launch_degrid(cb, ctx->s.grid, ctx->s.vis, false, st); });
    ch.degrid_tiled = ch.ms[2] <= ch.ms[3] ? 1 : 0;
    if (cb.L <= 32) {
      ch.ms[4] = time_ms(st, [&] { launch_gram(ctx, cb, ctx->s.img, nullptr, true, st); });
      ch.ms[5] = time_ms(st, [&] { launch_gram(ctx, cb, ctx->s.img, nullptr, false, st); });
      ch.gram_tc = ch.ms[4] <= ch.ms[5] ? 1 : 0;
    } else {
      ch.gram_tc = 0;
    }
    ensure_coef(ctx);
    float* th = dalloc<float>(cb.sara.I);
    try {
      ch.ms[6] = time_ms(st, [&] {
        launch_sara_analysis(ctx, cb, ctx->s.img, ctx->s.coef, st);
        launch_l21_weights(cb, ctx->s.coef, th, st);
      });
      const int cps[3] = {4, 8, 16};
      int best = 0;
      for (int k = 0; k < 3; ++k) {
        cb.prox_cps = cps[k];
        ch.ms[7 + k] = time_ms(st, [&] { launch_sara_fast(ctx, cb, ctx->s.img, nullptr, nullptr, nullptr, th, true, st); });
        if (ch.ms[7 + k] < ch.ms[7 + best]) best = k;
      }
      ch.prox_cps = cps[best];
      ch.sara_fast = ch.ms[7 + best] <= ch.ms[6] ? 1 : 0;
      FHS_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      cudaStreamSynchronize(st);
      cudaFree(th);
      throw;
    }
    cudaFree(th);
    tune_store(key, ch);
  }
  cb.tuned = ch.source;
  cb.degrid_tiled = ch.degrid_tiled;
  cb.gram_tc = ch.gram_tc;
  cb.sara_fast = ch.sara_fast;
  cb.prox_cps = ch.prox_cps;
  for (int k = 0; k < 10; ++k) cb.tune_ms[k] = ch.ms[k];
}
}  // namespace

// ====================================================================== C ABI
extern "C" {

fhs_status fhs_create(const fhs_cube_desc* cubes, int32_t ncubes, void* stream, fhs_ctx** out) {
  if (!out) { g_create_err = "out is NULL"; return FHS_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!cubes || ncubes < 1) { g_create_err = "need at least one cube"; return FHS_ERR_INVALID_ARG; }
  fhs_ctx* ctx = new fhs_ctx();
  ctx->stream = (cudaStream_t)stream;
  g_alloc_used = 0;
  try {
    upload_kb_poly(kb_poly());
    Filters filt;
    memset(&filt, 0, sizeof(filt));
    for (int b = 0; b < 8; ++b) {
      std::vector<double> h = daubechies(b + 1);
      int F = (int)h.size();
      for (int k = 0; k < F; ++k) {
        filt.h[b][k] = (float)h[k];
        filt.g[b][k] = (float)((k % 2 ? -1.0 : 1.0) * h[F - 1 - k]);
      }
    }
    FHS_CUDA(upload_filters(filt));
    ctx->cubes.resize(ncubes);
    const bool tune = g_tune_mode.load() != 0;
    std::vector<TuneChoice> choice(ncubes);
    std::vector<std::string> keys(ncubes);
    for (int c = 0; c < ncubes; ++c) {
      // the gridder tile fixes the visibility order: chosen (autotuner) before the build
      if (tune) {
        keys[c] = tune_key(cubes[c]);
        choice[c] = tune_before_build(cubes[c], ctx->stream);
      }
      build_cube(ctx->cubes[c], cubes[c], ctx->stream, choice[c].grid_tile);
    }
    // twiddle table exp(-2 pi i k / Kmax): Kmax is the least common multiple of the grid
    // sides (2^a 3^b each), so every transform length divides it
    int kmax = 1;
    for (const Cube& cb : ctx->cubes)
      for (int K : {cb.K1, cb.K2}) kmax = std::lcm(kmax, K);
    FHS_REQUIRE(kmax <= (1 << 16), FHS_ERR_UNSUPPORTED, "grid sides too far apart for one twiddle table");
    ctx->Kmax = kmax;
    std::vector<float2> tw(kmax);
    for (int k = 0; k < kmax; ++k) {
      double a = -2.0 * kPi * k / kmax;
      tw[k] = make_float2((float)cos(a), (float)sin(a));
    }
    ctx->d_tw = dalloc<float2>(kmax);
    upload(ctx->d_tw, tw.data(), tw.size(), ctx->stream);
    alloc_scratch(ctx);
    encode_degrid_maps(ctx);
    FHS_CUDA(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
    FHS_CUDA(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
    FHS_CUDA(cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming));
    FHS_CUDA(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
    FHS_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    FHS_CUDA(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    if (tune)
      for (int c = 0; c < ncubes; ++c) tune_after_build(ctx, c, choice[c], keys[c]);
    FHS_CUDA(cudaStreamSynchronize(ctx->stream));
  } catch (const Fail& e) {
    g_create_err = e.msg;
    for (Cube& cb : ctx->cubes) free_cube(cb);
    free_scratch(ctx->s);
    if (ctx->d_tw) cudaFree(ctx->d_tw);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    for (cudaEvent_t e2 : {ctx->ev_in, ctx->ev_out, ctx->ev_fork, ctx->ev_join})
      if (e2) cudaEventDestroy(e2);
    delete ctx;
    return e.st;
  }
  *out = ctx;
  return FHS_OK;
}

fhs_status fhs_destroy(fhs_ctx* ctx) {
  if (!ctx) return FHS_ERR_INVALID_ARG;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->gstream) cudaStreamSynchronize(ctx->gstream);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->aux) {
    cudaStreamSynchronize(ctx->aux);
    cudaStreamDestroy(ctx->aux);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  free_lanes(ctx, 1);
  if (ctx->ev_lanes_fork) cudaEventDestroy(ctx->ev_lanes_fork);
  for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
  for (Cube& cb : ctx->cubes) free_cube(cb);
  free_scratch(ctx->s);
  if (ctx->d_tw) cudaFree(ctx->d_tw);
  delete ctx;
  return FHS_OK;
}

fhs_status fhs_get_sizes(const fhs_ctx* cctx, int32_t cube, fhs_sizes* out) {
  fhs_ctx* ctx = const_cast<fhs_ctx*>(cctx);
  return guarded(ctx, [&] {
    FHS_REQUIRE(out, FHS_ERR_INVALID_ARG, "out is NULL");
    const Cube& cb = get_cube(ctx, cube);
    out->n_pix = (int64_t)cb.n1 * cb.n2;
    out->n_vis = cb.n_vis;
    out->n_coef = cb.sara.I;
    out->n_facet_pix = cb.n_facet_pix;
    out->n_facets = cb.Qy * cb.Qx;
    out->n_blocks = cb.L * cb.B;
  });
}

fhs_status fhs_sync(fhs_ctx* ctx) {
  return guarded(ctx, [&] {
    FHS_CUDA(cudaStreamSynchronize(ctx->stream));
    FHS_REQUIRE(read_device_status(true) == 0, FHS_ERR_TIMEOUT, "a bounded device-side wait gave up");
  });
}

const char* fhs_last_error(const fhs_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

fhs_status fhs_vis_permutation(const fhs_ctx* cctx, int32_t cube, int64_t* perm_host) {
  fhs_ctx* ctx = const_cast<fhs_ctx*>(cctx);
  return guarded(ctx, [&] {
    FHS_REQUIRE(perm_host, FHS_ERR_INVALID_ARG, "perm_host is NULL");
    const Cube& cb = get_cube(ctx, cube);
    memcpy(perm_host, cb.perm_host.data(), cb.n_vis * sizeof(int64_t));
  });
}

fhs_status fhs_vis_to_internal(fhs_ctx* ctx, int32_t cube, const float* user, float* internal) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(user && internal && user != internal, FHS_ERR_INVALID_ARG, "need distinct non-NULL arrays");
    const Cube& cb = get_cube(ctx, cube);
    launch_vis_gather(cb.d_perm, cb.n_vis, (const float2*)user, (float2*)internal, ctx->stream);
    check_launch("vis_to_internal");
  });
}

fhs_status fhs_vis_to_user(fhs_ctx* ctx, int32_t cube, const float* internal, float* user) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(user && internal && user != internal, FHS_ERR_INVALID_ARG, "need distinct non-NULL arrays");
    const Cube& cb = get_cube(ctx, cube);
    launch_vis_scatter(cb.d_perm, cb.n_vis, (const float2*)internal, (float2*)user, ctx->stream);
    check_launch("vis_to_user");
  });
}

fhs_status fhs_measure(fhs_ctx* ctx, int32_t cube, const float* x, float* y) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(x && y, FHS_ERR_INVALID_ARG, "NULL array");
    const Cube& cb = get_cube(ctx, cube);
    launch_measure(ctx, cb, x, (float2*)y, ctx->stream);
    check_launch("measure");
  });
}

fhs_status fhs_adjoint(fhs_ctx* ctx, int32_t cube, const float* v, float* x) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(x && v, FHS_ERR_INVALID_ARG, "NULL array");
    const Cube& cb = get_cube(ctx, cube);
    adjoint_into(ctx, cb, (const float2*)v, nullptr, nullptr, x, nullptr, false);
  });
}

fhs_status fhs_opnorm_sq(fhs_ctx* ctx, int32_t cube, int32_t max_iter, double rel_tol, double* out) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(out && max_iter >= 1, FHS_ERR_INVALID_ARG, "bad arguments");
    opnorm_sq(ctx, get_cube(ctx, cube), max_iter, rel_tol, out);
  });
}

fhs_status fhs_heuristic_params(fhs_ctx* ctx, int32_t cube, const double* sigma, int32_t power_iters, double rel_tol,
                                double* eta_out, double* eps_out, double* mu_out, double* mu_bar_out) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(sigma && power_iters >= 1 && std::isfinite(rel_tol) && rel_tol >= 0, FHS_ERR_INVALID_ARG,
                "bad arguments");
    FHS_REQUIRE(cube >= 0 && cube < (int32_t)ctx->cubes.size(), FHS_ERR_INVALID_ARG, "cube index out of range");
    Cube& cb = ctx->cubes[cube];
    const int L = cb.L, LB = cb.L * cb.B, Q = cb.Qy * cb.Qx;
    for (int l = 0; l < L; ++l)
      FHS_REQUIRE(std::isfinite(sigma[l]) && sigma[l] >= 0, FHS_ERR_INVALID_ARG, "sigma must be finite and >= 0");
    std::vector<double> opn(L);
    opnorm_sq(ctx, cb, power_iters, rel_tol, opn.data());
    cudaStream_t st = ctx->stream;
    // inputs and outputs in the FP64 reduction scratch (>= 2 L + L B + 1 + Q doubles)
    const size_t need = 2 * (size_t)L + LB + 1 + Q;
    FHS_REQUIRE(need <= ctx->s.red_elems, FHS_ERR_UNSUPPORTED, "too many blocks or facets for the scratch");
    double* d_in = ctx->s.red;
    double* d_out = d_in + 2 * L;
    std::vector<double> in(2 * L);
    for (int l = 0; l < L; ++l) { in[l] = sigma[l]; in[L + l] = opn[l]; }
    upload(d_in, in.data(), in.size(), st);
    launch_heuristics(cb, d_in, d_in + L, d_out, st);
    check_launch("heuristics");
    std::vector<double> h(LB + L + 1 + Q);
    FHS_CUDA(cudaMemcpyAsync(h.data(), d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    FHS_CUDA(cudaStreamSynchronize(st));
    for (double v : h) FHS_REQUIRE(std::isfinite(v), FHS_ERR_NONFINITE, "non-finite parameter");
    // host mirrors (used for the statistics and by later fhs_set_params calls)
    cb.eta.assign(h.begin(), h.begin() + L);
    cb.eps.assign(h.begin() + L, h.begin() + L + LB);
    cb.mu = h[L + LB];
    cb.mu_bar.assign(h.begin() + L + LB + 1, h.end());
    if (eta_out) std::copy(cb.eta.begin(), cb.eta.end(), eta_out);
    if (eps_out) std::copy(cb.eps.begin(), cb.eps.end(), eps_out);
    if (mu_out) *mu_out = cb.mu;
    if (mu_bar_out) std::copy(cb.mu_bar.begin(), cb.mu_bar.end(), mu_bar_out);
  });
}

fhs_status fhs_sara_analysis(fhs_ctx* ctx, int32_t cube, const float* x, float* coef) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(x && coef, FHS_ERR_INVALID_ARG, "NULL array");
    const Cube& cb = get_cube(ctx, cube);
    launch_sara_analysis(ctx, cb, x, coef, ctx->stream);
    check_launch("sara analysis");
  });
}

fhs_status fhs_sara_synthesis(fhs_ctx* ctx, int32_t cube, const float* coef, float* x) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(x && coef, FHS_ERR_INVALID_ARG, "NULL array");
    const Cube& cb = get_cube(ctx, cube);
    launch_sara_synthesis(ctx, cb, coef, x, 1.f, false, ctx->stream);
    check_launch("sara synthesis");
  });
}

fhs_status fhs_prox_l21_sara_facets(fhs_ctx* ctx, int32_t cube, const float* xcheck, float* W, const float* theta,
                                    float* A) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(xcheck && W && theta && A, FHS_ERR_INVALID_ARG, "NULL array");
    const Cube& cb = get_cube(ctx, cube);
    sara_dual(ctx, cb, xcheck, W, theta, A);
  });
}

fhs_status fhs_prox_nuclear_facets(fhs_ctx* ctx, int32_t cube, const float* xcheck, float* P, const float* theta_bar,
                                   float* A) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(xcheck && P && theta_bar && A, FHS_ERR_INVALID_ARG, "NULL array");
    const Cube& cb = get_cube(ctx, cube);
    launch_nuclear(ctx, cb, xcheck, P, theta_bar, A, false, nullptr, ctx->stream);
    check_launch("nuclear dual");
  });
}

fhs_status fhs_proj_l2ball_blocks(fhs_ctx* ctx, int32_t cube, const float* z, const float* y, float* v_out,
                                  double* dnorm_out) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(z && y && v_out, FHS_ERR_INVALID_ARG, "NULL array");
    const Cube& cb = get_cube(ctx, cube);
    cudaStream_t st = ctx->stream;
    int np = degrid_parts(cb);
    launch_l2ball_partials(cb, (const float2*)z, (const float2*)y, ctx->s.vis, ctx->s.red, np, st);
    launch_block_finalize(cb, ctx->s.red, np, ctx->s.blk_scale, ctx->s.blk_out, st);
    launch_l2ball_scale(cb, ctx->s.vis, ctx->s.blk_scale, (float2*)v_out, st);
    check_launch("l2 ball");
    if (dnorm_out) {
      FHS_CUDA(cudaMemcpyAsync(dnorm_out, ctx->s.blk_out, (size_t)cb.L * cb.B * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
      FHS_CUDA(cudaStreamSynchronize(st));
      for (int k = 0; k < cb.L * cb.B; ++k)
        FHS_REQUIRE(std::isfinite(dnorm_out[k]), FHS_ERR_NONFINITE, "non-finite block norm");
    }
  });
}

fhs_status fhs_reweight(fhs_ctx* ctx, int32_t cube, const float* x, float* theta, float* theta_bar) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(x && theta && theta_bar, FHS_ERR_INVALID_ARG, "NULL array");
    reweight_cube(ctx, get_cube(ctx, cube), x, theta, theta_bar);
  });
}

fhs_status fhs_pdfb_iter_host(fhs_ctx* ctx, const fhs_iterate* it, const float* const* y_host, float* const* X_host,
                              int32_t n_iter, fhs_iter_stats* stats) {
  fhs_status rc = guarded(ctx, [&] {
    FHS_REQUIRE(it && y_host && X_host && n_iter >= 0, FHS_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t st = ctx->stream;
    for (int c = 0; c < (int)ctx->cubes.size(); ++c) {
      const Cube& cb = ctx->cubes[c];
      FHS_REQUIRE(y_host[c] && X_host[c] && it[c].y, FHS_ERR_INVALID_ARG, "NULL array");
      // caller's order -> internal order through the visibility scratch
      FHS_CUDA(cudaMemcpyAsync(ctx->s.vis, y_host[c], (size_t)cb.n_vis * sizeof(float2), cudaMemcpyHostToDevice, st));
      launch_vis_gather(cb.d_perm, cb.n_vis, ctx->s.vis, (float2*)it[c].y, st);
      check_launch("vis_to_internal");
    }
  });
  if (rc != FHS_OK) return rc;
  rc = fhs_pdfb_iter(ctx, it, n_iter, stats);
  if (rc != FHS_OK) return rc;
  return guarded(ctx, [&] {
    cudaStream_t st = ctx->stream;
    for (int c = 0; c < (int)ctx->cubes.size(); ++c) {
      const Cube& cb = ctx->cubes[c];
      FHS_CUDA(cudaMemcpyAsync(X_host[c], it[c].X, (size_t)cb.L * cb.n1 * cb.n2 * sizeof(float),
                               cudaMemcpyDeviceToHost, st));
    }
    FHS_CUDA(cudaStreamSynchronize(st));
  });
}

fhs_status fhs_solve(fhs_ctx* ctx, const fhs_iterate* it, const fhs_solve_params* prm, fhs_solve_report* report) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(it && prm && report, FHS_ERR_INVALID_ARG, "NULL argument");
    FHS_REQUIRE(prm->p_min >= 1 && prm->p_max >= prm->p_min && prm->t_max >= 1 &&
                    prm->t_max <= FHS_MAX_SOLVE_CYCLES && std::isfinite(prm->xi_pdfb) && prm->xi_pdfb >= 0 &&
                    std::isfinite(prm->res_factor) && prm->res_factor >= 0 && std::isfinite(prm->xi_reweight) &&
                    prm->xi_reweight >= 0,
                FHS_ERR_INVALID_ARG, "solve parameters out of range");
    const int nc = (int)ctx->cubes.size();
    for (int c = 0; c < nc; ++c) {
      const fhs_iterate& a = it[c];
      FHS_REQUIRE(a.X && a.Xcheck && a.y && a.state.W && a.state.theta && a.state.P && a.state.theta_bar &&
                      a.state.v && a.state.u_prev,
                  FHS_ERR_INVALID_ARG, "NULL array in fhs_iterate");
    }
    ensure_coef(ctx);   // no allocation may happen inside a capture
    if (!ctx->solve_dev) ctx->solve_dev = dalloc<char>((size_t)nc * solve_state_bytes());
    cudaStream_t user = ctx->stream;
    // work queued on the caller's stream comes first
    FHS_CUDA(cudaEventRecord(ctx->ev_in, user));
    FHS_CUDA(cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0));
    struct Restore {      // the caller's stream and the kernel timer, whatever happens
      fhs_ctx* c;
      cudaStream_t s;
      ~Restore() { c->stream = s; c->timer_off = false; }
    } restore{ctx, user};
    ctx->timer_off = true;
    bool nonfinite = false;
    for (int c = 0; c < nc; ++c) {
      const uint64_t l0 = g_launches.load();
      SolveCounts cnt;
      cudaGraph_t g = build_solve_graph(ctx, c, it[c], *prm, ctx->gstream, cnt);
      ctx->stream = user;
      g_launches.fetch_sub(g_launches.load() - l0);    // captured, not launched
      cudaGraphExec_t ex = nullptr;
      cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      FHS_CUDA(e);
      e = cudaGraphLaunch(ex, ctx->gstream);
      if (e == cudaSuccess)
        e = read_solve_state((char*)ctx->solve_dev + (size_t)c * solve_state_bytes(), &report[c], ctx->gstream);
      cudaGraphExecDestroy(ex);
      FHS_CUDA(e);
      // kernels run: the begin part once, the cycle body per cycle, the iteration body
      // per PDFB iteration
      note_launches((int)(cnt.top + cnt.cycle * (uint64_t)report[c].cycles +
                          cnt.iteration * (uint64_t)report[c].iterations));
      nonfinite = nonfinite || report[c].nonfinite;
    }
    FHS_CUDA(cudaEventRecord(ctx->ev_out, ctx->gstream));
    FHS_CUDA(cudaStreamWaitEvent(user, ctx->ev_out, 0));
    FHS_REQUIRE(read_device_status(true) == 0, FHS_ERR_TIMEOUT, "a bounded device-side wait gave up");
    FHS_REQUIRE(!nonfinite, FHS_ERR_NONFINITE, "a PDFB statistic was NaN or Inf; the solve stopped there");
  });
}

fhs_status fhs_set_preconditioning(fhs_ctx* ctx, int32_t cube, int32_t n_sub, const float* U_user) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(cube >= 0 && cube < (int32_t)ctx->cubes.size(), FHS_ERR_INVALID_ARG, "cube index out of range");
    FHS_REQUIRE(n_sub >= 0 && n_sub <= 1000, FHS_ERR_INVALID_ARG, "n_sub must be in [0, 1000]");
    Cube& cb = ctx->cubes[cube];
    cudaStream_t st = ctx->stream;
    FHS_CUDA(cudaStreamSynchronize(st));
    ctx->param_version++;
    if (n_sub == 0) {
      cb.n_sub = 0;
      return;
    }
    const int64_t n = cb.n_vis;
    std::vector<float> U(n);
    std::vector<uint8_t> blk(n);
    if (n) FHS_CUDA(cudaMemcpy(blk.data(), cb.d_blk, n, cudaMemcpyDeviceToHost));
    if (U_user) {
      for (int64_t i = 0; i < n; ++i) {
        const float u = U_user[cb.perm_host[i]];
        FHS_REQUIRE(std::isfinite(u) && u > 0.f, FHS_ERR_INVALID_ARG, "U must be finite and > 0");
        U[i] = u;
      }
    } else {
      // inverse sampling density: 1 / (visibilities of the channel whose nearest cell of
      // the oversampled grid, round(omega K / 2 pi) mod K, is the visibility's own)
      std::vector<float2> uv(n);
      if (n) FHS_CUDA(cudaMemcpy(uv.data(), cb.d_uv, n * sizeof(float2), cudaMemcpyDeviceToHost));
      std::vector<int64_t> cell;
      std::vector<int64_t> sorted;
      for (int l = 0; l < cb.L; ++l) {
        const int64_t o = cb.vis_off[l], m = cb.vis_off[l + 1] - o;
        cell.resize(m);
        for (int64_t j = 0; j < m; ++j) {
          const double tr = floor((double)uv[o + j].y * cb.K1 / (2.0 * kPi) + 0.5);
          const double tc = floor((double)uv[o + j].x * cb.K2 / (2.0 * kPi) + 0.5);
          const int64_t r = (((int64_t)tr % cb.K1) + cb.K1) % cb.K1, c = (((int64_t)tc % cb.K2) + cb.K2) % cb.K2;
          cell[j] = r * cb.K2 + c;
        }
        sorted = cell;
        std::sort(sorted.begin(), sorted.end());
        for (int64_t j = 0; j < m; ++j) {
          auto rng = std::equal_range(sorted.begin(), sorted.end(), cell[j]);
          U[o + j] = (float)(1.0 / (double)(rng.second - rng.first));
        }
      }
    }
    std::vector<float> gmax(cb.L * cb.B, 0.f), gamma(cb.L * cb.B, 0.f);
    for (int l = 0; l < cb.L; ++l)
      for (int64_t i = cb.vis_off[l]; i < cb.vis_off[l + 1]; ++i) {
        float& g = gmax[l * cb.B + blk[i]];
        g = std::max(g, U[i]);
      }
    for (int k = 0; k < cb.L * cb.B; ++k) gamma[k] = gmax[k] > 0.f ? 1.f / gmax[k] : 0.f;
    if (!cb.d_U) cb.d_U = dalloc<float>(n);
    if (!cb.d_gamma) cb.d_gamma = dalloc<float>(gamma.size());
    if (!ctx->s.vis2) ctx->s.vis2 = dalloc<float2>(ctx->s.vis_elems);
    for (Lane& x : ctx->xl)
      if (!x.s.vis2) x.s.vis2 = dalloc<float2>(ctx->s.vis_elems);
    upload(cb.d_U, U.data(), U.size(), st);
    upload(cb.d_gamma, gamma.data(), gamma.size(), st);
    FHS_CUDA(cudaStreamSynchronize(st));
    cb.n_sub = n_sub;
  });
}

fhs_status fhs_set_dde(fhs_ctx* ctx, int32_t cube, int32_t S_d, int32_t n_kern, const float* kern,
                       const int32_t* kidx) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(cube >= 0 && cube < (int32_t)ctx->cubes.size(), FHS_ERR_INVALID_ARG, "cube index out of range");
    FHS_REQUIRE(S_d == 0 || (S_d >= 1 && S_d <= 2 * kDdeMaxR + 1 && (S_d & 1)), FHS_ERR_INVALID_ARG,
                "S_d must be 0 or odd in [1, 9]");
    Cube& cb = ctx->cubes[cube];
    cudaStream_t st = ctx->stream;
    FHS_CUDA(cudaStreamSynchronize(st));
    ctx->param_version++;
    if (S_d == 0) {
      cb.dde_R = -1;
      return;
    }
    FHS_REQUIRE(kern && kidx && n_kern >= 1, FHS_ERR_INVALID_ARG, "kernels and indices are required");
    FHS_REQUIRE(kTaps + S_d - 1 <= cb.tile, FHS_ERR_UNSUPPORTED, "extended footprint wider than a grid tile");
    const int sd2 = S_d * S_d;
    std::vector<float> l1(n_kern);
    for (int k = 0; k < n_kern; ++k) {
      double a = 0.0;
      for (int j = 0; j < 2 * sd2; ++j) {
        const float x = kern[(size_t)k * 2 * sd2 + j];
        FHS_REQUIRE(std::isfinite(x), FHS_ERR_INVALID_ARG, "non-finite DDE kernel coefficient");
        a += fabs((double)x);
      }
      l1[k] = (float)(a * (1.0 + 1.0 / (1 << 20)));     // rounded up: a bound of the tap values
    }
    const int64_t n = cb.n_vis;
    std::vector<int32_t> idx(n);
    for (int64_t i = 0; i < n; ++i) {
      const int32_t k = kidx[cb.perm_host[i]];
      FHS_REQUIRE(k >= 0 && k < n_kern, FHS_ERR_INVALID_ARG, "DDE kernel index out of range");
      idx[i] = k;
    }
    if (cb.d_dde_kern) { cudaFree(cb.d_dde_kern); cb.d_dde_kern = nullptr; }
    if (cb.d_dde_l1) { cudaFree(cb.d_dde_l1); cb.d_dde_l1 = nullptr; }
    cb.d_dde_kern = dalloc<float2>((size_t)n_kern * sd2);
    cb.d_dde_l1 = dalloc<float>(n_kern);
    if (!cb.d_dde_idx) cb.d_dde_idx = dalloc<int32_t>(n ? n : 1);
    if (!cb.d_dde_ncmax) cb.d_dde_ncmax = dalloc<int>((size_t)cb.L * cb.ntile_r * cb.ntile_c);
    upload(cb.d_dde_kern, reinterpret_cast<const float2*>(kern), (size_t)n_kern * sd2, st);
    upload(cb.d_dde_l1, l1.data(), l1.size(), st);
    if (n) upload(cb.d_dde_idx, idx.data(), idx.size(), st);
    cb.dde_R = (S_d - 1) / 2;
    cb.dde_nkern = n_kern;
    // the extended footprints covering each cell of a tile fix its fixed-point scale
    launch_grid_dde_count(cb, st);
    FHS_CUDA(cudaGetLastError());
    FHS_CUDA(cudaStreamSynchronize(st));
  });
}

fhs_status fhs_set_params(fhs_ctx* ctx, int32_t cube, double tau, double zeta, double kappa, const double* eta,
                          double mu, const double* mu_bar, const double* eps) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(eta && mu_bar && eps, FHS_ERR_INVALID_ARG, "NULL parameter array");
    FHS_REQUIRE(cube >= 0 && cube < (int32_t)ctx->cubes.size(), FHS_ERR_INVALID_ARG, "cube index out of range");
    Cube& cb = ctx->cubes[cube];
    FHS_REQUIRE(std::isfinite(tau) && std::isfinite(zeta) && std::isfinite(kappa) && std::isfinite(mu) && tau > 0 &&
                    zeta > 0 && kappa > 0 && mu >= 0,
                FHS_ERR_INVALID_ARG, "tau, zeta, kappa must be positive and mu non-negative");
    const int Q = cb.Qy * cb.Qx;
    for (int l = 0; l < cb.L; ++l) FHS_REQUIRE(std::isfinite(eta[l]) && eta[l] > 0, FHS_ERR_INVALID_ARG, "bad eta");
    for (int q = 0; q < Q; ++q) FHS_REQUIRE(std::isfinite(mu_bar[q]) && mu_bar[q] >= 0, FHS_ERR_INVALID_ARG, "bad mu_bar");
    for (int k = 0; k < cb.L * cb.B; ++k) FHS_REQUIRE(std::isfinite(eps[k]) && eps[k] >= 0, FHS_ERR_INVALID_ARG, "bad eps");
    cb.tau = tau; cb.zeta = zeta; cb.kappa = kappa; cb.mu = mu;
    cb.eta.assign(eta, eta + cb.L);
    cb.mu_bar.assign(mu_bar, mu_bar + Q);
    cb.eps.assign(eps, eps + cb.L * cb.B);
    std::vector<float> eta_f(cb.eta.begin(), cb.eta.end()), mub_f(cb.mu_bar.begin(), cb.mu_bar.end());
    FHS_CUDA(cudaStreamSynchronize(ctx->stream));
    upload(cb.d_eps, cb.eps.data(), cb.eps.size(), ctx->stream);
    upload(cb.d_eta, eta_f.data(), eta_f.size(), ctx->stream);
    upload(cb.d_mubar, mub_f.data(), mub_f.size(), ctx->stream);
    FHS_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

uint64_t fhs_kernel_launches(void) { return g_launches.load(); }

fhs_status fhs_checkpoint_save(fhs_ctx* ctx, const fhs_iterate* it, const char* path) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(path, FHS_ERR_INVALID_ARG, "NULL path");
    check_iterates(ctx, it);
    FileCloser fc{fopen(path, "wb")};
    FHS_REQUIRE(fc.f, FHS_ERR_INVALID_ARG, std::string("cannot open ") + path + " for writing");
    FHS_CUDA(cudaStreamSynchronize(ctx->stream));
    Fnv h;
    auto put = [&](const void* p, size_t n, bool hash) {
      FHS_REQUIRE(fwrite(p, 1, n, fc.f) == n, FHS_ERR_INVALID_ARG, "checkpoint write failed");
      if (hash) h.add(p, n);
    };
    put(kCkptMagic, sizeof(kCkptMagic), false);
    const int64_t nc = (int64_t)ctx->cubes.size();
    put(&nc, sizeof(nc), true);
    for (const Cube& cb : ctx->cubes) {
      const std::vector<int64_t> shp = ckpt_shape(cb);
      const std::vector<double> prm = ckpt_params(cb);
      put(shp.data(), shp.size() * 8, true);
      put(prm.data(), prm.size() * 8, true);
    }
    std::vector<unsigned char> buf(kCkptChunk);
    for (int c = 0; c < (int)nc; ++c)
      for (const CkptArray& a : ckpt_arrays(ctx->cubes[c], it[c]))
        for (size_t o = 0; o < a.bytes; o += kCkptChunk) {
          const size_t n = std::min(kCkptChunk, a.bytes - o);
          FHS_CUDA(cudaMemcpy(buf.data(), (const char*)a.dev + o, n, cudaMemcpyDeviceToHost));
          put(buf.data(), n, true);
        }
    put(&h.h, sizeof(h.h), false);
  });
}

fhs_status fhs_checkpoint_load(fhs_ctx* ctx, const fhs_iterate* it, const char* path) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(path, FHS_ERR_INVALID_ARG, "NULL path");
    check_iterates(ctx, it);
    FileCloser fc{fopen(path, "rb")};
    FHS_REQUIRE(fc.f, FHS_ERR_INVALID_ARG, std::string("cannot open ") + path);
    auto get = [&](void* p, size_t n) {
      FHS_REQUIRE(fread(p, 1, n, fc.f) == n, FHS_ERR_INVALID_ARG, "checkpoint truncated");
    };
    char magic[8];
    get(magic, 8);
    FHS_REQUIRE(memcmp(magic, kCkptMagic, 8) == 0, FHS_ERR_INVALID_ARG, "not a checkpoint of this library");
    // pass 1: the hash over the whole payload, before anything is changed
    const long start = ftell(fc.f);
    FHS_REQUIRE(fseek(fc.f, 0, SEEK_END) == 0, FHS_ERR_INVALID_ARG, "checkpoint not seekable");
    const long end = ftell(fc.f);
    FHS_REQUIRE(end - start >= 16, FHS_ERR_INVALID_ARG, "checkpoint truncated");
    fseek(fc.f, start, SEEK_SET);
    std::vector<unsigned char> buf(kCkptChunk);
    Fnv h;
    for (long left = end - start - 8; left > 0;) {
      const size_t n = (size_t)std::min<long>(left, (long)kCkptChunk);
      get(buf.data(), n);
      h.add(buf.data(), n);
      left -= (long)n;
    }
    uint64_t stored = 0;
    get(&stored, 8);
    FHS_REQUIRE(stored == h.h, FHS_ERR_INVALID_ARG, "checkpoint corrupt (hash mismatch)");
    // pass 2: shapes must match the context, then parameters and arrays
    fseek(fc.f, start, SEEK_SET);
    int64_t nc = 0;
    get(&nc, 8);
    FHS_REQUIRE(nc == (int64_t)ctx->cubes.size(), FHS_ERR_INVALID_ARG, "checkpoint has another number of cubes");
    std::vector<std::vector<double>> prms;
    for (Cube& cb : ctx->cubes) {
      std::vector<int64_t> shp(ckpt_shape(cb).size());
      get(shp.data(), shp.size() * 8);
      std::vector<int64_t> mine = ckpt_shape(cb);
      mine.back() = shp.back();     // n_sub may differ: the caller sets the preconditioner
      FHS_REQUIRE(shp == mine, FHS_ERR_INVALID_ARG, "checkpoint of a cube of another shape");
      std::vector<double> prm(ckpt_params(cb).size());
      get(prm.data(), prm.size() * 8);
      prms.push_back(prm);
    }
    for (int c = 0; c < (int)nc; ++c)
      for (const CkptArray& a : ckpt_arrays(ctx->cubes[c], it[c]))
        for (size_t o = 0; o < a.bytes; o += kCkptChunk) {
          const size_t n = std::min(kCkptChunk, a.bytes - o);
          get(buf.data(), n);
          FHS_CUDA(cudaMemcpy((char*)a.dev + o, buf.data(), n, cudaMemcpyHostToDevice));
        }
    for (int c = 0; c < (int)nc; ++c) {
      Cube& cb = ctx->cubes[c];
      const std::vector<double>& p = prms[c];
      const int L = cb.L, Q = cb.Qy * cb.Qx, LB = cb.L * cb.B;
      cb.tau = p[0]; cb.zeta = p[1]; cb.kappa = p[2]; cb.mu = p[3];
      cb.eta.assign(p.begin() + 4, p.begin() + 4 + L);
      cb.mu_bar.assign(p.begin() + 4 + L, p.begin() + 4 + L + Q);
      cb.eps.assign(p.begin() + 4 + L + Q, p.begin() + 4 + L + Q + LB);
      std::vector<float> eta_f(cb.eta.begin(), cb.eta.end()), mub_f(cb.mu_bar.begin(), cb.mu_bar.end());
      upload(cb.d_eps, cb.eps.data(), cb.eps.size(), ctx->stream);
      upload(cb.d_eta, eta_f.data(), eta_f.size(), ctx->stream);
      upload(cb.d_mubar, mub_f.data(), mub_f.size(), ctx->stream);
    }
    FHS_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->param_version++;
  });
}

fhs_status fhs_set_wait_limit(int64_t spins) {
  if (spins < -1) return FHS_ERR_INVALID_ARG;
  return set_wait_first((long long)spins) == cudaSuccess ? FHS_OK : FHS_ERR_CUDA;
}

fhs_status fhs_set_alloc_limit(uint64_t bytes) {
  g_alloc_limit.store(bytes);
  return FHS_OK;
}

fhs_status fhs_set_autotune(int32_t mode, const char* cache_path) {
  if (mode < 0 || mode > 2) return FHS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_mode.store(mode);
  g_tune_path = cache_path ? cache_path : "";
  return FHS_OK;
}

fhs_status fhs_get_tuning(const fhs_ctx* cctx, int32_t cube, fhs_tuning* out) {
  fhs_ctx* ctx = const_cast<fhs_ctx*>(cctx);
  return guarded(ctx, [&] {
    FHS_REQUIRE(out, FHS_ERR_INVALID_ARG, "out is NULL");
    const Cube& cb = get_cube(ctx, cube);
    out->grid_tile = cb.tile;
    out->degrid_tiled = cb.degrid_tiled;
    out->gram_tc = cb.gram_tc;
    out->sara_fast = cb.sara_fast;
    out->prox_ctas_per_sm = cb.prox_cps;
    out->source = cb.tuned;
    for (int k = 0; k < 10; ++k) out->ms[k] = cb.tune_ms[k];
  });
}

fhs_status fhs_set_kernel_timer(fhs_ctx* ctx, int32_t kernel) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(kernel == FHS_TIMER_NONE || kernel == FHS_TIMER_GRID || kernel == FHS_TIMER_DEGRID,
                FHS_ERR_INVALID_ARG, "unknown kernel timer");
    const size_t need = 2 * ctx->cubes.size();
    while (ctx->tev.size() < need) {
      cudaEvent_t e;
      FHS_CUDA(cudaEventCreate(&e));
      ctx->tev.push_back(e);
    }
    ctx->timer = kernel;
    ctx->timer_armed = false;
  });
}

fhs_status fhs_kernel_timer_read(fhs_ctx* ctx, double* ms_total, int32_t* launches) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(ms_total && launches, FHS_ERR_INVALID_ARG, "NULL output");
    FHS_REQUIRE(ctx->timer != FHS_TIMER_NONE && ctx->timer_armed, FHS_ERR_INVALID_ARG,
                "no kernel timer selected, or no iteration since the selection");
    const int nc = (int)ctx->cubes.size();
    double tot = 0.0;
    for (int c = 0; c < nc; ++c) {
      FHS_CUDA(cudaEventSynchronize(ctx->tev[2 * c + 1]));
      float ms = 0.f;
      FHS_CUDA(cudaEventElapsedTime(&ms, ctx->tev[2 * c], ctx->tev[2 * c + 1]));
      tot += ms;
    }
    *ms_total = tot;
    *launches = nc;
  });
}

fhs_status fhs_set_path(fhs_ctx* ctx, int32_t path) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(path == FHS_PATH_FAST || path == FHS_PATH_PLAIN, FHS_ERR_INVALID_ARG, "unknown path");
    ctx->path = path;
  });
}

fhs_status fhs_set_lanes(fhs_ctx* ctx, int32_t lanes) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(lanes >= 1 && lanes <= kMaxLanes, FHS_ERR_INVALID_ARG, "lanes must be in [1, 4]");
    if ((int)ctx->xl.size() + 1 > lanes) {
      if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
      ctx->graph_key.clear();
      free_lanes(ctx, lanes);
    }
    ctx->lanes = lanes;
  });
}

fhs_status fhs_get_lanes(const fhs_ctx* ctx, int32_t* lanes) {
  if (!ctx || !lanes) return FHS_ERR_INVALID_ARG;
  *lanes = lanes_in_use(ctx);
  return FHS_OK;
}

fhs_status fhs_pdfb_iter(fhs_ctx* ctx, const fhs_iterate* it, int32_t n_iter, fhs_iter_stats* stats) {
  return guarded(ctx, [&] {
    FHS_REQUIRE(it && n_iter >= 0, FHS_ERR_INVALID_ARG, "bad arguments");
    const int nc = (int)ctx->cubes.size();
    std::vector<const void*> key;
    key.push_back((const void*)(intptr_t)ctx->path);
    key.push_back((const void*)(intptr_t)ctx->timer);
    key.push_back((const void*)(uintptr_t)ctx->param_version);
    key.push_back((const void*)(intptr_t)ctx->lanes);
    for (int c = 0; c < nc; ++c) {
      const fhs_iterate& a = it[c];
      FHS_REQUIRE(a.X && a.Xcheck && a.y && a.state.W && a.state.theta && a.state.P && a.state.theta_bar &&
                      a.state.v && a.state.u_prev,
                  FHS_ERR_INVALID_ARG, "NULL array in fhs_iterate");
      const void* ps[] = {a.X, a.Xcheck, a.y, a.state.W, a.state.theta, a.state.P, a.state.theta_bar, a.state.v,
                          a.state.u_prev};
      key.insert(key.end(), ps, ps + 9);
    }
    if (n_iter == 0) return;
    if (ctx->path == FHS_PATH_PLAIN) {
      // the comparison arm: direct launches, no graph
      for (int p = 0; p < n_iter; ++p) pdfb_iteration(ctx, it);
    } else {
    // (re)capture one iteration of every cube into a CUDA graph when the arrays or the path change
    if (!ctx->graph_exec || key != ctx->graph_key) {
      if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
      ensure_coef(ctx);   // no allocation may happen inside the capture
      ensure_lanes(ctx);
      cudaStream_t user = ctx->stream;
      uint64_t before = g_launches.load();
      FHS_CUDA(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal));
      ctx->stream = ctx->gstream;
      try {
        pdfb_iteration(ctx, it);
      } catch (...) {
        ctx->stream = user;
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(ctx->gstream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      ctx->stream = user;
      cudaGraph_t g = nullptr;
      FHS_CUDA(cudaStreamEndCapture(ctx->gstream, &g));
      cudaError_t e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
      cudaGraphDestroy(g);
      FHS_CUDA(e);
      ctx->graph_kernels = g_launches.load() - before;
      g_launches.fetch_sub(ctx->graph_kernels);          // captured, not launched
      ctx->graph_key = key;
    }
    FHS_CUDA(cudaEventRecord(ctx->ev_in, ctx->stream));
    FHS_CUDA(cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0));
    for (int p = 0; p < n_iter; ++p) {
      FHS_CUDA(cudaGraphLaunch(ctx->graph_exec, ctx->gstream));
      note_launches((int)ctx->graph_kernels);
    }
    FHS_CUDA(cudaEventRecord(ctx->ev_out, ctx->gstream));
    FHS_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_out, 0));
    }
    if (ctx->timer != FHS_TIMER_NONE) ctx->timer_armed = true;
    if (!stats) return;
    std::vector<double> h(ctx->s.stat_stride * nc);
    FHS_CUDA(cudaMemcpyAsync(h.data(), ctx->s.stat, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    FHS_CUDA(cudaStreamSynchronize(ctx->stream));
    FHS_REQUIRE(read_device_status(true) == 0, FHS_ERR_TIMEOUT, "a bounded device-side wait gave up");
    for (int c = 0; c < nc; ++c) {
      const Cube& cb = ctx->cubes[c];
      const double* st = h.data() + ctx->s.stat_stride * c;
      const int pp = primal_parts(cb);
      const double* blk = st + 2 * pp;
      double dx2 = 0.0, x2 = 0.0;
      for (int k = 0; k < pp; ++k) { dx2 += st[2 * k]; x2 += st[2 * k + 1]; }
      double r2 = 0.0, e2 = 0.0, d2 = 0.0;
      for (int k = 0; k < cb.L * cb.B; ++k) {
        r2 += blk[cb.L * cb.B + k] * blk[cb.L * cb.B + k];
        d2 += blk[k] * blk[k];       // ||v + Phi x_check - y|| of the data duals
        e2 += cb.eps[k] * cb.eps[k];
      }
      FHS_REQUIRE(std::isfinite(dx2) && std::isfinite(x2) && std::isfinite(r2) && std::isfinite(d2),
                  FHS_ERR_NONFINITE, "non-finite iteration statistics");
      stats[c].xi = x2 > 0 ? sqrt(dx2 / x2) : INFINITY;
      stats[c].res_norm = sqrt(r2);
      stats[c].eps_norm = sqrt(e2);
    }
  });
}

}  // extern "C"
