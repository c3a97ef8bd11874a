// Fused SARA l2,1 dual (Algorithm 2 W update, Table 2 row 3) on GB300.
//
// Three kernels replace the level-by-level plain passes:
//   k_fa_prox   : per 16x16 coefficient tile of one (basis, level), two passes
//                 over the L channels: each stages the input tile with its
//                 filter halo and the tile's W values in shared memory
//                 (cp.async, double buffered, zero fill outside the signal) and
//                 filters along x then y; pass 1 accumulates ||z_i||^2 of
//                 z = W + Psi^dagger x across channels (and writes the LL band
//                 for the next level), pass 2 recomputes z and writes
//                 W <- z min(1, alpha_i / ||z_i||) (weights mode: pass 1 only,
//                 theta_i = mu / (||coef_i|| + mu)).  No coefficient buffer
//                 round trip through HBM.
//   k_fs_level  : synthesis of one level (4 -> 2) of one basis, per 32x32
//                 output tile and channel: both separable transpose passes in
//                 shared memory.
//   k_fs_final  : level-1 synthesis of all eight bases plus the Dirac block for
//                 a 32x32 output tile, accumulated in registers, A += kappa *
//                 result written once.
// Same conventions as sara.cu (zero-padded full convolution, odd phase, /3).




namespace fhs {

// uses c_filt of sara.cu (this file is included at the end of sara.cu)

constexpr int kTK = 16;          // analysis coefficient tile
constexpr int kTO = 32;          // synthesis output tile
constexpr int kInMax = 2 * kTK + kMaxFilt - 2;     // 46
constexpr int kKnMax = kTO / 2 + kMaxFilt / 2 + 1;  // 25

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

struct AnaArgs {
  const float* in;     // [L][m1][m2]
  float* ll_out;       // [L][mo1][mo2] or null at the last level
  float* W;            // [L][I]
  const float* theta;  // [I]
  float* theta_out;    // weights mode
  int64_t I;
  int64_t off[4];      // d0, d1, d2, LL4
  int L, m1, m2, mo1, mo2, basis, nsub;
  float alpha_scale, mu;
  int weights;
};

// Stage channel l: its input tile (with halo, zero outside the signal) and, in
// dual mode, this thread's W values of the channel into wst[s][tid].
__device__ __forceinline__ void fa_stage(const AnaArgs& a, float* tin, float* wst, int l, int r_in0, int c_in0,
                                         int IN, bool valid, int64_t pos) {
  const float* inl = a.in + (size_t)l * a.m1 * a.m2;
  for (int idx = threadIdx.x; idx < IN * IN; idx += blockDim.x) {
    int r = idx / IN, c = idx % IN;
    int gr = r_in0 + r, gc = c_in0 + c;
    bool v = gr >= 0 && gr < a.m1 && gc >= 0 && gc < a.m2;
    cp_async4(&tin[r * (kInMax + 1) + c], v ? inl + (size_t)gr * a.m2 + gc : inl, v);
  }
  const float* Wl = a.W ? a.W + (size_t)l * a.I : inl;
  for (int s = 0; s < a.nsub; ++s) {
    bool v = valid && !a.weights;
    cp_async4(&wst[s * (kTK * kTK) + threadIdx.x], v ? Wl + a.off[s] + pos : inl, v);
  }
  cp_async_commit();
}

// Coefficients of this thread's position for the staged channel: cf = (d0, d1, d2, LL) / 3;
// also returns the unscaled LL for the next level.
__device__ __forceinline__ void fa_filter(const float* tin, float* tlx, float* thx, int b, int F, int IN, int tk,
                                          int tc, bool valid, float cf[4], float& ll_out) {
  for (int idx = threadIdx.x; idx < IN * kTK; idx += blockDim.x) {
    int r = idx / kTK, kc = idx % kTK;
    const float* row = tin + r * (kInMax + 1) + 2 * kc + F - 1;   // input column 2 kc + F - 1 - t
    float sl = 0.f, sh = 0.f;
    for (int t = 0; t < F; ++t) {
      float x = row[-t];
      sl = fmaf(c_filt.h[b][t], x, sl);
      sh = fmaf(c_filt.g[b][t], x, sh);
    }
    tlx[r * (kTK + 1) + kc] = sl;
    thx[r * (kTK + 1) + kc] = sh;
  }
  __syncthreads();
  float ll = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
  if (valid) {
    for (int t = 0; t < F; ++t) {
      int r = 2 * tk + F - 1 - t;
      float vl = tlx[r * (kTK + 1) + tc], vh = thx[r * (kTK + 1) + tc];
      float h = c_filt.h[b][t], g = c_filt.g[b][t];
      ll = fmaf(h, vl, ll);
      d1 = fmaf(g, vl, d1);
      d0 = fmaf(h, vh, d0);
      d2 = fmaf(g, vh, d2);
    }
  }
  const float third = 1.f / 3.f;
  cf[0] = d0 * third; cf[1] = d1 * third; cf[2] = d2 * third; cf[3] = ll * third;
  ll_out = ll;
}

// Two phases over the L channels of a 16x16 coefficient tile: phase 1 forms
// z = W + Psi^dagger x for every channel and accumulates ||z_i||^2 (the LL band
// for the next level is written here); phase 2 stages the channels again (the
// tiles are L2-resident by then), recomputes z and writes W = z min(1, alpha/||z||).
// Keeping only the norms between the phases (instead of z for all channels)
// cuts shared memory to ~32 KB per CTA and lets 7 CTAs share an SM.
__global__ void __launch_bounds__(256) k_fa_prox(AnaArgs a) {
  extern __shared__ float sm[];
  const int b = a.basis;
  const int F = 2 * (b + 1);
  const int IN = 2 * kTK + F - 2;
  float* tinb[2] = {sm, sm + kInMax * (kInMax + 1)};
  float* tlx = sm + 2 * kInMax * (kInMax + 1);        // [kInMax][kTK+1]
  float* thx = tlx + kInMax * (kTK + 1);
  float* wstb[2] = {thx + kInMax * (kTK + 1), thx + kInMax * (kTK + 1) + 4 * kTK * kTK};
  const int k0 = blockIdx.y * kTK, c0 = blockIdx.x * kTK;
  const int r_in0 = 2 * k0 + 2 - F, c_in0 = 2 * c0 + 2 - F;
  const int tk = threadIdx.x / kTK, tc = threadIdx.x % kTK;
  const bool valid = (k0 + tk < a.mo1) && (c0 + tc < a.mo2);
  const int64_t pos = (int64_t)(k0 + tk) * a.mo2 + (c0 + tc);
  float n2[4] = {0.f, 0.f, 0.f, 0.f};
  float fac[4] = {1.f, 1.f, 1.f, 1.f};
  const int phases = a.weights ? 1 : 2;
  for (int ph = 0; ph < phases; ++ph) {
    fa_stage(a, tinb[0], wstb[0], 0, r_in0, c_in0, IN, valid, pos);
    for (int l = 0; l < a.L; ++l) {
      const int cur = l & 1;
      if (l + 1 < a.L) {
        fa_stage(a, tinb[cur ^ 1], wstb[cur ^ 1], l + 1, r_in0, c_in0, IN, valid, pos);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      float cf[4], ll;
      fa_filter(tinb[cur], tlx, thx, b, F, IN, tk, tc, valid, cf, ll);
      if (valid) {
        if (ph == 0 && a.ll_out) a.ll_out[(size_t)l * a.mo1 * a.mo2 + pos] = ll;
        const float* wst = wstb[cur];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (s < a.nsub) {
            float z = wst[s * (kTK * kTK) + threadIdx.x] + cf[s];   // W staged (0 in weights mode)
            if (ph == 0) n2[s] = fmaf(z, z, n2[s]);
            else a.W[(size_t)l * a.I + a.off[s] + pos] = z * fac[s];
          }
        }
      }
      __syncthreads();   // tin / tlx / wst of this channel are reused two stages later
    }
    if (ph == 0 && valid) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (s >= a.nsub) break;
        float nrm = sqrtf(n2[s]);
        if (a.weights) {
          a.theta_out[a.off[s] + pos] = a.mu / (nrm + a.mu);
        } else {
          float alpha = a.alpha_scale * a.theta[a.off[s] + pos];
          fac[s] = nrm > alpha ? alpha / nrm : 1.f;
        }
      }
    }
  }
}

// Dirac block of the dual: z = W + x / 3 per pixel, l2,1 across channels.
template <int LMAX>
__global__ void __launch_bounds__(256) k_fa_dirac(const float* __restrict__ x, float* __restrict__ W,
                                                  const float* __restrict__ theta, float* __restrict__ theta_out,
                                                  int64_t I, int64_t off, int64_t N, int L, float alpha_scale,
                                                  float mu, int weights) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  float z[LMAX];
  float n2 = 0.f;
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    if (l < L) {
      float v = x[(size_t)l * N + p] * (1.f / 3.f) + (weights ? 0.f : W[(size_t)l * I + off + p]);
      z[l] = v;
      n2 = fmaf(v, v, n2);
    }
  }
  float nrm = sqrtf(n2);
  if (weights) {
    theta_out[off + p] = mu / (nrm + mu);
    return;
  }
  float alpha = alpha_scale * theta[off + p];
  float f = nrm > alpha ? alpha / nrm : 1.f;
#pragma unroll
  for (int l = 0; l < LMAX; ++l)
    if (l < L) W[(size_t)l * I + off + p] = z[l] * f;
}

// ------------------------------------------------------------- synthesis
struct SynLevel {
  const float* ll;     // [L][mo1][mo2] synthesised coarser band, or null: LL4 from W
  const float* W;
  int64_t I;
  int64_t off[4];      // d0, d1, d2, LL4
  int mo1, mo2, m1, m2;
};

// Synthesis of one (basis, level) for the 32x32 output tile (r0, c0) of channel l
// into acc (4 values per thread: rows r0 + ty + 8q, column c0 + tx).
__device__ __forceinline__ void fs_tile(const SynLevel& s, int b, int l, int r0, int c0, float* sh, float acc[4]) {
  const int F = 2 * (b + 1);
  const int klo = r0 / 2, clo = c0 / 2;
  const int KN = kTO / 2 + F / 2;                    // coefficient rows / cols touching the tile
  float* tc = sh;                                    // [4][kKnMax][kKnMax+1]: LL, d0, d1, d2
  const int TS = kKnMax * (kKnMax + 1);
  float* lx = sh + 4 * TS;                           // [kTO][kKnMax+1]
  float* hx = lx + kTO * (kKnMax + 1);
  const float third = 1.f / 3.f;
  const float* Wl = s.W + (size_t)l * s.I;
  const float* lll = s.ll ? s.ll + (size_t)l * s.mo1 * s.mo2 : nullptr;
  for (int idx = threadIdx.x; idx < 4 * KN * KN; idx += blockDim.x) {
    int band = idx / (KN * KN), rem = idx % (KN * KN);
    int kr = rem / KN, kc = rem % KN;
    int gk = klo + kr, gc = clo + kc;
    float v = 0.f;
    if (gk < s.mo1 && gc < s.mo2) {
      int64_t pos = (int64_t)gk * s.mo2 + gc;
      if (band == 0) v = lll ? lll[pos] : Wl[s.off[3] + pos] * third;
      else v = Wl[s.off[band - 1] + pos] * third;
    }
    tc[band * TS + kr * (kKnMax + 1) + kc] = v;
  }
  __syncthreads();
  // y synthesis, polyphase: output row i = r0 + il (r0 even), m = il / 2, p = il % 2;
  // a[2m + p] = sum_{q < F/2} f[2q + 1 - p] c[m + q] (no bounds tests: the tile is zero-padded)
  for (int idx = threadIdx.x; idx < kTO * KN; idx += blockDim.x) {
    int il = idx / KN, kc = idx % KN;
    int p = il & 1, m = il >> 1;
    float sl = 0.f, sx = 0.f;
    for (int q = 0; q < F / 2; ++q) {
      int t = 2 * q + 1 - p;
      float h = c_filt.h[b][t], g = c_filt.g[b][t];
      int o = (m + q) * (kKnMax + 1) + kc;
      sl = fmaf(h, tc[o], fmaf(g, tc[2 * TS + o], sl));
      sx = fmaf(h, tc[TS + o], fmaf(g, tc[3 * TS + o], sx));
    }
    lx[il * (kKnMax + 1) + kc] = sl;
    hx[il * (kKnMax + 1) + kc] = sx;
  }
  __syncthreads();
  // x synthesis, polyphase, parity uniform per warp (see fs_pos)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = w & 1, m = lane & 15;
#pragma unroll
  for (int qq = 0; qq < 4; ++qq) {
    int il = (w >> 1) * 2 + (lane >> 4) + 8 * qq;
    float v = 0.f;
    for (int q = 0; q < F / 2; ++q) {
      int t = 2 * q + 1 - p;
      int o = il * (kKnMax + 1) + m + q;
      v = fmaf(c_filt.h[b][t], lx[o], fmaf(c_filt.g[b][t], hx[o], v));
    }
    acc[qq] += v;
  }
  __syncthreads();
}

// Output position of accumulator qq of this thread in the 32x32 tile.
__device__ __forceinline__ void fs_pos(int qq, int& il, int& jc) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  il = (w >> 1) * 2 + (lane >> 4) + 8 * qq;
  jc = 2 * (lane & 15) + (w & 1);
}

__global__ void __launch_bounds__(256) k_fs_level(SynLevel s, int b, float* __restrict__ out) {
  extern __shared__ float sh[];
  const int l = blockIdx.z;
  const int r0 = blockIdx.y * kTO, c0 = blockIdx.x * kTO;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  fs_tile(s, b, l, r0, c0, sh, acc);
  float* ol = out + (size_t)l * s.m1 * s.m2;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int il, jc;
    fs_pos(q, il, jc);
    int r = r0 + il, c = c0 + jc;
    if (r < s.m1 && c < s.m2) ol[(size_t)r * s.m2 + c] = acc[q];
  }
}

struct SynFinal {
  SynLevel lv[8];      // level-1 description of each basis (ll = its synthesised LL1)
  int64_t dirac_off;
  int n1, n2;
  float kappa;
};

__global__ void __launch_bounds__(256) k_fs_final(SynFinal s, float* __restrict__ A) {
  extern __shared__ float sh[];
  const int l = blockIdx.z;
  const int r0 = blockIdx.y * kTO, c0 = blockIdx.x * kTO;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int b = 0; b < 8; ++b) fs_tile(s.lv[b], b, l, r0, c0, sh, acc);
  const size_t N = (size_t)s.n1 * s.n2;
  const float* Wd = s.lv[0].W + (size_t)l * s.lv[0].I + s.dirac_off;
  float* Al = A + (size_t)l * N;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int il, jc;
    fs_pos(q, il, jc);
    int r = r0 + il, c = c0 + jc;
    if (r < s.n1 && c < s.n2) {
      size_t p = (size_t)r * s.n2 + c;
      float v = acc[q] + Wd[p] * (1.f / 3.f);
      Al[p] = fmaf(s.kappa, v, Al[p]);
    }
  }
}

// ------------------------------------------------------------- launchers
static size_t fa_smem(int, int) {
  return (size_t)(2 * kInMax * (kInMax + 1) + 2 * kInMax * (kTK + 1) + 2 * 4 * kTK * kTK) * sizeof(float);
}

static size_t fs_smem() { return (size_t)(4 * kKnMax * (kKnMax + 1) + 2 * kTO * (kKnMax + 1)) * sizeof(float); }

// Fused analysis + l2,1 dual (or weights) of every basis and level, then the
// fused synthesis accumulated into A (dual mode only).
void launch_sara_fast(fhs_ctx* ctx, const Cube& cb, const float* x, float* W, const float* theta, float* A,
                      float* theta_out, bool weights, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fa_prox, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_fs_level, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_fs_final, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    attr = true;
  }
  const SaraLayout& S = cb.sara;
  const int L = cb.L;
  const float alpha_scale = (float)(cb.mu / cb.kappa);
  float* llA = ctx->s.t2;
  float* llB = ctx->s.t3;
  for (int b = 0; b < 8; ++b) {
    const float* in = x;
    for (int j = 1; j <= kLevels; ++j) {
      AnaArgs a;
      a.in = in;
      a.ll_out = (j == kLevels) ? nullptr : ((j & 1) ? llA : llB);
      a.W = W;
      a.theta = theta;
      a.theta_out = theta_out;
      a.I = S.I;
      a.off[0] = S.off[b][j][0]; a.off[1] = S.off[b][j][1]; a.off[2] = S.off[b][j][2];
      a.off[3] = S.off[b][kLevels][3];
      a.L = L;
      a.m1 = S.rows[b][j - 1]; a.m2 = S.cols[b][j - 1];
      a.mo1 = S.rows[b][j]; a.mo2 = S.cols[b][j];
      a.basis = b;
      a.nsub = (j == kLevels) ? 4 : 3;
      a.alpha_scale = alpha_scale;
      a.mu = (float)cb.mu;
      a.weights = weights ? 1 : 0;
      dim3 g((a.mo2 + kTK - 1) / kTK, (a.mo1 + kTK - 1) / kTK);
      k_fa_prox<<<g, 256, fa_smem(L, a.nsub), st>>>(a);
      note_launches(1);
      in = a.ll_out;
    }
  }
  const int64_t N = (int64_t)cb.n1 * cb.n2;
  {
    const unsigned g = (unsigned)((N + 255) / 256);
    const int wm = weights ? 1 : 0;
    if (L <= 16)
      k_fa_dirac<16><<<g, 256, 0, st>>>(x, W, theta, theta_out, S.I, S.dirac_off, N, L, alpha_scale, (float)cb.mu, wm);
    else if (L <= 32)
      k_fa_dirac<32><<<g, 256, 0, st>>>(x, W, theta, theta_out, S.I, S.dirac_off, N, L, alpha_scale, (float)cb.mu, wm);
    else
      k_fa_dirac<64><<<g, 256, 0, st>>>(x, W, theta, theta_out, S.I, S.dirac_off, N, L, alpha_scale, (float)cb.mu, wm);
    note_launches(1);
  }
  if (weights) return;
  // synthesis: levels 4..2 per basis into its LL1 slot, then level 1 of all bases + Dirac into A
  SynFinal fin;
  float* slots = ctx->s.ll1;
  for (int b = 0; b < 8; ++b) {
    const float* ll = nullptr;
    for (int j = kLevels; j >= 2; --j) {
      SynLevel s;
      s.ll = ll;
      s.W = W;
      s.I = S.I;
      s.off[0] = S.off[b][j][0]; s.off[1] = S.off[b][j][1]; s.off[2] = S.off[b][j][2];
      s.off[3] = S.off[b][kLevels][3];
      s.mo1 = S.rows[b][j]; s.mo2 = S.cols[b][j];
      s.m1 = S.rows[b][j - 1]; s.m2 = S.cols[b][j - 1];
      float* out = (j == 2) ? slots + ctx->s.ll1_off[b] : ((j & 1) ? llA : llB);
      dim3 g((s.m2 + kTO - 1) / kTO, (s.m1 + kTO - 1) / kTO, L);
      k_fs_level<<<g, 256, fs_smem(), st>>>(s, b, out);
      note_launches(1);
      ll = out;
    }
    SynLevel& f = fin.lv[b];
    f.ll = slots + ctx->s.ll1_off[b];
    f.W = W;
    f.I = S.I;
    f.off[0] = S.off[b][1][0]; f.off[1] = S.off[b][1][1]; f.off[2] = S.off[b][1][2];
    f.off[3] = S.off[b][kLevels][3];
    f.mo1 = S.rows[b][1]; f.mo2 = S.cols[b][1];
    f.m1 = cb.n1; f.m2 = cb.n2;
  }
  fin.dirac_off = S.dirac_off;
  fin.n1 = cb.n1;
  fin.n2 = cb.n2;
  fin.kappa = (float)cb.kappa;
  dim3 g((cb.n2 + kTO - 1) / kTO, (cb.n1 + kTO - 1) / kTO, L);
  k_fs_final<<<g, 256, fs_smem(), st>>>(fin, A);
  note_launches(1);
}

}  // namespace fhs

namespace fhs {
bool sara_fast_supported(const Cube&) { return true; }
}  // namespace fhs
