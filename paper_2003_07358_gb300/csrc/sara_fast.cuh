// Fast SARA l2,1 dual (Algorithm 2 W update, Table 2 row 3) on GB300, included
// at the end of sara.cu (it uses that file's c_filt filter table).
//
//   k_ana1_all  : level 1 of all eight bases for a 32x32 coefficient tile of one
//                 channel from one staged db8 input window.
//   k_ana2_all  : one level (2..4) of every basis in one launch (k_ana2_one: one
//                 basis, for levels whose every basis fills the GPU alone), a 32x32
//                 coefficient tile of one channel per CTA: the input tile with
//                 its filter halo is staged in shared memory, filtered along x
//                 then y with register blocking (each thread produces 4 outputs
//                 from one window of F + 6 loaded values); writes the LL band for
//                 the next level and the detail bands (/3) to the coefficient buffer.
//   k_prox2     : the l2,1 dual over every coefficient of the sub-cube in one
//                 streaming pass (Dirac block read straight from x):
//                 W <- z min(1, alpha_i / ||z_i||), z = W + Psi^dagger x
//                 (weights mode: theta_i = mu / (||Psi^dagger x||_i + mu)).
//   k_syn2_all  : one synthesis level (4 -> 3, 3 -> 2, 2 -> 1) of every basis in
//                 one launch (k_syn2_one: one basis, as above), a 32x32 output
//                 tile of one channel per CTA,
//                 polyphase (even outputs take the odd taps and vice versa),
//                 register-blocked.
//   k_synfin    : level 1 of all eight bases and the Dirac block for a 32x32
//                 output tile, accumulated in registers; A += kappa * result.
// Same conventions as the plain kernels (zero-padded full convolution, odd
// phase, coefficients scaled by 1/3).

namespace fhs {

constexpr int kT2 = 32;                              // tile side (coefficients or outputs)
constexpr int kIn2 = 2 * kT2 + kMaxFilt - 2;         // 78: input rows/cols of an analysis tile
constexpr int kKn2 = kT2 / 2 + kMaxFilt / 2;         // 24: coefficient rows/cols of a synthesis tile

// Filter taps of basis F/2 - 1, read straight from the constant bank: with the tap
// index known at compile time (unrolled loops) every FMA takes the tap as a
// constant-bank operand, no register and no load.
template <int F>
struct FTaps {
  struct H { __device__ __forceinline__ float operator[](int t) const { return c_filt.h[F / 2 - 1][t]; } };
  struct G { __device__ __forceinline__ float operator[](int t) const { return c_filt.g[F / 2 - 1][t]; } };
  H h;
  G g;
  __device__ __forceinline__ void load() {}
};

// ------------------------------------------------------------- async copies
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ------------------------------------------------------------- analysis
// x then y pass of one (basis, level) for the coefficient tile (k0, c0) of one channel.
// Staged input element (r, c) of this filter's window is tin[r + o][c + o] (o > 0 when
// the window sits inside a wider one staged for a longer filter).  Writes the three
// detail bands (/3) to cl + off_d and the LL band to llo (next level's input) or, when
// llo is null, to cl + off_ll (/3).  Starts with a barrier so that tlx / thx may be
// reused from a previous call.
template <int F>
__device__ __forceinline__ void ana_tile(const float (*tin)[kIn2 + 1], int o, float (*tlx)[kT2 + 1],
                                         float (*thx)[kT2 + 1], float* __restrict__ cl, float* __restrict__ llo,
                                         int64_t off0, int64_t off1, int64_t off2, int64_t off_ll, int k0, int c0,
                                         int mo1, int mo2) {
  constexpr int IN = 2 * kT2 + F - 2;
  constexpr int WIN = F + 6;                          // window of a 4-output block
  FTaps<F> f;
  __syncthreads();
  // x: lx[r][kc] = sum_t h[t] tin[r][2 kc + F - 1 - t], 4 consecutive kc per item
  for (int item = threadIdx.x; item < IN * 8; item += 256) {
    const int r = item >> 3, kc0 = (item & 7) * 4;
    float v[WIN];
#pragma unroll
    for (int u = 0; u < WIN; ++u) v[u] = tin[r + o][2 * kc0 + u + o];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float sl = 0.f, sh = 0.f;
#pragma unroll
      for (int t = 0; t < F; ++t) {
        sl = fmaf(f.h[t], v[2 * m + F - 1 - t], sl);
        sh = fmaf(f.g[t], v[2 * m + F - 1 - t], sh);
      }
      tlx[r][kc0 + m] = sl;
      thx[r][kc0 + m] = sh;
    }
  }
  __syncthreads();
  // y: 4 consecutive coefficient rows per thread, all four bands
  const int kc = threadIdx.x & 31, kr0 = (threadIdx.x >> 5) * 4;
  float a[WIN], b[WIN];
#pragma unroll
  for (int u = 0; u < WIN; ++u) {
    a[u] = tlx[2 * kr0 + u][kc];
    b[u] = thx[2 * kr0 + u][kc];
  }
  const float third = 1.f / 3.f;
  const int gc = c0 + kc;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float ll = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
    for (int t = 0; t < F; ++t) {
      const float va = a[2 * m + F - 1 - t], vb = b[2 * m + F - 1 - t];
      ll = fmaf(f.h[t], va, ll);
      d1 = fmaf(f.g[t], va, d1);
      d0 = fmaf(f.h[t], vb, d0);
      d2 = fmaf(f.g[t], vb, d2);
    }
    const int gk = k0 + kr0 + m;
    if (gk < mo1 && gc < mo2) {
      const int64_t pos = (int64_t)gk * mo2 + gc;
      cl[off0 + pos] = d0 * third;
      cl[off1 + pos] = d1 * third;
      cl[off2 + pos] = d2 * third;
      if (llo) llo[pos] = ll;
      else cl[off_ll + pos] = ll * third;
    }
  }
}

// Stage rows [r0, r0 + IN) x columns [c0, c0 + IN) of one channel image (zero outside)
// with asynchronous copies, so that all of a thread's loads are in flight at once:
// lane = column, warp = row.
template <int IN>
__device__ __forceinline__ void ana_stage(float (*tin)[kIn2 + 1], const float* __restrict__ inl, int r0, int c0,
                                          int m1, int m2) {
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;
#pragma unroll
  for (int cj = 0; cj < (IN + 31) / 32; ++cj) {
    const int c = lane + 32 * cj, gc = c0 + c;
    if (c >= IN) continue;
    const bool vc = gc >= 0 && gc < m2;
#pragma unroll 4
    for (int r = wrp; r < IN; r += 8) {
      const int gr = r0 + r;
      const bool v = vc && gr >= 0 && gr < m1;
      cp_async4(&tin[r][c], v ? inl + (size_t)gr * m2 + gc : inl, v);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
}

// One level (2, 3 or 4) of every basis in one launch: blockIdx.x runs over the
// coefficient tiles of all bases (longest filters first), blockIdx.y over channels.
// The bases of a level are independent (each reads its own coarser LL band), so one
// launch per level replaces eight and the small levels fill the GPU together.
struct Ana2Basis {
  const float* in;     // LL band of the previous level [L][m1][m2]
  float* ll_out;       // LL band of this level [L][mo1][mo2], or null: LL4 into coef (/3)
  int64_t off[3];      // detail bands in the coefficient buffer
  int64_t off_ll;      // LL4 (last level only)
  int m1, m2, mo1, mo2;
  int tiles_x;         // coefficient tiles along a row of this basis
  int tile0;           // first linear tile of this basis
  int F;               // filter length
};
struct Ana2All {
  Ana2Basis b[8];
  int nb;
};

template <int F>
__device__ __forceinline__ void ana2_body(const Ana2Basis& B, int tile, int l, float* __restrict__ coef, int64_t I,
                                          float (*tin)[kIn2 + 1], float (*tlx)[kT2 + 1], float (*thx)[kT2 + 1]) {
  const int ty = tile / B.tiles_x, tx = tile - ty * B.tiles_x;
  const int k0 = ty * kT2, c0 = tx * kT2;
  ana_stage<2 * kT2 + F - 2>(tin, B.in + (size_t)l * B.m1 * B.m2, 2 * k0 + 2 - F, 2 * c0 + 2 - F, B.m1, B.m2);
  ana_tile<F>(tin, 0, tlx, thx, coef + (size_t)l * I, B.ll_out ? B.ll_out + (size_t)l * B.mo1 * B.mo2 : nullptr,
              B.off[0], B.off[1], B.off[2], B.off_ll, k0, c0, B.mo1, B.mo2);
}

__global__ void __launch_bounds__(256, 4) k_ana2_all(const Ana2All a, float* __restrict__ coef, int64_t I) {
  __shared__ float tin[kIn2][kIn2 + 1];
  __shared__ float tlx[kIn2][kT2 + 1];
  __shared__ float thx[kIn2][kT2 + 1];
  const int t = blockIdx.x, l = blockIdx.y;
  int bi = 0;
#pragma unroll 1
  for (int k = 1; k < a.nb; ++k)
    if (t >= a.b[k].tile0) bi = k;
  const Ana2Basis& B = a.b[bi];
  const int tile = t - B.tile0;
  switch (B.F) {
    case 2: ana2_body<2>(B, tile, l, coef, I, tin, tlx, thx); break;
    case 4: ana2_body<4>(B, tile, l, coef, I, tin, tlx, thx); break;
    case 6: ana2_body<6>(B, tile, l, coef, I, tin, tlx, thx); break;
    case 8: ana2_body<8>(B, tile, l, coef, I, tin, tlx, thx); break;
    case 10: ana2_body<10>(B, tile, l, coef, I, tin, tlx, thx); break;
    case 12: ana2_body<12>(B, tile, l, coef, I, tin, tlx, thx); break;
    case 14: ana2_body<14>(B, tile, l, coef, I, tin, tlx, thx); break;
    default: ana2_body<16>(B, tile, l, coef, I, tin, tlx, thx); break;
  }
}

// One basis of a level on its own (tiles along blockIdx.x, channels along blockIdx.y):
// used when every basis's tiles fill the GPU by themselves, where the per-filter
// register allocation keeps more CTAs per SM than the merged kernel.
template <int F>
__global__ void __launch_bounds__(256) k_ana2_one(const Ana2Basis B, float* __restrict__ coef, int64_t I) {
  __shared__ float tin[kIn2][kIn2 + 1];
  __shared__ float tlx[kIn2][kT2 + 1];
  __shared__ float thx[kIn2][kT2 + 1];
  ana2_body<F>(B, blockIdx.x, blockIdx.y, coef, I, tin, tlx, thx);
}

// Level 1 of all eight bases for a 32x32 coefficient tile of one channel: the input
// window of the longest filter (db8, 78 x 78) is staged once and each basis reads its
// own window inside it (offset 16 - F), instead of one launch and one staging per
// basis.  The LL1 band of basis b goes to its slot in the LL1 buffer (the input of
// its level 2).
struct Ana1 {
  int64_t off[8][3];   // level-1 detail-band offsets of each basis
  int mo1[8], mo2[8];  // level-1 coefficient rows / columns of each basis
  int64_t ll_off[8];   // LL1 slot of each basis in the LL1 buffer (units of floats)
};

template <int F>
__device__ __forceinline__ void ana1_basis(const Ana1& a, const float (*tin)[kIn2 + 1], float (*tlx)[kT2 + 1],
                                           float (*thx)[kT2 + 1], float* cl, float* ll1, int l, int k0, int c0) {
  constexpr int b = F / 2 - 1;
  ana_tile<F>(tin, kMaxFilt - F, tlx, thx, cl, ll1 + a.ll_off[b] + (size_t)l * a.mo1[b] * a.mo2[b], a.off[b][0],
              a.off[b][1], a.off[b][2], 0, k0, c0, a.mo1[b], a.mo2[b]);
}

__global__ void __launch_bounds__(256) k_ana1_all(const float* __restrict__ x, float* __restrict__ coef,
                                                  float* __restrict__ ll1, Ana1 a, int64_t I, int n1, int n2) {
  __shared__ float tin[kIn2][kIn2 + 1];
  __shared__ float tlx[kIn2][kT2 + 1];
  __shared__ float thx[kIn2][kT2 + 1];
  const int l = blockIdx.z;
  const int k0 = blockIdx.y * kT2, c0 = blockIdx.x * kT2;
  ana_stage<kIn2>(tin, x + (size_t)l * n1 * n2, 2 * k0 + 2 - kMaxFilt, 2 * c0 + 2 - kMaxFilt, n1, n2);
  float* cl = coef + (size_t)l * I;
  ana1_basis<2>(a, tin, tlx, thx, cl, ll1, l, k0, c0);
  ana1_basis<4>(a, tin, tlx, thx, cl, ll1, l, k0, c0);
  ana1_basis<6>(a, tin, tlx, thx, cl, ll1, l, k0, c0);
  ana1_basis<8>(a, tin, tlx, thx, cl, ll1, l, k0, c0);
  ana1_basis<10>(a, tin, tlx, thx, cl, ll1, l, k0, c0);
  ana1_basis<12>(a, tin, tlx, thx, cl, ll1, l, k0, c0);
  ana1_basis<14>(a, tin, tlx, thx, cl, ll1, l, k0, c0);
  ana1_basis<16>(a, tin, tlx, thx, cl, ll1, l, k0, c0);
}

// ---------------------------------------------------------- l2,1 dual
// One coefficient per thread; z of every channel is parked in shared memory
// (L x 256 floats) instead of registers, so the kernel runs at full occupancy
// with 2L independent loads in flight per thread.
__global__ void __launch_bounds__(256, 4) k_prox2(float* __restrict__ W, const float* __restrict__ coef,
                                               const float* __restrict__ x, const float* __restrict__ theta,
                                               float* __restrict__ theta_out, int64_t I, int64_t dirac_off, int64_t N,
                                               int L, float alpha_scale, float mu, int weights) {
  extern __shared__ float zs[];                         // [L][256]
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I; i += (int64_t)gridDim.x * blockDim.x) {
    const bool dirac = i >= dirac_off;
    float n2 = 0.f;
#pragma unroll 16
    for (int l = 0; l < L; ++l) {
      float c = dirac ? x[(size_t)l * N + (i - dirac_off)] * (1.f / 3.f) : coef[(size_t)l * I + i];
      float v = weights ? c : W[(size_t)l * I + i] + c;
      zs[l * 256 + threadIdx.x] = v;
      n2 = fmaf(v, v, n2);
    }
    const float nrm = sqrtf(n2);
    if (weights) {
      theta_out[i] = mu / (nrm + mu);
      continue;
    }
    const float alpha = alpha_scale * theta[i];
    const float fct = nrm > alpha ? alpha / nrm : 1.f;
#pragma unroll 16
    for (int l = 0; l < L; ++l) W[(size_t)l * I + i] = zs[l * 256 + threadIdx.x] * fct;
  }
}

// ------------------------------------------------------------ synthesis
struct Syn2 {
  const float* ll;     // synthesised coarser band [L][mo1][mo2], or null: LL4 from W (/3)
  const float* W;
  int64_t I;
  int64_t off[4];      // d0, d1, d2, LL4
  int mo1, mo2, m1, m2;
};

// Staging of the four coefficient bands (LL, d0, d1, d2; raw values, zero outside the
// level) of the synthesis tile (r0, c0) of channel l: window rows [r0/2, r0/2 + KN),
// columns [c0/2, c0/2 + KN), KN = 16 + F/2, by 4-byte asynchronous copies (lane =
// column, warp = row), band b at b kTS2e, rows at stride kKn2 + 1.
constexpr int kTS2e = kKn2 * (kKn2 + 1);             // 600

template <int F>
__device__ __forceinline__ void syn2_stage_e(const Syn2& s, int l, int r0, int c0, float* tc) {
  constexpr int KN = kT2 / 2 + F / 2;
  static_assert(KN <= 32, "one warp spans a staged row");
  const int kc = threadIdx.x & 31, kr0 = threadIdx.x >> 5;   // lane = column, warp = row (step 8)
  if (kc < KN) {
    const int klo = r0 / 2, gc = c0 / 2 + kc;
    // rows kr0, kr0 + 8, ... of this thread that lie inside the band (none if the column is out)
    const int nrows = gc < s.mo2 ? min((KN - kr0 + 7) / 8, max(0, (s.mo1 - klo - kr0 + 7) / 8)) : 0;
    const float* Wl = s.W + (size_t)l * s.I;
    const float* b0 = s.ll ? s.ll + (size_t)l * s.mo1 * s.mo2 : Wl + s.off[3];
    const int64_t start = (int64_t)(klo + kr0) * s.mo2 + gc, step = 8 * (int64_t)s.mo2;
    const float* bp[4] = {b0 + start, Wl + s.off[0] + start, Wl + s.off[1] + start, Wl + s.off[2] + start};
    float* dst = tc + kr0 * (kKn2 + 1) + kc;
#pragma unroll
    for (int band = 0; band < 4; ++band) {
      const float* src = bp[band];
#pragma unroll
      for (int j = 0; j < (KN + 7) / 8; ++j) {
        if (kr0 + 8 * j < KN) {
          const bool v = j < nrows;
          cp_async4(dst + band * kTS2e + 8 * j * (kKn2 + 1), v ? src : b0, v);
        }
        src += step;
      }
    }
  }
  cp_async_commit();
}

// Synthesis of one staged (basis, level) tile, added to acc[4]: outputs at row
// il = threadIdx.x >> 3, columns 4 * (threadIdx.x & 7) + q.  tl, t0, t1, t2: window
// element (0, 0) of the LL, d0, d1, d2 bands, rows at stride R.  Coefficients carry the
// 1/3 of the dictionary except a synthesised LL band (ll_scale = 1).
template <int F, int R>
__device__ __forceinline__ void syn2_compute(const float* tl, const float* t0, const float* t1, const float* t2,
                                             float* lx, float* hx, float ll_scale, float acc[4]) {
  constexpr int KN = kT2 / 2 + F / 2;
  constexpr int WIN = F / 2 + 1;
  FTaps<F> f;
  f.load();
  const float third = 1.f / 3.f;
  for (int item = threadIdx.x; item < KN * 8; item += 256) {
    const int kc = item % KN, mg = (item / KN) * 2;
    float vl[WIN + 1], v1[WIN + 1], v0[WIN + 1], v2[WIN + 1];
#pragma unroll
    for (int u = 0; u <= WIN; ++u) {
      const int o = (mg + u) * R + kc;
      vl[u] = tl[o];
      v0[u] = t0[o];
      v1[u] = t1[o];
      v2[u] = t2[o];
    }
    // raw coefficients; the dictionary's 1/3 (and ll_scale) applied once per output
#pragma unroll
    for (int mm = 0; mm < 2; ++mm) {
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float slh = 0.f, slg = 0.f, sxh = 0.f, sxg = 0.f;
#pragma unroll
        for (int q = 0; q < F / 2; ++q) {
          const float hh = f.h[2 * q + 1 - p], gg = f.g[2 * q + 1 - p];
          slh = fmaf(hh, vl[mm + q], slh);
          slg = fmaf(gg, v1[mm + q], slg);
          sxh = fmaf(hh, v0[mm + q], sxh);
          sxg = fmaf(gg, v2[mm + q], sxg);
        }
        const int il = 2 * (mg + mm) + p;
        lx[il * (kKn2 + 1) + kc] = fmaf(ll_scale, slh, third * slg);
        hx[il * (kKn2 + 1) + kc] = third * (sxh + sxg);
      }
    }
  }
  __syncthreads();
  {
    const int il = threadIdx.x >> 3, g4 = threadIdx.x & 7;
    const int mg = 2 * g4;
    float a[WIN + 1], b[WIN + 1];
#pragma unroll
    for (int u = 0; u <= WIN; ++u) {
      a[u] = lx[il * (kKn2 + 1) + mg + u];
      b[u] = hx[il * (kKn2 + 1) + mg + u];
    }
#pragma unroll
    for (int mm = 0; mm < 2; ++mm) {
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < F / 2; ++q)
          v = fmaf(f.h[2 * q + 1 - p], a[mm + q], fmaf(f.g[2 * q + 1 - p], b[mm + q], v));
        acc[2 * mm + p] += v;
      }
    }
  }
  __syncthreads();
}

// Staging and compute of basis b = F/2 - 1 (runtime b, compile-time F).
__device__ __forceinline__ void syn2_stage_any(int b, const Syn2& s, int l, int r0, int c0, float* tc) {
  switch (b) {
    case 0: syn2_stage_e<2>(s, l, r0, c0, tc); break;
    case 1: syn2_stage_e<4>(s, l, r0, c0, tc); break;
    case 2: syn2_stage_e<6>(s, l, r0, c0, tc); break;
    case 3: syn2_stage_e<8>(s, l, r0, c0, tc); break;
    case 4: syn2_stage_e<10>(s, l, r0, c0, tc); break;
    case 5: syn2_stage_e<12>(s, l, r0, c0, tc); break;
    case 6: syn2_stage_e<14>(s, l, r0, c0, tc); break;
    default: syn2_stage_e<16>(s, l, r0, c0, tc); break;
  }
}

template <int F>
__device__ __forceinline__ void syn2_compute_e(const float* tc, float* lx, float* hx, float lls, float acc[4]) {
  syn2_compute<F, kKn2 + 1>(tc, tc + kTS2e, tc + 2 * kTS2e, tc + 3 * kTS2e, lx, hx, lls, acc);
}

__device__ __forceinline__ void syn2_compute_any(int b, const float* tc, float* lx, float* hx, float lls,
                                                 float acc[4]) {
  switch (b) {
    case 0: syn2_compute_e<2>(tc, lx, hx, lls, acc); break;
    case 1: syn2_compute_e<4>(tc, lx, hx, lls, acc); break;
    case 2: syn2_compute_e<6>(tc, lx, hx, lls, acc); break;
    case 3: syn2_compute_e<8>(tc, lx, hx, lls, acc); break;
    case 4: syn2_compute_e<10>(tc, lx, hx, lls, acc); break;
    case 5: syn2_compute_e<12>(tc, lx, hx, lls, acc); break;
    case 6: syn2_compute_e<14>(tc, lx, hx, lls, acc); break;
    default: syn2_compute_e<16>(tc, lx, hx, lls, acc); break;
  }
}

// One synthesis level (4 -> 3, 3 -> 2 or 2 -> 1) of every basis in one launch, tiles of
// all bases along blockIdx.x (longest filters first), channels along blockIdx.y.
struct Syn2All {
  Syn2 s[8];
  float* out[8];       // synthesised LL band of the finer level [L][m1][m2]
  int tiles_x[8], tile0[8], F[8];
  int nb;
};

template <int F>
__device__ __forceinline__ void syn2_body(const Syn2& s, float* __restrict__ out, int tiles_x, int tile, int l,
                                          float* sh) {
  const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
  const int r0 = ty * kT2, c0 = tx * kT2;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  syn2_stage_e<F>(s, l, r0, c0, sh);
  cp_async_wait<0>();
  __syncthreads();
  syn2_compute<F, kKn2 + 1>(sh, sh + kTS2e, sh + 2 * kTS2e, sh + 3 * kTS2e, sh + 4 * kTS2e,
                            sh + 4 * kTS2e + kT2 * (kKn2 + 1), s.ll ? 1.f : 1.f / 3.f, acc);
  const int il = threadIdx.x >> 3, jc0 = 4 * (threadIdx.x & 7);
  const int r = r0 + il;
  if (r >= s.m1) return;
  float* ol = out + (size_t)l * s.m1 * s.m2 + (size_t)r * s.m2;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (c0 + jc0 + q < s.m2) ol[c0 + jc0 + q] = acc[q];
}

__global__ void __launch_bounds__(256) k_syn2_all(const Syn2All a) {
  __shared__ float sh[4 * kTS2e + 2 * kT2 * (kKn2 + 1)];
  const int t = blockIdx.x, l = blockIdx.y;
  int bi = 0;
#pragma unroll 1
  for (int k = 1; k < a.nb; ++k)
    if (t >= a.tile0[k]) bi = k;
  const int tile = t - a.tile0[bi];
  switch (a.F[bi]) {
    case 2: syn2_body<2>(a.s[bi], a.out[bi], a.tiles_x[bi], tile, l, sh); break;
    case 4: syn2_body<4>(a.s[bi], a.out[bi], a.tiles_x[bi], tile, l, sh); break;
    case 6: syn2_body<6>(a.s[bi], a.out[bi], a.tiles_x[bi], tile, l, sh); break;
    case 8: syn2_body<8>(a.s[bi], a.out[bi], a.tiles_x[bi], tile, l, sh); break;
    case 10: syn2_body<10>(a.s[bi], a.out[bi], a.tiles_x[bi], tile, l, sh); break;
    case 12: syn2_body<12>(a.s[bi], a.out[bi], a.tiles_x[bi], tile, l, sh); break;
    case 14: syn2_body<14>(a.s[bi], a.out[bi], a.tiles_x[bi], tile, l, sh); break;
    default: syn2_body<16>(a.s[bi], a.out[bi], a.tiles_x[bi], tile, l, sh); break;
  }
}

template <int F>
__global__ void __launch_bounds__(256) k_syn2_one(const Syn2 s, float* __restrict__ out, int tiles_x) {
  __shared__ float sh[4 * kTS2e + 2 * kT2 * (kKn2 + 1)];
  syn2_body<F>(s, out, tiles_x, blockIdx.x, blockIdx.y, sh);
}

// A level runs as one launch per basis when the smallest basis alone has at least two
// waves of CTAs (four per SM), else as one merged launch over all bases.
static bool sara_level_per_basis(const int* tiles, int L) {
  int64_t mn = INT64_MAX;
  for (int k = 0; k < 8; ++k) mn = std::min<int64_t>(mn, (int64_t)tiles[k] * L);
  return mn >= 2LL * 4 * num_sms();
}

#define FHS_F_SWITCH(F, KERNEL, GRID, ...)                               \
  switch (F) {                                                           \
    case 2: KERNEL<2><<<GRID, 256, 0, st>>>(__VA_ARGS__); break;         \
    case 4: KERNEL<4><<<GRID, 256, 0, st>>>(__VA_ARGS__); break;         \
    case 6: KERNEL<6><<<GRID, 256, 0, st>>>(__VA_ARGS__); break;         \
    case 8: KERNEL<8><<<GRID, 256, 0, st>>>(__VA_ARGS__); break;         \
    case 10: KERNEL<10><<<GRID, 256, 0, st>>>(__VA_ARGS__); break;       \
    case 12: KERNEL<12><<<GRID, 256, 0, st>>>(__VA_ARGS__); break;       \
    case 14: KERNEL<14><<<GRID, 256, 0, st>>>(__VA_ARGS__); break;       \
    default: KERNEL<16><<<GRID, 256, 0, st>>>(__VA_ARGS__); break;       \
  }

struct SynFin2 {
  Syn2 lv[8];          // level-1 description of each basis (ll = its synthesised LL1)
  int64_t dirac_off;
  int n1, n2;
  float kappa;
  int vec4;            // A, W, the Dirac block and n2 allow 16-byte accesses
};

// Level 1 of all bases: the tiles of basis b + 1 are staged (cp.async) while basis b
// is computed.
__global__ void __launch_bounds__(256, 3) k_synfin(SynFin2 s, float* __restrict__ A) {
  __shared__ float sh[2 * 4 * kTS2e + 2 * kT2 * (kKn2 + 1)];
  float* lx = sh + 8 * kTS2e;
  float* hx = lx + kT2 * (kKn2 + 1);
  const int l = blockIdx.z;
  const int r0 = blockIdx.y * kT2, c0 = blockIdx.x * kT2;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  syn2_stage_any(0, s.lv[0], l, r0, c0, sh);
#pragma unroll 1
  for (int b = 0; b < 8; ++b) {
    if (b + 1 < 8) {
      syn2_stage_any(b + 1, s.lv[b + 1], l, r0, c0, sh + ((b + 1) & 1) * 4 * kTS2e);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    syn2_compute_any(b, sh + (b & 1) * 4 * kTS2e, lx, hx, 1.f, acc);
  }
  const int il = threadIdx.x >> 3, jc0 = 4 * (threadIdx.x & 7);
  const int r = r0 + il;
  if (r >= s.n1) return;
  const size_t N = (size_t)s.n1 * s.n2;
  const size_t drow = (size_t)l * s.lv[0].I + s.dirac_off + (size_t)r * s.n2;
  const float* Wd = s.lv[0].W + drow;
  float* Al = A + (size_t)l * N + (size_t)r * s.n2;
  const int c = c0 + jc0;
  // four consecutive outputs: one 16-byte read-modify-write of A when the row and the
  // Dirac block allow it
  if (s.vec4 && c + 3 < s.n2) {
    const float4 wd = *reinterpret_cast<const float4*>(Wd + c);
    float4 a = *reinterpret_cast<const float4*>(Al + c);
    a.x = fmaf(s.kappa, acc[0] + wd.x * (1.f / 3.f), a.x);
    a.y = fmaf(s.kappa, acc[1] + wd.y * (1.f / 3.f), a.y);
    a.z = fmaf(s.kappa, acc[2] + wd.z * (1.f / 3.f), a.z);
    a.w = fmaf(s.kappa, acc[3] + wd.w * (1.f / 3.f), a.w);
    *reinterpret_cast<float4*>(Al + c) = a;
    return;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (c + q < s.n2) Al[c + q] = fmaf(s.kappa, acc[q] + Wd[c + q] * (1.f / 3.f), Al[c + q]);
}

// ------------------------------------------------------------- launchers
// Analysis of every basis and level into the coefficient buffer, the l2,1 dual (or
// weights), then (dual mode) the synthesis accumulated into A.
void launch_sara_fast(fhs_ctx* ctx, const Cube& cb, const float* x, float* W, const float* theta, float* A,
                      float* theta_out, bool weights, cudaStream_t st) {
  const SaraLayout& S = cb.sara;
  const int L = cb.L;
  float* coef = ctx->s.coef;
  // LL1, LL2 and LL3 slots of the eight bases (also used by the synthesis below)
  {
    int64_t o1 = 0, o2 = 0, o3 = 0;
    for (int b = 0; b < 8; ++b) {
      ctx->s.ll1_off[b] = o1;
      ctx->s.ll2_off[b] = o2;
      ctx->s.ll3_off[b] = o3;
      o1 += (int64_t)L * S.rows[b][1] * S.cols[b][1];
      o2 += (int64_t)L * S.rows[b][2] * S.cols[b][2];
      o3 += (int64_t)L * S.rows[b][3] * S.cols[b][3];
    }
  }
  // level 1 of every basis in one launch (grid over the longest filter's coefficients)
  {
    Ana1 a;
    for (int b = 0; b < 8; ++b) {
      for (int k = 0; k < 3; ++k) a.off[b][k] = S.off[b][1][k];
      a.mo1[b] = S.rows[b][1];
      a.mo2[b] = S.cols[b][1];
      a.ll_off[b] = ctx->s.ll1_off[b];
    }
    int r = 0, c = 0;
    for (int b = 0; b < 8; ++b) { r = std::max(r, S.rows[b][1]); c = std::max(c, S.cols[b][1]); }
    dim3 g((c + kT2 - 1) / kT2, (r + kT2 - 1) / kT2, L);
    k_ana1_all<<<g, 256, 0, st>>>(x, coef, ctx->s.ll1, a, S.I, cb.n1, cb.n2);
    note_launches(1);
  }
  // levels 2..4: one launch per level over the tiles of every basis (longest filters
  // first); LL2 and LL3 of each basis in its own slot of s.ll2 / s.ll3
  for (int j = 2; j <= kLevels; ++j) {
    Ana2All a;
    a.nb = 8;
    int t0 = 0;
    for (int k = 0; k < 8; ++k) {
      const int b = 7 - k;
      Ana2Basis& B = a.b[k];
      B.in = (j == 2) ? ctx->s.ll1 + ctx->s.ll1_off[b] : (j == 3) ? ctx->s.ll2 + ctx->s.ll2_off[b]
                                                                  : ctx->s.ll3 + ctx->s.ll3_off[b];
      B.ll_out = (j == 2) ? ctx->s.ll2 + ctx->s.ll2_off[b] : (j == 3) ? ctx->s.ll3 + ctx->s.ll3_off[b] : nullptr;
      for (int q = 0; q < 3; ++q) B.off[q] = S.off[b][j][q];
      B.off_ll = S.off[b][kLevels][3];
      B.m1 = S.rows[b][j - 1]; B.m2 = S.cols[b][j - 1];
      B.mo1 = S.rows[b][j]; B.mo2 = S.cols[b][j];
      B.tiles_x = (B.mo2 + kT2 - 1) / kT2;
      B.tile0 = t0;
      B.F = 2 * (b + 1);
      t0 += B.tiles_x * ((B.mo1 + kT2 - 1) / kT2);
    }
    int tiles[8];
    for (int k = 0; k < 8; ++k) tiles[k] = (k + 1 < 8 ? a.b[k + 1].tile0 : t0) - a.b[k].tile0;
    if (sara_level_per_basis(tiles, L)) {
      for (int k = 0; k < 8; ++k) {
        FHS_F_SWITCH(a.b[k].F, k_ana2_one, dim3(tiles[k], L), a.b[k], coef, S.I);
      }
      note_launches(8);
    } else {
      k_ana2_all<<<dim3(t0, L), 256, 0, st>>>(a, coef, S.I);
      note_launches(1);
    }
  }
  {
    const int64_t N = (int64_t)cb.n1 * cb.n2;
    const unsigned g = (unsigned)std::min<int64_t>((S.I + 255) / 256, (int64_t)num_sms() * cb.prox_cps);
    const float as = (float)(cb.mu / cb.kappa), mu = (float)cb.mu;
    const int wm = weights ? 1 : 0;
    const size_t smem = (size_t)L * 256 * sizeof(float);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_prox2, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxL * 256 * (int)sizeof(float));
      attr = true;
    }
    k_prox2<<<g, 256, smem, st>>>(W, coef, x, theta, theta_out, S.I, S.dirac_off, N, L, as, mu, wm);
    note_launches(1);
  }
  if (weights) return;
  SynFin2 fin;
  float* slots = ctx->s.ll1;
  // levels 4 -> 2: one launch per level over the tiles of every basis; the synthesised
  // LL3, LL2 and LL1 bands reuse the analysis slots (s.ll3, s.ll2, s.ll1)
  for (int j = kLevels; j >= 2; --j) {
    Syn2All a;
    a.nb = 8;
    int t0 = 0;
    for (int k = 0; k < 8; ++k) {
      const int b = 7 - k;
      Syn2& s = a.s[k];
      s.ll = (j == kLevels) ? nullptr : (j == 3) ? ctx->s.ll3 + ctx->s.ll3_off[b] : ctx->s.ll2 + ctx->s.ll2_off[b];
      s.W = W;
      s.I = S.I;
      s.off[0] = S.off[b][j][0]; s.off[1] = S.off[b][j][1]; s.off[2] = S.off[b][j][2];
      s.off[3] = S.off[b][kLevels][3];
      s.mo1 = S.rows[b][j]; s.mo2 = S.cols[b][j];
      s.m1 = S.rows[b][j - 1]; s.m2 = S.cols[b][j - 1];
      a.out[k] = (j == 2) ? slots + ctx->s.ll1_off[b] : (j == 3) ? ctx->s.ll2 + ctx->s.ll2_off[b]
                                                                 : ctx->s.ll3 + ctx->s.ll3_off[b];
      a.tiles_x[k] = (s.m2 + kT2 - 1) / kT2;
      a.tile0[k] = t0;
      a.F[k] = 2 * (b + 1);
      t0 += a.tiles_x[k] * ((s.m1 + kT2 - 1) / kT2);
    }
    int tiles[8];
    for (int k = 0; k < 8; ++k) tiles[k] = (k + 1 < 8 ? a.tile0[k + 1] : t0) - a.tile0[k];
    if (sara_level_per_basis(tiles, L)) {
      for (int k = 0; k < 8; ++k) {
        FHS_F_SWITCH(a.F[k], k_syn2_one, dim3(tiles[k], L), a.s[k], a.out[k], a.tiles_x[k]);
      }
      note_launches(8);
    } else {
      k_syn2_all<<<dim3(t0, L), 256, 0, st>>>(a);
      note_launches(1);
    }
  }
  for (int b = 0; b < 8; ++b) {
    Syn2& f = fin.lv[b];
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
  fin.vec4 = (cb.n2 % 4 == 0 && S.dirac_off % 4 == 0 && S.I % 4 == 0 && ((uintptr_t)A % 16) == 0 &&
              ((uintptr_t)W % 16) == 0) ? 1 : 0;
  dim3 g((cb.n2 + kT2 - 1) / kT2, (cb.n1 + kT2 - 1) / kT2, L);
  k_synfin<<<g, 256, 0, st>>>(fin, A);
  note_launches(1);
}

bool sara_fast_supported(const Cube&) { return true; }

}  // namespace fhs
