// Register-resident row DFT of length N = R1 * R2 * R3 (2048, 4096, 8192) for the
// fast path, included by nufft.cu inside namespace fhs.
//
// One CTA transforms one grid row with NT = R2 * R3 threads, each holding E = R1
// values, in three register passes with two shared-memory exchanges (against five
// Stockham passes of the shared-memory FFT):
//   n = b + NT a (b < NT, a < R1),  k = k_a + R1 (k_c + R2 k_d),  b = d + R3 c.
//   1. thread b: R1-point DFT over a of x[b + NT a] (coalesced loads straight
//      from the grid row), times w_N^{b k_a};
//   2. task (k_a, d): R2-point DFT over c, times w_NT^{d k_c};
//   3. task (k_a, k_c): R3-point DFT over d, stored to k (coalesced).
// Exchanges use a [R1][NT + 1] float2 buffer: lanes of a warp differ in k_a, so
// the padded row stride makes every exchange access two wavefronts (the minimum
// for 64-bit accesses).  Forward rows read only the n2 image columns (the others
// are zero); inverse rows store only those columns.

// exp(-2 pi i j / 32), j < 16
__constant__ float2 c_w32[16] = {
    {1.f, 0.f},                          {9.807852804e-01f, -1.950903220e-01f},
    {9.238795325e-01f, -3.826834324e-01f}, {8.314696123e-01f, -5.555702330e-01f},
    {7.071067812e-01f, -7.071067812e-01f}, {5.555702330e-01f, -8.314696123e-01f},
    {3.826834324e-01f, -9.238795325e-01f}, {1.950903220e-01f, -9.807852804e-01f},
    {0.f, -1.f},                           {-1.950903220e-01f, -9.807852804e-01f},
    {-3.826834324e-01f, -9.238795325e-01f}, {-5.555702330e-01f, -8.314696123e-01f},
    {-7.071067812e-01f, -7.071067812e-01f}, {-8.314696123e-01f, -5.555702330e-01f},
    {-9.238795325e-01f, -3.826834324e-01f}, {-9.807852804e-01f, -1.950903220e-01f},
};

// In-place R-point DFT of v (natural order in and out), radix-2 decimation in time
// down to the 8-, 4- and 2-point kernels; sign exp(-2 pi i / R), INV flips it.
template <int R, bool INV>
__device__ __forceinline__ void rdft(float2* v) {
  if constexpr (R == 2) {
    dft2(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4(v[0], v[1], v[2], v[3], INV);
  } else if constexpr (R == 8) {
    dft8(v, INV);
  } else {
    constexpr int H = R / 2;
    float2 e[H], o[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
      e[k] = v[2 * k];
      o[k] = v[2 * k + 1];
    }
    rdft<H, INV>(e);
    rdft<H, INV>(o);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      float2 t;
      if (k == 0) {
        t = o[0];
      } else if (2 * k == H) {               // w = -i (forward), +i (inverse)
        t = INV ? make_float2(-o[k].y, o[k].x) : make_float2(o[k].y, -o[k].x);
      } else {
        float2 w = c_w32[k * (32 / R)];
        if (INV) w.y = -w.y;
        t = cmul(o[k], w);
      }
      v[k] = cadd(e[k], t);
      v[k + H] = csub(e[k], t);
    }
  }
}

template <int N> struct RegRowCfg;
template <> struct RegRowCfg<2048> { static constexpr int R1 = 16, R2 = 16, R3 = 8; };
template <> struct RegRowCfg<4096> { static constexpr int R1 = 16, R2 = 16, R3 = 16; };
template <> struct RegRowCfg<8192> { static constexpr int R1 = 32, R2 = 16, R3 = 16; };

template <int N>
struct RegRow {
  static constexpr int R1 = RegRowCfg<N>::R1, R2 = RegRowCfg<N>::R2, R3 = RegRowCfg<N>::R3;
  static constexpr int NT = R2 * R3;
  static constexpr int LD = NT + 1;
  static constexpr int SMEM = R1 * LD * (int)sizeof(float2);
  static_assert(R1 * NT == N, "factorisation");
};

template <int N, bool INV>
__global__ void __launch_bounds__(RegRow<N>::NT, 2) k_rowr(float2* __restrict__ grid, int K1, int n2,
                                                           const float2* __restrict__ tw, int twstride) {
  using C = RegRow<N>;
  constexpr int NT = C::NT, R1 = C::R1, R2 = C::R2, R3 = C::R3, LD = C::LD;
  constexpr int LOG1 = ilog2c(R1);
  extern __shared__ float2 sm[];
  const int t = threadIdx.x;
  float2* row = grid + ((size_t)blockIdx.y * K1 + blockIdx.x) * N;
  const int h2 = n2 / 2;

  // ---- pass 1: R1-point DFT over a of x[t + NT a], twiddle w_N^{t k_a}
  {
    float2 v[R1];
#pragma unroll
    for (int a = 0; a < R1; ++a) {
      const int n = t + NT * a;
      const bool in = INV || n < h2 || n >= N - h2;
      v[a] = in ? row[n] : make_float2(0.f, 0.f);
    }
    rdft<R1, INV>(v);
    // w^(2^j), w = w_N^t, from the table; w^k as products over the set bits of k
    float2 wp[LOG1];
#pragma unroll
    for (int j = 0; j < LOG1; ++j) {
      float2 w = __ldg(&tw[(size_t)((t << j) & (N - 1)) * twstride]);
      if (INV) w.y = -w.y;
      wp[j] = w;
    }
#pragma unroll
    for (int k = 1; k < R1; ++k) {
      float2 w = make_float2(1.f, 0.f);
      bool first = true;
#pragma unroll
      for (int j = 0; j < LOG1; ++j) {
        if ((k >> j) & 1) {
          w = first ? wp[j] : cmul(w, wp[j]);
          first = false;
        }
      }
      v[k] = cmul(v[k], w);
    }
#pragma unroll
    for (int k = 0; k < R1; ++k) sm[k * LD + t] = v[k];
  }
  __syncthreads();

  // ---- pass 2: tasks (k_a, d), R2-point DFT over c of Y[d + R3 c][k_a], twiddle w_NT^{d k_c}
  constexpr int J2 = R1 * R3 / NT;
  {
    float2 u[J2][R2];
#pragma unroll
    for (int j = 0; j < J2; ++j) {
      const int s = t + NT * j;
      const int ka = s % R1, d = s / R1;
#pragma unroll
      for (int c = 0; c < R2; ++c) u[j][c] = sm[ka * LD + d + R3 * c];
      rdft<R2, INV>(u[j]);
#pragma unroll
      for (int kc = 1; kc < R2; ++kc) {
        float2 w = __ldg(&tw[(size_t)(((d * kc) & (NT - 1)) * R1) * twstride]);
        if (INV) w.y = -w.y;
        u[j][kc] = cmul(u[j][kc], w);
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < J2; ++j) {
      const int s = t + NT * j;
      const int ka = s % R1, d = s / R1;
#pragma unroll
      for (int kc = 0; kc < R2; ++kc) sm[ka * LD + d * R2 + kc] = u[j][kc];
    }
  }
  __syncthreads();

  // ---- pass 3: tasks (k_a, k_c), R3-point DFT over d; k = task + (N / R3) k_d
  constexpr int J3 = R1 * R2 / NT;
#pragma unroll
  for (int j = 0; j < J3; ++j) {
    const int s = t + NT * j;
    const int ka = s % R1, kc = s / R1;
    float2 z[R3];
#pragma unroll
    for (int d = 0; d < R3; ++d) z[d] = sm[ka * LD + d * R2 + kc];
    rdft<R3, INV>(z);
#pragma unroll
    for (int kd = 0; kd < R3; ++kd) {
      const int k = s + (N / R3) * kd;
      if (!INV || k < h2 || k >= N - h2) row[k] = z[kd];
    }
  }
}

// ------------------------------------------------------------------ columns
// Register-resident column DFT of length N = R1 * 8 (64, 128, 256) over 32 adjacent
// grid columns (one per lane) and 8 row groups (one per warp):
//   i = i0 + 8 m (i0 = warp, m < R1),  k = k_m + R1 k_i;
//   pass 1: R1-point DFT over m of the thread's column, times w_N^{i0 k_m};
//   pass 2: tasks k_m (warp-strided), 8-point DFT over i0.
// One exchange through a [R1][8][32] float2 buffer (lanes = columns: conflict-free).
// load(i) returns element i of the thread's column; store(k, v) writes output k.
template <int N> struct RegCol {
  static constexpr int R1 = N / 8;
  static constexpr int SMEM = N * 32 * (int)sizeof(float2);
};

template <int N, bool INV, class Load, class Store>
__device__ __forceinline__ void col_fft_reg(float2* sm, const float2* __restrict__ tw, int twstride, Load load,
                                            Store store) {
  constexpr int R1 = RegCol<N>::R1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = load(w + 8 * m);
    rdft<R1, INV>(v);
#pragma unroll
    for (int km = 1; km < R1; ++km) {
      float2 t = __ldg(&tw[(size_t)((w * km) & (N - 1)) * twstride]);
      if (INV) t.y = -t.y;
      v[km] = cmul(v[km], t);
    }
#pragma unroll
    for (int km = 0; km < R1; ++km) sm[(km * 8 + w) * 32 + lane] = v[km];
  }
  __syncthreads();
#pragma unroll
  for (int km = w; km < R1; km += 8) {
    float2 z[8];
#pragma unroll
    for (int i0 = 0; i0 < 8; ++i0) z[i0] = sm[(km * 8 + i0) * 32 + lane];
    rdft<8, INV>(z);
#pragma unroll
    for (int ki = 0; ki < 8; ++ki) store(km + R1 * ki, z[ki]);
  }
}

// Step A forward (Z fused) for group g, image columns c0 .. c0 + 31 (see k_colA_fwd).
template <int N>
__global__ void __launch_bounds__(256) k_colA_fwd_r(const float* __restrict__ x, float2* __restrict__ grid,
                                                    const float* __restrict__ sr, const float* __restrict__ sc,
                                                    int n1, int n2, int K1, int K2, int N2c,
                                                    const float2* __restrict__ tw, int twN, int twK) {
  extern __shared__ float2 sm[];
  const int l = blockIdx.z, g = blockIdx.y, cc = blockIdx.x * 32 + (threadIdx.x & 31);
  const float* xl = x + (size_t)l * n1 * n2;
  float2* gl = grid + (size_t)l * K1 * K2;
  const int h1 = n1 / 2, h2 = n2 / 2;
  const bool col_ok = cc < n2;
  const int c = cc < h2 ? cc + h2 : cc - h2;
  const float scc = col_ok ? sc[c] : 0.f;
  const int gcol = colmap(cc, n2, K2);
  auto load = [&](int i) {
    const int rho = N2c * i + g;
    const int r = rho < h1 ? rho + h1 : (rho >= K1 - h1 ? rho - (K1 - h1) : -1);
    float val = 0.f;
    if (r >= 0 && col_ok) val = xl[(size_t)r * n2 + c] * sr[r] * scc;
    return make_float2(val, 0.f);
  };
  auto store = [&](int k, float2 v) {
    if (!col_ok) return;
    if (N2c > 1) v = cmul(v, __ldg(&tw[(size_t)(g * k) * twK]));
    gl[(size_t)(N2c * k + g) * K2 + gcol] = v;
  };
  col_fft_reg<N, false>(sm, tw, twN, load, store);
}

// Step B (both directions): group k1, rows N k1 + i (see k_colB).
template <int N, bool INV>
__global__ void __launch_bounds__(256) k_colB_r(float2* __restrict__ grid, int n2, int K1, int K2,
                                                const float2* __restrict__ tw, int twN) {
  extern __shared__ float2 sm[];
  const int l = blockIdx.z, k1 = blockIdx.y, cc = blockIdx.x * 32 + (threadIdx.x & 31);
  float2* gl = grid + (size_t)l * K1 * K2 + (size_t)N * k1 * K2;
  const bool col_ok = cc < n2;
  const int gcol = colmap(cc, n2, K2);
  auto load = [&](int i) { return col_ok ? gl[(size_t)i * K2 + gcol] : make_float2(0.f, 0.f); };
  auto store = [&](int k, float2 v) {
    if (col_ok) gl[(size_t)k * K2 + gcol] = v;
  };
  col_fft_reg<N, INV>(sm, tw, twN, load, store);
}

// Step A^H with the crop fused (see k_colA_adj).
template <int N>
__global__ void __launch_bounds__(256) k_colA_adj_r(const float2* __restrict__ grid, float* __restrict__ out,
                                                    const float* __restrict__ sr, const float* __restrict__ sc,
                                                    const float* __restrict__ eta, int accumulate, int n1, int n2,
                                                    int K1, int K2, int N2c, const float2* __restrict__ tw, int twN,
                                                    int twK) {
  extern __shared__ float2 sm[];
  const int l = blockIdx.z, g = blockIdx.y, cc = blockIdx.x * 32 + (threadIdx.x & 31);
  const float2* gl = grid + (size_t)l * K1 * K2;
  const bool col_ok = cc < n2;
  const int gcol = colmap(cc, n2, K2);
  const int h1 = n1 / 2, h2 = n2 / 2;
  const int c = cc < h2 ? cc + h2 : cc - h2;
  const float e = (eta ? eta[l] : 1.f) * (col_ok ? sc[c] : 0.f);
  float* ol = out + (size_t)l * n1 * n2;
  auto load = [&](int i) {
    float2 v = make_float2(0.f, 0.f);
    if (col_ok) {
      v = gl[(size_t)(N2c * i + g) * K2 + gcol];
      if (N2c > 1) v = cmul(v, cconj(__ldg(&tw[(size_t)(g * i) * twK])));
    }
    return v;
  };
  auto store = [&](int k, float2 v) {
    const int rho = N2c * k + g;
    const int r = rho < h1 ? rho + h1 : (rho >= K1 - h1 ? rho - (K1 - h1) : -1);
    if (r < 0 || !col_ok) return;
    const float val = e * sr[r] * v.x;
    const size_t o = (size_t)r * n2 + c;
    ol[o] = accumulate ? ol[o] + val : val;
  };
  col_fft_reg<N, true>(sm, tw, twN, load, store);
}
