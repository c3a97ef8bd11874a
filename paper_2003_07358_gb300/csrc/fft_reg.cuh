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

// Packed column transform of the two-for-one path: [L][K1][n2/2] complex, rows in the
// column transform's physical order, frequency k at ((k & (N1c - 1)) << lg2) | (k >> lg1).
struct RowPack {
  const float2* P;
  int N1c, lg1, lg2;
};

// Frequency pair (k, K1 - k) of CTA c, enumerated so that consecutive CTAs take consecutive
// physical rows k1 N2c + k2 (k = k1 + N1c k2) and their partners consecutive rows in reverse:
// k1 = 0 with k2 <= N2c/2, then 0 < k1 < N1c/2 with every k2, then k1 = N1c/2 with
// k2 < N2c/2; K1/2 + 1 pairs in all, the self-conjugate rows 0 and K1/2 included.
__device__ __forceinline__ int pair_frequency(int c, int N1c, int N2c) {
  const int h = N2c / 2;
  int k1, k2;
  if (c <= h) { k1 = 0; k2 = c; }
  else if (c < h + 1 + (N1c / 2 - 1) * N2c) { const int e = c - (h + 1); k1 = 1 + e / N2c; k2 = e % N2c; }
  else { k1 = N1c / 2; k2 = c - (h + 1 + (N1c / 2 - 1) * N2c); }
  return k1 + N1c * k2;
}

template <int N, bool INV, class Store>
__device__ __forceinline__ void row_dft_reg(float2 (&v)[RegRow<N>::R1], float2* sm, const float2* __restrict__ tw,
                                            int twstride, Store store) {
  using C = RegRow<N>;
  constexpr int NT = C::NT, R1 = C::R1, R2 = C::R2, R3 = C::R3, LD = C::LD;
  constexpr int LOG1 = ilog2c(R1);
  const int t = threadIdx.x;
  {
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
    store(j, s, z);
  }
}

template <int N, bool INV>
__global__ void __launch_bounds__(RegRow<N>::NT, 2) k_rowr(float2* __restrict__ grid, int K1, int n2,
                                                           const float2* __restrict__ tw, int twstride) {
  using C = RegRow<N>;
  constexpr int NT = C::NT, R1 = C::R1, R3 = C::R3;
  extern __shared__ float2 sm[];
  const int t = threadIdx.x;
  float2* row = grid + ((size_t)blockIdx.y * K1 + blockIdx.x) * N;
  const int h2 = n2 / 2;
  float2 v[R1];
#pragma unroll
  for (int a = 0; a < R1; ++a) {
    const int n = t + NT * a;
    const bool in = INV || n < h2 || n >= N - h2;
    v[a] = in ? row[n] : make_float2(0.f, 0.f);
  }
  row_dft_reg<N, INV>(v, sm, tw, twstride, [&](int, int s, const float2* z) {
#pragma unroll
    for (int kd = 0; kd < R3; ++kd) {
      const int k = s + (N / R3) * kd;
      if (!INV || k < h2 || k >= N - h2) row[k] = z[kd];
    }
  });
}

// Forward row DFT of the frequency pair (k, K1 - k) from the packed column transform of
// the complex image columns y_j = x_{j + n2/2} + i x_j (j < n2/2, see k_colA_fwd_p).  The
// real columns' transforms follow from Hermitian symmetry, X_a[k] = (Y[k] + conj(Y[-k]))/2
// (grid column j) and X_b[k] = (Y[k] - conj(Y[-k]))/(2i) (grid column N - n2/2 + j); both
// packed rows are read by this CTA only (the second row's reloads hit L1).  Needs n2 = N/2.
template <int N>
__global__ void __launch_bounds__(RegRow<N>::NT, 2) k_rowr_fwd_p(float2* __restrict__ grid, int K1,
                                                                 const float2* __restrict__ tw, int twstride,
                                                                 RowPack pk) {
  using C = RegRow<N>;
  constexpr int NT = C::NT, R1 = C::R1, R3 = C::R3;
  constexpr int HP = N / 4;
  extern __shared__ float2 sm[];
  const int t = threadIdx.x;
  const int k = pair_frequency(blockIdx.x, pk.N1c, K1 / pk.N1c), km = (K1 - k) & (K1 - 1);
  const int prk = ((k & (pk.N1c - 1)) << pk.lg2) | (k >> pk.lg1);
  const int prm = ((km & (pk.N1c - 1)) << pk.lg2) | (km >> pk.lg1);
  const float2* yk = pk.P + ((size_t)blockIdx.y * K1 + prk) * HP;
  const float2* ym = pk.P + ((size_t)blockIdx.y * K1 + prm) * HP;
#pragma unroll 1
  for (int rr = 0; rr < (k == km ? 1 : 2); ++rr) {
    const float2* ya = rr ? ym : yk;                     // Y[+-k] and Y[-+k]
    const float2* yb = rr ? yk : ym;
    float2* row = grid + ((size_t)blockIdx.y * K1 + (rr ? prm : prk)) * N;
    if (rr) __syncthreads();                             // the exchange buffer is reused
    float2 v[R1];
#pragma unroll
    for (int a = 0; a < R1; ++a) {
      const int n = t + NT * a;
      v[a] = make_float2(0.f, 0.f);
      if (n < HP) {
        const float2 A = ya[n], B = yb[n];
        v[a] = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
      } else if (n >= N - HP) {
        const int j = n - (N - HP);
        const float2 A = ya[j], B = yb[j];
        v[a] = make_float2(0.5f * (A.y + B.y), -0.5f * (A.x - B.x));
      }
    }
    row_dft_reg<N, false>(v, sm, tw, twstride, [&](int, int s, const float2* z) {
#pragma unroll
      for (int kd = 0; kd < R3; ++kd) row[s + (N / R3) * kd] = z[kd];
    });
  }
}

// Inverse row DFT of the frequency pair (k, K1 - k) of CTA blockIdx.x (see pair_frequency), written
// as the packed input of the inverse column transform (two-for-one real output).  With A
// the row DFT^H outputs and image-column pair j (grid columns j and N - n2/2 + j):
//   c_j[k] = (A_j[k] + conj(A_j[-k])) / 2 + i (A_{N-n2/2+j}[k] + conj(A_{N-n2/2+j}[-k])) / 2,
// a Hermitian sequence plus i times another, so its column DFT^H is the real part of
// column j's plus i times the real part of column N - n2/2 + j's.  Row k's outputs of the
// two column ranges wait in shared memory while row -k is transformed.  Needs n2 = N / 2.
template <int N>
struct RegRowAdjP {
  static constexpr int J3 = RegRow<N>::R1 * RegRow<N>::R2 / RegRow<N>::NT;
  static constexpr int NA = RegRow<N>::R3 / 4;          // outputs per task in [0, N/4)
  static constexpr int SMEM = RegRow<N>::SMEM + J3 * NA * 2 * RegRow<N>::NT * (int)sizeof(float2);
};

template <int N>
__global__ void __launch_bounds__(RegRow<N>::NT, 2) k_rowr_adj_p(const float2* __restrict__ grid, float2* __restrict__ P,
                                                                 int K1, const float2* __restrict__ tw, int twstride,
                                                                 RowPack pk) {
  using C = RegRow<N>;
  constexpr int NT = C::NT, R1 = C::R1, R3 = C::R3, LD = C::LD;
  constexpr int NA = RegRowAdjP<N>::NA;
  constexpr int HP = N / 4;
  static_assert(NA * (N / R3) == HP, "a task's first NA outputs are the first image columns");
  extern __shared__ float2 sm[];
  float2* hold = sm + R1 * LD;                            // [J3][NA][2][NT]
  const int t = threadIdx.x;
  const int k = pair_frequency(blockIdx.x, pk.N1c, K1 / pk.N1c), km = (K1 - k) & (K1 - 1);
  const int prk = ((k & (pk.N1c - 1)) << pk.lg2) | (k >> pk.lg1);
  const int prm = ((km & (pk.N1c - 1)) << pk.lg2) | (km >> pk.lg1);
  const float2* gk = grid + ((size_t)blockIdx.y * K1 + prk) * N;
  const float2* gm = grid + ((size_t)blockIdx.y * K1 + prm) * N;
  float2* ck = P + ((size_t)blockIdx.y * K1 + prk) * HP;
  float2* cm = P + ((size_t)blockIdx.y * K1 + prm) * HP;
#pragma unroll 1
  for (int rr = 0; rr < 2; ++rr) {
    const float2* g = rr ? gm : gk;
    if (rr) __syncthreads();                              // the exchange buffer is reused
    float2 v[R1];
#pragma unroll
    for (int a = 0; a < R1; ++a) v[a] = g[t + NT * a];
    row_dft_reg<N, true>(v, sm, tw, twstride, [&](int j, int s, const float2* z) {
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        float2* hk = hold + ((j * NA + q) * 2) * NT + t;
        if (rr == 0) {                                    // row k: park both column ranges
          hk[0] = z[q];
          hk[NT] = z[R3 - NA + q];
        } else {                                          // row -k: combine
          const float2 ak = hk[0], bk = hk[NT];
          const float2 am = z[q], bm = z[R3 - NA + q];
          const float2 ha = make_float2(0.5f * (ak.x + am.x), 0.5f * (ak.y - am.y));   // Hermitian part, column j
          const float2 hb = make_float2(0.5f * (bk.x + bm.x), 0.5f * (bk.y - bm.y));   // column N - N/4 + j
          const int col = s + (N / R3) * q;
          ck[col] = make_float2(ha.x - hb.y, ha.y + hb.x);   // ha + i hb
          cm[col] = make_float2(ha.x + hb.y, hb.x - ha.y);   // conj(ha) + i conj(hb)
        }
      }
    });
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

// Step A forward with two image columns per complex column (two-for-one real DFT):
// packed column j < n2/2 holds x_{j + n2/2} + i x_j (image columns, Z fused), i.e. the
// image columns that the grid places at column j and at column K2 - n2/2 + j.  Output:
// P [L][K1][n2/2] in the same row order as the in-place step A.
template <int N>
__global__ void __launch_bounds__(256) k_colA_fwd_p(const float* __restrict__ x, float2* __restrict__ P,
                                                    const float* __restrict__ sr, const float* __restrict__ sc,
                                                    int n1, int n2, int K1, int N2c, const float2* __restrict__ tw,
                                                    int twN, int twK) {
  extern __shared__ float2 sm[];
  const int hp = n2 / 2;
  const int l = blockIdx.z, g = blockIdx.y, j = blockIdx.x * 32 + (threadIdx.x & 31);
  const float* xl = x + (size_t)l * n1 * n2;
  float2* pl = P + (size_t)l * K1 * hp;
  const int h1 = n1 / 2;
  const bool ok = j < hp;
  const int ca = j + hp, cb = j;                      // image columns of the real and imaginary parts
  const float sa = ok ? sc[ca] : 0.f, sb = ok ? sc[cb] : 0.f;
  auto load = [&](int i) {
    const int rho = N2c * i + g;
    const int r = rho < h1 ? rho + h1 : (rho >= K1 - h1 ? rho - (K1 - h1) : -1);
    float2 v = make_float2(0.f, 0.f);
    if (r >= 0 && ok) {
      const float s = sr[r];
      v = make_float2(xl[(size_t)r * n2 + ca] * s * sa, xl[(size_t)r * n2 + cb] * s * sb);
    }
    return v;
  };
  auto store = [&](int k, float2 v) {
    if (!ok) return;
    if (N2c > 1) v = cmul(v, __ldg(&tw[(size_t)(g * k) * twK]));
    pl[(size_t)(N2c * k + g) * hp + j] = v;
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

// Step A^H from the packed inverse column transform (two-for-one): packed column j holds
// (column j) + i (column K2 - n2/2 + j) of the grid, i.e. the image columns j + n2/2 and
// j; crop, Z^T, real parts and eta fused into the store.
template <int N>
__global__ void __launch_bounds__(256) k_colA_adj_p(const float2* __restrict__ P, float* __restrict__ out,
                                                    const float* __restrict__ sr, const float* __restrict__ sc,
                                                    const float* __restrict__ eta, int accumulate, int n1, int n2,
                                                    int K1, int N2c, const float2* __restrict__ tw, int twN, int twK) {
  extern __shared__ float2 sm[];
  const int hp = n2 / 2;
  const int l = blockIdx.z, g = blockIdx.y, j = blockIdx.x * 32 + (threadIdx.x & 31);
  const float2* pl = P + (size_t)l * K1 * hp;
  const bool ok = j < hp;
  const int ca = j + hp, cb = j;
  const float el = eta ? eta[l] : 1.f;
  const float ea = ok ? el * sc[ca] : 0.f, eb = ok ? el * sc[cb] : 0.f;
  float* ol = out + (size_t)l * n1 * n2;
  const int h1 = n1 / 2;
  auto load = [&](int i) {
    float2 v = make_float2(0.f, 0.f);
    if (ok) {
      v = pl[(size_t)(N2c * i + g) * hp + j];
      if (N2c > 1) v = cmul(v, cconj(__ldg(&tw[(size_t)(g * i) * twK])));
    }
    return v;
  };
  auto store = [&](int k, float2 v) {
    const int rho = N2c * k + g;
    const int r = rho < h1 ? rho + h1 : (rho >= K1 - h1 ? rho - (K1 - h1) : -1);
    if (r < 0 || !ok) return;
    const float s = sr[r];
    const size_t oa = (size_t)r * n2 + ca, ob = (size_t)r * n2 + cb;
    const float va = ea * s * v.x, vb = eb * s * v.y;
    ol[oa] = accumulate ? ol[oa] + va : va;
    ol[ob] = accumulate ? ol[ob] + vb : vb;
  };
  col_fft_reg<N, true>(sm, tw, twN, load, store);
}
